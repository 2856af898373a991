"""Seeded synthetic inputs: video feature volumes of the paper's shapes.

This module holds no arithmetic of the method itself (no affinity, no
convolution, no power iteration).  It only draws feature volumes and masks,
and it is the one piece shared by the CUDA path's tests/bench and the oracle's
tests: both sides consume the same bytes.

The paper evaluates on DAVIS-2016 (854x480 videos, tens of frames; Sec. 5)
and SegTrackv2.  Neither dataset is available here, so these seeded videos
stand in for them with the same shapes: a moving elliptical object over a
cluttered background, plus moving distractor blobs and Gaussian noise,
clamped to [0, 1] like a soft segmentation / flow-magnitude map.

Recipe (per video, numpy PCG64, ``seed = 19070273 + 1000*config + index``):
  * background: iid U(0, 0.3) per voxel;
  * object: ellipse with semi-axes (W/8, H/6), random orientation, centre
    uniform in the middle half of the frame, moving linearly at a speed
    U(2, 6) px/frame in a random direction and reflecting at the borders;
    interior iid U(0.7, 0.9) per voxel;
  * distractors: ``n_distractors`` ellipses of half the object's size,
    centre uniform over the frame, own speed U(2, 6), interior U(0.4, 0.6);
  * noise: + N(0, 0.05) everywhere, then clamp to [0, 1];
  * mask: the object's support (uint8 0/1).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

BASE_SEED = 19070273


def config_seed(config: int, index: int = 0) -> int:
    """Seed of video ``index`` of workload ``config``."""
    return BASE_SEED + 1000 * int(config) + int(index)


@dataclasses.dataclass(frozen=True)
class Workload:
    """One named workload: volume shape, Gaussian support and iteration count.

    Radii are half-extents: an ``a x b x c`` kernel (x-taps x y-taps x t-taps)
    has rx = (a-1)/2, ry = (b-1)/2, rt = (c-1)/2.
    """
    name: str
    nf: int
    h: int
    w: int
    rt: int
    ry: int
    rx: int
    sigma_t: float
    sigma_xy: float
    iters: int
    p: float
    alpha: float
    n_distractors: int
    config: int
    nchan: int = 1          # pairwise feature channels (Eq. 9)

    @property
    def n(self) -> int:
        return self.nf * self.h * self.w


# The five workloads (the paper's resolution 854x480; alpha = 1 and p = 0.1
# are the paper's unsupervised setting of Sec. 5; p = 1 for the
# differentiable workload because d(f^p)/df is unbounded at f = 0 for p < 1).
WORKLOADS = {
    "small_16x64x64": Workload("small_16x64x64", 16, 64, 64, 3, 3, 3, 1.5, 2.0,
                               30, 0.1, 1.0, 0, 1),
    "video_72x480x854": Workload("video_72x480x854", 72, 480, 854, 2, 5, 5, 1.5,
                                 3.0, 50, 0.1, 1.0, 2, 2),
    "video_72x480x854_lowp": Workload("video_72x480x854_lowp", 72, 480, 854, 2,
                                      5, 5, 1.5, 3.0, 50, 0.1, 1.0, 2, 3),
    "grad_48x480x854": Workload("grad_48x480x854", 48, 480, 854, 2, 5, 5, 1.5,
                                3.0, 40, 1.0, 1.0, 2, 5),
    # the uneven batch (shapes from batch_layout); nf/h/w here are unused
    "batch_24": Workload("batch_24", 0, 0, 0, 2, 4, 4, 1.5, 2.5, 50, 0.1, 1.0, 2, 4),
    # two pairwise channels (Eq. 9), as with the paper's forward and backward
    # optical-flow magnitudes: S = channel 0 = the video, channel 1 a second
    # seeded video of the same shape
    "video2ch_72x480x854": Workload("video2ch_72x480x854", 72, 480, 854, 2, 5, 5, 1.5, 3.0, 50,
                                    0.1, 1.0, 2, 6, nchan=2),
}

# Uneven batch: 24 videos, frames U{20..120}, resolution from this set,
# 9x9x5 kernel (sigma_xy = 2.5, sigma_t = 1.5).
BATCH_RESOLUTIONS = ((320, 240), (480, 360), (640, 360), (854, 480))
BATCH_CONFIG = 4
BATCH_VIDEOS = 24


def _ellipse_mask(h: int, w: int, cx: float, cy: float, ax: float, ay: float,
                  theta: float, yy: np.ndarray, xx: np.ndarray) -> np.ndarray:
    c, s = math.cos(theta), math.sin(theta)
    dx = xx - cx
    dy = yy - cy
    u = (c * dx + s * dy) / ax
    v = (-s * dx + c * dy) / ay
    return (u * u + v * v) <= 1.0


def _reflect(pos: float, lo: float, hi: float) -> float:
    """Reflect a coordinate into [lo, hi] (billiard motion)."""
    span = hi - lo
    if span <= 0:
        return lo
    q = (pos - lo) % (2 * span)
    return lo + (q if q <= span else 2 * span - q)


def make_video(nf: int, h: int, w: int, seed: int, n_distractors: int = 2):
    """Draw one seeded video.

    Returns ``(f, mask)``: ``f`` float32 ``[nf, h, w]`` in [0, 1] and ``mask``
    uint8 ``[nf, h, w]`` (object support).
    """
    rng = np.random.default_rng(seed)
    # Trajectories first (a fixed number of draws), then the per-frame fields.
    ax, ay = w / 8.0, h / 6.0
    obj = dict(cx=rng.uniform(w / 4, 3 * w / 4), cy=rng.uniform(h / 4, 3 * h / 4),
               theta=rng.uniform(0, math.pi), speed=rng.uniform(2, 6),
               phi=rng.uniform(0, 2 * math.pi), ax=ax, ay=ay)
    dis = []
    for _ in range(n_distractors):
        dis.append(dict(cx=rng.uniform(0, w), cy=rng.uniform(0, h),
                        theta=rng.uniform(0, math.pi), speed=rng.uniform(2, 6),
                        phi=rng.uniform(0, 2 * math.pi), ax=ax / 2, ay=ay / 2))
    f = np.empty((nf, h, w), np.float32)
    mask = np.empty((nf, h, w), np.uint8)
    yy, xx = np.mgrid[0:h, 0:w].astype(np.float32)
    for t in range(nf):
        frame = rng.random((h, w), dtype=np.float32) * np.float32(0.3)
        for d in dis:
            cx = _reflect(d["cx"] + t * d["speed"] * math.cos(d["phi"]), 0, w - 1)
            cy = _reflect(d["cy"] + t * d["speed"] * math.sin(d["phi"]), 0, h - 1)
            m = _ellipse_mask(h, w, cx, cy, d["ax"], d["ay"], d["theta"], yy, xx)
            vals = rng.random((h, w), dtype=np.float32) * np.float32(0.2) + np.float32(0.4)
            frame[m] = vals[m]
        cx = _reflect(obj["cx"] + t * obj["speed"] * math.cos(obj["phi"]), 0, w - 1)
        cy = _reflect(obj["cy"] + t * obj["speed"] * math.sin(obj["phi"]), 0, h - 1)
        m = _ellipse_mask(h, w, cx, cy, obj["ax"], obj["ay"], obj["theta"], yy, xx)
        vals = rng.random((h, w), dtype=np.float32) * np.float32(0.2) + np.float32(0.7)
        frame[m] = vals[m]
        frame += rng.standard_normal((h, w), dtype=np.float32) * np.float32(0.05)
        np.clip(frame, 0.0, 1.0, out=frame)
        f[t] = frame
        mask[t] = m
    return f, mask


def workload_video(name: str, index: int = 0):
    """The seeded feature volume (and object mask) of a named workload."""
    wl = WORKLOADS[name]
    return make_video(wl.nf, wl.h, wl.w, config_seed(wl.config, index),
                      wl.n_distractors)


def channel_seed(config: int, index: int, channel: int) -> int:
    """Seed of pairwise channel ``channel`` >= 1 of video ``index``."""
    return config_seed(config, index) + 7919 * int(channel)


def workload_features(name: str, index: int = 0):
    """(s, f) of a named workload: s = the seeded video; f = s for one
    channel, else [nchan, nf, h, w] with channel 0 = s and channel c a video
    drawn from ``channel_seed``."""
    wl = WORKLOADS[name]
    s, _ = make_video(wl.nf, wl.h, wl.w, config_seed(wl.config, index), wl.n_distractors)
    if wl.nchan == 1:
        return s, s
    chans = [s] + [make_video(wl.nf, wl.h, wl.w, channel_seed(wl.config, index, c),
                              wl.n_distractors)[0] for c in range(1, wl.nchan)]
    return s, np.ascontiguousarray(np.stack(chans))


def batch_layout(n_videos: int = BATCH_VIDEOS, config: int = BATCH_CONFIG):
    """Frame counts and resolutions of the uneven batch: list of (nf, h, w)."""
    rng = np.random.default_rng(config_seed(config, 999))
    dims = []
    for _ in range(n_videos):
        nf = int(rng.integers(20, 121))
        w, h = BATCH_RESOLUTIONS[int(rng.integers(0, len(BATCH_RESOLUTIONS)))]
        dims.append((nf, h, w))
    return dims


def batch_videos(n_videos: int = BATCH_VIDEOS, config: int = BATCH_CONFIG,
                 scale: float = 1.0):
    """The uneven batch: list of float32 volumes.  ``scale`` < 1 shrinks every
    video (frames and both spatial sizes) for quick tests."""
    out = []
    for i, (nf, h, w) in enumerate(batch_layout(n_videos, config)):
        nf_s = max(1, int(round(nf * scale)))
        h_s = max(1, int(round(h * scale)))
        w_s = max(1, int(round(w * scale)))
        f, _ = make_video(nf_s, h_s, w_s, config_seed(config, i), 2)
        out.append(f)
    return out


def random_volume(shape, seed: int, lo: float = 0.0, hi: float = 1.0):
    """iid uniform float32 volume, for unit tests of odd shapes."""
    rng = np.random.default_rng(seed)
    return (rng.random(shape, dtype=np.float64) * (hi - lo) + lo).astype(np.float32)
