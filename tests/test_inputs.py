"""The seeded input generator: determinism, ranges, shapes (CPU only)."""
import numpy as np

from paper_1907_02731_gb300 import inputs


def test_deterministic_and_in_range():
    a, ma = inputs.make_video(5, 48, 64, seed=123, n_distractors=2)
    b, mb = inputs.make_video(5, 48, 64, seed=123, n_distractors=2)
    c, _ = inputs.make_video(5, 48, 64, seed=124, n_distractors=2)
    assert a.dtype == np.float32 and a.shape == (5, 48, 64)
    assert np.array_equal(a, b) and np.array_equal(ma, mb)
    assert not np.array_equal(a, c)
    assert a.min() >= 0.0 and a.max() <= 1.0
    # object interior is brighter than the background on average
    assert a[ma == 1].mean() > 0.6 > 0.3 > a[ma == 0].mean()
    assert ma.sum() > 0


def test_small_workload_shape():
    f, m = inputs.workload_video("small_16x64x64")
    wl = inputs.WORKLOADS["small_16x64x64"]
    assert f.shape == (wl.nf, wl.h, wl.w) == (16, 64, 64)
    assert (wl.rt, wl.ry, wl.rx) == (3, 3, 3)


def test_batch_layout():
    dims = inputs.batch_layout()
    assert len(dims) == 24
    for nf, h, w in dims:
        assert 20 <= nf <= 120
        assert (w, h) in inputs.BATCH_RESOLUTIONS
    assert dims == inputs.batch_layout()
    vids = inputs.batch_videos(n_videos=3, scale=0.1)
    assert len(vids) == 3 and all(v.ndim == 3 for v in vids)


def test_workload_features_channels():
    """Eq. 9 workload: channel 0 is the video S, the other channel a distinct
    seeded video of the same shape; single-channel workloads return f = s."""
    from paper_1907_02731_gb300 import inputs
    wl = inputs.WORKLOADS["video2ch_72x480x854"]
    assert wl.nchan == 2
    small = dict(nf=3, h=20, w=30)
    import dataclasses
    inputs.WORKLOADS["_tiny2ch"] = dataclasses.replace(wl, name="_tiny2ch", **small)
    try:
        s, f = inputs.workload_features("_tiny2ch")
        s2, f2 = inputs.workload_features("_tiny2ch")
        assert f.shape == (2, 3, 20, 30) and f.dtype == np.float32
        np.testing.assert_array_equal(f[0], s)
        assert not np.array_equal(f[1], f[0])
        np.testing.assert_array_equal(f, f2)
    finally:
        del inputs.WORKLOADS["_tiny2ch"]
    s1, f1 = inputs.workload_features("small_16x64x64")
    assert f1 is s1
