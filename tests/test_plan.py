"""Host-side work decomposition of the specialised step kernel (CPU only):
every (tile, frame) unit is covered exactly once, each CTA gets the same
number of output frames up to one, and a video's segments are contiguous."""
import collections

import pytest

import paper_1907_02731_gb300 as sf
from paper_1907_02731_gb300 import build as sfbuild
from paper_1907_02731_gb300 import inputs

TX, TY = 112, 12


@pytest.fixture(scope="module", autouse=True)
def _lib():
    sfbuild.build()


def _check(dims, sms):
    segs, cta = sf.sfseg_plan_segments(dims, sms)
    n_cta = len(cta) - 1
    assert 1 <= n_cta <= sms and cta[0] == 0 and cta[-1] == len(segs)
    assert all(a <= b for a, b in zip(cta, cta[1:]))
    cover = collections.Counter()
    per_cta = []
    for c in range(n_cta):
        frames = 0
        for v, x0, y0, t0, t1 in segs[cta[c]:cta[c + 1]]:
            nf, h, w = dims[v]
            assert x0 % TX == 0 and y0 % TY == 0 and x0 < w and y0 < h
            assert 0 <= t0 < t1 <= nf
            for t in range(t0, t1):
                cover[(v, x0, y0, t)] += 1
            frames += t1 - t0
        per_cta.append(frames)
    expect = sum(nf * -(-w // TX) * -(-h // TY) for nf, h, w in dims)
    assert len(cover) == expect and set(cover.values()) == {1}
    assert max(per_cta) - min(per_cta) <= 1
    # whole-tile rounds per video: CTA c streams that video's tiles c, c + n_cta, ...
    for c in range(n_cta):
        k = cta[c]
        for v, (nf, h, w) in enumerate(dims):
            tv = [(x0, y0) for y0 in range(0, h, TY) for x0 in range(0, w, TX)]
            for r in range(len(tv) // n_cta):
                sv, x0, y0, t0, t1 = segs[k]
                assert (sv, (x0, y0), t0, t1) == (v, tv[c + r * n_cta], 0, nf)
                k += 1
    return segs, n_cta


def test_plan_full_video():
    segs, n_cta = _check([(72, 480, 854)], 152)
    assert n_cta == 152


def test_plan_uneven_batch():
    _check(inputs.batch_layout(), 152)


@pytest.mark.parametrize("dims", [[(1, 1, 1)], [(3, 5, 7)], [(16, 64, 64)], [(9, 200, 129), (2, 3, 4)]])
def test_plan_small(dims):
    segs, n_cta = _check(dims, 152)
    units = sum(nf * -(-w // TX) * -(-h // TY) for nf, h, w in dims)
    assert n_cta == max(1, min(152, units // 8))


def test_plan_rejects_empty():
    with pytest.raises(sf.SFSegError):
        sf.sfseg_plan_segments([(0, 4, 4)], 152)
