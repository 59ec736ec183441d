"""Pins of the oracle's target view and LR-consistency check (§3.2.1, §3.2.2, eq. lrc), CPU.

What fixes them, other than themselves:
  * the target view's eq. (c) equals 1 - numpy.corrcoef of explicitly built clamped blocks;
  * the target view equals the reference view of the mirrored pair with the roles of the
    images exchanged (a geometric identity, computed through the reference-view routines);
  * on a fronto-parallel shift both views recover the shift and the check keeps the pixels
    whose match is inside the image;
  * on a scene with a foreground block the check removes the background strip that the
    block hides in the target view (an occlusion built with a z-buffer), and keeps the rest;
  * the rule itself on hand-made maps (|difference| 1 passes, 2 fails, partner outside fails).
"""
import numpy as np
import pytest

import oracle


@pytest.fixture(scope="module", autouse=True)
def _built():
    oracle.build()


def _clamped_block(img, u, v, rw):
    H, W = img.shape
    ys = np.clip(np.arange(v - rw, v + rw + 1), 0, H - 1)
    xs = np.clip(np.arange(u - rw, u + rw + 1), 0, W - 1)
    return img[np.ix_(ys, xs)].astype(np.float64)


def test_target_cost_is_one_minus_corrcoef_of_the_swapped_blocks():
    rng = np.random.default_rng(21)
    ref = rng.integers(0, 256, (20, 30), dtype=np.uint8)
    tgt = rng.integers(0, 256, (20, 30), dtype=np.uint8)
    for (u, v, d) in ((5, 7, 0), (10, 3, 4), (27, 19, 6), (0, 0, 9), (29, 10, 2)):
        a = _clamped_block(tgt, u, v, 3).ravel()
        b = _clamped_block(ref, u + d, v, 3).ravel()
        want = 1.0 - np.corrcoef(a, b)[0, 1]
        assert oracle.cost_tar(ref, tgt, u, v, d, 7) == pytest.approx(want, abs=1e-12)


def test_target_view_is_the_mirrored_reference_view():
    rng = np.random.default_rng(22)
    H, W, D = 24, 40, 8
    ref = rng.integers(0, 256, (H, W), dtype=np.uint8)
    tgt = np.roll(ref, -3, axis=1)
    tgt = np.clip(tgt.astype(int) + rng.integers(-6, 7, (H, W)), 0, 255).astype(np.uint8)
    dt_, eb, es = oracle.target_view(ref, tgt, D, 5, 5, 3.0, 10.0)
    # the target view of (ref, tgt) is the reference view of (mirror(tgt), mirror(ref))
    fr = np.ascontiguousarray(tgt[:, ::-1])
    ft = np.ascontiguousarray(ref[:, ::-1])
    _, dm, ebm, esm = oracle.stereo(fr, ft, np.zeros(H, np.float32), D, 5, 5, 3.0, 10.0)
    dm, ebm, esm = dm[:, ::-1], ebm[:, ::-1], esm[:, ::-1]
    assert np.abs(eb - ebm).max() < 1e-12 and np.abs(es - esm).max() < 1e-12
    sure = (es - eb) > 1e-9
    assert np.array_equal(dt_[sure], dm[sure])


def _textured(rng, H, W):
    from scipy import ndimage
    t = ndimage.gaussian_filter(rng.normal(size=(H, W)), 1.0)
    return np.clip(np.rint(128 + 40 * t / t.std()), 0, 255).astype(np.uint8)


def test_fronto_parallel_shift_is_consistent():
    rng = np.random.default_rng(23)
    H, W, D, d0 = 30, 72, 12, 5
    ref = _textured(rng, H, W)
    tgt = np.empty_like(ref)
    for x in range(W):
        tgt[:, x] = ref[:, min(x + d0, W - 1)]
    _, dref, _, _ = oracle.stereo(ref, tgt, np.zeros(H, np.float32), D, 5, 7, 3.0, 10.0)
    dtar, _, _ = oracle.target_view(ref, tgt, D, 5, 7, 3.0, 10.0)
    m = 5                                      # block + bilateral radius
    inner = (slice(m, H - m), slice(d0 + m, W - d0 - m))
    assert np.all(dref[inner] == d0)
    assert np.all(dtar[m:H - m, m:W - d0 - m] == d0)
    ok = oracle.lr_check(dref, dtar)
    assert np.all(ok[inner] == 1)
    # a reference pixel whose match would lie left of the target image fails
    assert np.all(ok[:, :d0][dref[:, :d0] > np.arange(d0)[None, :]] == 0)


def test_occluded_strip_is_removed():
    """Background at disparity 3, a foreground block (columns 30..45) at disparity 9: in the
    target the block covers target columns 21..36, hiding the background pixels 24..29."""
    rng = np.random.default_rng(24)
    H, W, D = 40, 90, 14
    ref = _textured(rng, H, W)
    disp = np.full(W, 3)
    disp[30:46] = 9
    tgt = np.zeros_like(ref)
    zbuf = np.full(W, -1)
    for u in range(W):                         # the nearest (largest d) point wins a target column
        x = u - disp[u]
        if 0 <= x < W and disp[u] > zbuf[x]:
            zbuf[x] = disp[u]
            tgt[:, x] = ref[:, u]
    for x in range(W):
        if zbuf[x] < 0:
            tgt[:, x] = tgt[:, x - 1]
    _, dref, _, _ = oracle.stereo(ref, tgt, np.zeros(H, np.float32), D, 5, 7, 3.0, 10.0)
    dtar, _, _ = oracle.target_view(ref, tgt, D, 5, 7, 3.0, 10.0)
    ok = oracle.lr_check(dref, dtar)
    rows = slice(6, H - 6)
    occluded = ok[rows, 24:30]
    assert occluded.mean() <= 0.2, occluded.mean()
    far = np.r_[15:18, 55:75]                  # background away from every edge
    assert ok[rows][:, far].mean() >= 0.98
    assert ok[rows, 35:41].mean() >= 0.95      # inside the foreground


def test_the_rule_on_hand_made_maps():
    dref = np.array([[0, 1, 2, 3, 5, 7]], np.int32)
    dtar = np.array([[0, 2, 0, 1, 3, 9]], np.int32)
    # u=0: partner 0, |0-0| = 0 keep; u=1: partner 0, |1-0| = 1 keep; u=2: partner 0, |2-0| = 2 drop;
    # u=3: partner 0, 3 drop; u=4: partner -1 outside, drop; u=5: partner -2 outside, drop
    assert oracle.lr_check(dref, dtar).tolist() == [[1, 1, 0, 0, 0, 0]]
    assert oracle.lr_check(dref, dtar, delta_r=4.0).tolist() == [[1, 1, 1, 0, 0, 0]]
    assert oracle.lr_check(dref, dtar, delta_r=0.0).tolist() == [[1, 0, 0, 0, 0, 0]]
