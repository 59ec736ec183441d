"""Pins for the CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: a library routine
(numpy's Pearson correlation, scipy's correlate, numpy least squares / polyfit),
a closed form, an invariant, or a value the paper prints.  None of these needs a GPU.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from oracle import dt, metrics
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def rand_img(rng, h, w, lo=0, hi=256):
    return rng.integers(lo, hi, size=(h, w), dtype=np.uint8)


# --------------------------------------------------------------------------- warp (§3.1)

def test_warp_zero_shift_is_identity():
    rng = np.random.default_rng(1)
    t = rand_img(rng, 12, 37)
    assert np.array_equal(oracle.warp(t, np.zeros(12, np.float32)), t)


def test_warp_recovers_shifted_copy():
    rng = np.random.default_rng(2)
    ref = rand_img(rng, 9, 50)
    k = 7
    cols = np.minimum(np.arange(50) + k, 49)
    tgt = ref[:, cols]                       # the scene seen k pixels further left
    out = oracle.warp(tgt, np.full(9, k, np.float32))
    assert np.array_equal(out[:, k:50 - k], ref[:, k:50 - k])


@pytest.mark.parametrize("s,expect", [(2.5, 3), (2.49, 2), (-2.5, -2), (-2.51, -3), (0.0, 0),
                                      (0.49999997, 0), (-0.5, 0), (7.5, 8)])
def test_warp_rounding(s, expect):
    assert oracle.round_shift(np.float32(s)) == expect
    rng = np.random.default_rng(3)
    t = rand_img(rng, 1, 40)
    out = oracle.warp(t, np.array([s], np.float32))
    src = np.clip(np.arange(40) - expect, 0, 39)
    assert np.array_equal(out[0], t[0, src])


# --------------------------------------------------------------------------- cost, eq. (c)

def _blocks(ref, tgt, u, v, d, rw):
    H, W = ref.shape
    ys = np.clip(np.arange(v - rw, v + rw + 1), 0, H - 1)[:, None]
    xr = np.clip(np.arange(u - rw, u + rw + 1), 0, W - 1)[None, :]
    xt = np.clip(np.arange(u - rw, u + rw + 1) - d, 0, W - 1)[None, :]
    return ref[ys, xr].ravel().astype(np.float64), tgt[ys, xt].ravel().astype(np.float64)


def test_cost_equals_one_minus_pearson():
    """eq. (c) with population statistics is 1 - NCC; numpy's corrcoef is the reference."""
    rng = np.random.default_rng(4)
    ref = rand_img(rng, 24, 32)
    tgt = rand_img(rng, 24, 32)
    for rw in (1, 3, 4):
        for _ in range(60):
            u, v, d = rng.integers(0, 32), rng.integers(0, 24), rng.integers(0, 20)
            a, b = _blocks(ref, tgt, u, v, d, rw)
            expect = 1.0 - np.corrcoef(a, b)[0, 1]
            assert oracle.cost(ref, tgt, u, v, d, 2 * rw + 1) == pytest.approx(expect, abs=1e-12)


def test_cost_zero_at_true_disparity_and_range():
    rng = np.random.default_rng(5)
    ref = rand_img(rng, 20, 60)
    d0 = 6
    tgt = ref[:, np.minimum(np.arange(60) + d0, 59)]      # tgt(u) = ref(u + d0)
    c = oracle.cost_volume(ref, tgt, 16, 7)
    assert np.all(c >= -1e-12) and np.all(c <= 2 + 1e-12)
    inner = c[3:-3, 3 + d0:60 - 3 - d0, d0]
    assert np.max(np.abs(inner)) < 1e-12


def test_cost_affine_invariance_and_anticorrelation():
    rng = np.random.default_rng(6)
    ref = rand_img(rng, 16, 40, 0, 100)
    tgt = rand_img(rng, 16, 40, 0, 100)
    c1 = oracle.cost_volume(ref, tgt, 8, 5)
    c2 = oracle.cost_volume(ref, (2 * tgt.astype(np.int32) + 20).astype(np.uint8), 8, 5)
    assert np.max(np.abs(c1 - c2)) < 1e-12
    c3 = oracle.cost_volume(ref, (255 - ref.astype(np.int32)).astype(np.uint8), 1, 5)
    assert np.allclose(c3[..., 0], 2.0, atol=1e-12)


def test_cost_zero_variance_is_one():
    ref = np.full((10, 10), 77, np.uint8)
    rng = np.random.default_rng(7)
    tgt = rand_img(rng, 10, 10)
    assert np.all(oracle.cost_volume(ref, tgt, 4, 3) == 1.0)
    assert np.all(oracle.cost_volume(tgt, ref, 4, 3) == 1.0)


# ----------------------------------------------------------------- aggregation, eq. (fbs)

def test_weight_values():
    ref = np.array([[100, 110, 100], [100, 100, 100]], np.uint8)
    assert oracle.weight(ref, 0, 0, 0, 0, 1.5, 5.5) == 1.0
    # intensity difference equal to sigma1 and no spatial offset: exp(-1)
    assert oracle.weight(ref, 0, 0, 1, 0, 3.0, 10.0) == pytest.approx(math.exp(-1 - 1 / 9.0))
    assert oracle.weight(ref, 1, 0, 0, 1, 2.0, 7.0) == pytest.approx(
        oracle.weight(ref, 0, 1, 1, 0, 2.0, 7.0))


def test_aggregate_constant_volume_is_identity():
    rng = np.random.default_rng(8)
    ref = rand_img(rng, 15, 21)
    c = np.full((15, 21, 5), 0.37)
    E = oracle.aggregate(ref, c, 9, 3.0, 10.0)
    assert np.max(np.abs(E - 0.37)) < 1e-15


def test_aggregate_window_one_is_identity():
    rng = np.random.default_rng(9)
    ref = rand_img(rng, 11, 13)
    c = rng.random((11, 13, 4))
    assert np.array_equal(oracle.aggregate(ref, c, 1, 3.0, 10.0), c)


def test_aggregate_without_range_term_is_gaussian_filter():
    """With sigma1 -> inf the weights are spatial only: a normalised Gaussian, checked
    against scipy.ndimage.correlate on interior pixels."""
    from scipy import ndimage
    rng = np.random.default_rng(10)
    ref = rand_img(rng, 30, 34)
    c = rng.random((30, 34, 3))
    s0, rb = 2.0, 4
    E = oracle.aggregate(ref, c, 2 * rb + 1, s0, 1e30)
    yy, xx = np.mgrid[-rb:rb + 1, -rb:rb + 1]
    K = np.exp(-(xx * xx + yy * yy) / s0 ** 2)
    K /= K.sum()
    for d in range(3):
        ref_f = ndimage.correlate(c[..., d], K, mode="constant")
        assert np.max(np.abs(E[rb:-rb, rb:-rb, d] - ref_f[rb:-rb, rb:-rb])) < 1e-13


def test_aggregate_is_a_weighted_mean():
    rng = np.random.default_rng(11)
    ref = rand_img(rng, 14, 18)
    c = rng.random((14, 18, 6)) * 2
    E = oracle.aggregate(ref, c, 5, 1.5, 5.5)
    from scipy import ndimage
    lo = ndimage.minimum_filter(c, size=(5, 5, 1), mode="nearest")
    hi = ndimage.maximum_filter(c, size=(5, 5, 1), mode="nearest")
    assert np.all(E >= lo - 1e-12) and np.all(E <= hi + 1e-12)


# --------------------------------------------------------- WTA and eq. (subpixel), §3.2.2

def test_subpixel_recovers_parabola_vertex():
    D = 32
    d = np.arange(D, dtype=np.float64)
    for d0 in (10.3, 4.5, 20.0, 1.01, 29.7):
        E = (0.7 * (d - d0) ** 2 + 0.2)[None, None, :]
        disp, dstar, eb, es = oracle.wta(E, np.array([3.0], np.float32))
        assert disp[0, 0] == pytest.approx(d0 + 3.0, abs=1e-12)
        assert dstar[0, 0] == int(math.ceil(d0 - 0.5))     # a tie goes to the lower d


def test_wta_ties_edges_and_bounds():
    rng = np.random.default_rng(12)
    E = rng.random((6, 7, 20))
    E[0, 0, :] = 1.0
    E[0, 0, 5] = E[0, 0, 9] = 0.1          # tie: lowest d wins
    E[0, 1, :] = np.linspace(0, 1, 20)      # minimum at d = 0 -> no sub-pixel step
    E[0, 2, :] = np.linspace(1, 0, 20)      # minimum at d = D - 1
    disp, dstar, eb, es = oracle.wta(E, np.zeros(6, np.float32))
    assert dstar[0, 0] == 5
    assert disp[0, 1] == 0.0 and disp[0, 2] == 19.0
    assert np.all(np.abs(disp - dstar) <= 0.5 + 1e-12)
    assert np.array_equal(dstar, np.argmin(E, axis=2))
    srt = np.sort(E, axis=2)
    assert np.array_equal(eb, srt[..., 0]) and np.array_equal(es, srt[..., 1])


def test_identical_images_give_the_row_shift():
    rng = np.random.default_rng(13)
    img = synth.texture(rng, 40, 56)
    shift = np.linspace(-3, 5, 40).astype(np.float32)
    disp, dstar, _, _ = oracle.stereo(img, img, shift, 16, 5, 5, 3.0, 10.0)
    si = np.floor(shift.astype(np.float64) + 0.5)
    assert np.all(dstar == 0)
    assert np.array_equal(disp, np.broadcast_to(si[:, None], disp.shape))


def test_stereo_rows_equal_full_volume_path():
    """The banded entry point equals cost_volume -> aggregate -> wta on the whole image."""
    rng = np.random.default_rng(14)
    ref = synth.texture(rng, 24, 32)
    tgt = synth.texture(rng, 24, 32)
    shift = np.zeros(24, np.float32)
    c = oracle.cost_volume(ref, tgt, 8, 5)
    E = oracle.aggregate(ref, c, 7, 3.0, 10.0)
    full = oracle.wta(E, shift)
    band = oracle.stereo(ref, tgt, shift, 8, 5, 7, 3.0, 10.0, rows=(5, 17))
    for a, b in zip(full, band):
        assert np.array_equal(a[5:17], b)


@pytest.mark.slow
def test_noise_free_plane_recovers_ground_truth():
    """End-to-end quality: a noise-free planar road (no potholes) through warp, cost,
    aggregation, WTA and sub-pixel lands close to the ground truth."""
    s = synth.make_scene(160, 120, 32, 99, roll=math.radians(2.0), coeffs=(8.0, 0.1, 0.0),
                         n_potholes=0, sigma_n=0.0, warp=True, win=7, bil=9)
    tw = oracle.warp(s.tgt, s.shift)
    disp, _, _, _ = oracle.stereo(s.ref, tw, s.shift, 32, 7, 9, 3.0, 10.0)
    m = oracle.valid_mask(160, 120, 32, 7, 9, s.shift).astype(bool)
    assert m.mean() > 0.3
    err = (disp - s.gt_disp)[m]
    # the parabola step has the usual pixel-locking bias (errors up to ~0.5 px that
    # average out); a wrong sign or a wrong direction of d would cost whole pixels
    assert abs(np.mean(err)) < 0.05
    assert np.mean(np.abs(err)) < 0.25 and np.mean(np.abs(err) < 0.75) > 0.99


# ------------------------------------------------- disparity transformation, §3.3

def _plane_data(rng, n, psi, a0, a1, noise=0.0, W=400, H=300):
    u = rng.uniform(0, W, n)
    v = rng.uniform(0, H, n)
    y = v * math.cos(psi) - u * math.sin(psi)
    d = a0 + a1 * y + noise * rng.standard_normal(n)
    return d, u, v


def test_line_fit_at_zero_roll_is_polyfit():
    """eq. (alpha2): with psi = 0 the fit is the ordinary v-disparity line."""
    rng = np.random.default_rng(15)
    d, u, v = _plane_data(rng, 500, 0.1, 5.0, 0.12, noise=1.0)
    slope, icpt = np.polyfit(v, d, 1)
    a = dt.line_fit(d, u, v, 0.0)
    assert a[0] == pytest.approx(icpt, rel=1e-10) and a[1] == pytest.approx(slope, rel=1e-10)
    r = d - (icpt + slope * v)
    assert dt.energy_min(d, u, v, 0.0) == pytest.approx(r @ r, rel=1e-9)


def test_energy_min_equals_residual_of_fit_and_has_period_pi():
    rng = np.random.default_rng(16)
    d, u, v = _plane_data(rng, 300, -0.2, 3.0, 0.2, noise=0.5)
    for psi in (-1.2, -0.3, 0.0, 0.4, 1.5):
        a = dt.line_fit(d, u, v, psi)
        assert dt.energy_min(d, u, v, psi) == pytest.approx(dt.energy(d, u, v, psi, a), rel=1e-9)
        assert dt.energy_min(d, u, v, psi) == pytest.approx(
            dt.energy_min(d, u, v, psi + math.pi), rel=1e-9)


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(17)
    d, u, v = _plane_data(rng, 400, 0.07, 4.0, 0.15, noise=0.8)
    for psi in (-0.5, -0.05, 0.0, 0.03, 0.3, 1.0):
        h = 1e-6
        fd = (dt.energy_min(d, u, v, psi + h) - dt.energy_min(d, u, v, psi - h)) / (2 * h)
        g = dt.grad_energy_min(d, u, v, psi)
        assert g == pytest.approx(fd, rel=1e-5, abs=1e-6 * abs(dt.energy_min(d, u, v, psi)))


@pytest.mark.parametrize("psi_true", [-0.1, 0.0, 0.03, 0.2, -0.6])
def test_roll_estimate_reaches_the_plane_fit_closed_form(psi_true):
    """min over (psi, alpha) of eq. (E2) is the least-squares plane d ~ a + b u + c v,
    so psi* = atan(-b/c), alpha1 = c / cos(psi*), alpha0 = a."""
    rng = np.random.default_rng(18)
    d, u, v = _plane_data(rng, 3000, psi_true, 6.0, 0.12, noise=0.7, W=1920, H=1080)
    d = d - 3.0 * np.exp(-((u - 900) ** 2 + (v - 700) ** 2) / 5000.0)   # a dent
    A = np.stack([np.ones_like(u), u, v], axis=1)
    a, b, c = np.linalg.lstsq(A, d, rcond=None)[0]
    psi_star = math.atan(-b / c)
    res = dt.estimate_roll(d, u, v)
    assert res["status"] == dt.STATUS_OK
    delta_psi = math.pi / 1.8e6          # the paper's stopping threshold (§4.4.2)
    assert abs(res["psi"] - psi_star) < 0.1 * delta_psi
    assert res["alpha1"] == pytest.approx(c / math.cos(psi_star), rel=1e-6)
    assert res["alpha0"] == pytest.approx(a, rel=1e-6, abs=1e-6)
    resid = d - A @ np.array([a, b, c])
    assert res["e_min"] == pytest.approx(resid @ resid, rel=1e-9)


def test_noise_free_plane_transforms_to_a_constant():
    H, W, psi, a0, a1 = 60, 80, 0.05, 7.0, 0.11
    u = np.arange(W)[None, :]
    v = np.arange(H)[:, None]
    disp = a0 + a1 * (v * math.cos(psi) - u * math.sin(psi))
    out, res = dt.disparity_transform(disp, delta_t=2.5)
    # exact up to the stopping threshold delta_psi = pi / 1.8e6 of §4.4.2
    assert abs(res["psi"] - psi) < 0.1 * math.pi / 1.8e6
    assert res["alpha0"] == pytest.approx(a0, rel=1e-6) and res["alpha1"] == pytest.approx(a1, rel=1e-6)
    assert np.max(np.abs(out - 2.5)) < 1e-5
    assert metrics.sigma_d(out) < 1e-5


def test_roll_estimate_respects_iteration_cap():
    rng = np.random.default_rng(19)
    d, u, v = _plane_data(rng, 500, 0.3, 2.0, 0.1, noise=0.5)
    res = dt.estimate_roll(d, u, v, max_iters=1)
    assert res["status"] == dt.STATUS_NOT_CONVERGED and res["iters"] == 1


# ------------------------------------------------------------ printed constants, §4.4

def test_throughput_worked_example():
    g = json.load(open(os.path.join(GOLDEN, "throughput_example.json")))
    val = metrics.mde_per_s(g["u_max"], g["v_max"], g["d_max_implied"], g["seconds"])
    assert round(val, 3) == g["mde_per_s"]


def test_error_metrics_definitions():
    gt = np.zeros((4, 5))
    disp = gt.copy()
    disp[0, 0] = 3.0
    disp[1, 1] = -2.0
    assert metrics.error_pixel_percent(disp, gt, 2) == pytest.approx(5.0)
    assert metrics.error_pixel_percent(disp, gt, 1) == pytest.approx(10.0)
    assert metrics.rms_error(disp, gt) == pytest.approx(math.sqrt(13 / 20))


# ------------------------------------------------ geometric validity (readings of §3.2, §3.3)

def _valid_by_enumeration(W, H, D, rw, rb, shift_int):
    """Every read behind pixel (u, v), listed one by one: for each neighbour q of the k x k
    window (in the image or not), each offset j of the w x w block and each d in [0, D), the
    reference read at q + j, the warped-target read at q + j - [d, 0], and the original-target
    read behind the warp, at that column minus the integer shift of its row.  The pixel is
    valid exactly when none of those coordinates lies outside the image (none needs a clamp).
    The shift table is passed as integers, so no rounding enters this check."""
    valid = np.zeros((H, W), np.uint8)
    offs = range(-(rw + rb), rw + rb + 1)
    # all (neighbour offset, block offset) pairs along one axis, listed explicitly
    pairs = [(a, b) for a in range(-rb, rb + 1) for b in range(-rw, rw + 1)]
    assert sorted({a + b for a, b in pairs}) == list(offs)
    for v in range(H):
        for u in range(W):
            ok = True
            for qy, jy in pairs:
                y = v + qy + jy
                for qx, jx in pairs:
                    x = u + qx + jx
                    if not (0 <= x < W and 0 <= y < H):          # reference read
                        ok = False
                        break
                    for d in range(D):
                        xt = x - d
                        if not (0 <= xt < W):                     # warped-target read
                            ok = False
                            break
                        xo = xt - int(shift_int[y])
                        if not (0 <= xo < W):                     # original target behind the warp
                            ok = False
                            break
                    if not ok:
                        break
                if not ok:
                    break
            valid[v, u] = ok
    return valid


@pytest.mark.parametrize("W,H,D,rw,rb,seed", [
    (23, 13, 3, 1, 1, 0),
    (20, 11, 1, 0, 0, 1),     # D = 1, w = k = 1: only the shift can invalidate a pixel
    (26, 15, 4, 2, 1, 2),
    (24, 12, 2, 0, 2, 3),     # w = 1
    (22, 14, 5, 1, 0, 4),     # k = 1
    (30, 17, 6, 1, 2, 5),
])
def test_valid_mask_equals_enumeration_of_every_read(W, H, D, rw, rb, seed):
    rng = np.random.default_rng(seed)
    # negative, zero and large shifts, and half-integers whose rounding goes up
    base = rng.integers(-6, 7, size=H).astype(np.float64)
    base[rng.integers(0, H)] = 0.0
    base[rng.integers(0, H)] = W // 2           # large enough to empty a whole band
    half = rng.random(H) < 0.3
    s = np.where(half, base - 0.5, base)        # k - 0.5 rounds to k (halves go up)
    shift_int = base.astype(np.int64)
    got = oracle.valid_mask(W, H, D, 2 * rw + 1, 2 * rb + 1, s.astype(np.float32))
    want = _valid_by_enumeration(W, H, D, rw, rb, shift_int)
    assert np.array_equal(got, want), np.argwhere(got != want)[:8]


def test_valid_mask_constant_shift_band():
    # a constant shift s moves the valid band of every interior row by max(0, s) on the left
    # and by min(0, s) on the right; the band is empty once it no longer fits
    W, H, D, rw, rb = 40, 9, 5, 1, 1
    m = rw + rb
    for s in (-7, -1, 0, 3, 30):
        got = oracle.valid_mask(W, H, D, 2 * rw + 1, 2 * rb + 1, np.full(H, s, np.float32))
        lo, hi = m + D - 1 + max(0, s), W - 1 - m + min(0, s)
        want = np.zeros((H, W), np.uint8)
        if lo <= hi:
            want[m:H - m, lo:hi + 1] = 1
        assert np.array_equal(got, want), s


# ------------------------------------------------------------ eq. (sigma_d), §4.4.2

def test_sigma_d_hand_computed():
    # s = (1, 2, 3, 4, 5, 7): mean 11/3, squared deviations sum to 70/3, and eq. (sigma_d)
    # divides by m = 6: sigma_d = sqrt(35/9) = sqrt(35)/3 (a 1/(m-1) form would give sqrt(70/15))
    s = np.array([[1.0, 2.0, 3.0], [4.0, 5.0, 7.0]])
    assert metrics.sigma_d(s) == pytest.approx(math.sqrt(35.0) / 3.0, rel=1e-14)
    # the mask selects the elements that enter: (2, 4, 7) -> mean 13/3, deviations
    # (-7/3, -1/3, 8/3), squares sum to 114/9, divided by 3 -> sqrt(38)/3
    mask = np.array([[0, 1, 0], [1, 0, 1]], bool)
    assert metrics.sigma_d(s, mask) == pytest.approx(math.sqrt(38.0) / 3.0, rel=1e-14)
    # a constant offset does not change it; a scale multiplies it
    assert metrics.sigma_d(s + 100.0) == pytest.approx(math.sqrt(35.0) / 3.0, rel=1e-12)
    assert metrics.sigma_d(2.5 * s) == pytest.approx(2.5 * math.sqrt(35.0) / 3.0, rel=1e-14)
