"""Pins of the differentiable FP64 oracle (oracle/diff.py), CPU only.

What fixes it, other than itself:
  * its cost and aggregation equal the C oracle's eq. (c) and eq. (fbs), which is written
    independently and pinned by brute force and closed forms (test_oracle_pins.py);
  * soft-argmin closed forms (uniform cost, a symmetric bowl, the T -> 0 limit = WTA);
  * its energy equals oracle.dt's eq. (E2), and its psi-gradient at the line fit equals
    oracle.dt's eq. (d_e_min);
  * every adjoint agrees with central finite differences of the forward (h = 1e-6 relative);
  * the roll refinement reaches the closed-form plane fit.
"""
import math

import numpy as np
import pytest
import torch

import oracle
import oracle.dt as odt
import synth
from oracle import diff

WIN, BIL, S0, S1, T = 9, 11, 3.0, 10.0, 0.1


@pytest.fixture(scope="module", autouse=True)
def _built():
    oracle.build()


@pytest.fixture(scope="module")
def crop():
    s = synth.make_config_scene("grad")
    ref, tgt, sh = synth.crop_pair(s, 448, 300, 64, 48)
    return s, ref, tgt, sh


def test_crop_keeps_the_match_inside_the_window(crop):
    """The residual disparity left after the window's row shift lies inside [0, 16)."""
    s, ref, tgt, sh = crop
    off = int(math.floor(float(np.mean(s.shift[300:348]))))
    resid = s.gt_disp[300:348, 448:512] - off - np.floor(sh.astype(np.float64) + 0.5)[:, None]
    assert -1.0 < resid.min() and resid.max() < 15.0
    assert np.array_equal(ref, s.ref[300:348, 448:512])
    assert np.array_equal(tgt, s.tgt[300:348, 448 - off:512 - off])


def test_cost_and_aggregation_equal_the_c_oracle(crop):
    _, ref, tgt, sh = crop
    D = 16
    tw = oracle.warp(tgt, sh)
    c = oracle.cost_volume(ref, tw, D, WIN)
    ct = diff.cost_volume(torch.tensor(ref.astype(np.float64)),
                          diff.warp(torch.tensor(tgt.astype(np.float64)), sh), D, WIN).numpy()
    assert np.abs(ct.transpose(1, 2, 0) - c).max() < 1e-12
    E = oracle.aggregate(ref, c, BIL, S0, S1)
    Et = diff.aggregate(torch.tensor(ref.astype(np.float64)),
                        torch.tensor(np.ascontiguousarray(c.transpose(2, 0, 1))), BIL, S0, S1).numpy()
    assert np.abs(Et.transpose(1, 2, 0) - E).max() < 1e-13


def test_warp_equals_the_c_oracle():
    rng = np.random.default_rng(5)
    tgt = rng.integers(0, 256, (12, 40), dtype=np.uint8)
    sh = rng.uniform(-9, 9, 12).astype(np.float32)
    w = diff.warp(torch.tensor(tgt.astype(np.float64)), sh).numpy()
    assert np.array_equal(w, oracle.warp(tgt, sh).astype(np.float64))


def test_flat_window_costs_one_with_finite_gradients():
    rng = np.random.default_rng(1)
    ref = rng.uniform(0, 255, (16, 24))
    ref[2:12, 3:14] = 77.123456789      # a flat patch whose rounded mean need not be exact
    tgt = rng.uniform(0, 255, (16, 24))
    c = diff.cost_volume(torch.tensor(ref), torch.tensor(tgt), 4, 5).numpy()
    assert np.all(c[:, 6:9, 7:11] == 1.0)
    _, g_r, g_t = diff.disparity_vjp(ref, tgt, np.zeros(16, np.float32), 4, 5, 5, S0, S1, T,
                                     np.ones((16, 24)))
    assert np.all(np.isfinite(g_r)) and np.all(np.isfinite(g_t))
    # a 1 x 1 image: every clamped block is flat, every cost 1, every gradient 0
    x = np.array([[123.456789]])
    c1 = diff.cost_volume(torch.tensor(x), torch.tensor(x * 0.37), 3, 3).numpy()
    assert np.all(c1 == 1.0)
    _, g_r, g_t = diff.disparity_vjp(x, x * 0.37, np.zeros(1, np.float32), 3, 3, 3, S0, S1, T, np.ones((1, 1)))
    assert np.all(g_r == 0) and np.all(g_t == 0)


def test_soft_argmin_closed_forms():
    D, H, W = 24, 3, 5
    sh = np.array([0.0, 2.4, -3.6], np.float32)           # rounds to 0, 2, -4
    E = torch.full((D, H, W), 0.7, dtype=torch.float64)
    l = diff.soft_argmin(E, sh, T).numpy()
    assert np.allclose(l, (D - 1) / 2 + np.array([0, 2, -4])[:, None], atol=1e-12, rtol=0)
    # a bowl symmetric about an interior integer d0 has its soft-argmin exactly at d0
    d = torch.arange(D, dtype=torch.float64)[:, None, None]
    d0 = 11.0
    bowl = 0.02 * (d - d0) ** 2 * torch.ones((1, H, W), dtype=torch.float64)
    bowl[23] = 9.0    # break the symmetry only where the mirror image (d = -1) does not exist
    bowl = torch.where(d <= 2 * d0, bowl, torch.full_like(bowl, 50.0))
    l = diff.soft_argmin(bowl, np.zeros(H, np.float32), T).numpy()
    assert np.allclose(l, d0, atol=1e-9, rtol=0)


def test_small_temperature_is_winner_take_all(crop):
    _, ref, tgt, sh = crop
    D = 16
    tw = oracle.warp(tgt, sh)
    E = oracle.aggregate(ref, oracle.cost_volume(ref, tw, D, WIN), BIL, S0, S1)
    _, dstar, eb, es = oracle.wta(E, sh)
    sure = (es - eb) > 0.05
    Tsmall = 1e-3                  # exp(-0.05 / 1e-3) ~ 2e-22: the soft-argmin is the argmin
    l = diff.soft_argmin(torch.tensor(np.ascontiguousarray(E.transpose(2, 0, 1))), sh, Tsmall).numpy()
    si = np.floor(sh.astype(np.float64) + 0.5)[:, None]
    assert sure.mean() > 0.5
    assert np.allclose((l - si)[sure], dstar[sure], atol=1e-12, rtol=0)


def test_energy_equals_eq_e2_of_the_dt_oracle():
    rng = np.random.default_rng(3)
    H, W = 20, 30
    l = rng.uniform(5, 25, (H, W))
    mask = (rng.uniform(size=(H, W)) > 0.3).astype(np.float64)
    psi, a0, a1 = 0.07, 4.0, 0.3
    v, u = np.nonzero(mask)
    ref_val = odt.energy(l[v, u], u.astype(np.float64), v.astype(np.float64), psi, [a0, a1])
    assert diff.energy_value(l, mask, psi, a0, a1) == pytest.approx(ref_val, rel=1e-13)


def test_psi_gradient_at_the_line_fit_is_eq_d_e_min():
    rng = np.random.default_rng(4)
    H, W = 24, 40
    v, u = np.mgrid[0:H, 0:W].astype(np.float64)
    l = 6 + 0.2 * (v * math.cos(0.05) - u * math.sin(0.05)) + rng.normal(0, 0.3, (H, W))
    mask = np.ones((H, W))
    for psi in (-0.2, 0.0, 0.11):
        a0, a1 = diff.alpha_fit(l, mask, psi)
        _, _, g, g0, g1 = diff.energy_grads(l, mask, psi, a0, a1)
        gm = odt.grad_energy_min(l.ravel(), u.ravel(), v.ravel(), psi)
        assert g == pytest.approx(gm, rel=1e-9, abs=1e-9)
        # at the fit the alpha-gradients vanish (normal equations)
        assert abs(g0) < 1e-8 * np.abs(l).sum() and abs(g1) < 1e-8 * np.abs(l).sum() * W


def _fd(f, x0, h):
    return (f(x0 + h) - f(x0 - h)) / (2 * h)


def _rel(a, b, scale):
    return abs(a - b) / max(abs(b), scale)


@pytest.mark.parametrize("jit", [False, True])
def test_image_adjoints_match_central_differences(crop, jit):
    """dL/dref and dL/dtgt at interior, edge and corner pixels (the clamp folds and the
    warp scatter at the window edges), images on and off the integer grid."""
    _, ref, tgt, sh = crop
    D = 16
    H, W = ref.shape
    refd = synth.jitter(ref, 11) if jit else ref.astype(np.float64)
    tgtd = synth.jitter(tgt, 12) if jit else tgt.astype(np.float64)
    mask = oracle.valid_mask(W, H, D, WIN, BIL, sh).astype(np.float64)
    mask[::5, ::3] = 1.0
    l0 = diff.disparity_value(refd, tgtd, sh, D, WIN, BIL, S0, S1, T)
    a0, a1 = diff.alpha_fit(l0, mask, 0.02)
    args = (sh, D, WIN, BIL, S0, S1, T, mask, 0.02, a0, a1)
    L, _, g_r, g_t, _, _, _ = diff.loss_and_grads(refd, tgtd, *args)
    pts = [(0, 0), (0, W - 1), (H - 1, 0), (H - 1, W - 1), (23, 31), (10, 0), (5, 1), (40, W - 2),
           (17, W - 1), (47, 20), (30, 7)]
    scale_r, scale_t = 1e-3 * np.abs(g_r).max(), 1e-3 * np.abs(g_t).max()
    for (v, u) in pts:
        for img, g, scale, which in ((refd, g_r, scale_r, 0), (tgtd, g_t, scale_t, 1)):
            h = 1e-6 * max(abs(img[v, u]), 1.0)

            def f(x):
                im = img.copy()
                im[v, u] = x
                pair = (im, tgtd) if which == 0 else (refd, im)
                l = diff.disparity_value(*pair, sh, D, WIN, BIL, S0, S1, T)
                return diff.energy_value(l, mask, 0.02, a0, a1)

            fd = _fd(f, img[v, u], h)
            assert _rel(g[v, u], fd, scale) < 1e-5, (which, v, u, g[v, u], fd)


def test_parameter_adjoints_match_central_differences(crop):
    _, ref, tgt, sh = crop
    D = 16
    H, W = ref.shape
    l = diff.disparity_value(ref, tgt, sh, D, WIN, BIL, S0, S1, T)
    mask = oracle.valid_mask(W, H, D, WIN, BIL, sh).astype(np.float64)
    psi, a0, a1 = 0.031, 38.0, 0.11
    L, g_l, g_psi, g_a0, g_a1 = diff.energy_grads(l, mask, psi, a0, a1)
    assert _fd(lambda x: diff.energy_value(l, mask, x, a0, a1), psi, 1e-6 * abs(psi)) == \
        pytest.approx(g_psi, rel=1e-5)
    assert _fd(lambda x: diff.energy_value(l, mask, psi, x, a1), a0, 1e-6 * abs(a0)) == \
        pytest.approx(g_a0, rel=1e-5)
    assert _fd(lambda x: diff.energy_value(l, mask, psi, a0, x), a1, 1e-6 * abs(a1)) == \
        pytest.approx(g_a1, rel=1e-5)
    for (v, u) in ((0, 0), (20, 33), (47, 63)):
        def f(x):
            ll = l.copy()
            ll[v, u] = x
            return diff.energy_value(ll, mask, psi, a0, a1)
        fd = _fd(f, l[v, u], 1e-6 * abs(l[v, u]))
        assert _rel(g_l[v, u], fd, 1e-3 * np.abs(g_l).max()) < 1e-5


def _plane_fit_psi(l, mask):
    """The closed form of §3.3's minimum: the OLS plane l ~ a + b u + c v gives
    psi* = atan(-b / c), wrapped into (-pi/2, pi/2]."""
    v, u = np.nonzero(mask)
    A = np.stack([np.ones_like(u), u, v], axis=1).astype(np.float64)
    a, b, c = np.linalg.lstsq(A, l[v, u], rcond=None)[0]
    return math.atan(-b / c)


def test_refine_roll_reaches_the_plane_fit():
    rng = np.random.default_rng(8)
    H, W = 54, 96
    v, u = np.mgrid[0:H, 0:W].astype(np.float64)
    roll = math.radians(4.5)
    l = 7 + 0.14 * (v * math.cos(roll) - u * math.sin(roll)) + rng.normal(0, 0.4, (H, W))
    mask = (rng.uniform(size=(H, W)) > 0.1).astype(np.float64)
    traj = diff.refine_roll(l, mask, 0.0, 50)
    psi = traj[-1][0]
    assert len(traj) == 51
    assert abs(psi - _plane_fit_psi(l, mask)) < 1e-10
    res = odt.estimate_roll(l[mask != 0], u[mask != 0], v[mask != 0])
    assert abs(psi - res["psi"]) < 1e-8
    assert traj[-1][4] <= traj[0][4]


def test_refine_roll_on_the_soft_argmin_of_a_crop(crop):
    _, ref, tgt, sh = crop
    D = 16
    H, W = ref.shape
    l = diff.disparity_value(ref, tgt, sh, D, WIN, BIL, S0, S1, T)
    mask = oracle.valid_mask(W, H, D, WIN, BIL, sh).astype(np.float64)
    traj = diff.refine_roll(l, mask, 0.0, 50)
    assert abs(traj[-1][0] - _plane_fit_psi(l, mask)) < 1e-10


def test_linear_warp_closed_forms():
    rng = np.random.default_rng(31)
    tgt = rng.uniform(0, 255, (6, 20))
    sh = np.array([0, 3, -2, 7, 25, -30], np.float32)          # integers: the rounded warp exactly
    w = diff.warp_linear(torch.tensor(tgt), torch.tensor(sh.astype(np.float64))).numpy()
    assert np.array_equal(w, diff.warp(torch.tensor(tgt), sh).numpy())
    ramp = np.tile(np.arange(20, dtype=np.float64) * 3.0 + 1.0, (3, 1))    # 3x + 1
    sh = np.array([0.25, 2.5, -1.75], np.float32)
    w = diff.warp_linear(torch.tensor(ramp), torch.tensor(sh.astype(np.float64))).numpy()
    u = np.arange(20)[None, :] - sh.astype(np.float64)[:, None]
    inside = (u >= 0) & (u <= 19)
    assert np.allclose(w[inside], (3.0 * u + 1.0)[inside], atol=1e-12, rtol=0)
    assert np.all(w[u < 0] == 1.0) and np.all(w[u > 19] == 58.0)   # clamped to the edge pixels


def test_linear_warp_shift_gradient_matches_central_differences(crop):
    _, ref, tgt, sh = crop
    D = 16
    shf = (sh + np.linspace(-0.4, 0.35, sh.size)).astype(np.float32)   # fractional shifts
    gl = np.random.default_rng(32).normal(size=ref.shape)
    l, g_r, g_t, g_s = diff.disparity_linear_vjp(ref, tgt, shf, D, WIN, BIL, S0, S1, T, gl)
    scale = 1e-3 * np.abs(g_s).max()
    for v in (0, 7, 23, 47):
        h = 1e-4

        def S(x):
            s2 = shf.astype(np.float64).copy()
            s2[v] = x
            with torch.no_grad():
                lx = diff.disparity(torch.tensor(ref.astype(np.float64)), torch.tensor(tgt.astype(np.float64)),
                                    torch.tensor(s2), D, WIN, BIL, S0, S1, T, 1).numpy()
            return float((lx * gl).sum())

        fd = (S(float(shf[v]) + h) - S(float(shf[v]) - h)) / (2 * h)
        assert abs(g_s[v] - fd) <= 1e-5 * max(abs(fd), scale), (v, g_s[v], fd)
    # the target adjoint of the interpolating warp, at an interior and an edge pixel
    for (v, u) in ((20, 30), (5, 0), (40, 63)):
        h = 1e-6 * max(abs(float(tgt[v, u])), 1.0)

        def St(x):
            t2 = tgt.astype(np.float64).copy()
            t2[v, u] = x
            return float((diff.disparity_linear_value(ref, t2, shf, D, WIN, BIL, S0, S1, T) * gl).sum())

        fd = (St(tgt[v, u] + h) - St(tgt[v, u] - h)) / (2 * h)
        assert abs(g_t[v, u] - fd) <= 1e-5 * max(abs(fd), 1e-3 * np.abs(g_t).max())
