"""Differentiable path on the GPU (include/stereo_diff.h) against the FP64 oracle
(oracle/diff.py, whose adjoints are pinned to central finite differences).

Tolerances: the soft-argmin disparity within 1e-3 px of the oracle (dl/dE(p,d) =
-P(p,d) (d - lbar) / T, so the FP32 rounding of E, about 1e-6, reaches l amplified by up to
D / (2T) = 320 at D = 64, T = 0.1; 1e-3 px is also the bar of the transformed disparity); every gradient within
1e-3 of the largest oracle gradient of its kind, element by element (FP32 kernels against
an FP64 oracle); eq. (E2) within 1e-6 relative; the refined roll angle within 1e-8 rad of
the closed-form fit of the same disparity map."""
import math

import numpy as np
import pytest
import torch

import oracle
import oracle.dt as odt
import synth
from oracle import diff as odiff
from paper_1904_06017_gb300 import diff as sgd
import paper_1904_06017_gb300 as sg

pytestmark = pytest.mark.gpu

WIN, BIL, S0, S1, T = 9, 11, 3.0, 10.0, 0.1
L_TOL = 1e-3
G_TOL = 1e-3


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1904_06017_gb300 import build
    build.build()
    oracle.build()


@pytest.fixture(scope="module")
def scene():
    return synth.make_config_scene("grad")


def dev(x, dtype=torch.float32):
    return torch.tensor(np.ascontiguousarray(x), dtype=dtype, device="cuda")


def gpu_forward(refs, tgts, shifts, D, win=WIN, bil=BIL, s0=S0, s1=S1, temp=T, mode=0):
    """Batched forward through the C calls; returns (l [B,H,W] numpy, params, tensors, ws)."""
    r = dev(np.stack(refs))
    t = dev(np.stack(tgts))
    s = dev(np.stack(shifts))
    B, H, W = r.shape
    p = sgd.stereo_diff_params_default(width=W, height=H, batch=B, max_disp=D, win=win, bil=bil,
                                       sigma0=s0, sigma1=s1, temperature=temp, warp_mode=mode)
    ws = torch.empty(sgd.stereo_softargmin_workspace_bytes(p), dtype=torch.uint8, device="cuda")
    l = torch.empty((B, H, W), dtype=torch.float32, device="cuda")
    sgd.stereo_softargmin_fwd(p, r, t, s, l, ws)
    torch.cuda.synchronize()
    return l.cpu().numpy().astype(np.float64), p, (r, t, s), ws


def gpu_backward(p, rts, ws, gl, want_shift=False):
    r, t, s = rts
    gr = torch.empty_like(r)
    gt = torch.empty_like(t)
    gs = torch.full_like(s, 7.0) if want_shift else None
    sgd.stereo_softargmin_bwd(p, r, t, s, dev(gl), gr, gt, ws, grad_shift=gs)
    torch.cuda.synchronize()
    out = (gr.cpu().numpy().astype(np.float64), gt.cpu().numpy().astype(np.float64))
    return out + (gs.cpu().numpy().astype(np.float64),) if want_shift else out


def check_grad(g, go, name, floor=0.0):
    scale = np.abs(go).max()
    err = np.abs(g - go).max()
    print("  %s: max |g| %.4g, max err %.3g (%.2e of max)" % (name, scale, err, err / max(scale, 1e-30)))
    assert err <= max(G_TOL * scale, floor), (name, err, scale)


CASES = [
    # (u0, v0, W, H, D, jitter)
    (448, 300, 64, 48, 16, False),
    (440, 310, 77, 45, 20, True),        # ragged: neither side a multiple of a tile
    (400, 280, 96, 64, 64, False),       # the search range of the 960 x 540 workload
]


@pytest.mark.parametrize("case", CASES, ids=["64x48_D16", "77x45_D20_jit", "96x64_D64"])
def test_forward_and_adjoint_match_the_oracle(scene, case):
    u0, v0, W, H, D, jit = case
    ref, tgt, sh = synth.crop_pair(scene, u0, v0, W, H)
    refd = synth.jitter(ref, 21) if jit else ref.astype(np.float64)
    tgtd = synth.jitter(tgt, 22) if jit else tgt.astype(np.float64)
    l, p, rts, ws = gpu_forward([refd], [tgtd], [sh], D)
    gl = np.random.default_rng(7).normal(0.0, 1.0, (H, W))
    lo, gro, gto = odiff.disparity_vjp(refd, tgtd, sh, D, WIN, BIL, S0, S1, T, gl)
    err = np.abs(l[0] - lo).max()
    print("\n%s: max |l - l_oracle| = %.3g px" % (case, err))
    assert err <= L_TOL
    gr, gt = gpu_backward(p, rts, ws, gl[None].astype(np.float32))
    check_grad(gr[0], gro, "dS/dref")
    check_grad(gt[0], gto, "dS/dtgt")


def test_rounded_shift_at_the_rounding_ties(scene):
    """§3.1's s_i = floor(s + 0.5) taken exactly for shifts next to the ties, where s + 0.5
    rounded to float32 would round up (0.5 - 2^-25 + 0.5 is a tie that rounds to 1.0): the
    rounded warp and the add-back of s_i follow the oracle's exact rounding."""
    ref, tgt, _ = synth.crop_pair(scene, 500, 300, 48, 16)
    # one shift per row: values next to the ties of floor(s + 0.5), and the ties themselves
    shift = np.array([0.5 - 2.0 ** -25, -0.5 - 2.0 ** -24, 0.5, -0.5, 1.5 - 2.0 ** -23, -1.5,
                      2.5, -2.5 + 2.0 ** -22, 0.25 + 2.0 ** -26, 1e-30, -1e-30, 0.0,
                      4.5, -3.5 - 2.0 ** -22, 0.375, 7.5], dtype=np.float32)
    # the point of the test: rounding s + 0.5 to float32 first gets the first row wrong
    assert np.floor(shift[0] + np.float32(0.5)) == 1.0 and odiff.round_shift(shift)[0] == 0
    refd, tgtd = ref.astype(np.float64), tgt.astype(np.float64)
    l, *_ = gpu_forward([refd], [tgtd], [shift], 16)
    lo, *_ = odiff.disparity_vjp(refd, tgtd, shift, 16, WIN, BIL, S0, S1, T, np.zeros((16, 48)))
    assert np.abs(l[0] - lo).max() <= L_TOL


def test_energy_forward_and_adjoint_match_the_oracle():
    rng = np.random.default_rng(9)
    B, H, W = 3, 37, 53
    l = rng.uniform(10, 40, (B, H, W))
    mask = (rng.uniform(size=(B, H, W)) > 0.25).astype(np.uint8)
    theta = np.array([[0.05, 12.0, 0.21], [-0.3, 3.0, -0.07], [1.2, 20.0, 0.4]])
    ge = np.array([1.0, -0.5, 2.0])
    d = dev(l)
    th = dev(theta, torch.float64)
    m = dev(mask, torch.uint8)
    ws = torch.empty(sgd.stereo_dt_energy_workspace_bytes(B), dtype=torch.uint8, device="cuda")
    e = torch.empty(B, dtype=torch.float64, device="cuda")
    sgd.stereo_dt_energy_fwd(d, m, th, e, ws)
    gd = torch.empty_like(d)
    gth = torch.empty_like(th)
    sgd.stereo_dt_energy_bwd(d, m, th, dev(ge, torch.float64), gd, gth, ws)
    e, gd, gth = e.cpu().numpy(), gd.cpu().numpy(), gth.cpu().numpy()
    lf = l.astype(np.float32).astype(np.float64)       # the GPU reads float32 disparities
    for b in range(B):
        Lo, glo, gpo, ga0o, ga1o = odiff.energy_grads(lf[b], mask[b], *theta[b])
        assert e[b] == pytest.approx(Lo, rel=1e-6)
        check_grad(gd[b], ge[b] * glo, "dL/dl")
        assert gth[b] == pytest.approx(ge[b] * np.array([gpo, ga0o, ga1o]), rel=1e-4)


def test_autograd_chain_matches_oracle_and_finite_differences(scene):
    """L = E2(SoftArgmin(ref, tgt), theta) through torch.autograd: gradients in both images
    and theta against the oracle's adjoint and, at a few pixels, FP64 central differences."""
    ref, tgt, sh = synth.crop_pair(scene, 448, 300, 64, 48)
    D = 16
    H, W = ref.shape
    mask = oracle.valid_mask(W, H, D, WIN, BIL, sh)
    r = dev(ref).requires_grad_(True)
    t = dev(tgt).requires_grad_(True)
    l = sgd.soft_argmin_disparity(r, t, dev(sh), D, WIN, BIL, S0, S1, T)
    a0, a1 = odiff.alpha_fit(l.detach().cpu().numpy(), mask, 0.02)
    theta = torch.tensor([0.02, a0 + 0.3, a1 * 1.01], dtype=torch.float64, device="cuda",
                         requires_grad=True)
    L = sgd.dt_energy(l, theta, dev(mask, torch.uint8))
    L.backward()
    Lo, lo, gro, gto, gpo, ga0o, ga1o = odiff.loss_and_grads(ref, tgt, sh, D, WIN, BIL, S0, S1, T, mask,
                                                              0.02, a0 + 0.3, a1 * 1.01)
    assert float(L.detach()) == pytest.approx(Lo, rel=1e-4)
    gr = r.grad.cpu().numpy().astype(np.float64)
    gt = t.grad.cpu().numpy().astype(np.float64)
    check_grad(gr, gro, "dL/dref")
    check_grad(gt, gto, "dL/dtgt")
    gth = theta.grad.cpu().numpy()
    assert gth == pytest.approx(np.array([gpo, ga0o, ga1o]), rel=1e-3)
    refd, tgtd = ref.astype(np.float64), tgt.astype(np.float64)
    for (v, u) in ((0, 0), (23, 31), (47, 63), (10, 1)):
        for img, g, which in ((refd, gr, 0), (tgtd, gt, 1)):
            h = 1e-6 * max(abs(img[v, u]), 1.0)
            vals = []
            for x in (img[v, u] + h, img[v, u] - h):
                im = img.copy()
                im[v, u] = x
                pair = (im, tgtd) if which == 0 else (refd, im)
                lx = odiff.disparity_value(*pair, sh, D, WIN, BIL, S0, S1, T)
                vals.append(odiff.energy_value(lx, mask, 0.02, a0 + 0.3, a1 * 1.01))
            fd = (vals[0] - vals[1]) / (2 * h)
            assert abs(g[v, u] - fd) <= G_TOL * np.abs(g).max(), (which, v, u, g[v, u], fd)


def test_batch_equals_single_calls(scene):
    crops = [synth.crop_pair(scene, u0, v0, 70, 40) for (u0, v0) in ((300, 200), (500, 350), (650, 420))]
    D = 24
    l, p, rts, ws = gpu_forward([c[0] for c in crops], [c[1] for c in crops], [c[2] for c in crops], D)
    gl = np.random.default_rng(3).normal(size=l.shape).astype(np.float32)
    gr, gt = gpu_backward(p, rts, ws, gl)
    for b, (ref, tgt, sh) in enumerate(crops):
        l1, p1, rts1, ws1 = gpu_forward([ref], [tgt], [sh], D)
        g1r, g1t = gpu_backward(p1, rts1, ws1, gl[b:b + 1])
        assert np.array_equal(l1[0], l[b])
        assert np.array_equal(g1r[0], gr[b]) and np.array_equal(g1t[0], gt[b])


def test_repeated_calls_are_bit_identical(scene):
    ref, tgt, sh = synth.crop_pair(scene, 448, 300, 64, 48)
    gl = np.random.default_rng(4).normal(size=(1, 48, 64)).astype(np.float32)
    outs = []
    for _ in range(2):
        l, p, rts, ws = gpu_forward([ref], [tgt], [sh], 16)
        outs.append((l, *gpu_backward(p, rts, ws, gl)))
    for a, b in zip(*outs):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("W,H,D,win,bil", [(1, 1, 4, 3, 3), (5, 1, 3, 3, 5), (1, 7, 2, 5, 3),
                                           (40, 3, 8, 5, 5), (33, 35, 1, 9, 11), (36, 20, 12, 1, 1),
                                           (50, 30, 40, 15, 15)])
def test_degenerate_shapes_match_the_oracle(W, H, D, win, bil):
    rng = np.random.default_rng(W * 100 + H)
    ref = rng.uniform(0, 255, (H, W))
    tgt = rng.uniform(0, 255, (H, W))
    sh = rng.uniform(-3, 3, H).astype(np.float32)
    l, p, rts, ws = gpu_forward([ref], [tgt], [sh], D, win, bil)
    gl = rng.normal(size=(H, W))
    lo, gro, gto = odiff.disparity_vjp(ref, tgt, sh, D, win, bil, S0, S1, T, gl)
    assert np.abs(l[0] - lo).max() <= L_TOL
    gr, gt = gpu_backward(p, rts, ws, gl[None].astype(np.float32))
    if D == 1 or win == 1:
        # one disparity, or 1 x 1 windows (sigma = 0, c = 1): l is constant, no gradient
        assert np.all(gr == 0) and np.all(gt == 0)
        assert np.all(gro == 0) and np.all(gto == 0)
    else:
        # absolute floor: where W = 1 every disparity reads the same clamped target block, and
        # their adjoints cancel exactly in FP64 but leave FP32 rounding (~1e-8) on the GPU
        check_grad(gr[0], gro, "dS/dref", floor=1e-6)
        check_grad(gt[0], gto, "dS/dtgt", floor=1e-6)


def test_workspace_checks(scene):
    p = sgd.stereo_diff_params_default(width=64, height=48, max_disp=16)
    n = sgd.stereo_softargmin_workspace_bytes(p)
    x = torch.zeros((1, 48, 64), device="cuda")
    s = torch.zeros((1, 48), device="cuda")
    small = torch.empty(n - 256, dtype=torch.uint8, device="cuda")
    with pytest.raises(sg.StereoError) as e:
        sgd.stereo_softargmin_fwd(p, x, x, s, x, small)
    assert e.value.code == sg.STEREO_EINVAL


def _plane_fit_psi(l, mask):
    v, u = np.nonzero(mask)
    A = np.stack([np.ones_like(u), u, v], axis=1).astype(np.float64)
    a, b, c = np.linalg.lstsq(A, l[v, u], rcond=None)[0]
    return math.atan(-b / c)


def test_refine_roll_reaches_the_oracle_fit_on_the_full_workload(scene):
    """960 x 540, D = 64: soft-argmin on the GPU, 50 refinement steps from psi = 0, against
    the closed-form fit and oracle.dt's search on the same (copied) disparity map."""
    H, W, D = scene.height, scene.width, 64
    l, p, rts, ws = gpu_forward([scene.ref.astype(np.float64)], [scene.tgt.astype(np.float64)],
                                [scene.shift], D)
    mask = oracle.valid_mask(W, H, D, WIN, BIL, scene.shift)
    traj = sgd.refine_roll(dev(l[0]), dev(mask, torch.uint8), 0.0, 50).cpu().numpy()[0]
    lf = l[0]
    psi_star = _plane_fit_psi(lf, mask)
    print("\nroll %.6f deg; refined %.9f, closed form %.9f rad" % (math.degrees(scene.roll), traj[-1, 0],
                                                                  psi_star))
    assert abs(traj[-1, 0] - psi_star) < 1e-8
    v, u = np.nonzero(mask)
    res = odt.estimate_roll(lf[v, u], u.astype(np.float64), v.astype(np.float64))
    assert abs(traj[-1, 0] - res["psi"]) < 1e-7
    a = odiff.alpha_fit(lf, mask, traj[-1, 0])
    assert traj[-1, 1] == pytest.approx(a[0], rel=1e-9, abs=1e-9)
    assert traj[-1, 2] == pytest.approx(a[1], rel=1e-9)
    assert traj[-1, 4] <= traj[0, 4]
    # the step's gradient is the adjoint kernel's psi-gradient at (psi_0, alpha(psi_0))
    theta = torch.tensor(traj[0, :3], dtype=torch.float64, device="cuda", requires_grad=True)
    L = sgd.dt_energy(dev(lf), theta, dev(mask, torch.uint8))
    L.backward()
    assert float(theta.grad[0]) == pytest.approx(traj[0, 3], rel=1e-3)
    assert float(L.detach()) == pytest.approx(traj[0, 4], rel=1e-5)


def _local_window(x, y, R, D, W, H):
    """A window holding every input that the soft-argmin of the pixels in rows y +- R, columns
    x - R .. x + R + D - 1 reads (the pixels whose l depends on ref(y, x) or on the warped
    target at (y, x)): rows y +- 2R, columns x - 2R - (D-1) .. x + 2R + D - 1."""
    r0, r1 = y - 2 * R, y + 2 * R + 1
    c0, c1 = x - 2 * R - (D - 1), x + 2 * R + D
    assert r0 >= 0 and c0 >= 0 and r1 <= H and c1 <= W
    return r0, r1, c0, c1


def test_full_workload_batch_sampled_against_the_oracle():
    """The differentiation workload: 8 pairs of 960 x 540, D = 64, in one batched call.
    Sampled checks of l and of both image gradients against the oracle run on a window that
    holds everything those values depend on (S = sum gl l over the pixels that depend on the
    sampled input pixel; its gradient there equals the full-image one)."""
    scenes = [synth.make_config_scene("grad", pair=i) for i in range(8)]
    H, W, D = 540, 960, 64
    R = BIL // 2 + WIN // 2
    l, p, rts, ws = gpu_forward([s.ref.astype(np.float64) for s in scenes],
                                [s.tgt.astype(np.float64) for s in scenes], [s.shift for s in scenes], D)
    gl = np.random.default_rng(12).normal(size=(8, H, W)).astype(np.float32)
    gr, gt = gpu_backward(p, rts, ws, gl)
    assert np.all(np.isfinite(l)) and np.all(np.isfinite(gr)) and np.all(np.isfinite(gt))
    rng = np.random.default_rng(13)
    for b in (0, 5):
        s = scenes[b]
        tw = odiff.warp(torch.tensor(s.tgt.astype(np.float64)), s.shift).numpy()
        si = np.floor(s.shift.astype(np.float64) + 0.5)
        for _ in range(2):
            x = int(rng.integers(2 * R + D, W - 2 * R - D))
            y = int(rng.integers(2 * R, H - 2 * R - 1))
            r0, r1, c0, c1 = _local_window(x, y, R, D, W, H)
            ref_w = torch.tensor(s.ref[r0:r1, c0:c1].astype(np.float64), requires_grad=True)
            tw_w = torch.tensor(tw[r0:r1, c0:c1], requires_grad=True)
            c = odiff.cost_volume(ref_w, tw_w, D, WIN)
            E = odiff.aggregate(ref_w, c, BIL, S0, S1)
            lbar = odiff.soft_argmin(E, np.zeros(r1 - r0, np.float32), T)
            yy, xx = y - r0, x - c0
            inner = (slice(yy - R, yy + R + 1), slice(xx - R, xx + R + D))
            full = (slice(y - R, y + R + 1), slice(x - R, x + R + D))
            lo = lbar.detach().numpy()[inner] + si[y - R:y + R + 1][:, None]
            assert np.abs(l[b][full] - lo).max() <= L_TOL
            S = (lbar[inner] * torch.tensor(gl[b][full].astype(np.float64))).sum()
            S.backward()
            g_ref = float(ref_w.grad[yy, xx])
            g_tw = float(tw_w.grad[yy, xx])
            # the target pixel (y, x - s_i(y)) feeds exactly the warped pixel (y, x)
            xs = x - int(si[y])
            print("\npair %d (%d, %d): dS/dref %.6g vs %.6g, dS/dtgt %.6g vs %.6g" % (
                b, x, y, gr[b, y, x], g_ref, gt[b, y, xs], g_tw))
            assert abs(gr[b, y, x] - g_ref) <= G_TOL * np.abs(gr[b]).max()
            assert abs(gt[b, y, xs] - g_tw) <= G_TOL * np.abs(gt[b]).max()


def test_linear_warp_matches_the_oracle(scene):
    """Fractional row shifts read by interpolation: l, both image gradients and dS/ds(v)."""
    ref, tgt, sh = synth.crop_pair(scene, 448, 300, 64, 48)
    D = 16
    H, W = ref.shape
    shf = (sh + np.linspace(-0.45, 0.4, H)).astype(np.float32)
    l, p, rts, ws = gpu_forward([ref.astype(np.float64)], [tgt.astype(np.float64)], [shf], D,
                                mode=sgd.STEREO_WARP_LINEAR)
    gl = np.random.default_rng(17).normal(size=(H, W))
    lo, gro, gto, gso = odiff.disparity_linear_vjp(ref, tgt, shf, D, WIN, BIL, S0, S1, T, gl)
    assert np.abs(l[0] - lo).max() <= L_TOL
    gr, gt, gs = gpu_backward(p, rts, ws, gl[None].astype(np.float32), want_shift=True)
    check_grad(gr[0], gro, "dS/dref")
    check_grad(gt[0], gto, "dS/dtgt")
    check_grad(gs[0], gso, "dS/ds")


def test_rounded_warp_has_no_shift_gradient(scene):
    ref, tgt, sh = synth.crop_pair(scene, 448, 300, 64, 48)
    l, p, rts, ws = gpu_forward([ref.astype(np.float64)], [tgt.astype(np.float64)], [sh], 16)
    _, _, gs = gpu_backward(p, rts, ws, np.ones((1, 48, 64), np.float32), want_shift=True)
    assert np.all(gs == 0.0)


def test_warp_coefficients_refined_through_autograd(scene):
    """s(v) = c0 + c1 v (eq. relation_vd) computed by torch from two float64 parameters: the
    backward of SoftArgmin (linear warp) and DTEnergy reaches c0 and c1; checked against the
    oracle's FP64 chain and against its central differences."""
    ref, tgt, sh = synth.crop_pair(scene, 448, 300, 64, 48)
    D = 16
    H, W = ref.shape
    v = np.arange(H, dtype=np.float64)
    c1_0 = float(np.polyfit(v, sh.astype(np.float64), 1)[0])
    c0_0 = float(sh[0]) + 0.3
    c = torch.tensor([c0_0, c1_0], dtype=torch.float64, device="cuda", requires_grad=True)
    vt = torch.arange(H, dtype=torch.float64, device="cuda")
    s = c[0] + c[1] * vt
    r = dev(ref)
    t = dev(tgt)
    l = sgd.soft_argmin_disparity(r, t, s, D, WIN, BIL, S0, S1, T, warp_mode=sgd.STEREO_WARP_LINEAR)
    theta = torch.tensor([0.02, 30.0, 0.1], dtype=torch.float64, device="cuda")
    L = sgd.dt_energy(l, theta)
    L.backward()
    g = c.grad.cpu().numpy()

    def loss(c0, c1):
        sv = (c0 + c1 * v).astype(np.float32)
        lx = odiff.disparity_linear_value(ref, tgt, sv, D, WIN, BIL, S0, S1, T)
        return odiff.energy_value(lx, np.ones((H, W)), 0.02, 30.0, 0.1)

    ct = torch.tensor([c0_0, c1_0], dtype=torch.float64, requires_grad=True)
    so = ct[0] + ct[1] * torch.arange(H, dtype=torch.float64)
    lo = odiff.disparity(torch.tensor(ref.astype(np.float64)), torch.tensor(tgt.astype(np.float64)), so, D, WIN,
                         BIL, S0, S1, T, 1)
    odiff.dt_energy(lo, torch.ones((H, W), dtype=torch.float64), torch.tensor(0.02, dtype=torch.float64),
                    torch.tensor(30.0, dtype=torch.float64), torch.tensor(0.1, dtype=torch.float64)).backward()
    go = ct.grad.numpy()
    print("\ndL/dc0, dL/dc1: GPU %s, oracle %s" % (g, go))
    assert g == pytest.approx(go, rel=1e-3)
    h = 1e-3
    fd0 = (loss(c0_0 + h, c1_0) - loss(c0_0 - h, c1_0)) / (2 * h)
    assert go[0] == pytest.approx(fd0, rel=1e-3)
