"""Parity of the CUDA path (through the C ABI) with the CPU oracle, element by element,
on seeded synthetic inputs: warp bit-exact; costs and aggregated costs within 1e-4
relative; WTA d* bit-exact wherever the oracle's best and second-best aggregated costs
differ by more than 1e-3; sub-pixel disparity within 0.01 px; valid mask bit-exact;
transformed disparity within 1e-3 px."""
import math

import numpy as np
import pytest
import torch

import oracle
from oracle import dt
import paper_1904_06017_gb300 as sg
import synth
from gpu_helpers import (DT_TOL, check_disparity, check_rel, dev_f32, dev_img, pitch_of)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1904_06017_gb300 import build
    build.build()
    oracle.build()


def run_fused(ref, tgtw, shift, D, win, bil, s0, s1, pitch_extra=0):
    H, W = ref.shape
    pitch = pitch_of(W, pitch_extra)
    disp = torch.empty((H, W), dtype=torch.float32, device="cuda")
    wta = torch.empty((H, W), dtype=torch.int32, device="cuda")
    valid = torch.empty((H, W), dtype=torch.uint8, device="cuda")
    with sg.Stereo(W, H, D, win=win, bil=bil, sigma0=s0, sigma1=s1, pitch=pitch) as st:
        st.cost_aggregate_wta(dev_img(ref, pitch), dev_img(tgtw, pitch), dev_f32(shift), disp, wta, valid)
        st.check_device_status()
    return disp.cpu().numpy(), wta.cpu().numpy(), valid.cpu().numpy()


# ------------------------------------------------------------------------------ warp
# widths equal to the pitch (320, 1920) put the second aligned source word of the last
# interior segment at the end of the row; 40 rows of random shifts cover every byte offset
@pytest.mark.parametrize("W,H,extra", [(37, 5, 16), (64, 9, 16), (100, 17, 16), (333, 11, 16), (1, 3, 16),
                                         (320, 40, 0), (1920, 24, 0)])
def test_warp_bit_exact(W, H, extra):
    rng = np.random.default_rng(W * 7 + H)
    tgt = rng.integers(0, 256, (H, W), dtype=np.uint8)
    shift = rng.uniform(-25, 25, H).astype(np.float32)
    shift[0] = 2.5
    shift[-1] = -2.5
    if H > 3:   # next to the ties, where s + 0.5 rounded to float32 would round up
        shift[1], shift[2] = 0.5 - 2.0 ** -25, -0.5 - 2.0 ** -24
    pitch = pitch_of(W, extra)
    out = dev_img(np.zeros((H, W), np.uint8), pitch, fill=0xAB)
    with sg.Stereo(W, H, 8, win=3, bil=3, pitch=pitch) as st:
        st.warp_target(dev_img(tgt, pitch), dev_f32(shift), out)
    o = out.cpu().numpy()
    assert np.array_equal(o[:, :W], oracle.warp(tgt, shift))
    assert np.all(o[:, W:] == 0xAB)      # bytes past the row are left alone


# ------------------------------------------------------------- unfused stage kernels
@pytest.mark.parametrize("W,H,D,win,bil", [(64, 48, 16, 7, 9), (45, 29, 13, 3, 5), (70, 33, 24, 9, 11)])
def test_unfused_stages_match_oracle(W, H, D, win, bil):
    rng = np.random.default_rng(W + H + D)
    ref = synth.texture(rng, H, W)
    tgt = synth.texture(rng, H, W)
    tgt[:, 5:] = ref[:, :-5]              # partly a true match at d = 5
    shift = np.zeros(H, np.float32)
    c_o = oracle.cost_volume(ref, tgt, D, win)
    E_o, ws = oracle.aggregate(ref, c_o, bil, 3.0, 10.0, return_wsum=True)
    d_o, ds_o, eb, es = oracle.wta(E_o, shift)
    pitch = pitch_of(W)
    cost = torch.empty((H, W, D), dtype=torch.float32, device="cuda")
    agg = torch.empty_like(cost)
    disp = torch.empty((H, W), dtype=torch.float32, device="cuda")
    wta = torch.empty((H, W), dtype=torch.int32, device="cuda")
    best2 = torch.empty((H, W, 2), dtype=torch.float32, device="cuda")
    r = dev_img(ref, pitch)
    with sg.Stereo(W, H, D, win=win, bil=bil, sigma0=3.0, sigma1=10.0, pitch=pitch) as st:
        st.cost_volume(r, dev_img(tgt, pitch), cost)
        st.aggregate_volume(r, cost, agg)
        st.wta_volume(agg, dev_f32(shift), disp, wta, best2)
    check_rel(cost.cpu().numpy(), c_o)
    check_rel(agg.cpu().numpy(), E_o)
    b2 = best2.cpu().numpy()
    check_rel(b2[..., 0], eb)
    check_rel(b2[..., 1], es)
    check_disparity(disp.cpu().numpy(), wta.cpu().numpy(), d_o, ds_o, eb, es, min_sure=0.8)


# --------------------------------------------------------------------- fused kernel
def _fused_vs_oracle(s, D, win, bil, s0, s1, warp=True, pitch_extra=0, min_sure=0.9):
    tw = oracle.warp(s.tgt, s.shift) if warp else s.tgt
    disp, wta, valid = run_fused(s.ref, tw, s.shift, D, win, bil, s0, s1, pitch_extra)
    d_o, ds_o, eb, es = oracle.stereo(s.ref, tw, s.shift, D, win, bil, s0, s1)
    check_disparity(disp, wta, d_o, ds_o, eb, es, min_sure=min_sure)
    vm = oracle.valid_mask(s.width, s.height, D, win, bil, s.shift)
    assert np.array_equal(valid, vm)
    return disp, d_o


def test_fused_small_preset():
    s = synth.make_config_scene("small")
    p = s.params
    _fused_vs_oracle(s, p["D"], p["win"], p["bil"], p["sigma0"], p["sigma1"], warp=False)


def test_fused_paper_parameters():
    """sigma0 = 1.5, sigma1 = 5.5, 120-connected (11 x 11) neighbourhood (§4.4.1)."""
    s = synth.make_scene(200, 90, 32, 777, roll=math.radians(2.0), n_potholes=2, warp=True, win=9, bil=11)
    _fused_vs_oracle(s, 32, 9, 11, 1.5, 5.5, min_sure=0.8)


@pytest.mark.parametrize("W,H,D,win,bil", [(201, 75, 20, 5, 7), (65, 33, 12, 3, 1), (130, 70, 24, 3, 3),
                                           (97, 41, 17, 5, 5), (150, 66, 30, 11, 15), (129, 52, 40, 9, 13)])
def test_fused_ragged_sizes_and_windows(W, H, D, win, bil):
    s = synth.make_scene(W, H, D, 1000 + W + D, roll=math.radians(3.0), coeffs=(4.0, 0.1, 1e-4),
                         n_potholes=1, warp=True, win=win, bil=bil)
    _fused_vs_oracle(s, D, win, bil, 3.0, 10.0, pitch_extra=32, min_sure=0.6 if bil == 1 else 0.8)


@pytest.mark.parametrize("W,H,D,win,bil", [(130, 70, 24, 9, 11), (97, 41, 17, 5, 5), (70, 33, 1, 3, 3)])
def test_fused_best_and_second_cost(W, H, D, win, bil):
    """The optional best2 output: the normalised E of eq. (fbs) at d* and the smallest E over
    d != d*, against the oracle's, at every pixel (within the cost tolerance); with D = 1
    there is no second disparity and both sides give +inf."""
    s = synth.make_scene(W, H, D, 2000 + W + D, roll=math.radians(2.0), coeffs=(4.0, 0.1, 1e-4),
                         n_potholes=1, warp=True, win=win, bil=bil)
    tw = oracle.warp(s.tgt, s.shift)
    pitch = pitch_of(W)
    disp = torch.empty((H, W), dtype=torch.float32, device="cuda")
    best2 = torch.empty((H, W, 2), dtype=torch.float32, device="cuda")
    with sg.Stereo(W, H, D, win=win, bil=bil, sigma0=3.0, sigma1=10.0, pitch=pitch) as st:
        st.cost_aggregate_wta(dev_img(s.ref, pitch), dev_img(tw, pitch), dev_f32(s.shift), disp, best2=best2)
        st.check_device_status()
    b2 = best2.cpu().numpy().astype(np.float64)
    _, _, eb, es = oracle.stereo(s.ref, tw, s.shift, D, win, bil, 3.0, 10.0)
    check_rel(b2[..., 0], eb)
    fin = np.isfinite(es)
    assert np.array_equal(np.isfinite(b2[..., 1]), fin)
    if fin.any():
        check_rel(b2[..., 1][fin], es[fin])


def test_fused_single_disparity_and_tiny_image():
    rng = np.random.default_rng(5)
    ref = synth.texture(rng, 20, 30)
    tgt = synth.texture(rng, 20, 30)
    shift = np.linspace(-2, 3, 20).astype(np.float32)
    disp, wta, valid = run_fused(ref, tgt, shift, 1, 5, 5, 3.0, 10.0)
    si = np.floor(shift.astype(np.float64) + 0.5)
    assert np.all(wta == 0)
    assert np.array_equal(disp, np.broadcast_to(si[:, None], disp.shape).astype(np.float32))
    one = np.array([[17]], np.uint8)
    d1, w1, v1 = run_fused(one, one, np.zeros(1, np.float32), 4, 3, 3, 3.0, 10.0)
    assert w1[0, 0] == 0 and v1[0, 0] == 0


def test_fused_identical_images_give_row_shift():
    rng = np.random.default_rng(6)
    img = synth.texture(rng, 70, 90)
    shift = np.linspace(-4, 6, 70).astype(np.float32)
    disp, wta, _ = run_fused(img, img, shift, 24, 7, 9, 3.0, 10.0)
    si = np.floor(shift.astype(np.float64) + 0.5)
    assert np.all(wta == 0)
    assert np.array_equal(disp, np.broadcast_to(si[:, None], disp.shape).astype(np.float32))


def test_fused_maximum_disparity_and_window():
    s = synth.make_scene(300, 40, 256, 4242, roll=0.0, coeffs=(100.0, 0.0, 0.0), n_potholes=0,
                         warp=False, win=11, bil=15)
    _fused_vs_oracle(s, 256, 11, 15, 3.0, 10.0, warp=False, min_sure=0.3)


# ------------------------------------------------------ disparity transformation
def _plane_map(H, W, psi, a0, a1, noise, seed, dent=True):
    rng = np.random.default_rng(seed)
    u = np.arange(W)[None, :]
    v = np.arange(H)[:, None]
    d = a0 + a1 * (v * math.cos(psi) - u * math.sin(psi)) + noise * rng.standard_normal((H, W))
    if dent:
        d -= 4.0 * np.exp(-((u - 0.6 * W) ** 2 + (v - 0.7 * H) ** 2) / (0.01 * W * H))
    return d


@pytest.mark.parametrize("H,W,psi,psi_init", [(120, 160, 0.05, 0.0), (540, 960, -0.08, 0.0),
                                              (1080, 1920, 0.1, 0.3), (300, 200, 0.0, -0.2)])
def test_dt_matches_oracle_on_a_shared_map(H, W, psi, psi_init):
    dmap = _plane_map(H, W, psi, 5.0, 0.12, 0.5, H + W).astype(np.float32)
    rng = np.random.default_rng(1)
    mask = (rng.random((H, W)) > 0.2).astype(np.uint8)
    out = torch.empty((H, W), dtype=torch.float32, device="cuda")
    with sg.Stereo(W, H, 16, pitch=pitch_of(W)) as st:
        res = st.disparity_transform(dev_f32(dmap), torch.from_numpy(mask).cuda(), psi_init, 1.5, out)
    out_o, r_o = dt.disparity_transform(dmap.astype(np.float64), mask.astype(bool), psi_init=psi_init,
                                        delta_t=1.5)
    delta_psi = math.pi / 1.8e6
    assert res.status == sg.STEREO_OK and r_o["status"] == 0
    assert res.n == int(mask.sum())
    assert abs(res.psi - r_o["psi"]) < delta_psi
    assert res.alpha1 == pytest.approx(r_o["alpha1"], rel=1e-5)
    assert res.alpha0 == pytest.approx(r_o["alpha0"], rel=1e-5, abs=1e-4)
    assert res.e_min == pytest.approx(r_o["e_min"], rel=1e-6)
    assert np.max(np.abs(out.cpu().numpy() - out_o)) < DT_TOL


@pytest.mark.parametrize("H,W,psi,psi_init", [(120, 160, 0.05, 0.0), (540, 960, -0.08, 0.0),
                                              (1080, 1920, 0.1, 0.3), (300, 200, 0.0, -0.2),
                                              (240, 320, -0.6, 0.0)])
def test_dt_reaches_the_plane_fit_closed_form(H, W, psi, psi_init):
    """The minimum of eq. (E2) over (psi, alpha) has a closed form: alpha0 + alpha1 y(psi) spans
    every affine function of (u, v), so the least-squares plane l ~ a + b u + c v over the
    fitted pixels gives psi* = atan(-b / c), alpha1 = c / cos(psi*), alpha0 = a, and E_min(psi*)
    is the plane's residual.  The device search lands within 1e-8 rad of psi*.  (The oracle,
    which evaluates eq. (E_min2) on raw coordinates, stops up to about 5e-8 rad from psi* on
    the 1080p map: its energy differences there are at its FP64 rounding floor.)"""
    dmap = _plane_map(H, W, psi, 5.0, 0.12, 0.5, H + W).astype(np.float32)
    rng = np.random.default_rng(1)
    mask = (rng.random((H, W)) > 0.2).astype(np.uint8)
    out = torch.empty((H, W), dtype=torch.float32, device="cuda")
    with sg.Stereo(W, H, 16, pitch=pitch_of(W)) as st:
        res = st.disparity_transform(dev_f32(dmap), torch.from_numpy(mask).cuda(), psi_init, 0.0, out)
    vv, uu = np.nonzero(mask)
    A = np.stack([np.ones(len(uu)), uu.astype(np.float64), vv.astype(np.float64)], axis=1)
    dv = dmap[vv, uu].astype(np.float64)
    (a, b, c), *_ = np.linalg.lstsq(A, dv, rcond=None)
    psi_star = math.atan(-b / c)
    assert res.status == sg.STEREO_OK
    assert abs(res.psi - psi_star) < 1e-8
    assert res.alpha1 == pytest.approx(c / math.cos(psi_star), rel=1e-7)
    assert res.alpha0 == pytest.approx(a, rel=1e-7, abs=1e-7)
    resid = dv - A @ np.array([a, b, c])
    assert res.e_min == pytest.approx(float(resid @ resid), rel=1e-7)


@pytest.mark.parametrize("H,W,offset", [(23, 37, 0), (47, 61, 1), (11, 13, 0), (31, 33, 3)])
def test_dt_ragged_and_unaligned_maps(H, W, offset):
    """Maps whose pixel count is not a multiple of the 32-pixel load pieces, and maps (and masks)
    that start off a 16-byte boundary, take the per-pixel reads of the moments kernel: the same
    fit as the oracle's."""
    dmap = _plane_map(H, W, 0.07, 4.0, 0.15, 0.3, H * W + offset, dent=False).astype(np.float32)
    rng = np.random.default_rng(H + W)
    mask = (rng.random((H, W)) > 0.1).astype(np.uint8)
    N = H * W
    dbuf = torch.zeros(N + offset, dtype=torch.float32, device="cuda")
    mbuf = torch.zeros(N + offset, dtype=torch.uint8, device="cuda")
    dbuf[offset:] = torch.from_numpy(dmap.ravel()).cuda()
    mbuf[offset:] = torch.from_numpy(mask.ravel()).cuda()
    d_in, m_in = dbuf[offset:].view(H, W), mbuf[offset:].view(H, W)
    out = torch.empty((H, W), dtype=torch.float32, device="cuda")
    with sg.Stereo(W, H, 2, pitch=pitch_of(W)) as st:
        res = st.disparity_transform(d_in, m_in, 0.0, 0.5, out)
    out_o, r_o = dt.disparity_transform(dmap.astype(np.float64), mask.astype(bool), delta_t=0.5)
    assert res.status == sg.STEREO_OK and res.n == int(mask.sum())
    assert abs(res.psi - r_o["psi"]) < math.pi / 1.8e6
    assert res.alpha1 == pytest.approx(r_o["alpha1"], rel=1e-5)
    assert res.alpha0 == pytest.approx(r_o["alpha0"], rel=1e-5, abs=1e-4)
    assert np.max(np.abs(out.cpu().numpy() - out_o)) < DT_TOL


def test_dt_device_result_iteration_cap_and_empty_mask():
    H, W = 64, 80
    dmap = _plane_map(H, W, 0.2, 3.0, 0.1, 0.3, 9).astype(np.float32)
    out = torch.empty((H, W), dtype=torch.float32, device="cuda")
    resbuf = torch.zeros(64, dtype=torch.uint8, device="cuda")
    with sg.Stereo(W, H, 8, pitch=pitch_of(W), max_iters=1) as st:
        assert st.disparity_transform(dev_f32(dmap), None, 0.0, 0.0, out, res=resbuf) is None
        torch.cuda.synchronize()
        raw = resbuf.cpu().numpy().tobytes()[:48]
        r = sg.stereo_dt_result.from_buffer_copy(raw)
        assert r.status == sg.STEREO_ENOCONV and r.iters == 1 and r.n == H * W
        empty = torch.zeros((H, W), dtype=torch.uint8, device="cuda")
        r2 = st.disparity_transform(dev_f32(dmap), empty, 0.0, 0.0, out)
        assert r2.status == sg.STEREO_EINVAL and r2.n == 0


# ------------------------------------------------------------ end to end pipeline
@pytest.mark.slow
def test_pipeline_large_preset():
    """1024 x 768, D = 32, w = 9, k = 11, warp on: every stage against the oracle."""
    s = synth.make_config_scene("large")
    p = s.params
    H, W, D = s.height, s.width, p["D"]
    pitch = pitch_of(W)
    ref, tgt = dev_img(s.ref, pitch), dev_img(s.tgt, pitch)
    shift = dev_f32(s.shift)
    tw = torch.empty_like(tgt)
    disp = torch.empty((H, W), dtype=torch.float32, device="cuda")
    wta = torch.empty((H, W), dtype=torch.int32, device="cuda")
    valid = torch.empty((H, W), dtype=torch.uint8, device="cuda")
    out = torch.empty_like(disp)
    with sg.Stereo(W, H, D, win=p["win"], bil=p["bil"], sigma0=p["sigma0"], sigma1=p["sigma1"],
                   pitch=pitch) as st:
        st.warp_target(tgt, shift, tw)
        st.cost_aggregate_wta(ref, tw, shift, disp, wta, valid)
        res = st.disparity_transform(disp, valid, 0.0, 0.0, out)
        st.check_device_status()
    tw_o = oracle.warp(s.tgt, s.shift)
    assert np.array_equal(tw[:, :W].cpu().numpy(), tw_o)
    d_o, ds_o, eb, es = oracle.stereo(s.ref, tw_o, s.shift, D, p["win"], p["bil"], p["sigma0"], p["sigma1"])
    check_disparity(disp.cpu().numpy(), wta.cpu().numpy(), d_o, ds_o, eb, es)
    vm = oracle.valid_mask(W, H, D, p["win"], p["bil"], s.shift)
    assert np.array_equal(valid.cpu().numpy(), vm)
    dmap = disp.cpu().numpy().astype(np.float64)
    out_o, r_o = dt.disparity_transform(dmap, vm.astype(bool))
    assert abs(res.psi - r_o["psi"]) < math.pi / 1.8e6
    assert np.max(np.abs(out.cpu().numpy() - out_o)) < DT_TOL


@pytest.mark.slow
def test_full_hd_sampled_rows():
    """1920 x 1080, D = 128, w = 9, k = 11: the benchmark workload in the benchmark's
    launch configuration, checked on sampled row bands the oracle computes directly."""
    s = synth.make_config_scene("hd")
    p = s.params
    H, W, D = s.height, s.width, p["D"]
    tw_o = oracle.warp(s.tgt, s.shift)
    pitch = pitch_of(W)
    tw = torch.empty((H, pitch), dtype=torch.uint8, device="cuda")
    disp = torch.empty((H, W), dtype=torch.float32, device="cuda")
    wta = torch.empty((H, W), dtype=torch.int32, device="cuda")
    valid = torch.empty((H, W), dtype=torch.uint8, device="cuda")
    shift = dev_f32(s.shift)
    with sg.Stereo(W, H, D, win=p["win"], bil=p["bil"], sigma0=p["sigma0"], sigma1=p["sigma1"],
                   pitch=pitch) as st:
        st.warp_target(dev_img(s.tgt, pitch), shift, tw)
        st.cost_aggregate_wta(dev_img(s.ref, pitch), tw, shift, disp, wta, valid)
        st.check_device_status()
    assert np.array_equal(tw[:, :W].cpu().numpy(), tw_o)
    dg, wg = disp.cpu().numpy(), wta.cpu().numpy()
    for v0, v1 in [(0, 8), (530, 546), (1072, 1080)]:
        d_o, ds_o, eb, es = oracle.stereo(s.ref, tw_o, s.shift, D, p["win"], p["bil"], p["sigma0"],
                                          p["sigma1"], rows=(v0, v1))
        check_disparity(dg[v0:v1], wg[v0:v1], d_o, ds_o, eb, es, min_sure=0.7)
    vm = oracle.valid_mask(W, H, D, p["win"], p["bil"], s.shift)
    assert np.array_equal(valid.cpu().numpy(), vm)


# ------------------------------------------------------------------ diagnostics
def test_status_profile_and_argument_errors():
    rng = np.random.default_rng(3)
    W, H, D = 96, 40, 16
    ref = dev_img(synth.texture(rng, H, W))
    tgt = dev_img(synth.texture(rng, H, W))
    shift = torch.zeros(H, dtype=torch.float32, device="cuda")
    disp = torch.empty((H, W), dtype=torch.float32, device="cuda")
    with sg.Stereo(W, H, D, pitch=pitch_of(W)) as st:
        sg.stereo_profile_enable(st.ctx, True)
        for _ in range(3):
            st.cost_aggregate_wta(ref, tgt, shift, disp)
        n, ms = sg.stereo_profile_read(st.ctx)
        assert n == 3 and ms > 0
        st.check_device_status()
        bad = ref.view(-1)[1:].data_ptr()          # not 16-byte aligned
        with pytest.raises(sg.StereoError) as e:
            sg.stereo_cost_aggregate_wta(st.ctx, bad, tgt, shift, disp)
        assert e.value.code == sg.STEREO_EINVAL
        with pytest.raises(sg.StereoError) as e:
            sg.stereo_warp_target(st.ctx, tgt, shift, tgt)
        assert e.value.code == sg.STEREO_EINVAL
