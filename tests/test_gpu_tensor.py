"""Tensor-core aggregation of the FP16 / BF16 storage forms (mma.sync over 4 x 4 pixel
patches, FP32 accumulators), the default kernel of those forms for bil <= 13: 32 x 36 tiles
with weights rounded from the FP32 ones (k_fused_sc, plain mode); batches may also take 64 x 36
tiles with weights formed in 16-bit arithmetic (k_fused_tc, tile_wc 16).

Its costs and bilateral weights are rounded to the 16-bit type, so it is held to bounds
derived from that rounding rather than the FP32 path's 1e-3 gap.  FP16: a cost moves by at
most 2 * 2^-11 ~ 1e-3; a weight's exponent is formed from the exact integer intensity
difference with three roundings of 2^-11 (about 1.5e-3 |exponent| absolute) and the power by
ex2.approx on halves (relative error under 2^-9.9), so for the weighted-mean exponent of a
window (a few units) a weight is off by at most about 0.4 %, and the normalised aggregated
cost by at most 1e-3 + 0.004 * 2 ~ 9e-3.  The integer disparity must then equal the oracle's
wherever the oracle's best and second-best normalised costs differ by more than twice that,
2e-2.  BF16 (8-bit significands, four times the rounding, ex2 on bf16 pairs): 1e-1."""
import math

import numpy as np
import pytest
import torch

import oracle
import paper_1904_06017_gb300 as sg
import synth
from gpu_helpers import dev_f32, dev_img, pitch_of

pytestmark = pytest.mark.gpu

GAP = {sg.STEREO_F16: 2e-2, sg.STEREO_BF16: 1e-1}


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1904_06017_gb300 import build
    build.build()
    oracle.build()


def run_single(ref, tgtw, shift, D, win, bil, s0, s1, dtype, pitch_extra=0):
    H, W = ref.shape
    pitch = pitch_of(W, pitch_extra)
    disp = torch.empty((H, W), dtype=torch.float32, device="cuda")
    wta = torch.empty((H, W), dtype=torch.int32, device="cuda")
    valid = torch.empty((H, W), dtype=torch.uint8, device="cuda")
    with sg.Stereo(W, H, D, win=win, bil=bil, sigma0=s0, sigma1=s1, pitch=pitch, cost_dtype=dtype) as st:
        st.cost_aggregate_wta(dev_img(ref, pitch), dev_img(tgtw, pitch), dev_f32(shift), disp, wta, valid)
        st.check_device_status()
    return disp.cpu().numpy(), wta.cpu().numpy(), valid.cpu().numpy()


def check_vs_oracle(s, D, win, bil, s0, s1, dtype, min_sure):
    tw = oracle.warp(s.tgt, s.shift)
    disp, wta, valid = run_single(s.ref, tw, s.shift, D, win, bil, s0, s1, dtype, pitch_extra=16)
    d_o, ds_o, eb, es = oracle.stereo(s.ref, tw, s.shift, D, win, bil, s0, s1)
    sure = (es - eb) > GAP[dtype]
    assert sure.mean() >= min_sure, "too few well-separated pixels (%.3f)" % sure.mean()
    bad = int(np.count_nonzero(wta[sure] != ds_o[sure]))
    err = np.abs(disp.astype(np.float64) - d_o)[sure]
    print("\n%dx%d D=%d win=%d bil=%d dtype=%d: sure %.3f, WTA mismatches %d, sub-pixel error mean %.2e p99 %.2e"
          % (s.width, s.height, D, win, bil, dtype, sure.mean(), bad, err.mean(), np.percentile(err, 99)))
    assert bad == 0, "%d WTA mismatches on well-separated pixels" % bad
    assert np.array_equal(valid, oracle.valid_mask(s.width, s.height, D, win, bil, s.shift))
    return err


@pytest.mark.parametrize("dtype", [sg.STEREO_F16, sg.STEREO_BF16])
@pytest.mark.parametrize("W,H,D,win,bil", [(201, 75, 20, 5, 7), (65, 37, 12, 3, 1), (130, 70, 33, 3, 3),
                                           (97, 41, 17, 5, 5), (150, 80, 48, 7, 9), (129, 52, 40, 9, 11),
                                           (140, 90, 64, 9, 13), (70, 40, 24, 11, 15)])
def test_tensor_form_matches_oracle(W, H, D, win, bil, dtype):
    """Ragged tiles (widths and heights off the 64 x 36 grid), disparity ranges off the
    16-disparity chunk, every bilateral radius the form takes; bil = 15 runs the FP16 / BF16
    form without tensor cores."""
    s = synth.make_scene(W, H, D, 3000 + W + D, roll=math.radians(3.0), coeffs=(4.0, 0.1, 1e-4),
                         n_potholes=1, warp=True, win=win, bil=bil)
    # the BF16 gap leaves fewer pixels to compare
    min_sure = (0.5 if bil == 1 else 0.7) if dtype == sg.STEREO_F16 else 0.3
    err = check_vs_oracle(s, D, win, bil, 3.0, 10.0, dtype, min_sure=min_sure)
    assert err.mean() < (0.01 if dtype == sg.STEREO_F16 else 0.05)


@pytest.mark.parametrize("W,H,D,win,bil", [(300, 40, 256, 11, 11), (300, 40, 256, 9, 13), (300, 40, 256, 11, 13)])
def test_tensor_form_maximum_disparity(W, H, D, win, bil):
    """D = 256: the widest target strip; with w = 11, k = 13 the form's shared memory is at its
    largest (about 218 KB)."""
    s = synth.make_scene(W, H, D, 4242 + bil, roll=0.0, coeffs=(100.0, 0.0, 0.0), n_potholes=0,
                         warp=False, win=win, bil=bil)
    tw = s.tgt
    disp, wta, valid = run_single(s.ref, tw, s.shift, D, win, bil, 3.0, 10.0, sg.STEREO_F16)
    d_o, ds_o, eb, es = oracle.stereo(s.ref, tw, s.shift, D, win, bil, 3.0, 10.0)
    sure = (es - eb) > GAP[sg.STEREO_F16]
    assert sure.mean() >= 0.2
    assert int(np.count_nonzero(wta[sure] != ds_o[sure])) == 0
    assert np.array_equal(valid, oracle.valid_mask(W, H, D, win, bil, s.shift))


def test_tensor_form_range_kernel_limit():
    """sigma1 > 150 leaves the FP16 form on FP32 weights (the packed -s^2 would be subnormal);
    the result must still meet the FP16 bar."""
    s = synth.make_scene(120, 60, 24, 4300, roll=math.radians(2.0), warp=True, win=7, bil=9)
    check_vs_oracle(s, 24, 7, 9, 3.0, 200.0, sg.STEREO_F16, min_sure=0.5)


@pytest.mark.parametrize("dtype", [sg.STEREO_F16, sg.STEREO_BF16])
def test_tensor_form_best_and_second_cost(dtype):
    """The optional best2 output (normalised E at d* and the smallest E over d != d*) against
    the oracle: within the bound on the normalised E that sets the form's WTA gap (half the gap)."""
    W, H, D = 150, 80, 48
    s = synth.make_scene(W, H, D, 5150, roll=math.radians(2.0), warp=True, win=7, bil=9)
    tw = oracle.warp(s.tgt, s.shift)
    pitch = pitch_of(W)
    disp = torch.empty((H, W), dtype=torch.float32, device="cuda")
    best2 = torch.empty((H, W, 2), dtype=torch.float32, device="cuda")
    with sg.Stereo(W, H, D, win=7, bil=9, sigma0=3.0, sigma1=10.0, pitch=pitch, cost_dtype=dtype) as st:
        st.cost_aggregate_wta(dev_img(s.ref, pitch), dev_img(tw, pitch), dev_f32(s.shift), disp, best2=best2)
        st.check_device_status()
    b2 = best2.cpu().numpy().astype(np.float64)
    _, _, eb, es = oracle.stereo(s.ref, tw, s.shift, D, 7, 9, 3.0, 10.0)
    err = max(np.abs(b2[..., 0] - eb).max(), np.abs(b2[..., 1] - es).max())
    print("\nbest2 dtype=%d: max |E - oracle| = %.2e" % (dtype, err))
    assert err <= GAP[dtype] / 2


def _with_best2(ref, tgtw, shift, D, win, bil, dtype, best2):
    H, W = ref.shape
    pitch = pitch_of(W)
    disp = torch.full((H, W), float("nan"), dtype=torch.float32, device="cuda")
    wta = torch.full((H, W), -7, dtype=torch.int32, device="cuda")
    valid = torch.full((H, W), 9, dtype=torch.uint8, device="cuda")
    b2 = torch.empty((H, W, 2), dtype=torch.float32, device="cuda") if best2 else None
    with sg.Stereo(W, H, D, win=win, bil=bil, sigma0=3.0, sigma1=10.0, pitch=pitch, cost_dtype=dtype) as st:
        st.cost_aggregate_wta(dev_img(ref, pitch), dev_img(tgtw, pitch), dev_f32(shift), disp, wta, valid,
                              best2=b2)
        st.check_device_status()
    return disp.cpu().numpy(), wta.cpu().numpy(), valid.cpu().numpy()


@pytest.mark.parametrize("dtype", [sg.STEREO_F16, sg.STEREO_BF16])
@pytest.mark.parametrize("W,win,bil", [(150, 9, 11), (600, 5, 7), (300, 7, 13)])
def test_tensor_form_best2_keeps_the_wta(dtype, W, win, bil):
    """The 16-bit form's best2 instance carries the smallest E over d != d* beside the running
    WTA; the WTA itself must not move.  On target rows that repeat their column-0 value over runs
    of 1 column to the whole row (long tails of tied costs), both instances must give the same
    disparity, WTA and validity maps bit for bit."""
    H, D = 70, 96
    rng = np.random.default_rng(21 + W + bil)
    ref = synth.texture(rng, H, W)
    tgt = np.empty_like(ref)
    tgt[:, :W - 3] = ref[:, 3:]
    tgt[:, W - 3:] = ref[:, -1:]
    runs = np.minimum(rng.choice([1, 2, 5, 7, 8, 9, 31, 32, 33, 100, 255, 256, 257, 520, W], size=H), W)
    for v in range(H):
        tgt[v, :runs[v]] = tgt[v, 0]
    shift = np.zeros(H, np.float32)
    a = _with_best2(ref, tgt, shift, D, win, bil, dtype, False)
    b = _with_best2(ref, tgt, shift, D, win, bil, dtype, True)
    for x, y in zip(a, b):
        assert np.array_equal(x, y, equal_nan=x.dtype.kind == "f")


def test_best2_needs_a_form_that_carries_it():
    """bil = 15 leaves FP16 storage on the SIMT form, which has no best2 instantiation."""
    W, H, D = 70, 40, 24
    s = synth.make_scene(W, H, D, 5170, warp=True, win=7, bil=15)
    pitch = pitch_of(W)
    disp = torch.empty((H, W), dtype=torch.float32, device="cuda")
    best2 = torch.empty((H, W, 2), dtype=torch.float32, device="cuda")
    with sg.Stereo(W, H, D, win=7, bil=15, sigma0=3.0, sigma1=10.0, pitch=pitch, cost_dtype=sg.STEREO_F16) as st:
        with pytest.raises(sg.StereoError):
            st.cost_aggregate_wta(dev_img(s.ref, pitch), dev_img(s.tgt, pitch), dev_f32(s.shift), disp, best2=best2)
        st.cost_aggregate_wta(dev_img(s.ref, pitch), dev_img(s.tgt, pitch), dev_f32(s.shift), disp)
        st.check_device_status()


def test_tensor_form_paper_parameters():
    """sigma0 = 1.5, sigma1 = 5.5, 11 x 11 neighbourhood (§4.4.1)."""
    s = synth.make_scene(200, 90, 32, 778, roll=math.radians(2.0), n_potholes=2, warp=True, win=9, bil=11)
    check_vs_oracle(s, 32, 9, 11, 1.5, 5.5, sg.STEREO_F16, min_sure=0.7)


@pytest.mark.parametrize("dtype", [sg.STEREO_F16, sg.STEREO_BF16])
def test_tensor_form_degenerate_inputs(dtype):
    rng = np.random.default_rng(15)
    img = synth.texture(rng, 70, 90)
    shift = np.linspace(-4, 6, 70).astype(np.float32)
    si = np.floor(shift.astype(np.float64) + 0.5)
    # identical images: d* = 0 everywhere and the output is the integer row shift
    disp, wta, _ = run_single(img, img, shift, 24, 7, 9, 3.0, 10.0, dtype)
    assert np.all(wta == 0)
    assert np.array_equal(disp, np.broadcast_to(si[:, None], disp.shape).astype(np.float32))
    # one disparity
    tgt = synth.texture(rng, 70, 90)
    disp, wta, _ = run_single(img, tgt, shift, 1, 5, 5, 3.0, 10.0, dtype)
    assert np.all(wta == 0)
    # one pixel
    one = np.array([[17]], np.uint8)
    d1, w1, v1 = run_single(one, one, np.zeros(1, np.float32), 4, 3, 3, 3.0, 10.0, dtype)
    assert w1[0, 0] == 0 and v1[0, 0] == 0


SIZES = [(160, 120, 32), (211, 97, 16), (300, 180, 48), (96, 64, 24), (257, 140, 40)]


def _batch(ss, dtype, wc, dc):
    qs = []
    for s, (W, H, D) in zip(ss, SIZES):
        pitch = pitch_of(W)
        qs.append(dict(ref=dev_img(s.ref, pitch), tgt=dev_img(s.tgt, pitch), shift=dev_f32(s.shift),
                       tgt_warped=torch.zeros((H, pitch), dtype=torch.uint8, device="cuda"),
                       disp=torch.zeros((H, W), dtype=torch.float32, device="cuda"),
                       valid=torch.zeros((H, W), dtype=torch.uint8, device="cuda"),
                       disp_out=torch.zeros((H, W), dtype=torch.float32, device="cuda"),
                       res=torch.zeros(64, dtype=torch.uint8, device="cuda"), max_disp=D))
    with sg.StereoBatch(qs, win=7, bil=9, sigma0=3.0, sigma1=10.0, cost_dtype=dtype, tile_wc=wc, tile_dc=dc) as b:
        b.run()
        torch.cuda.synchronize()
        b.check_device_status()
        cfg = b.config()
    return [q["disp"].cpu().numpy() for q in qs], qs, cfg


@pytest.mark.parametrize("wc,dc", [(32, 32), (16, 16)])
def test_tensor_form_batch_equals_single_and_tracks_simt_form(wc, dc):
    """tile_wc 32: the 32 x 36 form with weights rounded from FP32 (the default single-pair
    context for bil <= 13); tile_wc 16: the 64 x 36 form with 16-bit weights."""
    ss = [synth.make_scene(W, H, D, 700 + i, roll=math.radians(2.0 * (i - 2)), coeffs=(6.0, 0.1, 0.0),
                           n_potholes=1, warp=True, win=7, bil=9) for i, (W, H, D) in enumerate(SIZES)]
    tc, qs, cfg = _batch(ss, sg.STEREO_F16, wc, dc)
    assert cfg["tile_wc"] == wc and cfg["tile_dc"] == dc
    if wc == 32:
        # the persistent batch launch gives what single-pair contexts give (same kernel, same tiles)
        for (W, H, D), q, d in zip(SIZES, qs, tc):
            tw = torch.empty_like(q["tgt"])
            disp = torch.empty((H, W), dtype=torch.float32, device="cuda")
            with sg.Stereo(W, H, D, win=7, bil=9, sigma0=3.0, sigma1=10.0, pitch=q["ref"].shape[1],
                           cost_dtype=sg.STEREO_F16) as st:
                st.warp_target(q["tgt"], q["shift"], tw)
                st.cost_aggregate_wta(q["ref"], tw, q["shift"], disp)
            assert np.array_equal(disp.cpu().numpy(), d)
    # against the FP16 form without tensor cores (FP32 weights): the rounded disparities
    # agree as closely as FP16 and FP32 storage do (a sub-pixel disparity near a half-integer
    # rounds either way), and disparities more than half a pixel apart are rarer still
    simt, _, cfg2 = _batch(ss, sg.STEREO_F16, 2, 12)
    assert cfg2["tile_wc"] == 2
    total = sum(a.size for a in tc)
    diff = sum(int(np.count_nonzero(np.rint(a) != np.rint(b))) for a, b in zip(tc, simt))
    far = sum(int(np.count_nonzero(np.abs(a - b) > 0.5)) for a, b in zip(tc, simt))
    print("\nFP16 tensor-core (tiles %d) vs FP16 SIMT aggregation: rounded disparities differ on %.2e, "
          "by more than 0.5 px on %.2e of pixels" % (wc, diff / total, far / total))
    assert diff / total <= 5e-3
    assert far / total <= 1e-3


def test_tensor_form_rejects_unsupported_parameters():
    ss = [synth.make_scene(W, H, D, 710 + i, warp=True, win=7, bil=9) for i, (W, H, D) in enumerate(SIZES)]
    with pytest.raises(sg.StereoError):
        _batch(ss, sg.STEREO_F32, 16, 16)
