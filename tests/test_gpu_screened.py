"""The screened FP32 fused form (stereo_params.fused_form = STEREO_FUSED_TENSOR, the FP32 default):
tensor-core screening of the aggregation with a certified error bound, then k_fused's FP32
arithmetic on the certified candidates.  Its outputs must equal the SIMT FP32 form's bit for bit
-- disparity, integer WTA, validity and the best2 values -- on every shape: ragged tiles, search
ranges off the 32-disparity chunk, every window pair the form takes, ties (a flat image, where
every disparity ties and the whole range is refined), and the 1920 x 1080 workloads (D = 128,
k = 11; D = 192, k = 13)."""
import numpy as np
import pytest
import torch

import oracle
import paper_1904_06017_gb300 as sg
import synth
from gpu_helpers import check_disparity, dev_f32, dev_img, pitch_of

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1904_06017_gb300 import build
    build.build()
    oracle.build()


def run(ref, tgtw, shift, D, win, bil, s0, s1, form, best2=False, pitch_extra=0):
    H, W = ref.shape
    pitch = pitch_of(W, pitch_extra)
    disp = torch.full((H, W), float("nan"), dtype=torch.float32, device="cuda")
    wta = torch.full((H, W), -7, dtype=torch.int32, device="cuda")
    valid = torch.full((H, W), 9, dtype=torch.uint8, device="cuda")
    b2 = torch.full((H, W, 2), float("nan"), dtype=torch.float32, device="cuda") if best2 else None
    with sg.Stereo(W, H, D, win=win, bil=bil, sigma0=s0, sigma1=s1, pitch=pitch, fused_form=form) as st:
        r, t, s = dev_img(ref, pitch), dev_img(tgtw, pitch), dev_f32(shift)
        if best2:
            sg.stereo_cost_aggregate_wta_ex(st.ctx, r, t, s, disp, wta, valid, b2)
        else:
            st.cost_aggregate_wta(r, t, s, disp, wta, valid)
        st.check_device_status()
    out = [disp.cpu().numpy(), wta.cpu().numpy(), valid.cpu().numpy()]
    if best2:
        out.append(b2.cpu().numpy())
    return out


def assert_same(a, b):
    for x, y in zip(a, b):
        assert x.dtype == y.dtype and x.shape == y.shape
        same = (x == y) | (np.isnan(x) & np.isnan(y)) if x.dtype.kind == "f" else (x == y)
        assert same.all(), "%d of %d elements differ (first at %s)" % (
            int((~same).sum()), same.size, np.argwhere(~same)[0])


def pair(W, H, shift_px, seed, noise=2.0):
    rng = np.random.default_rng(seed)
    ref = synth.texture(rng, H, W)
    tgt = np.empty_like(ref)
    tgt[:, :W - shift_px] = ref[:, shift_px:]
    tgt[:, W - shift_px:] = ref[:, -1:]
    tgt = np.clip(tgt.astype(np.float64) + rng.normal(0, noise, tgt.shape), 0, 255).round().astype(np.uint8)
    return ref, tgt, np.zeros(H, np.float32)


@pytest.mark.parametrize("W,H,D,win,bil", [
    (70, 41, 20, 7, 9),      # D off the 32-disparity chunk, ragged tiles
    (33, 37, 33, 9, 11),     # one tile wide plus a column, one tile high plus a row
    (100, 75, 64, 9, 11),
    (65, 50, 1, 5, 7),       # D = 1
    (90, 60, 48, 3, 1),      # bil = 1
    (80, 44, 40, 11, 3),     # the largest block
    (64, 72, 17, 5, 5),
    (96, 36, 100, 7, 11),
    (80, 44, 40, 11, 13),    # bil = 13: a window row fills the 16 k-slots, the largest block
    (70, 41, 20, 9, 13),
    (33, 50, 70, 3, 13),
    (300, 40, 256, 11, 13),  # D = 256 with the largest blocks: the layout at its largest
])
def test_screened_equals_simt_bit_for_bit(W, H, D, win, bil):
    ref, tgt, shift = pair(W, H, min(5, D - 1), W * 31 + H)
    a = run(ref, tgt, shift, D, win, bil, 3.0, 10.0, sg.STEREO_FUSED_SIMT)
    b = run(ref, tgt, shift, D, win, bil, 3.0, 10.0, sg.STEREO_FUSED_TENSOR, pitch_extra=16)
    assert_same(a, b)


def test_screened_road_scene_and_oracle():
    """The 320 x 240 road preset: bit-identical to the SIMT form, and the oracle's parity bar."""
    s = synth.make_config_scene("small")
    p = s.params
    tw = oracle.warp(s.tgt, s.shift)
    args = (s.ref, tw, s.shift, p["D"], p["win"], p["bil"], p["sigma0"], p["sigma1"])
    a = run(*args, sg.STEREO_FUSED_SIMT)
    b = run(*args, sg.STEREO_FUSED_AUTO)
    assert_same(a, b)
    d_o, ds_o, eb, es = oracle.stereo(*args)
    check_disparity(b[0], b[1], d_o, ds_o, eb, es)


def test_screened_paper_parameters_and_warp():
    s = synth.make_config_scene("paper")
    p = s.params
    tw = oracle.warp(s.tgt, s.shift)
    args = (s.ref, tw, s.shift, p["D"], p["win"], p["bil"], p["sigma0"], p["sigma1"])
    assert_same(run(*args, sg.STEREO_FUSED_SIMT), run(*args, sg.STEREO_FUSED_TENSOR))


def test_screened_flat_and_identical_images():
    """A flat image makes every cost 1 and every disparity a tie (the whole range refined);
    identical images put the minimum at d = 0 on every pixel."""
    H, W, D = 45, 77, 40
    flat = np.full((H, W), 117, np.uint8)
    shift = np.zeros(H, np.float32)
    assert_same(run(flat, flat, shift, D, 9, 11, 3.0, 10.0, sg.STEREO_FUSED_SIMT),
                run(flat, flat, shift, D, 9, 11, 3.0, 10.0, sg.STEREO_FUSED_TENSOR))
    rng = np.random.default_rng(5)
    img = synth.texture(rng, H, W)
    a = run(img, img, shift, D, 9, 11, 3.0, 10.0, sg.STEREO_FUSED_SIMT)
    b = run(img, img, shift, D, 9, 11, 3.0, 10.0, sg.STEREO_FUSED_TENSOR)
    assert_same(a, b)
    assert (b[1] == 0).all()
    # half flat, half textured: wide ranges next to narrow ones in the same tiles
    half = img.copy()
    half[:, W // 2:] = 60
    assert_same(run(half, half, shift, D, 7, 9, 3.0, 10.0, sg.STEREO_FUSED_SIMT),
                run(half, half, shift, D, 7, 9, 3.0, 10.0, sg.STEREO_FUSED_TENSOR))


@pytest.mark.parametrize("W", [150, 600])
def test_screened_rows_with_flat_left_runs(W):
    """Target rows that repeat their column-0 value over runs of 1 column to the whole row (the
    row table's run lengths, measured 256 columns per step, decide where the refinement clips
    the flat tail): the screened form must still equal the SIMT form bit for bit."""
    H, D = 70, 96
    rng = np.random.default_rng(11 + W)
    ref = synth.texture(rng, H, W)
    tgt = np.empty_like(ref)
    tgt[:, :W - 3] = ref[:, 3:]
    tgt[:, W - 3:] = ref[:, -1:]
    runs = rng.choice([1, 2, 5, 7, 8, 9, 31, 32, 33, 100, 255, 256, 257, 520, W], size=H)
    runs = np.minimum(runs, W)
    for v in range(H):
        tgt[v, :runs[v]] = tgt[v, 0]
    shift = np.zeros(H, np.float32)
    for win, bil in ((9, 11), (5, 7)):
        assert_same(run(ref, tgt, shift, D, win, bil, 3.0, 10.0, sg.STEREO_FUSED_SIMT),
                    run(ref, tgt, shift, D, win, bil, 3.0, 10.0, sg.STEREO_FUSED_TENSOR))


@pytest.mark.parametrize("W,H,D,win,bil", [(90, 50, 24, 7, 9), (64, 40, 40, 9, 11), (70, 45, 36, 9, 13)])
def test_screened_best2_equals_simt(W, H, D, win, bil):
    ref, tgt, shift = pair(W, H, 4, W + H)
    a = run(ref, tgt, shift, D, win, bil, 3.0, 10.0, sg.STEREO_FUSED_SIMT, best2=True)
    b = run(ref, tgt, shift, D, win, bil, 3.0, 10.0, sg.STEREO_FUSED_TENSOR, best2=True)
    assert_same(a, b)


@pytest.mark.parametrize("preset", ["hd", "precision"])
def test_screened_hd_workload_equals_simt(preset):
    """The benchmark workload, 1920 x 1080, D = 128, w = 9, k = 11, and the precision workload,
    1920 x 1080, D = 192, w = 9, k = 13: whole maps."""
    s = synth.make_config_scene(preset)
    p = s.params
    pitch = pitch_of(s.width)
    H, W = s.height, s.width
    outs = []
    for form in (sg.STEREO_FUSED_SIMT, sg.STEREO_FUSED_TENSOR):
        tw = torch.empty((H, pitch), dtype=torch.uint8, device="cuda")
        disp = torch.empty((H, W), dtype=torch.float32, device="cuda")
        wta = torch.empty((H, W), dtype=torch.int32, device="cuda")
        valid = torch.empty((H, W), dtype=torch.uint8, device="cuda")
        with sg.Stereo(W, H, p["D"], win=p["win"], bil=p["bil"], sigma0=p["sigma0"], sigma1=p["sigma1"],
                       pitch=pitch, fused_form=form) as st:
            sh = dev_f32(s.shift)
            st.warp_target(dev_img(s.tgt, pitch), sh, tw)
            st.cost_aggregate_wta(dev_img(s.ref, pitch), tw, sh, disp, wta, valid)
            st.check_device_status()
        outs.append([disp.cpu().numpy(), wta.cpu().numpy(), valid.cpu().numpy()])
    assert_same(outs[0], outs[1])


@pytest.mark.parametrize("W,H,D,win,bil", [(1280, 720, 100, 7, 9), (1000, 610, 45, 11, 13)])
def test_screened_several_tiles_per_cta(W, H, D, win, bil):
    """More tiles than SMs (the persistent kernel takes several in turn, each next tile's images
    staged during the current one's refinement), a search range off the 32-disparity chunk,
    ragged tiles at the right and bottom: still the SIMT form bit for bit."""
    ref, tgt, shift = pair(W, H, 7, W + D)
    a = run(ref, tgt, shift, D, win, bil, 3.0, 10.0, sg.STEREO_FUSED_SIMT)
    b = run(ref, tgt, shift, D, win, bil, 3.0, 10.0, sg.STEREO_FUSED_TENSOR)
    assert_same(a, b)


def test_tensor_form_rejected_where_it_does_not_apply():
    with pytest.raises(sg.StereoError) as e:
        sg.Stereo(64, 48, 16, win=9, bil=15, fused_form=sg.STEREO_FUSED_TENSOR)
    assert e.value.code == sg.STEREO_ENOTSUP
    with pytest.raises(sg.StereoError) as e:
        sg.Stereo(64, 48, 16, fused_form=7)
    assert e.value.code == sg.STEREO_EINVAL
