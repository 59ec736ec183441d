"""Target view and LR-consistency check (eq. lrc) on the GPU against the oracle.

The target-view WTA must equal the oracle's bit for bit wherever the oracle's best and
second-best target-view costs differ by more than 1e-3 (the reference view's bar); the kept
mask must equal the oracle's eq. (lrc) wherever both WTA decisions it compares are sure."""
import numpy as np
import pytest
import torch

import oracle
import paper_1904_06017_gb300 as sg
import synth
from gpu_helpers import dev_f32, dev_img, pitch_of

pytestmark = pytest.mark.gpu

GAP = 1e-3


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1904_06017_gb300 import build
    build.build()
    oracle.build()


def gpu_lr(ref, tgt, shift, D, win, bil, s0, s1, delta_r=1.0, warp=True):
    H, W = ref.shape
    pitch = pitch_of(W)
    r, t = dev_img(ref, pitch), dev_img(tgt, pitch)
    sh = dev_f32(shift)
    tw = torch.zeros((H, pitch), dtype=torch.uint8, device="cuda")
    disp = torch.empty((H, W), dtype=torch.float32, device="cuda")
    wref = torch.empty((H, W), dtype=torch.int32, device="cuda")
    wtgt = torch.full((H, W), -7, dtype=torch.int32, device="cuda")
    ok = torch.full((H, W), 9, dtype=torch.uint8, device="cuda")
    with sg.Stereo(W, H, D, win=win, bil=bil, sigma0=s0, sigma1=s1, pitch=pitch) as st:
        if warp:
            st.warp_target(t, sh, tw)
        else:
            tw.copy_(t)
        st.cost_aggregate_wta(r, tw, sh, disp, wref)
        st.lr_check(r, tw, sh, wref, ok, wtgt, delta_r)
        st.check_device_status()
    return wref.cpu().numpy(), wtgt.cpu().numpy(), ok.cpu().numpy(), tw[:, :W].cpu().numpy()


def compare(ref, tw, shift, wref, wtgt, ok, D, win, bil, s0, s1, rows=None, delta_r=1.0):
    H, W = ref.shape
    v0, v1 = (0, H) if rows is None else rows
    _, dref, ebr, esr = oracle.stereo(ref, tw, shift, D, win, bil, s0, s1, rows=(v0, v1))
    dtar, ebt, est = oracle.target_view(ref, tw, D, win, bil, s0, s1, rows=(v0, v1))
    sure_t = (est - ebt) > GAP
    assert sure_t.mean() > 0.5
    assert np.array_equal(wtgt[v0:v1][sure_t], dtar[sure_t])
    sure_r = (esr - ebr) > GAP
    okd = oracle.lr_check(dref, dtar, delta_r)
    # pixels whose reference decision and partner's target decision are both sure
    u = np.arange(W)[None, :]
    x = u - dref
    inside = (x >= 0) & (x < W)
    xs = np.clip(x, 0, W - 1)
    both = sure_r & (~inside | np.take_along_axis(sure_t, xs, axis=1))
    assert np.array_equal(ok[v0:v1][both], okd[both])
    return float(okd.mean()), float(both.mean())


def test_small_preset():
    s = synth.make_config_scene("small")
    p = s.params
    wref, wtgt, ok, tw = gpu_lr(s.ref, s.tgt, s.shift, p["D"], p["win"], p["bil"], p["sigma0"], p["sigma1"])
    kept, checked = compare(s.ref, tw, s.shift, wref, wtgt, ok, p["D"], p["win"], p["bil"], p["sigma0"],
                            p["sigma1"])
    print("\nsmall preset: kept %.3f, compared on %.3f of the pixels" % (kept, checked))
    assert set(np.unique(ok)) <= {0, 1}


def test_occluding_block():
    """Background at disparity 3, a foreground block at 9 (z-buffered target): the GPU drops
    the occluded strip exactly where the oracle does."""
    rng = np.random.default_rng(24)
    H, W, D = 60, 120, 16
    ref = synth.texture(rng, H, W)
    disp = np.full(W, 3)
    disp[40:64] = 9
    tgt = np.zeros_like(ref)
    zbuf = np.full(W, -1)
    for u in range(W):
        x = u - disp[u]
        if 0 <= x < W and disp[u] > zbuf[x]:
            zbuf[x] = disp[u]
            tgt[:, x] = ref[:, u]
    for x in range(W):
        if zbuf[x] < 0:
            tgt[:, x] = tgt[:, x - 1]
    sh = np.zeros(H, np.float32)
    wref, wtgt, ok, tw = gpu_lr(ref, tgt, sh, D, 5, 7, 3.0, 10.0, warp=False)
    compare(ref, tw, sh, wref, wtgt, ok, D, 5, 7, 3.0, 10.0)
    assert ok[8:H - 8, 34:40].mean() < 0.5          # most of the hidden background strip


@pytest.mark.parametrize("W,H,D,win,bil", [(77, 45, 20, 5, 7), (40, 33, 1, 3, 3), (130, 70, 48, 9, 11)])
def test_ragged_and_degenerate(W, H, D, win, bil):
    s = synth.make_scene(W, H, D, 4242 + W, roll=0.03, coeffs=(4.0, 0.08, 0.0), n_potholes=1, warp=True,
                         win=win, bil=bil)
    wref, wtgt, ok, tw = gpu_lr(s.ref, s.tgt, s.shift, D, win, bil, 3.0, 10.0)
    compare(s.ref, tw, s.shift, wref, wtgt, ok, D, win, bil, 3.0, 10.0)
    if D == 1:
        assert np.all(wtgt == 0) and np.all(ok == 1)


def test_threshold_is_applied():
    s = synth.make_config_scene("small")
    p = s.params
    res = {}
    for dr in (0.0, 1.0, 4.0):
        wref, wtgt, ok, tw = gpu_lr(s.ref, s.tgt, s.shift, p["D"], p["win"], p["bil"], p["sigma0"],
                                    p["sigma1"], delta_r=dr)
        res[dr] = ok
        assert np.array_equal(ok, oracle.lr_check(wref, wtgt, dr))
    assert res[0.0].sum() <= res[1.0].sum() <= res[4.0].sum()


def test_hd_workload_sampled_rows():
    s = synth.make_config_scene("hd")
    p = s.params
    wref, wtgt, ok, tw = gpu_lr(s.ref, s.tgt, s.shift, p["D"], p["win"], p["bil"], p["sigma0"], p["sigma1"])
    for rows in ((300, 308), (700, 706)):
        compare(s.ref, tw, s.shift, wref, wtgt, ok, p["D"], p["win"], p["bil"], p["sigma0"], p["sigma1"],
                rows=rows)


def test_errors():
    with sg.Stereo(64, 32, 8, win=5, bil=5) as st:
        x = torch.zeros((32, 64), dtype=torch.uint8, device="cuda")
        w = torch.zeros((32, 64), dtype=torch.int32, device="cuda")
        with pytest.raises(sg.StereoError) as e:
            st.lr_check(x, x, torch.zeros(32, device="cuda"), w, torch.zeros((32, 64), dtype=torch.uint8,
                                                                            device="cuda"), delta_r=-1.0)
        assert e.value.code == sg.STEREO_EINVAL
