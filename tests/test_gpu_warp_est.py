"""Self-estimated warp model on the GPU against the oracle (oracle/warp_est.py).

  * the coarse pass: block averages, full-range reference view and geometric validity equal
    the oracle's on the same coarse pair (WTA bit-exact where the oracle's gap exceeds 1e-3,
    sub-pixel within 0.01 px there, validity bit-exact);
  * the FP64 line fit equals the oracle's fit of the GPU's own coarse map (shared map);
  * end to end, c0 and c1 agree with the oracle's estimate;
  * the estimated shift table drives the full pipeline about as accurately as the
    generator's own table."""
import math

import numpy as np
import pytest
import torch

import oracle
from oracle import warp_est
import paper_1904_06017_gb300 as sg
import synth
from gpu_helpers import dev_img, pitch_of

pytestmark = pytest.mark.gpu
WIN, BIL = 5, 7


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1904_06017_gb300 import build
    build.build()
    oracle.build()


def run_est(s, D, F, delta_p=0.0):
    H, W = s.height, s.width
    pitch = pitch_of(W)
    coef = torch.zeros(3, dtype=torch.float64, device="cuda")
    shift = torch.zeros(H, dtype=torch.float32, device="cuda")
    with sg.WarpEstimator(W, H, D, factor=F, win=WIN, bil=BIL, sigma0=3.0, sigma1=10.0, pitch=pitch) as e:
        e.run(dev_img(s.ref, pitch), dev_img(s.tgt, pitch), coef, shift, delta_p)
        torch.cuda.synchronize()
        disp, valid = e.coarse()
    return coef.cpu().numpy(), shift.cpu().numpy(), disp.cpu().numpy(), valid.cpu().numpy()


@pytest.mark.parametrize("F", [2, 4])
def test_coarse_pass_and_fit_match_the_oracle(F):
    s = synth.make_config_scene("large")
    D = int(math.ceil(s.gt_road.max())) + 8
    coef, shift, disp, valid = run_est(s, D, F)
    rc, tc = warp_est.downsample(s.ref, F), warp_est.downsample(s.tgt, F)
    Dc = int(math.ceil(D / F))
    zero = np.zeros(rc.shape[0], np.float32)
    d_o, ds_o, eb, es = oracle.stereo(rc, tc, zero, Dc, WIN, BIL, 3.0, 10.0)
    v_o = oracle.valid_mask(rc.shape[1], rc.shape[0], Dc, WIN, BIL, zero)
    assert np.array_equal(valid, v_o)
    sure = (es - eb) > 1e-3
    assert sure.mean() > 0.8
    assert np.abs(disp.astype(np.float64) - d_o)[sure].max() <= 0.01
    # the fit of the GPU's own coarse map
    c0o, c1o, no = warp_est.fit_rows(disp.astype(np.float64), valid, F)
    assert coef[2] == no
    assert coef[0] == pytest.approx(c0o, rel=1e-9, abs=1e-9) and coef[1] == pytest.approx(c1o, rel=1e-9)
    # end to end against the oracle's own coarse pass
    c0e, c1e, _ = warp_est.estimate_warp(s.ref, s.tgt, D, F, WIN, BIL, 3.0, 10.0)
    print("\\nF=%d: GPU c0 %.5f c1 %.6f, oracle c0 %.5f c1 %.6f" % (F, coef[0], coef[1], c0e, c1e))
    assert abs(coef[0] - c0e) < 0.05 and abs(coef[1] - c1e) < 1e-4
    v = np.arange(s.height)
    assert np.allclose(shift, (coef[0] + coef[1] * v).astype(np.float32), atol=1e-4)


def test_estimated_warp_drives_the_pipeline():
    """The estimated table (with a margin delta_p below the fitted line) in the full pipeline.
    A row shift shears the target (each row of a block moves by its own s_i), so tables of
    different slope give different costs: the estimated table is held to the accuracy the
    generator's own table reaches (median |l - gt| within 0.15 px of it) and to its coverage."""
    s = synth.make_config_scene("large")
    H, W = s.height, s.width
    D = 48
    coef, shift, _, _ = run_est(s, int(math.ceil(s.gt_road.max())) + 8, 4, delta_p=24.0)
    pitch = pitch_of(W)
    outs = []
    for table in (shift, s.shift):
        sh = torch.from_numpy(np.ascontiguousarray(table, dtype=np.float32)).cuda()
        tw = torch.empty((H, pitch), dtype=torch.uint8, device="cuda")
        disp = torch.empty((H, W), dtype=torch.float32, device="cuda")
        valid = torch.empty((H, W), dtype=torch.uint8, device="cuda")
        with sg.Stereo(W, H, D, win=9, bil=11, sigma0=3.0, sigma1=10.0, pitch=pitch) as st:
            st.warp_target(dev_img(s.tgt, pitch), sh, tw)
            st.cost_aggregate_wta(dev_img(s.ref, pitch), tw, sh, disp, None, valid)
        d, vm = disp.cpu().numpy(), valid.cpu().numpy().astype(bool)
        outs.append((float(np.median(np.abs(d - s.gt_disp)[vm])), float(vm.mean())))
    (e1, c1), (e2, c2) = outs
    print("\nmedian |l - gt|: estimated table %.3f px on %.2f of the pixels, generator's %.3f px on %.2f" % (
        e1, c1, e2, c2))
    assert e1 <= e2 + 0.15 and e1 < 0.5
    assert c1 >= 0.95 * c2


def test_factor_one_and_argument_checks():
    s = synth.make_scene(96, 64, 16, 5, roll=0.0, coeffs=(4.0, 0.05, 0.0), n_potholes=0, warp=False)
    coef, shift, disp, valid = run_est(s, 16, 1)
    c0o, c1o, no = warp_est.fit_rows(disp.astype(np.float64), valid, 1)
    assert coef[1] == pytest.approx(c1o, rel=1e-9)
    with pytest.raises(sg.StereoError):
        sg.WarpEstimator(96, 64, 16, factor=9)
    with pytest.raises(sg.StereoError):
        sg.WarpEstimator(4, 64, 16, factor=8)
