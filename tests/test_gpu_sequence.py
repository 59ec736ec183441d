"""Video warm start and the lambda0 sweep of the roll search (§3.3, §4.4.2).

A sequence of frames of one road whose roll drifts: each frame's roll search starts from the
previous frame's angle (the paper's warm start from frame t-1).  On the GPU every search must
land where the oracle's search lands on the same disparity map (within delta_psi), the warm
start must not take more iterations than a cold start in total, and a sweep of lambda0 must
follow the oracle iteration for iteration (to within one step) and converge for every rate."""
import math

import numpy as np
import pytest
import torch

import oracle
from oracle import dt
import paper_1904_06017_gb300 as sg
import synth
from gpu_helpers import dev_f32, dev_img, pitch_of

pytestmark = pytest.mark.gpu
DELTA_PSI = math.pi / 1.8e6


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1904_06017_gb300 import build
    build.build()
    oracle.build()


@pytest.fixture(scope="module")
def frames():
    """Disparity maps and validity of 6 frames (640 x 360, D = 32) from the GPU path."""
    seq = synth.make_roll_sequence(6, 640, 360, 32, 90210, 1.0, 0.6, n_potholes=2, depth=(2.0, 5.0),
                                   warp=True, win=9, bil=11)
    H, W = 360, 640
    pitch = pitch_of(W)
    out = []
    with sg.Stereo(W, H, 32, win=9, bil=11, sigma0=3.0, sigma1=10.0, pitch=pitch) as st:
        for s in seq:
            tw = torch.empty((H, pitch), dtype=torch.uint8, device="cuda")
            disp = torch.empty((H, W), dtype=torch.float32, device="cuda")
            valid = torch.empty((H, W), dtype=torch.uint8, device="cuda")
            sh = dev_f32(s.shift)
            st.warp_target(dev_img(s.tgt, pitch), sh, tw)
            st.cost_aggregate_wta(dev_img(s.ref, pitch), tw, sh, disp, None, valid)
            out.append((s, disp, valid))
        torch.cuda.synchronize()
    return out


def run_dt(disp, valid, psi_init, lambda0=10.0):
    H, W = disp.shape
    o = torch.empty_like(disp)
    res = torch.zeros(64, dtype=torch.uint8, device="cuda")
    sg.stereo_disparity_transform_noalloc(W, H, disp, valid, psi_init, 0.0, o, res, lambda0=lambda0)
    torch.cuda.synchronize()
    return sg.stereo_dt_result.from_buffer_copy(res.cpu().numpy().tobytes()[:48])


def oracle_dt(disp, valid, psi_init, lambda0=10.0):
    d = disp.cpu().numpy().astype(np.float64)
    m = valid.cpu().numpy().astype(bool)
    v, u = np.nonzero(m)
    return dt.estimate_roll(d[v, u], u.astype(np.float64), v.astype(np.float64), psi_init=psi_init,
                            lambda0=lambda0)


def test_warm_start_follows_the_oracle_and_saves_iterations(frames):
    cold_it = warm_it = 0
    prev = 0.0
    for t, (s, disp, valid) in enumerate(frames):
        cold = run_dt(disp, valid, 0.0)
        warm = run_dt(disp, valid, prev)
        oc = oracle_dt(disp, valid, 0.0)
        ow = oracle_dt(disp, valid, prev)
        for r, o in ((cold, oc), (warm, ow)):
            assert r.status == sg.STEREO_OK and o["status"] == 0
            assert abs(r.psi - o["psi"]) < DELTA_PSI
            assert abs(r.iters - o["iters"]) <= 1
        assert abs(warm.psi - cold.psi) < DELTA_PSI
        print("frame %d: roll %.3f deg, psi %.5f deg, iterations cold %d warm %d" % (
            t, math.degrees(s.roll), math.degrees(warm.psi), cold.iters, warm.iters))
        cold_it += cold.iters
        warm_it += warm.iters
        prev = warm.psi
    assert warm_it <= cold_it


@pytest.mark.parametrize("lambda0", [0.01, 0.1, 1.0, 10.0, 100.0, 1000.0])
def test_lambda0_sweep(frames, lambda0):
    s, disp, valid = frames[3]
    r = run_dt(disp, valid, 0.0, lambda0)
    o = oracle_dt(disp, valid, 0.0, lambda0)
    print("lambda0 %g: iterations %d (oracle %d), psi %.6f" % (lambda0, r.iters, o["iters"], r.psi))
    assert r.status == sg.STEREO_OK and o["status"] == 0
    assert abs(r.psi - o["psi"]) < DELTA_PSI
    assert abs(r.iters - o["iters"]) <= 1
