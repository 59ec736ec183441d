"""The disparity transformation entry point that allocates no device memory.

It is meant for callers that cannot allocate (a framework that owns the device heap, a
real-time loop that must not block in cudaMalloc, a plug-in forbidden to allocate after
start-up).  This file is collected last on purpose.  It runs the no-allocation call twice
in a row, through the C ABI, on the same map as the context-based
stereo_disparity_transform, and requires the same roll angle, line and transformed map
within the tolerances of the other parity tests.  It must pass in a fresh process as
well as after the other tests (the call keeps its scratch in a fixed device array that
every call shares)."""
import math

import numpy as np
import pytest
import torch

import paper_1904_06017_gb300 as sg
from gpu_helpers import DT_TOL

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1904_06017_gb300 import build
    build.build()


def _map(H, W, psi, seed):
    rng = np.random.default_rng(seed)
    u = np.arange(W)[None, :]
    v = np.arange(H)[:, None]
    d = 6.0 + 0.11 * (v * math.cos(psi) - u * math.sin(psi)) + 0.4 * rng.standard_normal((H, W))
    d -= 3.0 * np.exp(-((u - 0.3 * W) ** 2 + (v - 0.6 * H) ** 2) / (0.02 * W * H))
    return d.astype(np.float32), (rng.random((H, W)) > 0.1).astype(np.uint8)


@pytest.mark.parametrize("H,W,psi", [(540, 960, 0.06), (1080, 1920, -0.09)])
def test_noalloc_matches_context_call_twice(H, W, psi):
    dmap, mask = _map(H, W, psi, H + W)
    disp = torch.from_numpy(dmap).cuda()
    m = torch.from_numpy(mask).cuda()
    ref_out = torch.empty_like(disp)
    with sg.Stereo(W, H, 16, pitch=(W + 15) // 16 * 16) as st:
        ref = st.disparity_transform(disp, m, 0.0, 1.0, ref_out)
    assert ref.status == sg.STEREO_OK

    delta_psi = st.params.delta_psi
    outs = [torch.full_like(disp, float("nan")) for _ in range(2)]
    ress = [torch.zeros(64, dtype=torch.uint8, device="cuda") for _ in range(2)]
    free_after = []
    for k in range(2):
        sg.stereo_disparity_transform_noalloc(W, H, disp, m, 0.0, 1.0, outs[k], res=ress[k],
                                              lambda0=st.params.lambda0, delta_psi=delta_psi,
                                              max_iters=st.params.max_iters)
        torch.cuda.synchronize()
        free_after.append(torch.cuda.mem_get_info()[0])
    for k in range(2):
        r = sg.stereo_dt_result.from_buffer_copy(ress[k].cpu().numpy().tobytes()[:48])
        assert r.status == sg.STEREO_OK and r.n == ref.n
        assert abs(r.psi - ref.psi) < delta_psi
        assert r.alpha1 == pytest.approx(ref.alpha1, rel=1e-6)
        assert r.alpha0 == pytest.approx(ref.alpha0, rel=1e-6, abs=1e-6)
        assert np.max(np.abs(outs[k].cpu().numpy() - ref_out.cpu().numpy())) < DT_TOL
    # the second call left the device's free memory where the first call left it
    assert free_after[1] == free_after[0]


def test_noalloc_rejects_oversized_maps_and_null_pointers():
    lib = sg.load_library()
    disp = torch.zeros(16, dtype=torch.float32, device="cuda")
    rc = lib.stereo_disparity_transform_noalloc(20000, 4, disp.data_ptr(), None, 0.0, 0.0, 10.0, 1e-6,
                                                100, disp.data_ptr(), None, None)
    assert rc == sg.STEREO_EINVAL and "16384" in sg.stereo_last_error()
    rc = lib.stereo_disparity_transform_noalloc(4, 4, None, None, 0.0, 0.0, 10.0, 1e-6, 100, None, None, None)
    assert rc == sg.STEREO_EINVAL
