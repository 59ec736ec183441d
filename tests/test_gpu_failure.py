"""Failure detection of the fused kernels' bounded staging wait, without any GPU fault.

The test hook stereo_debug_stall_staging makes every CTA arm its staging barrier without
issuing a copy, so the bounded wait runs out (after about a millisecond, with nothing in
flight) and the CTA sets the device status word and returns.  The host must read
STEREO_ETIMEOUT, the word must be cleared by that read, and the same context must give the
oracle's disparities once the hook is off."""
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


@pytest.mark.parametrize("dtype", [sg.STEREO_F32, sg.STEREO_F16])
def test_expired_staging_wait_reports_timeout_and_context_recovers(dtype):
    H, W, D, win, bil = 72, 150, 24, 7, 9
    rng = np.random.default_rng(31)
    ref = synth.texture(rng, H, W)
    tgt = np.empty_like(ref)
    tgt[:, :-4] = ref[:, 4:]
    tgt[:, -4:] = ref[:, -1:]
    shift = np.zeros(H, np.float32)
    pitch = pitch_of(W)
    r, t, s = dev_img(ref, pitch), dev_img(tgt, pitch), dev_f32(shift)
    disp = torch.full((H, W), -1.0, dtype=torch.float32, device="cuda")
    wta = torch.empty((H, W), dtype=torch.int32, device="cuda")
    valid = torch.empty((H, W), dtype=torch.uint8, device="cuda")
    with sg.Stereo(W, H, D, win=win, bil=bil, sigma0=3.0, sigma1=10.0, pitch=pitch, cost_dtype=dtype) as st:
        st.check_device_status()                      # starts clear
        sg.stereo_debug_stall_staging(st.ctx, True)
        st.cost_aggregate_wta(r, t, s, disp, wta, valid)
        with pytest.raises(sg.StereoError) as e:
            st.check_device_status()
        assert e.value.code == sg.STEREO_ETIMEOUT
        st.check_device_status()                      # the read cleared the word
        # no tile was staged, so no output was written
        assert torch.all(disp == -1.0).item()
        sg.stereo_debug_stall_staging(st.ctx, False)
        st.cost_aggregate_wta(r, t, s, disp, wta, valid)
        st.check_device_status()
    d_o, ds_o, eb, es = oracle.stereo(ref, tgt, shift, D, win, bil, 3.0, 10.0)
    if dtype == sg.STEREO_F32:
        check_disparity(disp.cpu().numpy(), wta.cpu().numpy(), d_o, ds_o, eb, es)
    else:
        # the FP16 form's derived WTA gap (2e-2, as in the tensor-form tests)
        check_disparity(disp.cpu().numpy(), wta.cpu().numpy(), d_o, ds_o, eb, es, tol=0.1, gap=2e-2,
                        min_sure=0.5)


def test_stall_hook_rejects_null_context():
    lib = sg.load_library()
    assert lib.stereo_debug_stall_staging(None, 1) == sg.STEREO_EINVAL
