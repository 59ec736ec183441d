"""Helpers shared by the GPU tests: device images with a row pitch, and the
parity criteria of the hot path (applied to oracle and library outputs)."""
import numpy as np
import torch

# Tolerances of the parity tests.
WTA_GAP = 1e-3        # d* must match wherever the oracle's best and second-best E differ by more
SUBPIX_TOL = 0.01     # px, sub-pixel disparity
COST_REL = 1e-4       # FP32 cost / aggregated cost, relative (floor 1e-2 on the magnitude)
DT_TOL = 1e-3         # px, transformed disparity


def pitch_of(width, extra=0):
    return (width + 15) // 16 * 16 + extra


def dev_img(a, pitch=None, fill=0):
    a = np.ascontiguousarray(a, dtype=np.uint8)
    H, W = a.shape
    pitch = pitch_of(W) if pitch is None else pitch
    t = torch.full((H, pitch), fill, dtype=torch.uint8, device="cuda")
    t[:, :W] = torch.from_numpy(a).cuda()
    return t


def dev_f32(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def check_disparity(disp, wta, d_o, ds_o, eb, es, tol=SUBPIX_TOL, gap=WTA_GAP, min_sure=0.9):
    """d* bit-exact where the oracle's gap exceeds `gap`; |disp - oracle| <= tol there."""
    sure = (es - eb) > gap
    assert sure.mean() >= min_sure, "too few well-separated pixels (%.3f)" % sure.mean()
    if wta is not None:
        bad = np.count_nonzero(wta[sure] != ds_o[sure])
        assert bad == 0, "%d WTA mismatches on well-separated pixels" % bad
    err = np.abs(disp.astype(np.float64) - d_o)[sure]
    assert err.max() <= tol, "sub-pixel error %g > %g" % (err.max(), tol)
    return sure


def check_rel(gpu, ref, rel=COST_REL, floor=1e-2):
    gpu = np.asarray(gpu, np.float64)
    ref = np.asarray(ref, np.float64)
    bound = rel * np.maximum(np.abs(ref), floor)
    excess = np.abs(gpu - ref) - bound
    assert np.all(excess <= 0), "max relative error %g" % np.max(np.abs(gpu - ref) / np.maximum(np.abs(ref), floor))
