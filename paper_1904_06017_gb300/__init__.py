"""GB300 (sm_103a) road-stereo library: Python binding of the C ABI in include/stereo.h
(and, in ``paper_1904_06017_gb300.diff``, of include/stereo_diff.h).

Thin marshalling only: every function has the name of the C entry point it calls,
turns tensors into device pointers and streams into cudaStream_t handles, and raises
``StereoError`` on a non-zero status.  All arithmetic runs in the CUDA kernels of
``libstereo_gb300.so``; there is no CPU or PyTorch fallback, and importing a function
that needs the library fails loudly when it has not been built.

Hot path (Fan et al., arXiv 1904.06017): stereo_warp_target (§3.1) ->
stereo_cost_aggregate_wta (eq. c, eq. fbs, WTA, eq. subpixel; §3.2) ->
stereo_disparity_transform (§3.3).
"""
from __future__ import annotations

import ctypes
import os

__all__ = [
    "StereoError", "stereo_params", "stereo_dt_result", "load_library", "library_path",
    "stereo_params_default", "stereo_create", "stereo_destroy", "stereo_row_shift_affine",
    "stereo_warp_target", "stereo_cost_aggregate_wta", "stereo_cost_aggregate_wta_ex", "stereo_disparity_transform",
    "stereo_cost_volume", "stereo_aggregate_volume", "stereo_wta_volume",
    "stereo_check_device_status", "stereo_debug_stall_staging", "stereo_profile_enable", "stereo_profile_read",
    "stereo_fp32_peak_probe", "stereo_last_error", "stereo_version", "Stereo",
    "stereo_disparity_transform_noalloc", "stereo_lr_check", "WarpEstimator", "stereo_pair_desc",
    "stereo_batch_params",
    "stereo_batch_params_default", "stereo_batch_create", "stereo_batch_run", "stereo_batch_config",
    "stereo_batch_check_device_status", "stereo_batch_destroy", "StereoBatch",
    "STEREO_OK", "STEREO_EINVAL", "STEREO_ENOMEM", "STEREO_ECUDA", "STEREO_ETIMEOUT",
    "STEREO_ENOCONV", "STEREO_ENOTSUP", "STEREO_F32", "STEREO_F16", "STEREO_BF16",
    "STEREO_FUSED_AUTO", "STEREO_FUSED_SIMT", "STEREO_FUSED_TENSOR",
]

STEREO_OK = 0
STEREO_EINVAL = -1
STEREO_ENOMEM = -2
STEREO_ECUDA = -3
STEREO_ETIMEOUT = -4
STEREO_ENOCONV = -5
STEREO_ENOTSUP = -6
STEREO_F32, STEREO_F16, STEREO_BF16 = 0, 1, 2
STEREO_FUSED_AUTO, STEREO_FUSED_SIMT, STEREO_FUSED_TENSOR = 0, 1, 2

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "_lib", "libstereo_gb300.so")
_lib = None


class StereoError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (status %d)" % (msg, code))
        self.code = code


class stereo_params(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int32), ("height", ctypes.c_int32), ("pitch", ctypes.c_int32),
                ("max_disp", ctypes.c_int32), ("win", ctypes.c_int32), ("bil", ctypes.c_int32),
                ("sigma0", ctypes.c_float), ("sigma1", ctypes.c_float),
                ("cost_dtype", ctypes.c_int32), ("lambda0", ctypes.c_double),
                ("delta_psi", ctypes.c_double), ("max_iters", ctypes.c_int32), ("fused_form", ctypes.c_int32)]


class stereo_dt_result(ctypes.Structure):
    _fields_ = [("psi", ctypes.c_double), ("alpha0", ctypes.c_double), ("alpha1", ctypes.c_double),
                ("e_min", ctypes.c_double), ("iters", ctypes.c_int32), ("status", ctypes.c_int32),
                ("n", ctypes.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class stereo_pair_desc(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int32), ("height", ctypes.c_int32), ("pitch", ctypes.c_int32),
                ("max_disp", ctypes.c_int32), ("ref_dev", ctypes.c_void_p), ("tgt_dev", ctypes.c_void_p),
                ("shift_dev", ctypes.c_void_p), ("tgt_warped_dev", ctypes.c_void_p),
                ("disp_dev", ctypes.c_void_p), ("valid_dev", ctypes.c_void_p),
                ("disp_out_dev", ctypes.c_void_p), ("res_dev", ctypes.c_void_p),
                ("psi_init", ctypes.c_double), ("delta_t", ctypes.c_float), ("wta_dev", ctypes.c_void_p)]


class stereo_batch_params(ctypes.Structure):
    _fields_ = [("win", ctypes.c_int32), ("bil", ctypes.c_int32), ("sigma0", ctypes.c_float),
                ("sigma1", ctypes.c_float), ("cost_dtype", ctypes.c_int32), ("lambda0", ctypes.c_double),
                ("delta_psi", ctypes.c_double), ("max_iters", ctypes.c_int32), ("tile_wc", ctypes.c_int32),
                ("tile_dc", ctypes.c_int32)]


def library_path() -> str:
    return _LIB_PATH


def load_library():
    """Load libstereo_gb300.so (build it first with ``paper_1904_06017_gb300.build``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_LIB_PATH):
        raise ImportError("libstereo_gb300.so is not built (%s); run "
                          "`python -c 'import __graft_entry__ as g; g.build()'`" % _LIB_PATH)
    lib = ctypes.CDLL(_LIB_PATH)
    P, I32, D, F = ctypes.c_void_p, ctypes.c_int32, ctypes.c_double, ctypes.c_float
    sigs = {
        "stereo_params_default": [P],
        "stereo_create": [P, P],
        "stereo_destroy": [P],
        "stereo_row_shift_affine": [I32, D, D, D, P],
        "stereo_warp_target": [P, P, P, P, P],
        "stereo_cost_aggregate_wta": [P, P, P, P, P, P, P, P],
        "stereo_cost_aggregate_wta_ex": [P, P, P, P, P, P, P, P, P],
        "stereo_disparity_transform": [P, P, P, D, F, P, P, P],
        "stereo_cost_volume": [P, P, P, P, P],
        "stereo_aggregate_volume": [P, P, P, P, P],
        "stereo_wta_volume": [P, P, P, P, P, P, P],
        "stereo_check_device_status": [P, P],
        "stereo_debug_stall_staging": [P, I32],
        "stereo_profile_enable": [P, I32],
        "stereo_profile_read": [P, P, P],
        "stereo_fp32_peak_probe": [I32, P, P],
        "stereo_disparity_transform_noalloc": [I32, I32, P, P, D, F, D, D, I32, P, P, P],
        "stereo_batch_params_default": [P],
        "stereo_batch_create": [P, I32, P, P],
        "stereo_batch_run": [P, P],
        "stereo_batch_config": [P, P, P, P, P],
        "stereo_batch_check_device_status": [P],
        "stereo_batch_destroy": [P],
        "stereo_lr_check": [P, P, P, P, P, P, P, F, P],
        "stereo_warp_est_create": [I32, I32, I32, I32, I32, I32, I32, F, F, P],
        "stereo_warp_est_run": [P, P, P, D, P, P, P],
        "stereo_warp_est_coarse": [P, P, P, P, P],
        "stereo_warp_est_destroy": [P],
        "stereo_diff_params_default": [P],
        "stereo_softargmin_workspace_bytes": [P, P],
        "stereo_softargmin_fwd": [P, P, P, P, P, P, ctypes.c_size_t, P],
        "stereo_softargmin_bwd": [P, P, P, P, P, P, P, P, P, ctypes.c_size_t, P],
        "stereo_dt_energy_workspace_bytes": [I32, P],
        "stereo_dt_energy_fwd": [I32, I32, I32, P, P, P, P, P, ctypes.c_size_t, P],
        "stereo_dt_energy_bwd": [I32, I32, I32, P, P, P, P, P, P, P, ctypes.c_size_t, P],
        "stereo_dt_refine_roll": [I32, I32, I32, P, P, D, I32, P, P, ctypes.c_size_t, P],
    }
    for name, args in sigs.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int
    lib.stereo_last_error.restype = ctypes.c_char_p
    lib.stereo_last_error.argtypes = []
    lib.stereo_version.restype = ctypes.c_char_p
    lib.stereo_version.argtypes = []
    _lib = lib
    return lib


def _check(rc):
    if rc != STEREO_OK:
        raise StereoError(rc, load_library().stereo_last_error().decode())
    return rc


def _ptr(x):
    """Device pointer of a CUDA tensor (or a raw integer address); None is NULL."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        if not x.is_cuda:
            raise StereoError(STEREO_EINVAL, "tensor must be on a CUDA device")
        if not x.is_contiguous():
            raise StereoError(STEREO_EINVAL, "tensor must be contiguous")
        return x.data_ptr()
    raise TypeError("expected a CUDA tensor, an integer address or None")


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def stereo_version() -> str:
    return load_library().stereo_version().decode()


def stereo_last_error() -> str:
    return load_library().stereo_last_error().decode()


def stereo_params_default(**overrides) -> stereo_params:
    p = stereo_params()
    _check(load_library().stereo_params_default(ctypes.byref(p)))
    for k, v in overrides.items():
        setattr(p, k, v)
    return p


def stereo_create(params: stereo_params):
    ctx = ctypes.c_void_p()
    _check(load_library().stereo_create(ctypes.byref(params), ctypes.byref(ctx)))
    return ctx


def stereo_destroy(ctx):
    _check(load_library().stereo_destroy(ctx))


def stereo_row_shift_affine(height, c0, c1, delta_p):
    import numpy as np
    out = np.empty(int(height), dtype=np.float32)
    _check(load_library().stereo_row_shift_affine(int(height), float(c0), float(c1), float(delta_p),
                                                  out.ctypes.data_as(ctypes.c_void_p)))
    return out


def stereo_warp_target(ctx, tgt, shift, tgt_warped, stream=None):
    _check(load_library().stereo_warp_target(ctx, _ptr(tgt), _ptr(shift), _ptr(tgt_warped),
                                             _stream(stream)))


def stereo_cost_aggregate_wta(ctx, ref, tgt_warped, shift, disp, wta=None, valid=None, stream=None):
    _check(load_library().stereo_cost_aggregate_wta(ctx, _ptr(ref), _ptr(tgt_warped), _ptr(shift),
                                                    _ptr(disp), _ptr(wta), _ptr(valid),
                                                    _stream(stream)))


def stereo_cost_aggregate_wta_ex(ctx, ref, tgt_warped, shift, disp, wta=None, valid=None, best2=None,
                                 stream=None):
    _check(load_library().stereo_cost_aggregate_wta_ex(ctx, _ptr(ref), _ptr(tgt_warped), _ptr(shift),
                                                       _ptr(disp), _ptr(wta), _ptr(valid), _ptr(best2),
                                                       _stream(stream)))


def stereo_disparity_transform(ctx, disp, mask, psi_init, delta_t, disp_out, res=None, stream=None):
    """res: None -> the call synchronises and returns a stereo_dt_result (host);
    a CUDA uint8 tensor of >= 48 bytes -> the result stays on the device (asynchronous)."""
    lib = load_library()
    if res is None:
        r = stereo_dt_result()
        _check(lib.stereo_disparity_transform(ctx, _ptr(disp), _ptr(mask), float(psi_init),
                                              float(delta_t), _ptr(disp_out), ctypes.byref(r),
                                              _stream(stream)))
        return r
    _check(lib.stereo_disparity_transform(ctx, _ptr(disp), _ptr(mask), float(psi_init), float(delta_t),
                                          _ptr(disp_out), _ptr(res), _stream(stream)))
    return None


def stereo_disparity_transform_noalloc(width, height, disp, mask, psi_init, delta_t, disp_out,
                                       res=None, lambda0=10.0, delta_psi=None, max_iters=100,
                                       stream=None):
    """The disparity transformation for callers that cannot allocate device memory:
    no context, scratch in a fixed device array of the library (see include/stereo.h).
    res: None, or a CUDA uint8 tensor of >= 48 bytes that receives the stereo_dt_result."""
    import math
    if delta_psi is None:
        delta_psi = math.pi / 1.8e6
    _check(load_library().stereo_disparity_transform_noalloc(
        int(width), int(height), _ptr(disp), _ptr(mask), float(psi_init), float(delta_t),
        float(lambda0), float(delta_psi), int(max_iters), _ptr(disp_out), _ptr(res), _stream(stream)))


def stereo_lr_check(ctx, ref, tgt_warped, shift, wta_ref, lr_ok, wta_tgt=None, delta_r=1.0, stream=None):
    """Target view and eq. (lrc) for a pair whose reference view already ran (wta_ref is
    that call's int32 WTA output); lr_ok receives 1 where a pixel is kept."""
    _check(load_library().stereo_lr_check(ctx, _ptr(ref), _ptr(tgt_warped), _ptr(shift), _ptr(wta_ref),
                                          _ptr(wta_tgt), _ptr(lr_ok), float(delta_r), _stream(stream)))


def stereo_cost_volume(ctx, ref, tgt_warped, cost, stream=None):
    _check(load_library().stereo_cost_volume(ctx, _ptr(ref), _ptr(tgt_warped), _ptr(cost),
                                             _stream(stream)))


def stereo_aggregate_volume(ctx, ref, cost, agg, stream=None):
    _check(load_library().stereo_aggregate_volume(ctx, _ptr(ref), _ptr(cost), _ptr(agg),
                                                  _stream(stream)))


def stereo_wta_volume(ctx, agg, shift, disp, wta=None, best2=None, stream=None):
    _check(load_library().stereo_wta_volume(ctx, _ptr(agg), _ptr(shift), _ptr(disp), _ptr(wta),
                                            _ptr(best2), _stream(stream)))


def stereo_check_device_status(ctx, stream=None):
    _check(load_library().stereo_check_device_status(ctx, _stream(stream)))


def stereo_debug_stall_staging(ctx, on=True):
    _check(load_library().stereo_debug_stall_staging(ctx, 1 if on else 0))


def stereo_profile_enable(ctx, on=True):
    _check(load_library().stereo_profile_enable(ctx, 1 if on else 0))


def stereo_profile_read(ctx):
    n = ctypes.c_int32()
    ms = ctypes.c_double()
    _check(load_library().stereo_profile_read(ctx, ctypes.byref(n), ctypes.byref(ms)))
    return int(n.value), float(ms.value)


def stereo_fp32_peak_probe(blocks_per_sm=2):
    gs = ctypes.c_double()
    gp = ctypes.c_double()
    _check(load_library().stereo_fp32_peak_probe(int(blocks_per_sm), ctypes.byref(gs), ctypes.byref(gp)))
    return float(gs.value), float(gp.value)


class Stereo:
    """Owns one context; methods are the C calls with this context bound."""

    def __init__(self, width, height, max_disp, win=9, bil=11, sigma0=1.5, sigma1=5.5,
                 pitch=None, cost_dtype=STEREO_F32, **extra):
        pitch = pitch if pitch is not None else (width + 15) // 16 * 16
        self.params = stereo_params_default(width=width, height=height, pitch=pitch,
                                            max_disp=max_disp, win=win, bil=bil, sigma0=sigma0,
                                            sigma1=sigma1, cost_dtype=cost_dtype, **extra)
        self.ctx = stereo_create(self.params)

    def close(self):
        if self.ctx is not None:
            stereo_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def warp_target(self, tgt, shift, out, stream=None):
        stereo_warp_target(self.ctx, tgt, shift, out, stream)

    def cost_aggregate_wta(self, ref, tgt_warped, shift, disp, wta=None, valid=None, stream=None, best2=None):
        """best2 (float32 [H, W, 2], optional): normalised E at d* and the smallest E over d != d*."""
        if best2 is None:
            stereo_cost_aggregate_wta(self.ctx, ref, tgt_warped, shift, disp, wta, valid, stream)
        else:
            stereo_cost_aggregate_wta_ex(self.ctx, ref, tgt_warped, shift, disp, wta, valid, best2, stream)

    def disparity_transform(self, disp, mask, psi_init, delta_t, out, res=None, stream=None):
        return stereo_disparity_transform(self.ctx, disp, mask, psi_init, delta_t, out, res, stream)

    def lr_check(self, ref, tgt_warped, shift, wta_ref, lr_ok, wta_tgt=None, delta_r=1.0, stream=None):
        stereo_lr_check(self.ctx, ref, tgt_warped, shift, wta_ref, lr_ok, wta_tgt, delta_r, stream)

    def cost_volume(self, ref, tgt_warped, cost, stream=None):
        stereo_cost_volume(self.ctx, ref, tgt_warped, cost, stream)

    def aggregate_volume(self, ref, cost, agg, stream=None):
        stereo_aggregate_volume(self.ctx, ref, cost, agg, stream)

    def wta_volume(self, agg, shift, disp, wta=None, best2=None, stream=None):
        stereo_wta_volume(self.ctx, agg, shift, disp, wta, best2, stream)

    def check_device_status(self, stream=None):
        stereo_check_device_status(self.ctx, stream)


# ---------------------------------------------------------------------------- batches

def stereo_batch_params_default(**overrides) -> stereo_batch_params:
    p = stereo_batch_params()
    _check(load_library().stereo_batch_params_default(ctypes.byref(p)))
    for k, v in overrides.items():
        setattr(p, k, v)
    return p


def stereo_batch_create(params: stereo_batch_params, pairs):
    """pairs: a sequence of stereo_pair_desc (device pointers filled in)."""
    arr = (stereo_pair_desc * len(pairs))(*pairs)
    b = ctypes.c_void_p()
    _check(load_library().stereo_batch_create(ctypes.byref(params), len(pairs), arr, ctypes.byref(b)))
    return b


def stereo_batch_run(batch, stream=None):
    _check(load_library().stereo_batch_run(batch, _stream(stream)))


def stereo_batch_config(batch):
    wc, dc, n, src = (ctypes.c_int32() for _ in range(4))
    _check(load_library().stereo_batch_config(batch, ctypes.byref(wc), ctypes.byref(dc), ctypes.byref(n),
                                              ctypes.byref(src)))
    return {"tile_wc": wc.value, "tile_dc": dc.value, "items": n.value,
            "source": {0: "parameters", 1: "autotune cache", 2: "autotune timing"}[src.value]}


def stereo_batch_check_device_status(batch):
    _check(load_library().stereo_batch_check_device_status(batch))


def stereo_batch_destroy(batch):
    _check(load_library().stereo_batch_destroy(batch))


class StereoBatch:
    """Owns one batch.  ``pairs`` is a list of dicts of CUDA tensors with keys ref, tgt,
    shift, tgt_warped, disp, valid, disp_out, res (uint8 tensor of >= 48 bytes) and ints
    max_disp (and optionally psi_init, delta_t, and wta: an int32 [H][W] tensor that receives
    the integer WTA disparity); images are [H][pitch] uint8 tensors."""

    def __init__(self, pairs, win=9, bil=11, sigma0=1.5, sigma1=5.5, cost_dtype=STEREO_F32,
                 tile_wc=0, tile_dc=0, **extra):
        self.params = stereo_batch_params_default(win=win, bil=bil, sigma0=sigma0, sigma1=sigma1,
                                                  cost_dtype=cost_dtype, tile_wc=tile_wc,
                                                  tile_dc=tile_dc, **extra)
        descs = []
        for q in pairs:
            H, pitch = q["ref"].shape
            W = q["disp"].shape[1]
            descs.append(stereo_pair_desc(W, H, pitch, int(q["max_disp"]), _ptr(q["ref"]), _ptr(q["tgt"]),
                                          _ptr(q["shift"]), _ptr(q["tgt_warped"]), _ptr(q["disp"]),
                                          _ptr(q["valid"]), _ptr(q["disp_out"]), _ptr(q["res"]),
                                          float(q.get("psi_init", 0.0)), float(q.get("delta_t", 0.0)),
                                          _ptr(q.get("wta"))))
        self.pairs = pairs      # keep the tensors alive
        self.batch = stereo_batch_create(self.params, descs)

    def run(self, stream=None):
        stereo_batch_run(self.batch, stream)

    def config(self):
        return stereo_batch_config(self.batch)

    def check_device_status(self):
        stereo_batch_check_device_status(self.batch)

    def close(self):
        if getattr(self, "batch", None) is not None:
            stereo_batch_destroy(self.batch)
            self.batch = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------- self-estimated warp model

class WarpEstimator:
    """stereo_warp_est_*: the row-shift model du(v) = c0 + c1 v (eq. relation_vd) estimated
    from a coarse full-range stereo pass over the unwarped pair."""

    def __init__(self, width, height, max_disp, factor=4, win=5, bil=7, sigma0=3.0, sigma1=10.0, pitch=None):
        pitch = pitch if pitch is not None else (width + 15) // 16 * 16
        e = ctypes.c_void_p()
        _check(load_library().stereo_warp_est_create(int(width), int(height), int(pitch), int(max_disp),
                                                     int(factor), int(win), int(bil), float(sigma0),
                                                     float(sigma1), ctypes.byref(e)))
        self.est = e
        self.height = int(height)

    def run(self, ref, tgt, coef, shift=None, delta_p=0.0, stream=None):
        """coef: CUDA float64 tensor of 3 (c0, c1, n); shift: CUDA float32 [height] or None."""
        _check(load_library().stereo_warp_est_run(self.est, _ptr(ref), _ptr(tgt), float(delta_p), _ptr(coef),
                                                  _ptr(shift), _stream(stream)))

    def coarse(self):
        """(disp, valid) of the last run: copies of the object's coarse map as CUDA tensors."""
        import torch
        d = ctypes.c_void_p()
        v = ctypes.c_void_p()
        wc = ctypes.c_int32()
        hc = ctypes.c_int32()
        _check(load_library().stereo_warp_est_coarse(self.est, ctypes.byref(d), ctypes.byref(v), ctypes.byref(wc),
                                                     ctypes.byref(hc)))
        n = wc.value * hc.value
        disp = torch.as_tensor(_DeviceBuffer(d.value, 4 * n), device="cuda").view(torch.float32)
        valid = torch.as_tensor(_DeviceBuffer(v.value, n), device="cuda")
        return disp.reshape(hc.value, wc.value).clone(), valid.reshape(hc.value, wc.value).clone()

    def close(self):
        if getattr(self, "est", None) is not None:
            _check(load_library().stereo_warp_est_destroy(self.est))
            self.est = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class _DeviceBuffer:
    """A raw device allocation seen as a uint8 tensor (the CUDA array interface)."""

    def __init__(self, ptr, nbytes):
        self.__cuda_array_interface__ = {"shape": (int(nbytes),), "typestr": "|u1", "data": (int(ptr), False),
                                         "version": 2}
