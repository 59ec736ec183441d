"""The CPU oracle of the road-stereo hot path.  TEST INFRASTRUCTURE ONLY.

Plain FP64 restatements of what the paper defines, used to check the GPU library:
``stereo_oracle.c`` (warp, eq. c, eq. omega_s / eq. fbs, WTA and eq. subpixel) behind
ctypes, and ``dt.py`` (the disparity transformation, §3.3) in numpy.  Only the tests,
the smoke check and the benchmark's CPU-baseline leg import this package; the
library under ``paper_1904_06017_gb300`` never does, and nothing here imports it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

from . import dt, metrics  # noqa: F401

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "stereo_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libstereo_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (-O2, OpenMP, strict IEEE arithmetic)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-fno-fast-math",
                               "-ffp-contract=off", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        I = ctypes.c_int
        Dd = ctypes.c_double
        _lib.oracle_round_shift.argtypes = [Dd]
        _lib.oracle_round_shift.restype = I
        _lib.oracle_set_threads.argtypes = [I]
        _lib.oracle_get_threads.restype = I
        _lib.oracle_warp.argtypes = [I, I, I, P, P, P, I]
        _lib.oracle_cost.argtypes = [P, P, I, I, I, I, I, I, I]
        _lib.oracle_cost.restype = Dd
        _lib.oracle_cost_volume.argtypes = [P, P, I, I, I, I, I, P]
        _lib.oracle_aggregate.argtypes = [P, I, I, I, I, I, Dd, Dd, P, P, P]
        _lib.oracle_weight.argtypes = [P, I, I, I, I, I, Dd, Dd]
        _lib.oracle_weight.restype = Dd
        _lib.oracle_wta_rows.argtypes = [I, I, P, P, I, I, P, P, P, P]
        _lib.oracle_stereo_rows.argtypes = [P, P, P, I, I, I, I, I, I, Dd, Dd, I, I, P, P, P, P]
        _lib.oracle_stereo_rows.restype = I
        _lib.oracle_valid_mask.argtypes = [I, I, I, I, I, P, P]
        _lib.oracle_cost_tar.argtypes = [P, P, I, I, I, I, I, I, I]
        _lib.oracle_cost_tar.restype = Dd
        _lib.oracle_target_view_rows.argtypes = [P, P, I, I, I, I, I, I, Dd, Dd, I, I, P, P, P]
        _lib.oracle_target_view_rows.restype = I
        _lib.oracle_lr_check.argtypes = [I, I, P, P, Dd, P]
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _u8(img):
    return np.ascontiguousarray(img, dtype=np.uint8)


def set_threads(n: int) -> None:
    lib().oracle_set_threads(int(n))


def get_threads() -> int:
    return int(lib().oracle_get_threads())


def round_shift(s: float) -> int:
    return int(lib().oracle_round_shift(float(s)))


def warp(tgt, shift):
    """§3.1 row-shift warp of the target image (uint8 H x W)."""
    tgt = _u8(tgt)
    H, W = tgt.shape
    shift = np.ascontiguousarray(shift, dtype=np.float32)
    out = np.empty_like(tgt)
    lib().oracle_warp(W, H, W, _ptr(tgt), _ptr(shift), _ptr(out), W)
    return out


def cost(ref, tgtw, u, v, d, win):
    """eq. (c) at one pixel and disparity."""
    ref, tgtw = _u8(ref), _u8(tgtw)
    H, W = ref.shape
    return float(lib().oracle_cost(_ptr(ref), _ptr(tgtw), W, H, W, int(u), int(v), int(d),
                                   win // 2))


def cost_volume(ref, tgtw, D, win):
    """eq. (c) for every pixel and d: float64 [H][W][D]."""
    ref, tgtw = _u8(ref), _u8(tgtw)
    H, W = ref.shape
    c = np.empty((H, W, D), dtype=np.float64)
    lib().oracle_cost_volume(_ptr(ref), _ptr(tgtw), W, H, W, int(D), win // 2, _ptr(c))
    return c


def weight(ref, up, vp, uq, vq, sigma0, sigma1):
    """eq. (omega_s) between reference pixels p and q."""
    ref = _u8(ref)
    H, W = ref.shape
    return float(lib().oracle_weight(_ptr(ref), W, up, vp, uq, vq, sigma0, sigma1))


def aggregate(ref, c, bil, sigma0, sigma1, return_wsum=False):
    """eq. (fbs) over a float64 [H][W][D] volume."""
    ref = _u8(ref)
    H, W = ref.shape
    c = np.ascontiguousarray(c, dtype=np.float64)
    D = c.shape[2]
    E = np.empty_like(c)
    ws = np.empty((H, W), dtype=np.float64)
    lib().oracle_aggregate(_ptr(ref), W, H, W, D, bil // 2, float(sigma0), float(sigma1),
                           _ptr(c), _ptr(E), _ptr(ws))
    return (E, ws) if return_wsum else E


def wta(E, shift):
    """WTA + eq. (subpixel) on an aggregated volume [H][W][D].
    Returns (disp, dstar, e_best, e_second)."""
    E = np.ascontiguousarray(E, dtype=np.float64)
    H, W, D = E.shape
    shift = np.ascontiguousarray(shift, dtype=np.float32)
    disp = np.empty((H, W), np.float64)
    dstar = np.empty((H, W), np.int32)
    eb = np.empty((H, W), np.float64)
    es = np.empty((H, W), np.float64)
    lib().oracle_wta_rows(W, D, _ptr(E), _ptr(shift), 0, H, _ptr(disp), _ptr(dstar), _ptr(eb),
                          _ptr(es))
    return disp, dstar, eb, es


def stereo(ref, tgtw, shift, D, win, bil, sigma0, sigma1, rows=None):
    """Cost + aggregation + WTA + sub-pixel for rows [v0, v1) (default: all rows) of a
    pair whose target is already warped.  Returns (disp, dstar, e_best, e_second)."""
    ref, tgtw = _u8(ref), _u8(tgtw)
    H, W = ref.shape
    v0, v1 = (0, H) if rows is None else rows
    shift = np.ascontiguousarray(shift, dtype=np.float32)
    n = v1 - v0
    disp = np.empty((n, W), np.float64)
    dstar = np.empty((n, W), np.int32)
    eb = np.empty((n, W), np.float64)
    es = np.empty((n, W), np.float64)
    rc = lib().oracle_stereo_rows(_ptr(ref), _ptr(tgtw), _ptr(shift), W, H, W, int(D), win // 2,
                                  bil // 2, float(sigma0), float(sigma1), int(v0), int(v1),
                                  _ptr(disp), _ptr(dstar), _ptr(eb), _ptr(es))
    if rc != 0:
        raise MemoryError("oracle_stereo_rows: out of memory")
    return disp, dstar, eb, es


def valid_mask(W, H, D, win, bil, shift):
    """Pixels whose reads behind every disparity stay inside the images (uint8 H x W)."""
    shift = np.ascontiguousarray(shift, dtype=np.float32)
    m = np.empty((H, W), np.uint8)
    lib().oracle_valid_mask(int(W), int(H), int(D), win // 2, bil // 2, _ptr(shift), _ptr(m))
    return m


def cost_tar(ref, tgtw, u, v, d, win):
    """The target view's eq. (c) at target pixel (u, v) and disparity d: the target block
    around (u, v) against the reference block around (u + d, v)."""
    ref, tgtw = _u8(ref), _u8(tgtw)
    H, W = ref.shape
    return float(lib().oracle_cost_tar(_ptr(ref), _ptr(tgtw), W, H, W, int(u), int(v), int(d), win // 2))


def target_view(ref, tgtw, D, win, bil, sigma0, sigma1, rows=None):
    """Target-view WTA (the second cost volume of §3.2.1, the warped target as the
    aggregation guide) for rows [v0, v1).  Returns (dstar, e_best, e_second), each
    [v1 - v0][W], u a column of the warped target."""
    ref, tgtw = _u8(ref), _u8(tgtw)
    H, W = ref.shape
    v0, v1 = (0, H) if rows is None else rows
    n = v1 - v0
    dstar = np.empty((n, W), np.int32)
    eb = np.empty((n, W), np.float64)
    es = np.empty((n, W), np.float64)
    rc = lib().oracle_target_view_rows(_ptr(ref), _ptr(tgtw), W, H, W, int(D), win // 2, bil // 2,
                                       float(sigma0), float(sigma1), int(v0), int(v1), _ptr(dstar),
                                       _ptr(eb), _ptr(es))
    if rc != 0:
        raise MemoryError("oracle_target_view_rows: out of memory")
    return dstar, eb, es


def lr_check(dref, dtar, delta_r=1.0):
    """eq. (lrc) on integer disparity maps of the warped pair: 1 where the pixel is kept."""
    dref = np.ascontiguousarray(dref, dtype=np.int32)
    dtar = np.ascontiguousarray(dtar, dtype=np.int32)
    H, W = dref.shape
    ok = np.empty((H, W), np.uint8)
    lib().oracle_lr_check(W, H, _ptr(dref), _ptr(dtar), float(delta_r), _ptr(ok))
    return ok
