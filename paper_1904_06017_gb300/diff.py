"""Differentiable stereo path: binding of include/stereo_diff.h and torch.autograd Functions.

The paper picks the disparity by winner-take-all (§3.2.2) and differentiates only the
disparity-transformation energy in the roll angle (eq. d_e_min).  Here the hard argmin is
replaced by a soft-argmin at temperature T over the bilateral-aggregated cost of eq. (c)
and eq. (fbs), and the energy of eq. (E2) is differentiable in the disparity map, the roll
angle and the line coefficients:

    l = SoftArgmin.apply(ref, tgt, shift, D, win, bil, sigma0, sigma1, T)    # [B, H, W]
    L = DTEnergy.apply(l, theta, mask)                                       # [B]; theta [B, 3]
    L.sum().backward()            # gradients into ref, tgt (float32) and theta (float64)

With warp_mode = STEREO_WARP_LINEAR the row shifts are read by interpolation and the shift
tensor receives a gradient as well, so warp coefficients from which torch computes s(v)
(eq. relation_vd: s(v) = c0 + c1 v - delta_p) are refined by the same backward pass.

Both Functions marshal tensors into the C calls; the forward and backward arithmetic is
the library's CUDA kernels, and there is no CPU path.  ``refine_roll`` runs the library's
gradient refinement of the roll angle.
"""
from __future__ import annotations

import ctypes

import torch

from . import STEREO_EINVAL, StereoError, _check, _ptr, _stream, load_library

__all__ = ["STEREO_WARP_ROUND", "STEREO_WARP_LINEAR", "stereo_diff_params", "stereo_diff_params_default",
           "stereo_softargmin_workspace_bytes", "stereo_softargmin_fwd", "stereo_softargmin_bwd", "stereo_dt_energy_workspace_bytes",
           "stereo_dt_energy_fwd", "stereo_dt_energy_bwd", "stereo_dt_refine_roll", "SoftArgmin",
           "DTEnergy", "soft_argmin_disparity", "dt_energy", "refine_roll"]


class stereo_diff_params(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int32), ("height", ctypes.c_int32), ("batch", ctypes.c_int32),
                ("max_disp", ctypes.c_int32), ("win", ctypes.c_int32), ("bil", ctypes.c_int32),
                ("sigma0", ctypes.c_float), ("sigma1", ctypes.c_float), ("temperature", ctypes.c_float),
                ("warp_mode", ctypes.c_int32)]


STEREO_WARP_ROUND, STEREO_WARP_LINEAR = 0, 1


def stereo_diff_params_default(**overrides) -> stereo_diff_params:
    p = stereo_diff_params()
    _check(load_library().stereo_diff_params_default(ctypes.byref(p)))
    for k, v in overrides.items():
        setattr(p, k, v)
    return p


def stereo_softargmin_workspace_bytes(params: stereo_diff_params) -> int:
    n = ctypes.c_size_t()
    _check(load_library().stereo_softargmin_workspace_bytes(ctypes.byref(params), ctypes.byref(n)))
    return int(n.value)


def _nbytes(t):
    return t.numel() * t.element_size()


def stereo_softargmin_fwd(params, ref, tgt, shift, disp, workspace, stream=None):
    _check(load_library().stereo_softargmin_fwd(ctypes.byref(params), _ptr(ref), _ptr(tgt), _ptr(shift),
                                                _ptr(disp), _ptr(workspace), _nbytes(workspace),
                                                _stream(stream)))


def stereo_softargmin_bwd(params, ref, tgt, shift, grad_disp, grad_ref, grad_tgt, workspace, stream=None,
                          grad_shift=None):
    _check(load_library().stereo_softargmin_bwd(ctypes.byref(params), _ptr(ref), _ptr(tgt), _ptr(shift),
                                                _ptr(grad_disp), _ptr(grad_ref), _ptr(grad_tgt),
                                                _ptr(grad_shift), _ptr(workspace), _nbytes(workspace),
                                                _stream(stream)))


def stereo_dt_energy_workspace_bytes(batch: int) -> int:
    n = ctypes.c_size_t()
    _check(load_library().stereo_dt_energy_workspace_bytes(int(batch), ctypes.byref(n)))
    return int(n.value)


def _bhw(disp):
    if disp.dim() != 3:
        raise StereoError(STEREO_EINVAL, "disparity must be [batch, height, width]")
    B, H, W = disp.shape
    return int(W), int(H), int(B)


def stereo_dt_energy_fwd(disp, mask, theta, energy, workspace, stream=None):
    W, H, B = _bhw(disp)
    _check(load_library().stereo_dt_energy_fwd(W, H, B, _ptr(disp), _ptr(mask), _ptr(theta), _ptr(energy),
                                               _ptr(workspace), _nbytes(workspace), _stream(stream)))


def stereo_dt_energy_bwd(disp, mask, theta, grad_energy, grad_disp, grad_theta, workspace, stream=None):
    W, H, B = _bhw(disp)
    _check(load_library().stereo_dt_energy_bwd(W, H, B, _ptr(disp), _ptr(mask), _ptr(theta),
                                               _ptr(grad_energy), _ptr(grad_disp), _ptr(grad_theta),
                                               _ptr(workspace), _nbytes(workspace), _stream(stream)))


def stereo_dt_refine_roll(disp, mask, psi_init, steps, traj, workspace, stream=None):
    W, H, B = _bhw(disp)
    _check(load_library().stereo_dt_refine_roll(W, H, B, _ptr(disp), _ptr(mask), float(psi_init), int(steps),
                                                _ptr(traj), _ptr(workspace), _nbytes(workspace),
                                                _stream(stream)))


def _batched(x, dims):
    """Add the batch dimension to an unbatched tensor."""
    return x.unsqueeze(0) if x.dim() == dims - 1 else x


def _f32(x):
    if not x.is_cuda:
        raise StereoError(STEREO_EINVAL, "tensor must be on a CUDA device")
    return x.detach().to(torch.float32).contiguous()


class SoftArgmin(torch.autograd.Function):
    """l = sum_d d softmax_d(-E(p,d)/T) + s_i(v) over float32 images [B, H, W] with row-shift
    tables [B, H]; differentiable in ref and tgt, and with warp_mode = STEREO_WARP_LINEAR
    (fractional shifts read by interpolation, s(v) added back unrounded) in the shifts too."""

    @staticmethod
    def forward(ctx, ref, tgt, shift, max_disp, win=9, bil=11, sigma0=1.5, sigma1=5.5, temperature=0.1,
                warp_mode=STEREO_WARP_ROUND):
        r, t, s = _f32(ref), _f32(tgt), _f32(shift)
        B, H, W = r.shape
        p = stereo_diff_params_default(width=W, height=H, batch=B, max_disp=int(max_disp), win=int(win),
                                       bil=int(bil), sigma0=float(sigma0), sigma1=float(sigma1),
                                       temperature=float(temperature), warp_mode=int(warp_mode))
        ws = torch.empty(stereo_softargmin_workspace_bytes(p), dtype=torch.uint8, device=r.device)
        disp = torch.empty((B, H, W), dtype=torch.float32, device=r.device)
        stereo_softargmin_fwd(p, r, t, s, disp, ws)
        ctx.params = p
        ctx.save_for_backward(r, t, s, ws)
        return disp

    @staticmethod
    def backward(ctx, grad_disp):
        r, t, s, ws = ctx.saved_tensors
        need_r, need_t, need_s = ctx.needs_input_grad[0], ctx.needs_input_grad[1], ctx.needs_input_grad[2]
        gr = torch.empty_like(r) if need_r else None
        gt = torch.empty_like(t) if need_t else None
        gs = torch.empty_like(s) if need_s else None
        if need_r or need_t or need_s:
            stereo_softargmin_bwd(ctx.params, r, t, s, grad_disp.to(torch.float32).contiguous(), gr, gt, ws,
                                  grad_shift=gs)
        return gr, gt, gs, None, None, None, None, None, None, None


class DTEnergy(torch.autograd.Function):
    """eq. (E2) per pair for disparities [B, H, W] and theta = (psi, alpha0, alpha1) [B, 3]
    (float64); mask uint8 [B, H, W] or None.  Returns float64 [B]."""

    @staticmethod
    def forward(ctx, disp, theta, mask=None):
        d = _f32(disp)
        th = theta.detach().to(torch.float64).contiguous()
        m = None if mask is None else mask.to(torch.uint8).contiguous()
        ws = torch.empty(stereo_dt_energy_workspace_bytes(d.shape[0]), dtype=torch.uint8, device=d.device)
        e = torch.empty(d.shape[0], dtype=torch.float64, device=d.device)
        stereo_dt_energy_fwd(d, m, th, e, ws)
        ctx.save_for_backward(d, th, m if m is not None else torch.empty(0, device=d.device), ws)
        ctx.has_mask = m is not None
        return e

    @staticmethod
    def backward(ctx, grad_e):
        d, th, m, ws = ctx.saved_tensors
        gd = torch.empty_like(d) if ctx.needs_input_grad[0] else None
        gth = torch.empty_like(th) if ctx.needs_input_grad[1] else None
        stereo_dt_energy_bwd(d, m if ctx.has_mask else None, th, grad_e.to(torch.float64).contiguous(), gd,
                             gth, ws)
        return gd, gth, None


def soft_argmin_disparity(ref, tgt, shift, max_disp, win=9, bil=11, sigma0=1.5, sigma1=5.5,
                          temperature=0.1, warp_mode=STEREO_WARP_ROUND):
    """SoftArgmin on [H, W] or [B, H, W] images (the output has the input's batch form)."""
    unbatched = ref.dim() == 2
    out = SoftArgmin.apply(_batched(ref, 3), _batched(tgt, 3), _batched(shift, 2), max_disp, win, bil,
                           sigma0, sigma1, temperature, warp_mode)
    return out[0] if unbatched else out


def dt_energy(disp, theta, mask=None):
    """DTEnergy on [H, W] or [B, H, W] maps; theta [3] or [B, 3]."""
    unbatched = disp.dim() == 2
    e = DTEnergy.apply(_batched(disp, 3), _batched(theta, 2), None if mask is None else _batched(mask, 3))
    return e[0] if unbatched else e


def refine_roll(disp, mask=None, psi_init=0.0, steps=50):
    """Roll refinement by gradient on the device (stereo_dt_refine_roll).  Returns the
    trajectory [B, steps + 1, 5] of (psi, alpha0, alpha1, dL/dpsi, L) as float64."""
    d = _f32(_batched(disp, 3))
    m = None if mask is None else _batched(mask, 3).to(torch.uint8).contiguous()
    ws = torch.empty(stereo_dt_energy_workspace_bytes(d.shape[0]), dtype=torch.uint8, device=d.device)
    traj = torch.empty((d.shape[0], int(steps) + 1, 5), dtype=torch.float64, device=d.device)
    stereo_dt_refine_roll(d, m, psi_init, steps, traj, ws)
    return traj
