"""Differentiable form of the stereo path, FP64 on the CPU.  TEST INFRASTRUCTURE ONLY.

The paper picks the disparity by winner-take-all (§3.2.2) and differentiates only the
disparity-transformation energy, and only with respect to the roll angle (eq. d_e_min).
To differentiate the whole path the hard argmin is replaced by a soft-argmin over the
aggregated cost:

    c(q,d)  = 1 - NCC of the w x w blocks (eq. c), clamp-to-edge reads, on float images
    E(p,d)  = sum_q w(p,q) c(q,d) / sum_q w(p,q)                    (eq. omega_s, eq. fbs)
    P(p,d)  = softmax_d(-E(p,d) / T),   l(p) = sum_d d P(p,d) + s_i(v)
    L       = sum_p m(p) (l(p) - alpha0 - alpha1 y_p(psi))^2                      (eq. E2)

with y_p(psi) = v cos(psi) - u sin(psi) (eq. y).  Every step is a plain PyTorch float64
operation, so torch.autograd gives the exact adjoint; the tests pin it to central finite
differences.  The target enters through the row-shift warp of §3.1 (a gather whose adjoint
is the matching scatter), so gradients reach the original target image.  With the
linear-interpolation warp (warp_mode 1) a fractional shift s(v) is read between the two
neighbouring target columns and added back unrounded, so gradients reach s(v) as well.

refine_roll() is gradient descent on the roll angle with the line fit eliminated
(alpha = alpha(psi) of eq. alpha3 at every step, so the psi-gradient of eq. E2 is the
gradient of eq. E_min2, eq. d_e_min), each step scaled by the Gauss-Newton curvature of
E_min.  The paper's own search (eq. e_min_gd, eq. adaptive_lambda) lives in oracle.dt.
"""
from __future__ import annotations

import math

import numpy as np
import torch


def round_shift(shift):
    """§3.1: the row shift rounded to the nearest integer, floor(s + 0.5), from float32."""
    s = np.asarray(shift, dtype=np.float32).astype(np.float64)
    return np.floor(s + 0.5).astype(np.int64)


def warp(tgt, shift):
    """§3.1 row-shift warp of a float image: out(u, v) = tgt(clamp(u - s_i(v)), v)."""
    H, W = tgt.shape
    si = torch.from_numpy(round_shift(shift))
    cols = torch.clamp(torch.arange(W)[None, :] - si[:, None], 0, W - 1)
    return torch.gather(tgt, 1, cols)


def warp_linear(tgt, shift):
    """§3.1 with a fractional shift read by linear interpolation: the point u - s(v) of target
    row v, out = (1 - f) tgt(clamp(x0)) + f tgt(clamp(x0 + 1)) with x0 = floor(u - s), f the
    fraction.  `shift` is a float64 tensor (it may require grad) holding float32 values."""
    H, W = tgt.shape
    x = torch.arange(W, dtype=torch.float64)[None, :] - shift[:, None]
    x0 = torch.floor(x.detach())
    f = x - x0
    i0 = torch.clamp(x0.long(), 0, W - 1)
    i1 = torch.clamp(x0.long() + 1, 0, W - 1)
    return (1.0 - f) * torch.gather(tgt, 1, i0) + f * torch.gather(tgt, 1, i1)


def _window_sd(blocks):
    """Population standard deviation of each w x w block and whether the block is flat
    (all its values equal, i.e. sigma = 0 exactly).  A flat block gets sigma = 1 so that its
    unused branch has a finite derivative."""
    flat = blocks.amax(dim=(2, 3)) == blocks.amin(dim=(2, 3))
    c = blocks - blocks.mean(dim=(2, 3), keepdim=True)
    var = (c * c).mean(dim=(2, 3))
    return torch.sqrt(torch.where(flat, torch.ones_like(var), var)), flat, c


def cost_volume(ref, tgtw, D, win):
    """eq. (c) on float images: c[d, v, u], population statistics, clamped reads; a window
    pair with sigma_ref * sigma_tgt = 0 (a block whose values are all equal) gets c = 1
    (NCC := 0)."""
    H, W = ref.shape
    rw = win // 2
    offs = torch.arange(-rw, rw + 1)
    ys = torch.clamp(torch.arange(H)[:, None] + offs[None, :], 0, H - 1)     # [H, w]
    xs = torch.clamp(torch.arange(W)[:, None] + offs[None, :], 0, W - 1)     # [W, w]
    a = ref[ys[:, None, :, None], xs[None, :, None, :]]                      # [H, W, w, w]
    sa, fa, ca = _window_sd(a)
    out = []
    for d in range(D):
        xt = torch.clamp(torch.arange(W)[:, None] - d + offs[None, :], 0, W - 1)
        b = tgtw[ys[:, None, :, None], xt[None, :, None, :]]
        sb, fb, cb = _window_sd(b)
        ncc = (ca * cb).mean(dim=(2, 3)) / (sa * sb)
        out.append(1.0 - torch.where(fa | fb, torch.zeros_like(ncc), ncc))
    return torch.stack(out, 0)


def aggregate(ref, c, bil, sigma0, sigma1):
    """eq. (omega_s), eq. (fbs): E[d, v, u]; neighbours outside the image are left out."""
    D, H, W = c.shape
    rb = bil // 2
    num = torch.zeros_like(c)
    den = torch.zeros((H, W), dtype=c.dtype)
    for dv in range(-rb, rb + 1):
        for du in range(-rb, rb + 1):
            v0, v1 = max(0, -dv), min(H, H - dv)
            u0, u1 = max(0, -du), min(W, W - du)
            if v0 >= v1 or u0 >= u1:
                continue
            ip = ref[v0:v1, u0:u1]
            iq = ref[v0 + dv:v1 + dv, u0 + du:u1 + du]
            w = torch.exp(-(du * du + dv * dv) / sigma0 ** 2 - (ip - iq) ** 2 / sigma1 ** 2)
            wfull = torch.zeros((H, W), dtype=c.dtype)
            wfull[v0:v1, u0:u1] = w
            cq = torch.zeros_like(c)
            cq[:, v0:v1, u0:u1] = c[:, v0 + dv:v1 + dv, u0 + du:u1 + du]
            den = den + wfull
            num = num + wfull[None] * cq
    return num / den[None]


def soft_argmin(E, shift, T):
    """l(p) = sum_d d softmax_d(-E(p,d)/T) + s_i(v)."""
    D = E.shape[0]
    P = torch.softmax(-E / T, dim=0)
    d = torch.arange(D, dtype=E.dtype)[:, None, None]
    si = torch.from_numpy(round_shift(shift)).to(E.dtype)
    return (P * d).sum(0) + si[:, None]


def dt_energy(l, mask, psi, alpha0, alpha1):
    """eq. (E2) over the masked pixels, raw pixel coordinates (u column, v row)."""
    H, W = l.shape
    u = torch.arange(W, dtype=l.dtype)[None, :]
    v = torch.arange(H, dtype=l.dtype)[:, None]
    y = v * torch.cos(psi) - u * torch.sin(psi)
    r = (l - alpha0 - alpha1 * y) * mask
    return (r * r).sum()


def soft_argmin_linear(E, shift, T):
    """l(p) = sum_d d softmax_d(-E(p,d)/T) + s(v) with the fractional shift added back."""
    D = E.shape[0]
    P = torch.softmax(-E / T, dim=0)
    d = torch.arange(D, dtype=E.dtype)[:, None, None]
    return (P * d).sum(0) + shift[:, None]


def disparity(ref, tgt, shift, D, win, bil, sigma0, sigma1, T, warp_mode=0):
    """Warp, cost, aggregation and soft-argmin: l [H, W].  warp_mode 0: the rounded shift of
    §3.1 (`shift` a float32 array); 1: the linear-interpolation warp (`shift` a float64 tensor)."""
    if warp_mode == 1:
        c = cost_volume(ref, warp_linear(tgt, shift), D, win)
        return soft_argmin_linear(aggregate(ref, c, bil, sigma0, sigma1), shift, T)
    c = cost_volume(ref, warp(tgt, shift), D, win)
    return soft_argmin(aggregate(ref, c, bil, sigma0, sigma1), shift, T)


def _t(x, grad=False):
    return torch.tensor(np.asarray(x, np.float64), dtype=torch.float64, requires_grad=grad)


def disparity_value(ref, tgt, shift, D, win, bil, sigma0, sigma1, T):
    """l as a float64 numpy array."""
    with torch.no_grad():
        return disparity(_t(ref), _t(tgt), shift, D, win, bil, sigma0, sigma1, T).numpy()


def disparity_vjp(ref, tgt, shift, D, win, bil, sigma0, sigma1, T, grad_l):
    """(l, dS/dref, dS/dtgt) for S = sum_p grad_l(p) l(p): the vector-Jacobian product."""
    r, t = _t(ref, True), _t(tgt, True)
    l = disparity(r, t, shift, D, win, bil, sigma0, sigma1, T)
    (l * _t(grad_l)).sum().backward()
    return l.detach().numpy(), r.grad.numpy(), t.grad.numpy()


def _shift_t(shift, grad=False):
    return torch.tensor(np.asarray(shift, np.float32).astype(np.float64), dtype=torch.float64,
                        requires_grad=grad)


def disparity_linear_value(ref, tgt, shift, D, win, bil, sigma0, sigma1, T):
    """l with the linear-interpolation warp, as a float64 numpy array."""
    with torch.no_grad():
        return disparity(_t(ref), _t(tgt), _shift_t(shift), D, win, bil, sigma0, sigma1, T, 1).numpy()


def disparity_linear_vjp(ref, tgt, shift, D, win, bil, sigma0, sigma1, T, grad_l):
    """(l, dS/dref, dS/dtgt, dS/dshift) with the linear-interpolation warp."""
    r, t, s = _t(ref, True), _t(tgt, True), _shift_t(shift, True)
    l = disparity(r, t, s, D, win, bil, sigma0, sigma1, T, 1)
    (l * _t(grad_l)).sum().backward()
    return l.detach().numpy(), r.grad.numpy(), t.grad.numpy(), s.grad.numpy()


def energy_value(l, mask, psi, alpha0, alpha1):
    with torch.no_grad():
        return float(dt_energy(_t(l), _t(mask), _t(psi), _t(alpha0), _t(alpha1)))


def energy_grads(l, mask, psi, alpha0, alpha1):
    """(L, dL/dl, dL/dpsi, dL/dalpha0, dL/dalpha1) of eq. (E2)."""
    lt, p, a0, a1 = _t(l, True), _t(psi, True), _t(alpha0, True), _t(alpha1, True)
    L = dt_energy(lt, _t(mask), p, a0, a1)
    L.backward()
    return float(L.detach()), lt.grad.numpy(), float(p.grad), float(a0.grad), float(a1.grad)


def loss_and_grads(ref, tgt, shift, D, win, bil, sigma0, sigma1, T, mask, psi, alpha0, alpha1):
    """The whole differentiable path: (L, l, dL/dref, dL/dtgt, dL/dpsi, dL/dalpha0, dL/dalpha1)."""
    r, t = _t(ref, True), _t(tgt, True)
    p, a0, a1 = _t(psi, True), _t(alpha0, True), _t(alpha1, True)
    l = disparity(r, t, shift, D, win, bil, sigma0, sigma1, T)
    L = dt_energy(l, _t(mask), p, a0, a1)
    L.backward()
    return (float(L.detach()), l.detach().numpy(), r.grad.numpy(), t.grad.numpy(), float(p.grad),
            float(a0.grad), float(a1.grad))


def _wrap(psi):
    """Into (-pi/2, pi/2]: E_t,min has period pi (eq. e_min_min)."""
    psi = math.fmod(psi, math.pi)
    if psi > math.pi / 2:
        psi -= math.pi
    elif psi <= -math.pi / 2:
        psi += math.pi
    return psi


def alpha_fit(l, mask, psi):
    """eq. (alpha3) over the masked pixels: the least-squares (alpha0, alpha1) at psi."""
    H, W = l.shape
    v, u = np.nonzero(np.asarray(mask) != 0)
    y = v * math.cos(psi) - u * math.sin(psi)
    Y = np.stack([np.ones_like(y), y], axis=1)
    return np.linalg.lstsq(Y, np.asarray(l, np.float64)[v, u], rcond=None)[0]


def refine_roll(l, mask, psi0=0.0, steps=50):
    """Gradient descent on psi with alpha = alpha(psi) re-fitted at every step.  The step is
    g / H: g = dL/dpsi at (psi, alpha(psi)) taken by autograd, H = 2 alpha1^2 |x~|^2 where
    x~ is x(psi) = u cos(psi) + v sin(psi) with its projection on [1, y(psi)] removed (the
    Gauss-Newton curvature of E_min).  Returns the trajectory [(psi, alpha0, alpha1, g, L)]
    of steps + 1 entries."""
    v, u = np.nonzero(np.asarray(mask) != 0)
    traj = []
    psi = float(psi0)
    for k in range(steps + 1):
        a0, a1 = alpha_fit(l, mask, psi)
        L, _, g, _, _ = energy_grads(l, mask, psi, a0, a1)
        traj.append((psi, float(a0), float(a1), g, L))
        if k == steps:
            break
        x = u * math.cos(psi) + v * math.sin(psi)
        y = v * math.cos(psi) - u * math.sin(psi)
        Y = np.stack([np.ones_like(y), y], axis=1)
        xt = x - Y @ np.linalg.lstsq(Y, x, rcond=None)[0]
        H = 2.0 * a1 * a1 * float(xt @ xt)
        if not H > 0:
            break
        psi = _wrap(psi - g / H)
    return traj
