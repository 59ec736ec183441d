"""Disparity-transformation oracle (§3.3), FP64 numpy.  TEST INFRASTRUCTURE ONLY.

Follows the paper's equations in their printed order with explicit matrices:
eq. (x), eq. (y) rotate the pixel coordinates; eq. (alpha3) / eq. (J) give the
least-squares line alpha(psi) = J(psi) d with J = (Y^T Y)^-1 Y^T; eq. (E_min2) gives
the minimum energy; eq. (d_e_min) / eq. (M) give its derivative
-2 d^T (I - Y J) dY J d; eq. (e_min_gd) with the adaptive rate of eq. (adaptive_lambda)
searches psi; eq. (disparity_transformation) maps every disparity.
u and v are the raw 0-based column and row of each pixel, as in the paper.

Readings where the paper is silent (the GPU library takes the same ones):
  * the rate lambda is applied to the energy divided by the number of pixels n
    (lambda0 = 10 of §4.4.2 then means the same thing for any map size);
  * "backtracking line search" (§3.3): a step that raises the energy is halved
    until it does not (at most 60 times); the next rate comes from
    eq. (adaptive_lambda) and is kept only when positive and finite;
  * psi is wrapped into (-pi/2, pi/2] after every step (eq. e_min_min);
  * the search stops when |psi_k+1 - psi_k| < delta_psi, or when the derivative
    vanishes, or after max_iters steps (status NOT_CONVERGED).
"""
from __future__ import annotations

import math

import numpy as np

STATUS_OK = 0
STATUS_NOT_CONVERGED = -5


def rotate(u, v, psi):
    """eq. (x), eq. (y): coordinates rotated by the roll angle psi."""
    x = u * math.cos(psi) + v * math.sin(psi)
    y = v * math.cos(psi) - u * math.sin(psi)
    return x, y


def _design(u, v, psi):
    _, y = rotate(u, v, psi)
    return np.stack([np.ones_like(y), y], axis=1)          # Y(psi) = [1, y(psi)]


def line_fit(d, u, v, psi):
    """eq. (alpha3), eq. (J): alpha(psi) = J(psi) d with J = (Y^T Y)^-1 Y^T."""
    Y = _design(u, v, psi)
    J = np.linalg.solve(Y.T @ Y, Y.T)
    return J @ d


def energy_min(d, u, v, psi):
    """eq. (E_min2): E_t,min(psi) = d^T d - d^T Y (Y^T Y)^-1 Y^T d."""
    Y = _design(u, v, psi)
    return float(d @ d - d @ (Y @ np.linalg.solve(Y.T @ Y, Y.T @ d)))


def energy(d, u, v, psi, alpha):
    """eq. (E2): E_t(psi) = ||d - Y(psi) alpha||^2 for a given alpha."""
    r = d - _design(u, v, psi) @ np.asarray(alpha, dtype=np.float64)
    return float(r @ r)


def grad_energy_min(d, u, v, psi):
    """eq. (d_e_min), eq. (M): -2 d^T W(psi) d, W = (I - Y J) dY J, where
    dY = dY/dpsi = [0, -x(psi)] (the derivative of eq. (y))."""
    x, _ = rotate(u, v, psi)
    Y = _design(u, v, psi)
    J = np.linalg.solve(Y.T @ Y, Y.T)
    dY = np.stack([np.zeros_like(x), -x], axis=1)
    t = dY @ (J @ d)                  # dY J d
    wd = t - Y @ (J @ t)              # (I - Y J) dY J d
    return float(-2.0 * (d @ wd))


def wrap(psi: float) -> float:
    """Map an angle into (-pi/2, pi/2] (eq. e_min_min); E_t,min has period pi."""
    psi = math.fmod(psi, math.pi)
    if psi > 0.5 * math.pi:
        psi -= math.pi
    elif psi <= -0.5 * math.pi:
        psi += math.pi
    return psi


def estimate_roll(d, u, v, psi_init=0.0, lambda0=10.0, delta_psi=math.pi / 1.8e6,
                  max_iters=100, max_halvings=60):
    """eq. (e_min_gd) with eq. (adaptive_lambda): gradient descent on E_t,min(psi)."""
    d = np.asarray(d, dtype=np.float64)
    u = np.asarray(u, dtype=np.float64)
    v = np.asarray(v, dtype=np.float64)
    n = float(d.size)

    def ebar(p):
        return energy_min(d, u, v, p) / n

    def gbar(p):
        return grad_energy_min(d, u, v, p) / n

    psi = wrap(float(psi_init))
    lam = float(lambda0)
    e_cur = ebar(psi)
    g = gbar(psi)
    status = STATUS_NOT_CONVERGED
    it = 0
    for it in range(1, max_iters + 1):
        step = lam * g
        psi_new = wrap(psi - step)
        e_new = ebar(psi_new)
        h = 0
        while e_new > e_cur and h < max_halvings:      # backtracking
            lam *= 0.5
            step = lam * g
            psi_new = wrap(psi - step)
            e_new = ebar(psi_new)
            h += 1
        g_new = gbar(psi_new)
        done = abs(step) < delta_psi or g_new == 0.0 or g_new == g
        lam_next = lam * g / (g - g_new) if g != g_new else lam   # eq. (adaptive_lambda)
        psi, e_cur, g = psi_new, e_new, g_new
        if done:
            status = STATUS_OK
            break
        if math.isfinite(lam_next) and lam_next > 0.0:
            lam = lam_next
    alpha = line_fit(d, u, v, psi)
    return dict(psi=psi, alpha0=float(alpha[0]), alpha1=float(alpha[1]),
                e_min=energy_min(d, u, v, psi), iters=it, status=status)


def transform(disp, psi, alpha0, alpha1, delta_t=0.0):
    """eq. (disparity_transformation):
    l'(p) = l(p) - alpha0 + alpha1 (u sin(psi) - v cos(psi)) + delta_t."""
    disp = np.asarray(disp, dtype=np.float64)
    H, W = disp.shape
    u = np.arange(W, dtype=np.float64)[None, :]
    v = np.arange(H, dtype=np.float64)[:, None]
    return disp - alpha0 + alpha1 * (u * math.sin(psi) - v * math.cos(psi)) + delta_t


def disparity_transform(disp, mask=None, psi_init=0.0, delta_t=0.0, lambda0=10.0,
                        delta_psi=math.pi / 1.8e6, max_iters=100):
    """§3.3 end to end on a disparity map: roll estimate over the masked pixels,
    line fit at that roll, transform of every pixel.  Returns (map, result dict)."""
    disp = np.asarray(disp, dtype=np.float64)
    if mask is None:
        mask = np.ones(disp.shape, dtype=bool)
    vv, uu = np.nonzero(np.asarray(mask))
    res = estimate_roll(disp[vv, uu], uu.astype(np.float64), vv.astype(np.float64),
                        psi_init, lambda0, delta_psi, max_iters)
    return transform(disp, res["psi"], res["alpha0"], res["alpha1"], delta_t), res
