"""Accuracy and throughput measures printed in the paper (§4.4).  TEST INFRASTRUCTURE ONLY."""
from __future__ import annotations

import numpy as np


def error_pixel_percent(disp, gt, eps_d, mask=None):
    """eq. (e_pep) with eq. (delta_function): percent of pixels whose |error| > eps_d."""
    err = np.abs(np.asarray(disp, np.float64) - np.asarray(gt, np.float64))
    if mask is not None:
        err = err[np.asarray(mask, bool)]
    return 100.0 * float(np.mean(err > eps_d))


def rms_error(disp, gt, mask=None):
    """eq. (e_rms): root mean squared disparity error."""
    err = np.asarray(disp, np.float64) - np.asarray(gt, np.float64)
    if mask is not None:
        err = err[np.asarray(mask, bool)]
    return float(np.sqrt(np.mean(err * err)))


def sigma_d(transformed, mask=None):
    """eq. (sigma_d): standard deviation of the transformed disparities."""
    s = np.asarray(transformed, np.float64)
    if mask is not None:
        s = s[np.asarray(mask, bool)]
    m = s.size
    return float(np.sqrt(np.sum((s - s.sum() / m) ** 2) / m))


def mde_per_s(u_max, v_max, d_max, seconds):
    """Millions of disparity evaluations per second (§4.4.1)."""
    return u_max * v_max * d_max / seconds * 1e-6
