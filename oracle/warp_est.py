"""Self-estimated warp model, FP64 / integer numpy.  TEST INFRASTRUCTURE ONLY.

The paper takes the perspective transformation of §3.1 from correspondences it does not
specify, with the road disparity affine in the row, du(v) = c0 + c1 v (eq. relation_vd).
Here the two coefficients come from a coarse first pass over the unwarped pair:

  1. both images are averaged over F x F blocks (the block sum plus F^2/2, divided by F^2 in
     integers: the mean rounded half up); a remainder of fewer than F rows or columns is left
     out;
  2. the reference view (eq. c, eq. fbs, WTA, eq. subpixel; the oracle of stereo_oracle.c) runs
     on the coarse pair over the full range of Dc = ceil(D / F) disparities, no warp;
  3. least squares over the coarse pixels the geometric validity keeps: F l_c(u_c, v_c) =
     a + b v_c, then c1 = b / F and c0 = a - c1 (F - 1) / 2 (a coarse row v_c covers full rows
     F v_c .. F v_c + F - 1, centred on F v_c + (F - 1) / 2).
"""
from __future__ import annotations

import math

import numpy as np

from . import stereo as _stereo, valid_mask as _valid_mask


def downsample(img, F):
    """Block means of F x F blocks, rounded half up, as uint8 [H // F][W // F]."""
    img = np.asarray(img, dtype=np.int64)
    Hc, Wc = img.shape[0] // F, img.shape[1] // F
    blocks = img[:Hc * F, :Wc * F].reshape(Hc, F, Wc, F).sum(axis=(1, 3))
    return ((blocks + (F * F) // 2) // (F * F)).astype(np.uint8)


def coarse_disparity(ref, tgt, D, F, win, bil, sigma0, sigma1):
    """Steps 1-2: (coarse disparity map in coarse pixels, validity) of the unwarped pair."""
    rc, tc = downsample(ref, F), downsample(tgt, F)
    Dc = int(math.ceil(D / F))
    Hc = rc.shape[0]
    zero = np.zeros(Hc, np.float32)
    disp, _, _, _ = _stereo(rc, tc, zero, Dc, win, bil, sigma0, sigma1)
    valid = _valid_mask(rc.shape[1], Hc, Dc, win, bil, zero)
    return disp, valid


def fit_rows(disp_c, valid_c, F):
    """Step 3: (c0, c1, n) of du(v) = c0 + c1 v in full-resolution units."""
    vc, _ = np.nonzero(valid_c)
    d = F * disp_c[valid_c != 0]
    if d.size < 2:
        return float("nan"), float("nan"), int(d.size)
    A = np.stack([np.ones_like(vc, dtype=np.float64), vc.astype(np.float64)], axis=1)
    a, b = np.linalg.lstsq(A, d, rcond=None)[0]
    c1 = b / F
    return float(a - c1 * (F - 1) / 2.0), float(c1), int(d.size)


def estimate_warp(ref, tgt, D, F, win, bil, sigma0, sigma1):
    """(c0, c1, n) of the road disparity du(v) = c0 + c1 v estimated from the pair."""
    disp, valid = coarse_disparity(ref, tgt, D, F, win, bil, sigma0, sigma1)
    return fit_rows(disp, valid, F)
