"""Pins of the self-estimated warp model (oracle/warp_est.py), CPU.

  * the block average is the rounded-half-up mean of every F x F block (brute force);
  * the fit equals numpy.polyfit of the full-resolution disparity against the block-centre row;
  * on a pair whose road disparity is exactly affine in the row (no roll, no quadratic term,
    no potholes) the estimate returns the road's own coefficients;
  * on the 1024 x 768 road workload (roll, quadratic term, potholes) the fitted line stays
    close to the centre-column road disparity the generator's shift table follows.
"""
import math

import numpy as np
import pytest

import oracle
import synth
from oracle import warp_est


@pytest.fixture(scope="module", autouse=True)
def _built():
    oracle.build()


def test_block_average_rounds_half_up():
    rng = np.random.default_rng(41)
    img = rng.integers(0, 256, (13, 22), dtype=np.uint8)
    for F in (1, 2, 3, 4):
        out = warp_est.downsample(img, F)
        assert out.shape == (13 // F, 22 // F)
        for vc in range(out.shape[0]):
            for uc in range(out.shape[1]):
                s = int(img[vc * F:(vc + 1) * F, uc * F:(uc + 1) * F].astype(int).sum())
                assert out[vc, uc] == math.floor(s / (F * F) + 0.5)


def test_fit_is_polyfit_on_block_centres():
    rng = np.random.default_rng(42)
    Hc, Wc, F = 30, 40, 4
    disp = rng.uniform(2, 20, (Hc, Wc))
    valid = (rng.uniform(size=(Hc, Wc)) > 0.3).astype(np.uint8)
    c0, c1, n = warp_est.fit_rows(disp, valid, F)
    vc, _ = np.nonzero(valid)
    b, a = np.polyfit(F * vc + (F - 1) / 2.0, F * disp[valid != 0], 1)
    assert n == int(valid.sum())
    assert c1 == pytest.approx(b, rel=1e-12) and c0 == pytest.approx(a, rel=1e-12)


def test_affine_road_is_recovered():
    s = synth.make_scene(640, 480, 64, 777, roll=0.0, coeffs=(8.0, 0.09, 0.0), n_potholes=0, warp=False,
                         sigma_n=1.0)
    c0, c1, n = warp_est.estimate_warp(s.ref, s.tgt, 64, 4, 5, 7, 3.0, 10.0)
    assert n > 5000
    assert abs(c1 - 0.09) < 0.004 and abs(c0 - 8.0) < 0.6, (c0, c1)


def test_road_workload_line_follows_the_road():
    """eq. (relation_vd) is affine, while the generator's road is quadratic in the row and
    rolled: the estimate must stay near the best affine line through the road itself (its
    fit sees only the columns the geometric validity keeps, hence the slack) and leave a
    residual spread within 4 px of that line's own."""
    s = synth.make_config_scene("large")
    D = int(math.ceil(s.gt_road.max())) + 8
    c0, c1, n = warp_est.estimate_warp(s.ref, s.tgt, D, 4, 5, 7, 3.0, 10.0)
    v = np.arange(s.height)
    vv = np.repeat(v, s.width)
    b, a = np.polyfit(vv, s.gt_road.ravel(), 1)            # the road's own least-squares line
    assert abs(c1 - b) < 0.01 and np.median(np.abs(c0 + c1 * v - (a + b * v))) < 3.0, (c0, c1, a, b)
    resid = s.gt_disp - (c0 + c1 * v)[:, None]
    best = s.gt_disp - (a + b * v)[:, None]
    assert np.ptp(resid) <= np.ptp(best) + 4.0
