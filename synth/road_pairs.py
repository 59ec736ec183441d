"""Seeded synthetic road-scene stereo pairs.

These stand in for the paper's UAV, KITTI and EISATS data (§4.2, §4.4), none of which
is available here.  The module draws a band-limited texture, a ground-truth road
disparity (a quadratic in the rotated row coordinate y = v cos(psi) - u sin(psi) of
eq. (y), with u measured from the centre column) minus elliptical pothole depressions,
and renders the target view from that disparity.  It holds none of the stereo
method's own arithmetic: no matching cost, no aggregation, no warp by row shift,
no fit.  Both the CPU oracle and the GPU path take their inputs from here.

Recipe (all draws from one ``numpy.random.Generator(PCG64(seed))``):

* texture: white N(0,1) noise, Gaussian blur sigma_blur = 1 px, rescaled to
  mean 128 / std 40, rounded and clipped to uint8;
* road disparity: d(u,v) = a0 + a1*y + a2*y^2 with y = v cos(roll) - (u-uc) sin(roll);
* potholes: d -= depth * (1 - rho^2) inside each ellipse (rho < 1);
* target: for every target column x solve u = x + d(u, v) by fixed-point
  iteration, sample the reference linearly along the row at u, add N(0, sigma_n^2),
  round and clip;
* row shift table: s(v) = road disparity at the centre column (no potholes)
  minus delta_p, delta_p chosen so that the residual disparity d - round(s) is
  non-negative with a small margin; all-zero when the config asks for no warp.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math

import numpy as np
from scipy import ndimage

SEED_BASE = 1904060170


@dataclass
class RoadScene:
    ref: np.ndarray          # (H, W) uint8 reference (left) image
    tgt: np.ndarray          # (H, W) uint8 target (right) image
    gt_disp: np.ndarray      # (H, W) float64 ground-truth disparity u_ref - u_tar
    gt_road: np.ndarray      # (H, W) float64 road disparity without potholes
    shift: np.ndarray        # (H,) float32 row shift s(v) for the perspective warp
    roll: float              # roll angle in radians
    coeffs: tuple            # (a0, a1, a2)
    delta_p: float           # constant subtracted from the road disparity in s(v)
    potholes: list = field(default_factory=list)  # (uc, vc, ra, rb, depth)
    params: dict = field(default_factory=dict)    # D, win, bil, sigma0, sigma1, ...

    @property
    def height(self) -> int:
        return int(self.ref.shape[0])

    @property
    def width(self) -> int:
        return int(self.ref.shape[1])


# Workload presets.  Sizes, search ranges and windows follow the configurations the
# method is measured on; sigma0 / sigma1 default to 3 / 10 where a preset does not
# name them, and "paper" is the paper's own filter (sigma0 = 1.5, sigma1 = 5.5,
# 120-connected neighbourhood, i.e. an 11 x 11 window; §4.4.1).
CONFIGS = {
    "small": dict(index=0, width=320, height=240, D=64, win=7, bil=9, sigma0=3.0, sigma1=10.0,
                  roll_deg=(3.0, 3.0), n_potholes=2, depth=(2.0, 4.0), sigma_n=2.0, warp=False),
    "large": dict(index=1, width=1024, height=768, D=32, win=9, bil=11, sigma0=3.0, sigma1=10.0,
                  roll_deg=(0.0, 5.0), n_potholes=4, depth=(3.0, 10.0), sigma_n=2.0, warp=True),
    "batch": dict(index=2, sizes=((640, 480), (960, 540), (1280, 720), (1920, 1080)),
                  Ds=(32, 64, 128), n_pairs=64, win=9, bil=11, sigma0=3.0, sigma1=10.0,
                  roll_deg=(-6.0, 6.0), n_potholes=4, depth=(3.0, 10.0), sigma_n=2.0, warp=True),
    "precision": dict(index=3, width=1920, height=1080, D=192, win=9, bil=13, sigma0=3.0,
                      sigma1=10.0, roll_deg=(3.0, 3.0), n_potholes=4, depth=(3.0, 10.0),
                      sigma_n=2.0, warp=True),
    "grad": dict(index=4, width=960, height=540, D=64, win=9, bil=11, sigma0=3.0, sigma1=10.0,
                 roll_deg=(-6.0, 6.0), n_potholes=4, depth=(3.0, 10.0), sigma_n=2.0, warp=True,
                 n_pairs=8, temperature=0.1),
    "hd": dict(index=5, width=1920, height=1080, D=128, win=9, bil=11, sigma0=3.0, sigma1=10.0,
               roll_deg=(3.0, 3.0), n_potholes=4, depth=(3.0, 10.0), sigma_n=2.0, warp=True),
    "paper": dict(index=6, width=640, height=360, D=32, win=9, bil=11, sigma0=1.5, sigma1=5.5,
                  roll_deg=(-3.0, 3.0), n_potholes=3, depth=(2.0, 6.0), sigma_n=2.0, warp=True),
}


def texture(rng: np.random.Generator, height: int, width: int, sigma_blur: float = 1.0,
            mean: float = 128.0, std: float = 40.0) -> np.ndarray:
    """Band-limited Gaussian noise texture, uint8."""
    n = rng.standard_normal((height, width))
    b = ndimage.gaussian_filter(n, sigma_blur, mode="reflect")
    b = (b - b.mean()) / b.std()
    return np.clip(np.rint(mean + std * b), 0, 255).astype(np.uint8)


def _road(u, v, width, roll, coeffs):
    a0, a1, a2 = coeffs
    uc = 0.5 * (width - 1)
    y = v * math.cos(roll) - (u - uc) * math.sin(roll)
    return a0 + a1 * y + a2 * y * y


def _pothole_depth(u, v, potholes):
    """Depth of the pothole depressions at (u, v); v is constant along each row, so each
    pothole only touches the band of rows with |v - pv| < rb (elsewhere rho^2 >= 1)."""
    shape = np.broadcast(u, v).shape
    ub = np.broadcast_to(u, shape)
    vb = np.broadcast_to(v, shape)
    out = np.zeros(shape)
    vrow = vb[:, 0]
    for (pu, pv, ra, rb, depth) in potholes:
        rows = np.nonzero(np.abs(vrow - pv) < rb)[0]
        if rows.size == 0:
            continue
        r0, r1 = int(rows[0]), int(rows[-1]) + 1
        rho2 = ((ub[r0:r1] - pu) / ra) ** 2 + ((vb[r0:r1] - pv) / rb) ** 2
        out[r0:r1] += np.where(rho2 < 1.0, depth * (1.0 - rho2), 0.0)
    return out


def make_scene(width: int, height: int, D: int, seed: int, *, roll: float | None = None,
               roll_deg=(3.0, 3.0), coeffs=(5.0, 0.12, 1e-4), n_potholes: int = 2,
               depth=(2.0, 4.0), sigma_n: float = 2.0, warp: bool = True,
               win: int = 9, bil: int = 11, sigma0: float = 3.0, sigma1: float = 10.0,
               margin: int = 2, **_unused) -> RoadScene:
    """Draw one road-scene pair; every random number comes from ``seed``."""
    rng = np.random.Generator(np.random.PCG64(seed))
    if roll is None:
        lo, hi = roll_deg
        roll = math.radians(lo if lo == hi else rng.uniform(lo, hi))
    ref = texture(rng, height, width)

    potholes = []
    for _ in range(n_potholes):
        ra = rng.uniform(0.04, 0.10) * width
        rb = rng.uniform(0.03, 0.08) * height
        pu = rng.uniform(ra + 0.05 * width, width - ra - 0.05 * width)
        pv = rng.uniform(max(rb, 0.35 * height), height - rb - 0.05 * height)
        potholes.append((pu, pv, ra, rb, rng.uniform(*depth)))

    u = np.arange(width, dtype=np.float64)[None, :]
    v = np.arange(height, dtype=np.float64)[:, None]
    gt_road = _road(u, v, width, roll, coeffs) * np.ones((height, 1))
    gt = gt_road - _pothole_depth(u, v, potholes)

    # Render the target: target column x shows the reference point u with u - d(u,v) = x.
    x = np.broadcast_to(u, (height, width))
    vv = np.broadcast_to(v, (height, width))
    uu = x + (_road(x, vv, width, roll, coeffs) - _pothole_depth(x, vv, potholes))
    for _ in range(4):
        uu = x + (_road(uu, vv, width, roll, coeffs) - _pothole_depth(uu, vv, potholes))
    uc = np.clip(uu, 0.0, width - 1.0)
    u0 = np.floor(uc).astype(np.int64)
    u1 = np.minimum(u0 + 1, width - 1)
    f = uc - u0
    rows = np.arange(height)[:, None]
    refd = ref.astype(np.float64)
    sample = (1.0 - f) * refd[rows, u0] + f * refd[rows, u1]
    sample += rng.normal(0.0, sigma_n, size=sample.shape)
    tgt = np.clip(np.rint(sample), 0, 255).astype(np.uint8)

    if warp:
        centre = _road(0.5 * (width - 1), np.arange(height, dtype=np.float64), width, roll, coeffs)
        dev = gt - centre[:, None]
        delta_p = float(math.ceil(max(0.0, -dev.min())) + margin)
        shift = (centre - delta_p).astype(np.float32)
    else:
        delta_p = 0.0
        shift = np.zeros(height, dtype=np.float32)

    params = dict(D=D, win=win, bil=bil, sigma0=sigma0, sigma1=sigma1)
    return RoadScene(ref=ref, tgt=tgt, gt_disp=gt, gt_road=gt_road, shift=shift, roll=roll,
                     coeffs=tuple(coeffs), delta_p=delta_p, potholes=potholes, params=params)


def make_config_scene(name: str, pair: int = 0) -> RoadScene:
    """The scene of a named preset (``pair`` selects one pair of a multi-pair preset)."""
    cfg = dict(CONFIGS[name])
    seed = SEED_BASE + cfg["index"] + 1000 * pair
    if name == "batch":
        return make_batch_scenes(1, first=pair)[0]
    w, h, D = cfg.pop("width"), cfg.pop("height"), cfg.pop("D")
    return make_scene(w, h, D, seed, **cfg)


def make_batch_scenes(n: int | None = None, first: int = 0) -> list:
    """Pairs of uneven sizes and search ranges (the batched workload)."""
    cfg = CONFIGS["batch"]
    n = cfg["n_pairs"] if n is None else n
    jobs = []
    for i in range(first, first + n):
        rng = np.random.Generator(np.random.PCG64(SEED_BASE + cfg["index"] + 7919 * (i + 1)))
        w, h = cfg["sizes"][int(rng.integers(len(cfg["sizes"])))]
        D = int(cfg["Ds"][int(rng.integers(len(cfg["Ds"])))])
        seed = SEED_BASE + cfg["index"] + 1000 * i
        kw = {k: cfg[k] for k in ("win", "bil", "sigma0", "sigma1", "roll_deg", "n_potholes",
                                  "depth", "sigma_n", "warp")}
        jobs.append((w, h, D, seed, kw))
    # every scene draws from its own generator, so threads change nothing but the wall time
    from concurrent.futures import ThreadPoolExecutor
    with ThreadPoolExecutor(max_workers=8) as ex:
        return list(ex.map(lambda j: make_scene(j[0], j[1], j[2], j[3], **j[4]), jobs))


def crop_pair(scene: RoadScene, u0: int, v0: int, width: int, height: int, offset: int | None = None):
    """A width x height window of a pair, for checks that must stay small.

    The reference is cut at column u0, the target at column u0 - offset, and the row-shift
    table of those rows is lowered by the same whole number of pixels, so that the target
    content a reference pixel matches stays inside the window.  ``offset`` defaults to the
    whole part of the mean shift over the rows.  Returns (ref, tgt, shift) as uint8, uint8,
    float32 arrays."""
    s = scene.shift[v0:v0 + height]
    off = int(math.floor(float(np.mean(s)))) if offset is None else int(offset)
    if not (0 <= u0 - off and u0 + width <= scene.width and 0 <= v0 and v0 + height <= scene.height):
        raise ValueError("window outside the pair")
    ref = np.ascontiguousarray(scene.ref[v0:v0 + height, u0:u0 + width])
    tgt = np.ascontiguousarray(scene.tgt[v0:v0 + height, u0 - off:u0 - off + width])
    return ref, tgt, (s - np.float32(off)).astype(np.float32)


def jitter(img: np.ndarray, seed: int, amp: float = 0.5) -> np.ndarray:
    """img as float64 plus uniform noise in [-amp, amp): grey levels off the integer grid."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return img.astype(np.float64) + rng.uniform(-amp, amp, size=img.shape)


def make_roll_sequence(n_frames: int, width: int, height: int, D: int, seed: int, roll0_deg: float,
                       drift_deg: float, **kw) -> list:
    """A video of one road: n_frames pairs drawn from the same seed (same texture, potholes
    and noise), the roll angle moving by drift_deg per frame from roll0_deg."""
    return [make_scene(width, height, D, seed, roll=math.radians(roll0_deg + t * drift_deg), **kw)
            for t in range(n_frames)]
