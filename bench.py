#!/usr/bin/env python3
"""Benchmark of the road-stereo hot path on GB300.

One step = the whole hot path on one 1920 x 1080 stereo pair, D = 128, w = 9, k = 11:
perspective warp (§3.1) -> fused cost + bilateral aggregation + WTA + sub-pixel
(eq. c, eq. fbs, eq. subpixel) -> disparity transformation (§3.3), inputs resident in
device memory.  L2 is flushed (a 256 MiB write) before every timed step, outside its
events.  Prints one JSON line (rank 0).  ``--impl reference`` times the CPU oracle
instead, on bounded row bands of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Gpix·disp/s of cost+bilateral+WTA and stereo pairs/s at 1080p, D=128, vs plain FP32"
UNIT = "Gpix*disp/s"
WORKLOAD = "road-stereo 1920x1080 D=128 w=9 k=11 sigma0=3 sigma1=10, warp + fused cost/agg/WTA + DT"
SM_COUNT_GB300 = 152
FP32_LANES_PER_SM = 128
SM_MAX_MHZ = 2070.0
# DRAM traffic of one fused-kernel launch on this workload, from the ncu capture summarised
# in profiles/ (dram__bytes_read.sum + dram__bytes_write.sum); valid only for the kernel
# source with this SHA-256 prefix.
FUSED_TRAFFIC = {"sha256": "972b7216c2da1f86", "bytes": 39214848}
FUSED_SOURCES = ("internal.cuh", "k_fused_common.cuh", "k_cost.cuh", "k_fused_tc.cuh", "k_fused_sc.cuh",
                 "k_fused_sc.cu")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-diff", action="store_true")
    ap.add_argument("--no-precision", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def measured_peaks():
    """The measured GB300 peak rates in MEASURED_PEAKS.json (empty when the file is absent)."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def kernel_sha():
    h = hashlib.sha256()
    for f in FUSED_SOURCES:
        h.update(open(os.path.join(ROOT, "paper_1904_06017_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms in the background, with the
    sampler's timestamps, so that the samples of any interval (the timed steps) can be told
    from the rest.  Started before the warm-up so that a short timed region still has samples."""
    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    REASONS = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None
        self.marks = {}

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def mark(self, name):
        """Wall-clock time of an event (local time, as nvidia-smi's timestamps)."""
        self.marks[name] = time.time()

    @staticmethod
    def _when(ts):
        import datetime
        for fmt in ("%Y/%m/%d %H:%M:%S.%f", "%Y/%m/%d %H:%M:%S"):
            try:
                return datetime.datetime.strptime(ts, fmt).timestamp()
            except ValueError:
                pass
        return None

    def _summary(self, rows):
        sm = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        mx = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        reasons = sorted({self.REASONS[i] for r in rows for i in range(4) if r[6 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}

    def stop(self, t0=None, t1=None):
        """Summary of the samples between marks t0 and t1 (all samples if unset), plus the
        summary of every sample taken under load (from the first mark on)."""
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 10:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        when = [self._when(r[0]) for r in rows]
        lo, hi = self.marks.get(t0), self.marks.get(t1)
        timed = [r for r, w in zip(rows, when) if w is not None and lo is not None and hi is not None
                 and lo - 0.1 <= w <= hi + 0.1]
        first = min(self.marks.values()) if self.marks else None
        load = [r for r, w in zip(rows, when) if w is not None and first is not None and w >= first]
        out = self._summary(timed if timed else load if load else rows)
        out["window"] = "timed steps" if timed else "whole GPU phase of the bench"
        out["under_load"] = self._summary(load if load else rows)
        out["under_load"]["window"] = "warm-up, timed steps, end-to-end and storage-variant legs"
        return out


def max_over_ranks(x, world, device="cpu"):
    """The largest of the ranks' values (the slowest rank's time); x itself at world = 1."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world, steps, units_per_step, t_max_ms):
    """Whole-job throughput in units/s (x1e-9): every rank processed `steps` steps of
    `units_per_step` units; the job took the slowest rank's time."""
    return world * steps * units_per_step / (t_max_ms * 1e-3) / 1e9


def make_inputs():
    import synth
    s = synth.make_config_scene("hd")
    return s


def cpu_baseline_sample(s, seconds):
    """The oracle on a bounded band of rows of the same pair, on all host cores."""
    import numpy as np
    import oracle
    p = s.params
    H, W, D = s.height, s.width, p["D"]
    tw = oracle.warp(s.tgt, s.shift)
    rows = 16
    v0 = H // 2 - rows // 2
    oracle.stereo(s.ref, tw, s.shift, D, p["win"], p["bil"], p["sigma0"], p["sigma1"], rows=(v0, v0 + 8))
    t = time.perf_counter()
    oracle.stereo(s.ref, tw, s.shift, D, p["win"], p["bil"], p["sigma0"], p["sigma1"], rows=(v0, v0 + rows))
    dt16 = time.perf_counter() - t
    rows = int(max(16, min(H - 2 * 16, round(rows * seconds / max(dt16, 1e-3)))))
    v0 = max(0, H // 2 - rows // 2)
    t = time.perf_counter()
    oracle.stereo(s.ref, tw, s.shift, D, p["win"], p["bil"], p["sigma0"], p["sigma1"], rows=(v0, v0 + rows))
    el = time.perf_counter() - t
    val = rows * W * D / el / 1e9
    return {"value": val, "unit": UNIT, "cores": oracle.get_threads(), "kind": "oracle",
            "sample": "rows %d..%d of the 1920x1080 D=128 pair (%d x %d x %d disparity evaluations), "
                      "FP64 C oracle (cost, aggregation, WTA, sub-pixel), %.1f s" % (v0, v0 + rows, rows, W, D, el)}


REFERENCE_BUDGET_S = 150.0


def reference_rows(s, n_steps, budget_s=REFERENCE_BUDGET_S):
    """Rows per reference step (1..16) so that n_steps steps take about budget_s seconds."""
    import oracle
    p = s.params
    tw = oracle.warp(s.tgt, s.shift)
    v0 = s.height // 2
    t = time.perf_counter()
    oracle.stereo(s.ref, tw, s.shift, p["D"], p["win"], p["bil"], p["sigma0"], p["sigma1"], rows=(v0, v0 + 2))
    per_row = (time.perf_counter() - t) / 2
    return int(max(1, min(16, budget_s / max(n_steps, 1) / max(per_row, 1e-6))))


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import numpy as np
    import oracle
    from oracle import dt
    oracle.build()
    s = make_inputs()
    p = s.params
    H, W, D = s.height, s.width, p["D"]
    rows = reference_rows(s, args.warmup + args.steps)
    times = []
    for it in range(args.warmup + args.steps):
        v0 = 16 + (it * 37) % (H - 32 - rows)
        t = time.perf_counter()
        tw = oracle.warp(s.tgt, s.shift)
        disp, _, _, _ = oracle.stereo(s.ref, tw, s.shift, D, p["win"], p["bil"], p["sigma0"], p["sigma1"],
                                      rows=(v0, v0 + rows))
        uu, vv = np.meshgrid(np.arange(W, dtype=np.float64), np.arange(v0, v0 + rows, dtype=np.float64))
        dt.estimate_roll(disp.ravel(), uu.ravel(), vv.ravel())
        el = time.perf_counter() - t
        if it >= args.warmup:
            times.append(el)
    tot = sum(times)
    val = args.steps * rows * W * D / tot / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": 0,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD + " (oracle on %d-row bands)" % rows,
                                            "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": oracle.get_threads(), "kind": "oracle",
                             "sample": "per step: warp of the full target, then cost/aggregation/WTA/"
                                       "sub-pixel on a %d-row band and the roll fit of that band" % rows},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def bench_batch(args, dev, stream, flush):
    """The batched workload: 64 pairs of uneven sizes and search ranges in one persistent
    launch inside a captured CUDA graph (autotuned tiles), FP32 costs, and the same batch
    with FP16 cost storage.  Its inputs (about 3 GB of images and staging) exceed L2."""
    import numpy as np
    import torch
    import paper_1904_06017_gb300 as sg
    import synth
    scenes = synth.make_batch_scenes()
    cfg = synth.CONFIGS["batch"]
    pairs = []
    for s in scenes:
        H, W, D = s.height, s.width, s.params["D"]
        pitch = (W + 15) // 16 * 16
        def img(a):
            t = torch.zeros((H, pitch), dtype=torch.uint8)
            t[:, :W] = torch.from_numpy(a)
            return t.to(dev)
        pairs.append(dict(ref=img(s.ref), tgt=img(s.tgt), shift=torch.from_numpy(s.shift).to(dev),
                          tgt_warped=torch.empty((H, pitch), dtype=torch.uint8, device=dev),
                          disp=torch.empty((H, W), dtype=torch.float32, device=dev),
                          wta=torch.empty((H, W), dtype=torch.int32, device=dev),
                          valid=torch.empty((H, W), dtype=torch.uint8, device=dev),
                          disp_out=torch.empty((H, W), dtype=torch.float32, device=dev),
                          res=torch.zeros(64, dtype=torch.uint8, device=dev), max_disp=D))
    units = sum(s.height * s.width * s.params["D"] for s in scenes)
    out = {"pairs": len(scenes), "sizes": sorted({"%dx%d" % (s.width, s.height) for s in scenes}),
           "search_ranges": sorted({s.params["D"] for s in scenes}), "win": cfg["win"], "bil": cfg["bil"]}
    steps = max(3, min(args.steps, 20))
    disp32 = wta32 = None
    for name, dtype in (("f32", sg.STEREO_F32), ("f16", sg.STEREO_F16)):
        b = sg.StereoBatch(pairs, win=cfg["win"], bil=cfg["bil"], sigma0=cfg["sigma0"], sigma1=cfg["sigma1"],
                           cost_dtype=dtype)
        for _ in range(2):
            b.run(stream)
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for i in range(steps):
            ev[i][0].record(stream)
            b.run(stream)
            ev[i][1].record(stream)
        torch.cuda.synchronize()
        b.check_device_status()
        ms = sum(a.elapsed_time(c) for a, c in ev) / steps
        disp = [q["disp"].cpu().numpy() for q in pairs]
        wta = [q["wta"].cpu().numpy() for q in pairs]
        valid = [q["valid"].cpu().numpy().astype(bool) for q in pairs]
        rec = {"ms_per_batch": ms, "pairs_per_s": len(scenes) * 1e3 / ms,
               "gpix_disp_per_s": units / ms / 1e6, "graph_runs": steps, "tiles": b.config()}
        if disp32 is None:
            disp32, wta32 = disp, wta
        else:
            npx = sum(a.size for a in disp32)
            moved = sum(int(np.count_nonzero(np.abs(a - c) > 0.5)) for a, c in zip(disp32, disp))
            rec["disp_diff_gt_half_px_vs_f32"] = moved / npx
            # the integer WTA disparity d*: the fraction of pixels whose d* differs from the
            # batched FP32 form's (the pass line is 0.1 %), over all pixels and over valid ones
            rec["wta_disagree_vs_f32"] = sum(int(np.count_nonzero(a != c)) for a, c in zip(wta32, wta)) / npx
            nv = sum(int(m.sum()) for m in valid)
            rec["wta_disagree_vs_f32_valid"] = (sum(int(np.count_nonzero((a != c) & m))
                                                    for a, c, m in zip(wta32, wta, valid)) / max(nv, 1))
            rec["wta_disagree_pass"] = rec["wta_disagree_vs_f32"] <= 1e-3
        out[name] = rec
        b.close()
    del pairs
    torch.cuda.empty_cache()
    return out


def bench_precision(args, dev, stream, flush, peak):
    """The precision workload: one 1920 x 1080 pair, D = 192, w = 9, k = 13, with the cost
    volume stored as FP32, FP16 and BF16 (FP32 accumulators in every form).  One step = warp
    -> fused cost/aggregation/WTA -> disparity transformation, L2 flushed before each step.
    Reports each form's step time, throughput, the fused kernel's share of the FP32 roofline
    (the same algorithmic work in every form) and its integer-WTA disagreement with FP32."""
    import numpy as np
    import torch
    import paper_1904_06017_gb300 as sg
    import synth
    s = synth.make_config_scene("precision")
    p = s.params
    H, W, D, win, bil = s.height, s.width, p["D"], p["win"], p["bil"]
    pitch = (W + 15) // 16 * 16

    def img(a):
        t = torch.zeros((H, pitch), dtype=torch.uint8)
        t[:, :W] = torch.from_numpy(a)
        return t.to(dev)

    ref, tgt, shift = img(s.ref), img(s.tgt), torch.from_numpy(s.shift).to(dev)
    tw = torch.empty_like(tgt)
    disp = torch.empty((H, W), dtype=torch.float32, device=dev)
    valid = torch.empty((H, W), dtype=torch.uint8, device=dev)
    out = torch.empty_like(disp)
    res = torch.zeros(64, dtype=torch.uint8, device=dev)
    flops_per_unit = 2.0 * bil * bil + 11.0 + 2.0 * bil * bil / D + 1.0
    flops = flops_per_unit * W * H * D
    n = max(3, min(args.steps, 20))
    rec = {"workload": "1920x1080 D=192 w=9 k=13 sigma0=3 sigma1=10", "flops_per_pixel_disparity": flops_per_unit}
    wta32 = None
    for name, dtype in (("f32", sg.STEREO_F32), ("f16", sg.STEREO_F16), ("bf16", sg.STEREO_BF16)):
        sv = sg.Stereo(W, H, D, win=win, bil=bil, sigma0=p["sigma0"], sigma1=p["sigma1"], pitch=pitch,
                       cost_dtype=dtype)
        wta = torch.empty((H, W), dtype=torch.int32, device=dev)
        sv.warp_target(tgt, shift, tw)
        sv.cost_aggregate_wta(ref, tw, shift, disp, wta, valid)
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n)]
        sg.stereo_profile_enable(sv.ctx, True)
        for i in range(n):
            flush.fill_(i & 0xFF)
            ev[i][0].record(stream)
            sv.warp_target(tgt, shift, tw)
            sv.cost_aggregate_wta(ref, tw, shift, disp, None, valid)
            sv.disparity_transform(disp, valid, 0.0, 0.0, out, res=res)
            ev[i][1].record(stream)
        torch.cuda.synchronize()
        nf, fms = sg.stereo_profile_read(sv.ctx)
        sg.stereo_profile_enable(sv.ctx, False)
        sv.check_device_status()
        sv.close()
        ms = sum(a.elapsed_time(b) for a, b in ev) / n
        fused = fms / max(nf, 1)
        w = wta.cpu().numpy()
        vm = valid.cpu().numpy().astype(bool)
        if wta32 is None:
            wta32 = w
        r = {"ms_per_step": ms, "gpix_disp_per_s": W * H * D / ms / 1e6, "pairs_per_s": 1e3 / ms,
             "fused_ms": fused, "fused_tflops": flops / (fused * 1e-3) / 1e12,
             "fused_frac_of_fp32_roofline": flops / (fused * 1e-3) / 1e12 / peak, "steps": n}
        if name != "f32":
            r["wta_disagree_vs_f32"] = float(np.mean(w != wta32))
            r["wta_disagree_vs_f32_valid"] = float(np.mean((w != wta32)[vm])) if vm.any() else None
        rec[name] = r
    return rec


def bench_diff(args, dev, stream, flush):
    """The differentiation workload: 8 pairs of 960 x 540, D = 64, w = 9, k = 11, T = 0.1.
    One step = soft-argmin forward, eq. (E2) forward, and the backward of both (gradients
    in both images and theta), through torch.autograd; plus 50 steps of roll refinement.
    Its workspace (about 3.4 GB) exceeds L2."""
    import numpy as np
    import torch
    from paper_1904_06017_gb300 import diff as sgd
    import synth
    cfg = synth.CONFIGS["grad"]
    B, W, H, D = cfg["n_pairs"], cfg["width"], cfg["height"], cfg["D"]
    scenes = [synth.make_config_scene("grad", pair=i) for i in range(B)]
    ref = torch.tensor(np.stack([s.ref for s in scenes]).astype(np.float32), device=dev, requires_grad=True)
    tgt = torch.tensor(np.stack([s.tgt for s in scenes]).astype(np.float32), device=dev, requires_grad=True)
    shift = torch.tensor(np.stack([s.shift for s in scenes]), device=dev)
    theta = torch.zeros((B, 3), dtype=torch.float64, device=dev)
    theta[:, 1], theta[:, 2] = 30.0, 0.1
    theta.requires_grad_(True)
    kw = dict(win=cfg["win"], bil=cfg["bil"], sigma0=cfg["sigma0"], sigma1=cfg["sigma1"],
              temperature=cfg["temperature"])

    def fwd():
        return sgd.SoftArgmin.apply(ref, tgt, shift, D, kw["win"], kw["bil"], kw["sigma0"], kw["sigma1"],
                                    kw["temperature"])

    def step():
        ref.grad = tgt.grad = theta.grad = None
        l = fwd()
        sgd.DTEnergy.apply(l, theta, None).sum().backward()
        return l

    for _ in range(2):
        step()
    torch.cuda.synchronize()
    n = max(3, min(args.steps, 10))
    e_f = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n)]
    e_s = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n)]
    for i in range(n):
        flush.fill_(i & 0xFF)
        e_f[i][0].record(stream)
        with torch.no_grad():
            l = fwd()
        e_f[i][1].record(stream)
        flush.fill_(i & 0xFF)
        e_s[i][0].record(stream)
        l = step()
        e_s[i][1].record(stream)
    torch.cuda.synchronize()
    fwd_ms = sum(a.elapsed_time(b) for a, b in e_f) / n
    step_ms = sum(a.elapsed_time(b) for a, b in e_s) / n
    # the fit mask: the library's geometric validity of each pair (no read behind any d
    # clamped), from the plain fused path on the same pair
    import paper_1904_06017_gb300 as sg
    pitch = (W + 15) // 16 * 16
    mask = torch.empty((B, H, W), dtype=torch.uint8, device=dev)
    search_psi = []
    with sg.Stereo(W, H, D, win=kw["win"], bil=kw["bil"], sigma0=kw["sigma0"], sigma1=kw["sigma1"],
                   pitch=pitch) as st:
        for b, sc in enumerate(scenes):
            def img(a):
                t = torch.zeros((H, pitch), dtype=torch.uint8)
                t[:, :W] = torch.from_numpy(a)
                return t.to(dev)
            rb, tb = img(sc.ref), img(sc.tgt)
            tw = torch.empty_like(tb)
            dtmp = torch.empty((H, W), dtype=torch.float32, device=dev)
            st.warp_target(tb, shift[b], tw)
            st.cost_aggregate_wta(rb, tw, shift[b], dtmp, None, mask[b])
            # the paper's roll search (the A7 kernel) on the same soft-argmin map and mask
            r = st.disparity_transform(l[b].detach().contiguous(), mask[b], 0.0, 0.0, dtmp)
            search_psi.append(r.psi)
        st.check_device_status()
    sgd.refine_roll(l.detach(), mask, 0.0, 50)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    traj = sgd.refine_roll(l.detach(), mask, 0.0, 50)
    e1.record(stream)
    torch.cuda.synchronize()
    psi = traj[:, -1, 0].cpu().numpy()
    # closed form on the same map and mask: the least-squares plane l = a + b u + c v gives
    # psi* = atan(-b / c) in (-pi/2, pi/2] (alpha0 + alpha1 y(psi) spans every plane)
    lh, mh = l.detach().double().cpu().numpy(), mask.cpu().numpy().astype(bool)
    vv, uu = np.mgrid[0:H, 0:W]
    plane_psi = []
    for b in range(B):
        m = mh[b]
        A = np.stack([np.ones(int(m.sum())), uu[m], vv[m]], 1).astype(np.float64)
        coef = np.linalg.lstsq(A, lh[b][m], rcond=None)[0]
        plane_psi.append(math.atan(-coef[1] / coef[2]))
    units = B * W * H * D
    k2 = cfg["bil"] ** 2
    return {"pairs": B, "size": "%dx%d" % (W, H), "max_disp": D, "temperature": cfg["temperature"],
            "forward_ms": fwd_ms, "forward_backward_ms": step_ms, "backward_ms": step_ms - fwd_ms,
            "forward_gpix_disp_per_s": units / fwd_ms / 1e6,
            "forward_backward_gpix_disp_per_s": units / step_ms / 1e6,
            "aggregation_flops_per_step": 2.0 * k2 * units * (1 + 2 + 2),
            "aggregation_tflops_effective": 2.0 * k2 * units * 5 / (step_ms * 1e-3) / 1e12,
            "refine_roll_50_steps_ms": e0.elapsed_time(e1),
            "fit_mask": "geometric validity from the library's fused path (%.1f %% of pixels)"
                        % (100.0 * float(mh.mean())),
            "refined_psi_deg": [float(np.degrees(x)) for x in psi],
            "search_psi_deg": [float(np.degrees(x)) for x in search_psi],
            "plane_fit_psi_deg": [float(np.degrees(x)) for x in plane_psi],
            "refined_minus_plane_fit_rad": [float(a - c) for a, c in zip(psi, plane_psi)],
            "search_minus_plane_fit_rad": [float(a - c) for a, c in zip(search_psi, plane_psi)],
            "true_roll_deg": [float(np.degrees(s.roll)) for s in scenes],
            "plane_fit_minus_true_roll_deg": [float(np.degrees(c - s.roll)) for c, s in zip(plane_psi, scenes)],
            "grad_finite": bool(torch.isfinite(ref.grad).all() and torch.isfinite(tgt.grad).all()),
            "steps": n}


def run_ours(args):
    import numpy as np
    import torch
    import paper_1904_06017_gb300 as sg
    from paper_1904_06017_gb300 import build as sgbuild

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    sgbuild.build()
    dev = torch.device("cuda", torch.cuda.current_device())

    s = make_inputs()
    p = s.params
    H, W, D, win, bil = s.height, s.width, p["D"], p["win"], p["bil"]
    pitch = (W + 15) // 16 * 16

    def img(a):
        t = torch.zeros((H, pitch), dtype=torch.uint8)
        t[:, :W] = torch.from_numpy(a)
        return t

    ref_h, tgt_h = img(s.ref).pin_memory(), img(s.tgt).pin_memory()
    shift_h = torch.from_numpy(s.shift).pin_memory()
    ref, tgt, shift = ref_h.to(dev), tgt_h.to(dev), shift_h.to(dev)
    tw = torch.empty_like(tgt)
    disp = torch.empty((H, W), dtype=torch.float32, device=dev)
    valid = torch.empty((H, W), dtype=torch.uint8, device=dev)
    out = torch.empty_like(disp)
    res = torch.zeros(64, dtype=torch.uint8, device=dev)
    out_h = torch.empty((H, W), dtype=torch.float32).pin_memory()
    res_h = torch.empty(64, dtype=torch.uint8).pin_memory()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    st = sg.Stereo(W, H, D, win=win, bil=bil, sigma0=p["sigma0"], sigma1=p["sigma1"], pitch=pitch)
    stream = torch.cuda.current_stream()
    launches_per_step = 7   # k_warp, k_prep, k_row_tables, k_fused, k_dt_moments, k_dt_solve, k_dt_apply

    def step():
        st.warp_target(tgt, shift, tw)
        st.cost_aggregate_wta(ref, tw, shift, disp, None, valid)
        st.disparity_transform(disp, valid, 0.0, 0.0, out, res=res)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    time.sleep(0.3)            # the sampler's first reading precedes the warm-up
    clocks.mark("warmup")
    for _ in range(args.warmup):
        step()
    st.check_device_status()

    # ---- device-resident timing, L2 flushed before each step (outside the events)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    sg.stereo_profile_enable(st.ctx, True)
    barrier()
    clocks.mark("timed_start")
    for i in range(args.steps):
        flush.fill_(i & 0xFF)
        ev[i][0].record(stream)
        step()
        ev[i][1].record(stream)
    barrier()
    clocks.mark("timed_end")
    n_fused, fused_ms = sg.stereo_profile_read(st.ctx)
    sg.stereo_profile_enable(st.ctx, False)
    st.check_device_status()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    t_max = max_over_ranks(sum(step_ms), world, dev)
    value = job_throughput(world, args.steps, W * H * D, t_max)
    pairs_per_s = job_throughput(world, args.steps, 1, t_max) * 1e9

    # ---- end to end through the public API: pinned host inputs in, transformed map out.  As a
    # pipeline would run it: two sets of device inputs and outputs, the copies on their own
    # stream, so the upload of step i + 1 and the read-back of step i - 1 overlap step i.  The
    # timed interval runs from before the first upload to after the last read-back and holds
    # every step's copies and its L2 flush.
    cs, xs = torch.cuda.Stream(), torch.cuda.Stream()   # compute, copies
    slot = [dict(ref=torch.empty_like(ref), tgt=torch.empty_like(tgt), shift=torch.empty_like(shift),
                 out=torch.empty_like(out), res=torch.empty_like(res),
                 out_h=torch.empty_like(out_h).pin_memory(), res_h=torch.empty_like(res_h).pin_memory())
            for _ in range(2)]
    ev_in = [torch.cuda.Event() for _ in range(args.steps)]
    ev_done = [torch.cuda.Event() for _ in range(args.steps)]
    ev_out = [torch.cuda.Event() for _ in range(args.steps)]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def upload(i):
        b = slot[i % 2]
        with torch.cuda.stream(xs):
            if i >= 2:
                xs.wait_event(ev_done[i - 2])    # step i - 2 has finished reading this slot
            b["ref"].copy_(ref_h, non_blocking=True)
            b["tgt"].copy_(tgt_h, non_blocking=True)
            b["shift"].copy_(shift_h, non_blocking=True)
            ev_in[i].record(xs)

    torch.cuda.synchronize()
    e0.record(xs)
    upload(0)
    for i in range(args.steps):
        b = slot[i % 2]
        if i + 1 < args.steps:
            upload(i + 1)
        with torch.cuda.stream(cs):
            cs.wait_event(ev_in[i])
            if i >= 2:
                cs.wait_event(ev_out[i - 2])      # the read-back of step i - 2 has left this slot
            flush.fill_(i & 0xFF)
            st.warp_target(b["tgt"], b["shift"], tw, stream=cs)
            st.cost_aggregate_wta(b["ref"], tw, b["shift"], disp, None, valid, stream=cs)
            st.disparity_transform(disp, valid, 0.0, 0.0, b["out"], res=b["res"], stream=cs)
            ev_done[i].record(cs)
        with torch.cuda.stream(xs):
            xs.wait_event(ev_done[i])
            b["out_h"].copy_(b["out"], non_blocking=True)
            b["res_h"].copy_(b["res"], non_blocking=True)
            ev_out[i].record(xs)
    e1.record(xs)
    torch.cuda.synchronize()
    e_ms = max_over_ranks(e0.elapsed_time(e1), world, dev)
    e2e = {"value": job_throughput(world, args.steps, W * H * D, e_ms), "unit": UNIT,
           "h2d_bytes_per_step": 2 * H * pitch + 4 * H, "d2h_bytes_per_step": 4 * H * W + 64,
           "pairs_per_s": job_throughput(world, args.steps, 1, e_ms) * 1e9,
           "pipeline": "two buffer sets; copies on their own stream overlap the neighbouring steps' compute"}
    res.copy_(slot[(args.steps - 1) % 2]["res"])
    r = sg.stereo_dt_result.from_buffer_copy(res.cpu().numpy().tobytes()[:48])

    # ---- cost-storage variants on the same pair: FP16 / BF16 storage vs the FP32 path
    variants = {}
    wta_ref = None
    nvar = max(3, min(args.steps, 50))
    for name, dtype, form in (("f32", sg.STEREO_F32, sg.STEREO_FUSED_AUTO),
                              ("f32_simt", sg.STEREO_F32, sg.STEREO_FUSED_SIMT),
                              ("f16", sg.STEREO_F16, sg.STEREO_FUSED_AUTO), ("bf16", sg.STEREO_BF16, sg.STEREO_FUSED_AUTO)):
        sv = sg.Stereo(W, H, D, win=win, bil=bil, sigma0=p["sigma0"], sigma1=p["sigma1"], pitch=pitch,
                       cost_dtype=dtype, fused_form=form)
        wta_v = torch.empty((H, W), dtype=torch.int32, device=dev)
        sv.warp_target(tgt, shift, tw)
        sv.cost_aggregate_wta(ref, tw, shift, disp, wta_v, valid)
        evv = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(nvar)]
        sg.stereo_profile_enable(sv.ctx, True)
        for i in range(nvar):
            flush.fill_(i & 0xFF)
            evv[i][0].record(stream)
            sv.warp_target(tgt, shift, tw)
            sv.cost_aggregate_wta(ref, tw, shift, disp, None, valid)
            sv.disparity_transform(disp, valid, 0.0, 0.0, out, res=res)
            evv[i][1].record(stream)
        torch.cuda.synchronize()
        nf, fms = sg.stereo_profile_read(sv.ctx)
        sv.check_device_status()
        sv.close()
        ms = sum(a.elapsed_time(b) for a, b in evv) / nvar
        wv = wta_v.cpu().numpy()
        if wta_ref is None:
            wta_ref = wv
        variants[name] = {"ms_per_step": ms, "pairs_per_s": 1e3 / ms, "gpix_disp_per_s": W * H * D / ms / 1e6,
                          "fused_ms": fms / max(nf, 1), "steps": nvar,
                          "wta_disagree_vs_f32": float(np.mean(wv != wta_ref))}

    # ---- target view + LR-consistency check (eq. lrc) on the same pair
    wta_r = torch.empty((H, W), dtype=torch.int32, device=dev)
    lr_ok = torch.empty((H, W), dtype=torch.uint8, device=dev)
    st.warp_target(tgt, shift, tw)
    st.cost_aggregate_wta(ref, tw, shift, disp, wta_r, valid)
    st.lr_check(ref, tw, shift, wta_r, lr_ok)
    evl = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(nvar)]
    for i in range(nvar):
        flush.fill_(i & 0xFF)
        evl[i][0].record(stream)
        st.lr_check(ref, tw, shift, wta_r, lr_ok)
        evl[i][1].record(stream)
    torch.cuda.synchronize()
    st.check_device_status()
    vm = valid.bool()
    lr = {"ms_per_call": sum(a.elapsed_time(b) for a, b in evl) / nvar, "calls": nvar, "delta_r": 1.0,
          "kept_fraction": float(lr_ok.float().mean()),
          "kept_fraction_of_valid": float(lr_ok[vm].float().mean()) if bool(vm.any()) else None}

    clk = clocks.stop("timed_start", "timed_end")

    if rank != 0:
        st.close()
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return 0

    # ---- roofline of the fused kernel: algorithmic flops per (pixel, d) F = 2k^2 (aggregation)
    # + 11 (cost from window sums) + 2k^2/D (weights and their sum, once per pixel) + 1 (WTA)
    fused_avg_ms = fused_ms / max(n_fused, 1)
    flops_per_unit = 2.0 * bil * bil + 11.0 + 2.0 * bil * bil / D + 1.0
    agg_flops = flops_per_unit * W * H * D
    achieved = agg_flops / (fused_avg_ms * 1e-3) / 1e12
    peak = SM_COUNT_GB300 * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ * 1e6 / 1e12
    traffic = FUSED_TRAFFIC["bytes"] if FUSED_TRAFFIC["sha256"] == kernel_sha() else None
    probe_s, probe_p = sg.stereo_fp32_peak_probe(2)
    roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "traffic": traffic,
            "kernel": "k_fused_sc (cost + bilateral aggregation + WTA + sub-pixel: tensor-core screening with a "
                      "certified bound, FP32 refinement; outputs bit for bit those of the SIMT FP32 kernel)",
            "flops_per_launch": agg_flops, "flops_per_pixel_disparity": flops_per_unit,
            "avg_launch_ms": fused_avg_ms, "launches": n_fused,
            "peak_basis": "152 SMs x 128 FP32 lanes x 2 flop x 2070 MHz (nominal, derived)",
            "fp32_probe_tflops": {"scalar_fma": probe_s / 1e3, "packed_f32x2_fma": probe_p / 1e3},
            "fused_gpix_disp_per_s": W * H * D / (fused_avg_ms * 1e-3) / 1e9}
    # the FP16 / BF16 forms do the same algorithmic work: their share of the same FP32 roofline
    for v in variants.values():
        v["fused_frac_of_fp32_roofline"] = agg_flops / (v["fused_ms"] * 1e-3) / 1e12 / peak
    # the tensor-core forms' executed mma work: per 4 x 4 patch, chunk of 32 disparities and
    # window row, four m16n8k16 (4096 flop each), including the zero-weight K slots (32 x 36
    # tiles of 72 patches; bil <= 13)
    peaks = measured_peaks()
    nks = 4 + 2 * (bil // 2)
    mma_flops = ((W + 31) // 32) * ((H + 35) // 36) * 72 * ((D + 31) // 32) * nks * 4 * 4096.0
    for name in ("f16", "bf16"):
        t_tf = mma_flops / (variants[name]["fused_ms"] * 1e-3) / 1e12
        variants[name]["tensor_mma"] = {
            "tflops": t_tf, "peak": peaks.get("bf16_tflops"), "unit": "TFLOP/s",
            "frac": t_tf / peaks["bf16_tflops"] if peaks.get("bf16_tflops") else None,
            "peak_basis": "measured dense bf16 (same rate for fp16), MEASURED_PEAKS.json",
            "note": "the form is bound by the cost phase and shared memory, not the tensor pipe"}
    variants["kernel"] = {"f32": "k_fused_sc (screened FP32 form; the default)",
                          "f32_simt": "k_fused (the SIMT FP32 form: FP32 weights and accumulators on the CUDA cores)",
                          "f16": "k_fused_sc, plain mode (tensor-core aggregation of the FP16 costs, FP32 accumulators)",
                          "bf16": "k_fused_sc, plain mode (tensor-core aggregation of the BF16 costs, FP32 accumulators)"}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "width": W, "height": H, "max_disp": D, "win": win, "bil": bil,
                       "pairs_per_step_per_gpu": 1, "l2": "flushed before each step (256 MiB write, untimed)"},
            "pairs_per_s": pairs_per_s, "e2e": e2e, "gpu_launches": launches_per_step * args.steps,
            "roofline": roof, "clocks": clk, "cost_storage_variants": variants, "lr_check": lr,
            "dt": {"psi": r.psi, "alpha0": r.alpha0, "alpha1": r.alpha1, "iters": r.iters, "status": r.status,
                   "true_roll": s.roll}}
    if not args.no_batch:
        try:
            line["batch"] = bench_batch(args, dev, stream, flush)
        except Exception as exc:   # the headline line above stands on its own
            line["batch"] = {"error": str(exc)[:300]}
    if not args.no_precision:
        try:
            line["precision"] = bench_precision(args, dev, stream, flush, peak)
        except Exception as exc:   # the headline line above stands on its own
            line["precision"] = {"error": str(exc)[:300]}
    if not args.no_diff:
        try:
            line["differentiation"] = bench_diff(args, dev, stream, flush)
        except Exception as exc:   # the headline line above stands on its own
            line["differentiation"] = {"error": str(exc)[:300]}
    if not args.no_cpu_baseline and world == 1:
        line["cpu_baseline"] = cpu_baseline_sample(s, args.cpu_seconds)
    st.close()
    print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
