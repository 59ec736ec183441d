"""Batches of uneven pairs: one persistent fused launch over all pairs inside a captured
CUDA graph.  Every pair's outputs must equal (bit for bit) what the single-pair calls give,
for every tile configuration the autotuner can choose, and after a graph replay on new
image contents; one pair is also checked against the oracle."""
import math
import os

import numpy as np
import pytest
import torch

import oracle
import paper_1904_06017_gb300 as sg
import synth
from gpu_helpers import check_disparity, dev_f32, dev_img, pitch_of

pytestmark = pytest.mark.gpu

SIZES = [(160, 120, 32), (211, 97, 16), (300, 180, 48), (96, 64, 24), (257, 140, 40)]


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1904_06017_gb300 import build
    build.build()
    oracle.build()


def scenes(seed0=500):
    return [synth.make_scene(W, H, D, seed0 + i, roll=math.radians(2.0 * (i - 2)), coeffs=(6.0, 0.1, 0.0),
                             n_potholes=1, warp=True, win=7, bil=9) for i, (W, H, D) in enumerate(SIZES)]


def buffers(s, D):
    H, W = s.height, s.width
    pitch = pitch_of(W)
    return dict(ref=dev_img(s.ref, pitch), tgt=dev_img(s.tgt, pitch), shift=dev_f32(s.shift),
                tgt_warped=torch.zeros((H, pitch), dtype=torch.uint8, device="cuda"),
                disp=torch.zeros((H, W), dtype=torch.float32, device="cuda"),
                valid=torch.zeros((H, W), dtype=torch.uint8, device="cuda"),
                disp_out=torch.zeros((H, W), dtype=torch.float32, device="cuda"),
                res=torch.zeros(64, dtype=torch.uint8, device="cuda"), max_disp=D)


def single(q, W, H, D, dtype=sg.STEREO_F32):
    pitch = q["ref"].shape[1]
    tw = torch.empty_like(q["tgt"])
    disp = torch.empty((H, W), dtype=torch.float32, device="cuda")
    valid = torch.empty((H, W), dtype=torch.uint8, device="cuda")
    out = torch.empty_like(disp)
    with sg.Stereo(W, H, D, win=7, bil=9, sigma0=3.0, sigma1=10.0, pitch=pitch, cost_dtype=dtype) as st:
        st.warp_target(q["tgt"], q["shift"], tw)
        st.cost_aggregate_wta(q["ref"], tw, q["shift"], disp, None, valid)
        r = st.disparity_transform(disp, valid, 0.0, 0.0, out)
    return disp.cpu().numpy(), valid.cpu().numpy(), out.cpu().numpy(), r


def run_batch(ss, dtype=sg.STEREO_F32, wc=2, dc=12, win=7, bil=9):
    qs = [buffers(s, D) for s, (_, _, D) in zip(ss, SIZES)]
    with sg.StereoBatch(qs, win=win, bil=bil, sigma0=3.0, sigma1=10.0, cost_dtype=dtype, tile_wc=wc,
                        tile_dc=dc) as b:
        b.run()
        torch.cuda.synchronize()
        b.check_device_status()
        cfg = b.config()
    outs = [(q["disp"].cpu().numpy(), q["valid"].cpu().numpy(), q["disp_out"].cpu().numpy(),
             sg.stereo_dt_result.from_buffer_copy(q["res"].cpu().numpy().tobytes()[:48])) for q in qs]
    return outs, cfg, qs


def test_batch_equals_single_pair_calls():
    ss = scenes()
    outs, cfg, qs = run_batch(ss)
    assert cfg["tile_wc"] == 2 and cfg["tile_dc"] == 12 and cfg["source"] == "parameters"
    for (W, H, D), q, (d, v, o, r) in zip(SIZES, qs, outs):
        d1, v1, o1, r1 = single(q, W, H, D)
        assert np.array_equal(d, d1) and np.array_equal(v, v1)
        assert r.status == r1.status and r.psi == r1.psi and np.array_equal(o, o1)
    s = ss[2]
    tw = oracle.warp(s.tgt, s.shift)
    d_o, ds_o, eb, es = oracle.stereo(s.ref, tw, s.shift, SIZES[2][2], 7, 9, 3.0, 10.0)
    check_disparity(outs[2][0], None, d_o, ds_o, eb, es, min_sure=0.8)


@pytest.mark.parametrize("wc,dc", [(1, 12), (4, 12), (2, 4), (8, 12), (32, 32)])
def test_every_tile_configuration_gives_the_same_result(wc, dc):
    """5 x 5 windows, where the 128 x 16 tile's shared memory fits too; wc = 8 is the
    warp-specialised kernel (producer and consumer warps, two cost buffers); wc = 32 the
    screened form (screening kernel, then the refinement kernel over the same work list)."""
    ss = scenes()
    ref, _, _ = run_batch(ss, win=5, bil=5)
    got, cfg, _ = run_batch(ss, wc=wc, dc=dc, win=5, bil=5)
    assert cfg["tile_wc"] == wc and cfg["tile_dc"] == dc
    for a, b in zip(ref, got):
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])


@pytest.mark.parametrize("wc", [2, 8, 32])
def test_many_tiles_per_cta_with_mixed_search_ranges(wc):
    """More tiles than CTAs, pairs of different search ranges interleaved in the work list:
    every CTA moves between pairs whose shared-memory layouts differ."""
    sizes = [(640, 480, 32), (960, 540, 64), (640, 480, 128), (960, 540, 32)] * 4
    ss = [synth.make_scene(W, H, D, 700 + i, roll=0.02, coeffs=(6.0, 0.1, 0.0), n_potholes=0, warp=True,
                           win=5, bil=5) for i, (W, H, D) in enumerate(sizes)]
    qs = [buffers(s, D) for s, (_, _, D) in zip(ss, sizes)]
    with sg.StereoBatch(qs, win=5, bil=5, sigma0=3.0, sigma1=10.0, tile_wc=wc, tile_dc=32 if wc == 32 else 12) as b:
        assert b.config()["items"] > 4 * 152
        b.run()
        torch.cuda.synchronize()
        b.check_device_status()
    for (W, H, D), q in zip(sizes[:4], qs[:4]):
        pitch = q["ref"].shape[1]
        tw = torch.empty_like(q["tgt"])
        disp = torch.empty((H, W), dtype=torch.float32, device="cuda")
        with sg.Stereo(W, H, D, win=5, bil=5, sigma0=3.0, sigma1=10.0, pitch=pitch) as st:
            st.warp_target(q["tgt"], q["shift"], tw)
            st.cost_aggregate_wta(q["ref"], tw, q["shift"], disp)
        assert np.array_equal(q["disp"].cpu().numpy(), disp.cpu().numpy())


def test_warp_specialised_kernel_at_the_default_windows():
    """7 x 7 blocks, 9 x 9 bilateral window: the producer/consumer kernel equals the one-phase
    kernel bit for bit (same integer costs, same FP32 accumulation order per pixel)."""
    ss = scenes()
    ref, _, _ = run_batch(ss)
    got, cfg, _ = run_batch(ss, wc=8, dc=12)
    assert cfg["tile_wc"] == 8
    for a, b in zip(ref, got):
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])


def test_autotuner_and_its_cache(tmp_path, monkeypatch):
    cache = tmp_path / "tune.json"
    monkeypatch.setenv("STEREO_AUTOTUNE_CACHE", str(cache))
    ss = scenes()
    ref, _, _ = run_batch(ss)
    got, cfg, _ = run_batch(ss, wc=0, dc=0)
    assert cfg["source"] == "autotune timing" and cache.exists()
    import json
    entries = json.loads(cache.read_text())
    assert len(entries) == 1 and list(entries.values())[0]["wc"] == cfg["tile_wc"]
    got2, cfg2, _ = run_batch(ss, wc=0, dc=0)
    assert cfg2["source"] == "autotune cache" and cfg2["tile_wc"] == cfg["tile_wc"]
    for a, b in zip(ref, got2):
        assert np.array_equal(a[0], b[0])


def test_graph_replay_sees_new_inputs_and_fp16_batch():
    ss = scenes()
    qs = [buffers(s, D) for s, (_, _, D) in zip(ss, SIZES)]
    with sg.StereoBatch(qs, win=7, bil=9, sigma0=3.0, sigma1=10.0, tile_wc=2, tile_dc=12) as b:
        b.run()
        torch.cuda.synchronize()
        # new contents in the same buffers: swap in other scenes of the same sizes
        ss2 = scenes(seed0=900)
        for q, s in zip(qs, ss2):
            q["ref"][:, :s.width].copy_(torch.from_numpy(s.ref))
            q["tgt"][:, :s.width].copy_(torch.from_numpy(s.tgt))
            q["shift"].copy_(torch.from_numpy(s.shift))
        b.run()
        b.run()
        torch.cuda.synchronize()
        for (W, H, D), q in zip(SIZES, qs):
            d1, v1, o1, _ = single(q, W, H, D)
            assert np.array_equal(q["disp"].cpu().numpy(), d1) and np.array_equal(q["disp_out"].cpu().numpy(), o1)
    h, _, _ = run_batch(ss, dtype=sg.STEREO_F16)
    f, _, _ = run_batch(ss)
    total = sum(a[0].size for a in f)
    diff = sum(int(np.count_nonzero(np.rint(a[0]) != np.rint(b[0]))) for a, b in zip(f, h))
    assert diff / total <= 5e-3
