"""bench.py's multi-rank host logic on CPU: two gloo ranks (world_size 2), no GPU.

Under torchrun every rank times its own pairs; the job's time is the slowest rank's and the
job's throughput counts the units of all ranks.  The reference arm runs on rank 0 only."""
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, times, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t_max = bench.max_over_ranks(times[rank], world, "cpu")
    out.put((rank, t_max, bench.job_throughput(world, 10, 1000, t_max)))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_and_job_throughput_with_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    times = [12.5, 40.0]        # ms: rank 1 is the slow one
    procs = [ctx.Process(target=_rank, args=(r, 2, port, times, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t_max, value in res:
        assert t_max == 40.0
        # 2 ranks x 10 steps x 1000 units in 40 ms
        assert value == pytest.approx(2 * 10 * 1000 / 0.040 / 1e9)


def test_single_rank_is_the_local_value():
    assert bench.max_over_ranks(7.25, 1) == 7.25
    assert bench.job_throughput(1, 4, 2e9, 1000.0) == pytest.approx(8.0)


def test_reference_arm_runs_on_rank_0_only(tmp_path):
    """A rank other than 0 of `bench.py --impl reference` exits 0 at once, printing nothing."""
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0
    assert r.stdout.strip() == ""


def test_reference_rows_fit_the_budget():
    import synth
    import oracle
    oracle.build()
    s = synth.make_scene(256, 64, 16, 5, warp=True)
    assert 1 <= bench.reference_rows(s, 1000, budget_s=0.01) <= 2
    assert bench.reference_rows(s, 1, budget_s=1e6) == 16


def test_reference_arm_prints_the_contract_line():
    """Rank 0 of `bench.py --impl reference` times the oracle on bands of the benchmark pair and
    prints one JSON line in the same metric, unit and direction as the GPU arm, with the
    oracle's run described under cpu_baseline and an end-to-end figure equal to its value."""
    import json
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "1"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["higher_is_better"] is True and d["steps"] == 1 and d["warmup"] == 1
    assert d["value"] > 0 and d["ms_per_step"] > 0 and d["vs_baseline"] is None
    assert d["config"]["workload"].startswith("road-stereo 1920x1080 D=128")
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0
