"""The multi-process path of the benchmark, on CPU: two gloo ranks on 127.0.0.1.

With N GPUs every rank runs an independent replica of the workload (weak scaling, no
data-path collective); the benchmark takes the slowest rank's time and counts the units of
all ranks.  These tests run that reduction with world size 2, and check that the reference
arm leaves every rank but 0 without work.
"""
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, times, out):
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        t = bench.max_over_ranks(times[rank], dist, torch.device("cpu"))
        dist.barrier()
        out.put((rank, t, bench.whole_job_rate(ws, 1000, t)))
    finally:
        dist.destroy_process_group()


def test_slowest_rank_time_and_whole_job_rate_world_size_2():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    times = [2.0, 5.0]
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, times, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[0] for r in res] == [0, 1]
    for _, t, rate in res:
        assert t == 5.0              # every rank sees the slowest rank's time
        assert rate == 2 * 1000 / 5.0  # units of both ranks over that time


def test_single_process_reduction_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, None, None) == 3.5
    assert bench.whole_job_rate(1, 700, 2.0) == 350.0


def test_reference_arm_on_other_ranks_exits_without_work():
    env = dict(os.environ, RANK="1", LOCAL_RANK="1", WORLD_SIZE="2", MASTER_ADDR="127.0.0.1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "0"], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""


def test_reference_arm_prints_the_contract_line():
    """One rank, one bench step of the oracle: the JSON line carries the contract's keys, the
    same workload description as the GPU arm, and no unformatted field."""
    import json
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    line = json.loads(r.stdout.strip().splitlines()[-1])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"):
        assert key in line
    assert line["impl"] == "reference" and line["value"] > 0 and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
    sys.path.insert(0, ROOT)
    import bench
    import synth
    assert line["config"] == bench.workload_config(synth.WORKLOADS["c2"])
    assert "%" not in json.dumps(line["config"])


def test_cpu_baseline_entry():
    """The GPU arm's cpu_baseline entry: the oracle timed on a bounded sample of the workload."""
    sys.path.insert(0, ROOT)
    import bench
    import synth
    cb = bench.cpu_baseline(synth.WORKLOADS["c2"], target_s=0.5)
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["value"] > 0 and cb["unit"] == bench.UNIT
    assert cb["sample"].startswith("1 of the 100 FP64 time steps")
