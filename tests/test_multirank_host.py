"""The N > 1 path of bench.py without a GPU: replicas on world_size 2 with
the gloo backend.  Each rank runs the whole workload on its own device; the
job's time is the slowest rank's and its bytes are the sum over ranks; the
reference arm runs on rank 0 only."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r, local = bench.dist_env()
        ms, nbytes = bench.reduce_over_ranks(dist, torch.device("cpu"), 10.0 + 5.0 * rank, 100.0 * (rank + 1))
        dist.barrier()
        q.put((r, w, local, ms, nbytes))
    finally:
        dist.destroy_process_group()


def test_two_replicas_take_the_slowest_time_and_all_bytes():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    results = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[0] for r in results] == [0, 1]
    for rank, world, local, ms, nbytes in results:
        assert world == 2 and local == rank
        assert ms == 15.0 and nbytes == 300.0


def test_single_process_passes_through():
    import bench
    assert bench.reduce_over_ranks(None, None, 12.5, 7.0) == (12.5, 7.0)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setattr("sys.argv", ["bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0"])
    args = bench.parse()
    assert bench.run_reference(args) is None        # returns at once, no work


def test_reference_arm_line_on_a_small_square():
    """bench.py --impl reference, run as the driver runs it (a process of its
    own, no GPU), prints one JSON line with the contract's keys; the oracle
    sample is timed on one thread and moves no host<->device bytes."""
    import json
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = {k: v for k, v in os.environ.items() if k not in ("RANK", "WORLD_SIZE", "LOCAL_RANK")}
    res = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--n", "129",
                          "--steps", "2", "--warmup", "3"], cwd=root, env=env, capture_output=True, text=True,
                         timeout=600)
    assert res.returncode == 0, res.stderr[-2000:]
    lines = [ln for ln in res.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, res.stdout
    d = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["n_gpus"] == 1 and d["steps"] == 2 and d["warmup"] == 3
    assert d["unit"] == "GB/s" and d["higher_is_better"] is True and d["value"] > 0.0
    assert d["config"]["workload"] == "square129_jitter0.2_nu1_tri"
    assert d["config"]["n_nodes"] == 129 * 129 and d["config"]["n_elements"] == 2 * 128 * 128
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
