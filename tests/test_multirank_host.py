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
