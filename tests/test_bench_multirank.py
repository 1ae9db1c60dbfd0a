"""Multi-rank host logic of bench.py on CPU (gloo, world size 2).

Under torchrun every rank runs an independent replica; the job's time is the
slowest rank's and the reported value counts every rank's units.  Two gloo
ranks with different local times check both.
"""

import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ws, r, local = bench.dist_env()
        local_ms = 100.0 * (rank + 1)            # rank 1 is the slower replica
        ms = bench.max_over_ranks(local_ms, dist)
        value = bench.whole_job_rate(ws, 3, 1.0e9, ms)
        out[rank] = (ws, r, local, ms, value)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_replicas_max_time_and_whole_job_value():
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        ws, r, local, ms, value = res[rank]
        assert (ws, r, local) == (world, rank, rank)
        assert ms == 200.0                          # slowest rank's time on every rank
        assert value == pytest.approx(2 * 3 * 1.0e9 / 0.2)


def test_single_process_needs_no_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(12.5, None) == 12.5
    assert bench.whole_job_rate(1, 2, 1e6, 1000.0) == pytest.approx(2e6)


def test_served_phase_failure_is_reported_not_raised():
    """The served phase runs in a child process; its failure comes back as an error field
    (here: no CUDA device on this machine) and leaves the caller unaffected."""
    if torch.cuda.is_available():
        pytest.skip("checks the failure path on a machine without a GPU")
    sys.path.insert(0, ROOT)
    import bench
    out = bench.served_isolated(2, 2.0, 0, timeout_s=240)
    assert set(out) == {"error"} and "exited" in out["error"]
