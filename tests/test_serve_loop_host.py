"""Request loop (paper_2208_10978_gb300.serve.Server) on the host, with its device work faked.

The loop's threads, admission core, resident-table ledger and teardown are
real; only the three device hooks (stream creation and the two evaluation
calls) are replaced by host stand-ins, so no GPU is needed:

* close() while requests are queued and one is inside an evaluation waits for
  that evaluation, then resolves every request that never ran with an error;
* close() while a worker is stuck inside a call keeps the admission core and
  the resident tables (a worker may still use them) and raises; once the
  worker returns, close() succeeds;
* with a budget that holds few problems' tables, unused problems are released
  least recently used first, the loop drops their handles, and the ledger
  never exceeds the budget.
"""

import threading
import time

import numpy as np
import pytest

import paper_2208_10978_gb300 as q2
from paper_2208_10978_gb300 import serve
from synth.workloads import uccsd_energy


class HostServer(serve.Server):
    """Server whose evaluations are host stand-ins gated by an event."""

    def __init__(self, *a, gate=None, **kw):
        self.gate = gate or threading.Event()
        self.calls = []
        super().__init__(*a, **kw)

    def _device_index(self, device):
        return 0

    def _make_stream(self):
        return None

    def _run_large(self, job, stream, ws):
        self.calls.append(job.rid)
        assert self.gate.wait(timeout=30)
        return 1.0 + job.rid, None, ws

    def _run_batch(self, batch, stream, ws):
        assert self.gate.wait(timeout=30)
        return np.array([2.0 + j.rid for j in batch]), [None] * len(batch), ws


@pytest.fixture(scope="module")
def problems():
    out = []
    for seed in range(4):
        w = uccsd_energy(14, 7, seed=seed, kind="spin_conserving")
        out.append(serve.problem_from_workload(w, key=1000 + seed))
    return out


def test_close_waits_for_running_and_fails_queued(problems):
    gate = threading.Event()
    srv = HostServer(budget_bytes=2**34, max_slots=1, n_streams=1, gate=gate)
    p = problems[0]
    futs = [srv.submit(i, p, np.zeros(p.n_params), False) for i in range(5)]
    deadline = time.time() + 10
    while not srv.calls and time.time() < deadline:
        time.sleep(0.01)
    assert srv.calls == [0]                       # one request inside an evaluation, four queued
    closer = threading.Thread(target=srv.close, kwargs={"timeout_s": 20})
    closer.start()
    time.sleep(0.2)
    assert closer.is_alive()                      # close() waits for the running evaluation
    gate.set()
    closer.join(timeout=30)
    assert not closer.is_alive()
    res = [f.result(timeout=5) for f in futs]
    assert res[0].status == q2.Q2_OK and res[0].energy == 1.0
    closed = [r for r in res if r.status != q2.Q2_OK]
    assert closed and all("server closed" in r.error for r in closed)
    assert all(r.status == q2.Q2_OK for r in res if r.rid in srv.calls)
    assert srv._core is None and not srv._tables
    with pytest.raises(RuntimeError):
        srv.submit(99, p, np.zeros(p.n_params), False)


def test_close_keeps_core_while_a_worker_is_stuck(problems):
    gate = threading.Event()
    srv = HostServer(budget_bytes=2**34, max_slots=2, n_streams=1, gate=gate)
    p = problems[1]
    fut = srv.submit(1, p, np.zeros(p.n_params), True)
    deadline = time.time() + 10
    while not srv.calls and time.time() < deadline:
        time.sleep(0.01)
    with pytest.raises(RuntimeError, match="still running"):
        srv.close(timeout_s=0.3)
    assert srv._core is not None and p.key in srv._tables
    assert srv.stats()["running"] == 1
    gate.set()                                    # the worker returns and completes on the kept core
    assert fut.result(timeout=10).status == q2.Q2_OK
    srv.close(timeout_s=10)
    assert srv._core is None


def test_unused_problem_tables_are_released_lru(problems):
    gate = threading.Event()
    gate.set()
    probe = HostServer(budget_bytes=2**34, max_slots=1, n_streams=1, gate=gate)
    hs = probe._handles(problems[0])
    work = probe.footprint(problems[0], False, hs)
    tables = probe.table_bytes(hs)
    probe.close(timeout_s=10)
    assert tables > 0 and work > 0
    budget = work + int(2.5 * tables)             # room for two problems' tables at most
    srv = HostServer(budget_bytes=budget, max_slots=1, n_streams=1, gate=gate)
    try:
        results = []
        for i in range(12):
            p = problems[i % 4]
            results.append(srv.submit(i, p, np.zeros(p.n_params), False).result(timeout=30))
            assert len(srv._tables) <= 3
        st = srv.stats()
    finally:
        srv.close(timeout_s=10)
    assert all(r.status == q2.Q2_OK for r in results)
    assert st["evictions"] >= 8 and st["resident_problems"] <= 2
    assert st["high_water_bytes"] <= budget and st["table_bytes"] <= 2.5 * tables


def test_a_dead_loop_fails_new_requests_at_once(problems):
    """When a loop dies on an error it cannot report per request (for instance a sticky device
    error), every pending request is resolved with that error and later requests fail at once
    instead of waiting in the queue."""

    class Dying(HostServer):
        def _run_large(self, job, stream, ws):
            raise RuntimeError("device context lost")

    srv = Dying(budget_bytes=2**34, max_slots=4, n_streams=1)
    p = problems[2]
    try:
        first = srv.submit(1, p, np.zeros(p.n_params), False).result(timeout=10)
        assert first.status != q2.Q2_OK and "device context lost" in first.error
        later = srv.submit(2, p, np.zeros(p.n_params), False).result(timeout=1)
        assert later.status != q2.Q2_OK and "server loop stopped" in later.error
    finally:
        srv._threads = [t for t in srv._threads if t.is_alive()]
        srv.close(timeout_s=10)
