"""Admission core of the request loop (include/q2_serve.h), on the host.

FIFO admission by bytes against the budget with a slot limit, later requests
passing a head that does not fit, queue timeouts, release on completion and
latency percentiles; every wait is simulated with caller-supplied times.
"""

import ctypes

import pytest

import paper_2208_10978_gb300 as q2
from paper_2208_10978_gb300.serve import _setup_core


@pytest.fixture
def core():
    L = _setup_core()
    made = []

    def make(budget, slots, timeout):
        h = ctypes.c_void_p()
        assert L.q2_server_create(budget, slots, timeout, ctypes.byref(h)) == 0
        made.append(h)
        return h
    yield L, make
    for h in made:
        L.q2_server_destroy(h)


def _admit(L, h, t, cap=64):
    ids = (ctypes.c_int64 * cap)()
    k = L.q2_server_admit(h, t, ids, cap)
    return [ids[i] for i in range(k)]


def _expire(L, h, t, cap=64):
    ids = (ctypes.c_int64 * cap)()
    k = L.q2_server_expire(h, t, ids, cap)
    return [ids[i] for i in range(k)]


def _stats(L, h):
    out = (ctypes.c_double * 11)()
    assert L.q2_server_stats(h, out) == 0
    return list(out)


def test_admission_by_bytes_and_slots(core):
    L, make = core
    h = make(100, 3, 10.0)
    for rid, b in [(1, 60), (2, 50), (3, 30), (4, 10), (5, 5)]:
        assert L.q2_server_submit(h, rid, b, 0.0) == 0
    # 1 fits (60); 2 does not (110 > 100) and is passed; 3 fits (90); 4 fits (100); slots full
    assert _admit(L, h, 0.1) == [1, 3, 4]
    s = _stats(L, h)
    assert s[6] == 100 and s[7] == 100 and s[5] == 3 and s[4] == 2
    assert _admit(L, h, 0.2) == []
    assert L.q2_server_complete(h, 1, 1.0) == 0
    assert _admit(L, h, 1.1) == [2]            # 40 + 50 = 90 <= 100, FIFO head first
    assert L.q2_server_complete(h, 3, 2.0) == 0
    assert _admit(L, h, 2.1) == [5]
    for rid, t in [(2, 3.0), (4, 3.0), (5, 3.5)]:
        assert L.q2_server_complete(h, rid, t) == 0
    s = _stats(L, h)
    assert s[2] == 5 and s[6] == 0 and s[7] == 100
    assert s[8] == pytest.approx(3.0) and s[9] == pytest.approx(3.5)


def test_high_water_never_exceeds_budget(core):
    import random
    L, make = core
    h = make(1000, 8, 1e9)
    rnd = random.Random(0)
    running = []
    rid = 0
    for step in range(400):
        t = float(step)
        for _ in range(rnd.randint(0, 3)):
            rid += 1
            assert L.q2_server_submit(h, rid, rnd.randint(1, 600), t) == 0
        running += _admit(L, h, t)
        assert _stats(L, h)[6] <= 1000
        if running and rnd.random() < 0.6:
            done = running.pop(rnd.randrange(len(running)))
            assert L.q2_server_complete(h, done, t + 0.5) == 0
    assert _stats(L, h)[7] <= 1000


def test_queue_timeout_and_errors(core):
    L, make = core
    h = make(100, 1, 5.0)
    assert L.q2_server_submit(h, 1, 80, 0.0) == 0
    assert L.q2_server_submit(h, 2, 80, 1.0) == 0
    assert L.q2_server_submit(h, 3, 101, 1.0) == q2.Q2_ERR_OOM       # larger than the budget
    assert L.q2_server_submit(h, 1, 10, 1.0) == q2.Q2_ERR_INVALID    # repeated id
    assert _admit(L, h, 1.0) == [1]
    assert _expire(L, h, 5.5) == []                                 # waited 4.5 s
    assert _expire(L, h, 6.5) == [2]                                # waited 5.5 s > 5
    assert L.q2_server_complete(h, 2, 7.0) == q2.Q2_ERR_INVALID     # never admitted
    assert _stats(L, h)[3] == 1
