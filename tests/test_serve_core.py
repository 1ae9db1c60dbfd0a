"""Admission core of the request loop (include/q2_serve.h), on the host.

FIFO admission by bytes against the budget with a slot limit, later requests
passing a head that does not fit, queue timeouts, release on completion and
latency percentiles; resident problem tables charged once per problem and
released least recently used first when room is needed; every wait is
simulated with caller-supplied times.
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
    out = (ctypes.c_double * 14)()
    assert L.q2_server_stats(h, out) == 0
    return list(out)


def test_admission_by_bytes_and_slots(core):
    L, make = core
    h = make(100, 3, 10.0)
    for rid, b in [(1, 60), (2, 50), (3, 30), (4, 10), (5, 5)]:
        assert L.q2_server_submit(h, rid, b, rid, 0, 0.0) == 0
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
            assert L.q2_server_submit(h, rid, rnd.randint(1, 600), rnd.randint(0, 20), rnd.randint(0, 50), t) == 0
        running += _admit(L, h, t)
        assert _stats(L, h)[6] <= 1000
        _evicted(L, h)
        if running and rnd.random() < 0.6:
            done = running.pop(rnd.randrange(len(running)))
            assert L.q2_server_complete(h, done, t + 0.5) == 0
    assert _stats(L, h)[7] <= 1000


def test_queue_timeout_and_errors(core):
    L, make = core
    h = make(100, 1, 5.0)
    assert L.q2_server_submit(h, 1, 80, 1, 0, 0.0) == 0
    assert L.q2_server_submit(h, 2, 80, 2, 0, 1.0) == 0
    assert L.q2_server_submit(h, 3, 101, 3, 0, 1.0) == q2.Q2_ERR_OOM       # larger than the budget
    assert L.q2_server_submit(h, 4, 60, 4, 41, 1.0) == q2.Q2_ERR_OOM      # with its tables
    assert L.q2_server_submit(h, 1, 10, 1, 0, 1.0) == q2.Q2_ERR_INVALID    # repeated id
    assert _admit(L, h, 1.0) == [1]
    assert _expire(L, h, 5.5) == []                                 # waited 4.5 s
    assert _expire(L, h, 6.5) == [2]                                # waited 5.5 s > 5
    assert L.q2_server_complete(h, 2, 7.0) == q2.Q2_ERR_INVALID     # never admitted
    assert _stats(L, h)[3] == 1


def _evicted(L, h, cap=64):
    ids = (ctypes.c_int64 * cap)()
    k = L.q2_server_take_evicted(h, ids, cap)
    return [ids[i] for i in range(k)]


def test_tables_charged_once_per_problem_and_evicted_lru(core):
    L, make = core
    h = make(100, 8, 1e9)
    # problem 7 (tables 20) twice, problem 8 (tables 30): 7's tables count once
    assert L.q2_server_submit(h, 1, 10, 7, 20, 0.0) == 0
    assert L.q2_server_submit(h, 2, 10, 7, 20, 0.0) == 0
    assert L.q2_server_submit(h, 3, 10, 8, 30, 0.0) == 0
    assert _admit(L, h, 0.1) == [1, 2, 3]
    s = _stats(L, h)
    assert s[6] == 10 + 10 + 10 + 20 + 30 and s[11] == 50 and s[12] == 2
    for rid, t in [(1, 1.0), (2, 1.0), (3, 2.0)]:
        assert L.q2_server_complete(h, rid, t) == 0
    s = _stats(L, h)
    assert s[6] == 50 and s[11] == 50              # tables stay resident after their requests
    assert _evicted(L, h) == []
    # a request for a new problem 9 (tables 40, workspace 30) needs 120 > 100:
    # the least recently used unused problem (7, last used at 1.0) is released first
    assert L.q2_server_submit(h, 4, 30, 9, 40, 3.0) == 0
    assert _admit(L, h, 3.1) == [4]
    assert _evicted(L, h) == [7]
    s = _stats(L, h)
    assert s[6] == 30 + 30 + 40 and s[11] == 70 and s[13] == 1
    # problem 8 is still resident: a request for it is charged its workspace only
    assert L.q2_server_submit(h, 5, 0, 8, 30, 3.5) == 0
    assert _admit(L, h, 3.6) == [5]
    assert _evicted(L, h) == []
    assert L.q2_server_complete(h, 5, 4.0) == 0
    # problem 9 is in use (request 4 running): it is never released; 8 is
    assert L.q2_server_submit(h, 6, 30, 10, 0, 5.0) == 0
    assert _admit(L, h, 5.1) == [6]
    assert _evicted(L, h) == [8]
    assert _stats(L, h)[7] <= 100


def test_queued_problem_tables_are_not_released(core):
    L, make = core
    h = make(100, 1, 1e9)
    assert L.q2_server_submit(h, 1, 50, 1, 40, 0.0) == 0
    assert _admit(L, h, 0.0) == [1]
    assert L.q2_server_complete(h, 1, 1.0) == 0       # problem 1 resident (40), unused
    assert L.q2_server_submit(h, 2, 10, 1, 40, 2.0) == 0   # queued again: problem 1 in use
    assert L.q2_server_submit(h, 3, 70, 2, 0, 2.0) == 0
    # slot limit 1: request 2 is admitted; 3 cannot be (slot), and 1's tables are never released
    assert _admit(L, h, 2.1) == [2]
    assert _evicted(L, h) == []
    assert L.q2_server_complete(h, 2, 3.0) == 0
    assert _admit(L, h, 3.1) == [3]                    # 40 + 70 > 100: problem 1 (now unused) released
    assert _evicted(L, h) == [1]
