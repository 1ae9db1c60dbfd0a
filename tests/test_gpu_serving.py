"""Serving path: batched small-state kernel and the continuous-batching loop.

* q2_batch_energy_grad (one persistent launch, one CTA per request) agrees
  with q2_vqe_energy_grad (tile kernels) and the oracle;
* a request's result is bit-for-bit the same alone and inside a batch;
* a stream of overlapping requests (10..18 qubits, 40% with gradient) served
  through paper_2208_10978_gb300.serve gives, request by request, the same
  result as evaluating it alone; complex64 served energies agree with the
  complex128 path within 1e-5 Ha; the ledger never exceeds its budget;
* a starved queue reports timeouts instead of waiting forever.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2208_10978_gb300 as q2
from paper_2208_10978_gb300 import serve
from oracle import statevector as sv
from synth.workloads import uccsd_energy, served_stream

pytestmark = pytest.mark.gpu


def _handles(w):
    return q2.Ansatz.from_uccsd(w.ansatz), q2.Hamiltonian(w.n, w.ham.x, w.ham.z, w.ham.c)


@pytest.mark.parametrize("dtype", ["complex128", "complex64"])
def test_batch_matches_tile_path_and_oracle(dtype):
    ws = [uccsd_energy(n, n // 2, seed=s) for n, s in [(8, 0), (10, 1), (12, 2), (8, 3), (6, 4)]]
    hs = [_handles(w) for w in ws]
    rng = np.random.default_rng(9)
    thetas = [rng.normal(0, 0.2, size=w.ansatz.n_params) for w in ws]
    wg = [True, False, True, True, False]
    e, g, _ = q2.batch_energy_grad([h[0] for h in hs], [h[1] for h in hs], thetas, wg, dtype=dtype)
    tol_e, tol_g = (1e-11, 1e-10) if dtype == "complex128" else (1e-5, 1e-4)
    for b, (w, h) in enumerate(zip(ws, hs)):
        e_t, g_t, _ = q2.vqe_energy_grad(h[0], h[1], thetas[b], dtype="complex128", want_grad=wg[b])
        assert abs(e[b] - e_t) < tol_e
        if wg[b]:
            assert np.max(np.abs(g[b] - g_t)) < tol_g
        else:
            assert g[b] is None
    a = ws[0].ansatz
    e_ref, gphi = sv.energy_and_gradient(8, 4, a.x, a.z, a.angles(thetas[0]), ws[0].ham.x, ws[0].ham.z, ws[0].ham.c)
    assert abs(e[0] - e_ref) < tol_e
    assert np.max(np.abs(g[0] - sv.fold_to_theta(gphi, a.param, a.coef, a.n_params))) < tol_g


def test_batch_result_same_alone_and_in_batch():
    ws = [uccsd_energy(n, n // 2, seed=s) for n, s in [(12, 5), (10, 6), (8, 7), (12, 8)] * 8]
    hs = [_handles(w) for w in ws[:4]] * 8
    rng = np.random.default_rng(3)
    thetas = [rng.normal(0, 0.2, size=w.ansatz.n_params) for w in ws]
    wg = [bool(i % 3) for i in range(len(ws))]
    e, g, _ = q2.batch_energy_grad([h[0] for h in hs], [h[1] for h in hs], thetas, wg)
    for b in (0, 5, 13, 31):
        e1, g1, _ = q2.batch_energy_grad([hs[b][0]], [hs[b][1]], [thetas[b]], [wg[b]])
        assert e1[0] == e[b]
        if wg[b]:
            assert np.array_equal(g1[0], g[b])


@pytest.fixture(scope="module")
def stream_problems():
    reqs = [r for r in served_stream(seed=1, n_requests=400, rate_per_s=400.0,
                                     n_choices=(10, 12, 14, 16, 18))][:40]
    problems, thetas = {}, {}
    for r in reqs:
        if r.problem_seed not in problems:
            w = uccsd_energy(r.n, r.n_elec, seed=r.problem_seed % 100000)
            problems[r.problem_seed] = serve.problem_from_workload(w, key=r.problem_seed)
            thetas[r.problem_seed] = w.theta
    return reqs, problems, thetas


def test_served_stream_same_as_alone(stream_problems):
    reqs, problems, thetas = stream_problems
    budget = 8 * 2**30
    srv = serve.Server(dtype="complex64", budget_bytes=budget, max_slots=16, n_streams=4)
    try:
        results, wall = serve.serve_stream(srv, reqs, problems, thetas, speed=1.0, wait_s=300)
        st = srv.stats()
    finally:
        srv.close()
    bad = [(r.rid, r.status, r.path, r.error) for r in results.values() if r.status != q2.Q2_OK]
    assert not bad, bad[:4]
    assert st["completed"] == len(reqs) and st["high_water_bytes"] <= budget
    assert st["p99_s"] >= st["p50_s"] > 0
    paths = {r.path for r in results.values()}
    assert paths == {"batch", "stream"}
    # requests overlapped on the device: some started before others finished
    spans = sorted((r.t_submit, r.t_done) for r in results.values())
    assert any(spans[i + 1][0] < spans[i][1] for i in range(len(spans) - 1))
    cache = {}
    for r in reqs:
        p = problems[r.problem_seed]
        if p.key not in cache:
            cache[p.key] = (q2.Ansatz(p.n, p.n_elec, p.rot_x, p.rot_z, p.rot_param, p.rot_coef, p.n_params),
                            q2.Hamiltonian(p.n, p.ham_x, p.ham_z, p.ham_c))
        e1, g1 = serve.evaluate_alone(p, thetas[r.problem_seed], r.want_grad, "complex64", cache[p.key])
        got = results[r.rid]
        assert abs(got.energy - e1) <= 1e-12 * max(1.0, abs(e1)), r.rid
        if r.want_grad:
            assert np.max(np.abs(got.grad - g1)) <= 1e-12
        e2, _ = serve.evaluate_alone(p, thetas[r.problem_seed], False, "complex128", cache[p.key])
        assert abs(got.energy - e2) < 1e-5


def test_starved_queue_times_out(stream_problems):
    reqs, problems, thetas = stream_problems
    big = next(p for p in problems.values() if p.n == 18)
    srv = serve.Server(dtype="complex64", budget_bytes=8 * 2**30, max_slots=1, n_streams=1,
                       queue_timeout_s=0.001)
    try:
        futs = [srv.submit(1000 + i, big, thetas[big.key], True) for i in range(6)]
        res = [f.result(timeout=120) for f in futs]
    finally:
        srv.close()
    status = [r.status for r in res]
    assert q2.Q2_ERR_TIMEOUT in status and q2.Q2_OK in status
