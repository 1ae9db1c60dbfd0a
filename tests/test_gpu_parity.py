"""CUDA path vs the oracle, element by element, through the C ABI.

Sizes span several tiles and a ragged tail (n = 13 with 12-qubit tiles is
two tiles; tile sizes are also shrunk to 8 qubits to force many passes at
small n).  Every state is normalised.  Tolerances, applied as written (no
extra factors):
  complex128: <= 1e-12 max-abs per amplitude and <= 1e-10 Ha in energy (the
    stated FP64 bars);
  complex64: <= 1e-5 Ha in energy (the stated FP32 bar) and <= 2e-6 max-abs
    per amplitude, derived from FP32 rounding: a normalised amplitude is at
    most 1, each combined rotation adds at most a few units of 2^-24
    relative error, and a few hundred sequential rotations per amplitude give
    well under 1e-5 relative, far under 2e-6 absolute at the amplitudes of
    these states (2^-n/2 typical).
  lambda = H psi, per amplitude relative to max(1, max |lambda|): 1e-12
    (complex128; 120 terms of |c| ~ 1 summed in FP64) and 2e-5 (complex64; the
    same sums in FP32, 120 x 2^-24 ~ 7e-6 worst case).
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2208_10978_gb300 as q2
from oracle import statevector as sv
from oracle import c_oracle
from synth.workloads import uccsd_energy

pytestmark = pytest.mark.gpu

TOL_AMP = {"complex128": 1e-12, "complex64": 2e-6}
TOL_E = {"complex128": 1e-10, "complex64": 1e-5}


@pytest.fixture(autouse=True)
def _default_tiles():
    q2.set_tile_qubits("complex64", 12)
    q2.set_tile_qubits("complex128", 11)
    yield
    q2.set_tile_qubits("complex64", 12)
    q2.set_tile_qubits("complex128", 11)


def to_dev(psi, dtype):
    return torch.from_numpy(np.asarray(psi, dtype=np.complex128)).to("cuda", getattr(torch, dtype))


def to_host(t):
    torch.cuda.synchronize()
    return t.to("cpu", torch.complex128).numpy()


@pytest.mark.parametrize("dtype", ["complex64", "complex128"])
@pytest.mark.parametrize("n,ne", [(1, 0), (1, 1), (3, 2), (8, 4), (13, 7)])
def test_init_hf_exact(dtype, n, ne):
    psi = q2.new_state(n, dtype)
    psi.fill_(3.0)
    q2.state_init_hf(psi, n, ne)
    assert np.array_equal(to_host(psi), sv.hf_state(n, ne))


@pytest.mark.parametrize("dtype", ["complex64", "complex128"])
@pytest.mark.parametrize("n", [1, 2, 3, 4])
def test_single_rotation_exhaustive(dtype, n):
    rng = np.random.default_rng(n)
    psi0 = rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)
    psi0 /= np.linalg.norm(psi0)
    for x in range(1 << n):
        for z in range(1 << n):
            phi = rng.uniform(-3, 3)
            psi = to_dev(psi0, dtype)
            q2.apply_pauli_rotations(psi, n, [x], [z], [phi])
            ref = sv.apply_rotation(psi0, x, z, phi)
            assert np.max(np.abs(to_host(psi) - ref)) < TOL_AMP[dtype], (x, z)


def _random_rotations(rng, n, k):
    x = rng.integers(0, 1 << n, size=k).astype(np.uint64)
    x[rng.random(k) < 0.1] = 0
    z = rng.integers(0, 1 << n, size=k).astype(np.uint64)
    for i in range(1, k):
        if rng.random() < 0.5:
            x[i] = x[i - 1]
    return x, z, rng.uniform(-3, 3, size=k)


@pytest.mark.parametrize("dtype", ["complex64", "complex128"])
@pytest.mark.parametrize("n,tile", [(9, 8), (13, None), (16, None), (16, 8), (17, 12)])
def test_random_rotations_match_oracle(dtype, n, tile):
    if tile:
        q2.set_tile_qubits(dtype, tile)
    rng = np.random.default_rng(10 * n + (tile or 0))
    x, z, phi = _random_rotations(rng, n, 150)
    psi0 = rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)
    psi0 /= np.linalg.norm(psi0)
    psi = to_dev(psi0, dtype)
    q2.apply_pauli_rotations(psi, n, x, z, phi)
    ref = c_oracle.apply_rotations(psi0, n, x, z, phi)
    assert np.max(np.abs(to_host(psi) - ref)) < TOL_AMP[dtype]


@pytest.mark.parametrize("dtype", ["complex64", "complex128"])
@pytest.mark.parametrize("n,ne,tile", [(8, 4, None), (12, 6, None), (12, 6, 8), (14, 7, None)])
def test_uccsd_state_and_energy(dtype, n, ne, tile):
    if tile:
        q2.set_tile_qubits(dtype, tile)
    w = uccsd_energy(n, ne, seed=0)
    a = w.ansatz
    psi = q2.new_state(n, dtype)
    q2.state_init_hf(psi, n, ne)
    q2.apply_pauli_rotations(psi, n, a.x, a.z, w.angles())
    ref = c_oracle.apply_rotations(c_oracle.hf_state(n, ne), n, a.x, a.z, w.angles())
    assert np.max(np.abs(to_host(psi) - ref)) < TOL_AMP[dtype]
    ham = q2.Hamiltonian(n, w.ham.x, w.ham.z, w.ham.c)
    e, nrm = ham.expectation(psi)
    e_ref, n_ref = c_oracle.expectation(ref, n, w.ham.x, w.ham.z, w.ham.c)
    assert abs(e - e_ref / n_ref) < TOL_E[dtype]
    assert abs(nrm - 1) < (1e-13 if dtype == "complex128" else 1e-5)


@pytest.mark.parametrize("dtype", ["complex64", "complex128"])
@pytest.mark.parametrize("n,tile", [(10, None), (14, None), (14, 8), (3, None)])
def test_expectation_and_happly_generic(dtype, n, tile):
    if tile:
        q2.set_tile_qubits(dtype, tile)
    rng = np.random.default_rng(300 + n)
    k = 120
    x = rng.integers(0, 1 << n, size=k).astype(np.uint64)
    x[:12] = 0
    x[60:75] = x[60]
    z = rng.integers(0, 1 << n, size=k).astype(np.uint64)
    c = rng.normal(size=k)
    psi0 = rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)
    psi0 /= np.linalg.norm(psi0)
    psi = to_dev(psi0, dtype)
    ham = q2.Hamiltonian(n, x, z, c)
    e, nrm = ham.expectation(psi)
    e_ref, n_ref = c_oracle.expectation(psi0, n, x, z, c)
    assert abs(e - e_ref / n_ref) < TOL_E[dtype]
    lam = torch.empty_like(psi)
    ham.apply(psi, lam)
    q2.async_status()
    lam_ref = c_oracle.apply_hamiltonian(psi0, n, x, z, c)
    scale = 1e-12 if dtype == "complex128" else 2e-5
    assert np.max(np.abs(to_host(lam) - lam_ref)) < scale * max(1.0, np.max(np.abs(lam_ref)))


@pytest.mark.parametrize("dtype", ["complex128", "complex64"])
@pytest.mark.parametrize("n,ne,tile", [(8, 4, None), (10, 4, None), (12, 6, 8)])
def test_vqe_energy_grad_matches_oracle(dtype, n, ne, tile):
    if tile:
        q2.set_tile_qubits(dtype, tile)
    w = uccsd_energy(n, ne, seed=2)
    a = w.ansatz
    ans = q2.Ansatz.from_uccsd(a)
    ham = q2.Hamiltonian(n, w.ham.x, w.ham.z, w.ham.c)
    theta = np.random.default_rng(1).normal(0, 0.3, size=a.n_params)
    e, g, _ = q2.vqe_energy_grad(ans, ham, theta, dtype=dtype, want_grad=True)
    e0, g0, _ = q2.vqe_energy_grad(ans, ham, theta, dtype=dtype, want_grad=False)
    e_ref, gphi = c_oracle.energy_and_gradient(n, ne, a.x, a.z, a.angles(theta), w.ham.x, w.ham.z, w.ham.c)
    g_ref = sv.fold_to_theta(gphi, a.param, a.coef, a.n_params)
    assert abs(e - e_ref) < TOL_E[dtype]
    assert abs(e0 - e_ref) < TOL_E[dtype]
    assert np.max(np.abs(g - g_ref)) < (1e-9 if dtype == "complex128" else 1e-4)


@pytest.mark.parametrize("dtype", ["complex128", "complex64"])
@pytest.mark.parametrize("shared", [True, False])
def test_vqe_gradient_generic_rotations(dtype, shared):
    """Ansatz of arbitrary Pauli strings (x = 0, even- and odd-Y groups), with
    runs of equal xmasks sharing one parameter (one-parameter groups: the
    register-blocked reverse sweep) or each rotation its own parameter."""
    n, ne = 11, 5
    rng = np.random.default_rng(17 + shared)
    k = 90
    x = rng.integers(0, 1 << n, size=k).astype(np.uint64)
    x[rng.random(k) < 0.1] = 0
    for i in range(1, k):
        if rng.random() < 0.6:
            x[i] = x[i - 1]
    z = rng.integers(0, 1 << n, size=k).astype(np.uint64)
    if shared:
        param = np.cumsum(np.concatenate([[0], (x[1:] != x[:-1]).astype(np.int64)])).astype(np.int32)
    else:
        param = np.arange(k, dtype=np.int32)
    n_params = int(param.max()) + 1
    coef = rng.choice([-1.0, -0.5, 0.25, 1.0], size=k)
    ans = q2.Ansatz(n, ne, x, z, param, coef, n_params)
    w = uccsd_energy(10, 5, seed=4)
    hx = np.concatenate([w.ham.x, [0, 1 << 10]]).astype(np.uint64)
    hz = np.concatenate([w.ham.z, [1 << 10, 0]]).astype(np.uint64)
    hc = np.concatenate([w.ham.c, [0.3, -0.2]])
    ham = q2.Hamiltonian(n, hx, hz, hc)
    theta = rng.normal(0, 0.4, size=n_params)
    e, g, _ = q2.vqe_energy_grad(ans, ham, theta, dtype=dtype, want_grad=True)
    phi = coef * theta[param]
    e_ref, gphi = c_oracle.energy_and_gradient(n, ne, x, z, phi, hx, hz, hc)
    g_ref = sv.fold_to_theta(gphi, param, coef, n_params)
    assert abs(e - e_ref) < TOL_E[dtype]
    assert np.max(np.abs(g - g_ref)) < (1e-9 if dtype == "complex128" else 1e-4)


@pytest.mark.parametrize("kind", ["spin_conserving", "paper_spin_adapted"])
def test_excitation_set_variants(kind):
    """The spin-conserving and the paper's spin-adapted generator sets (Sec. "Variational
    quantum circuit ansatz", Table 1) run through the same kernels: energy and dE/dtheta
    against the oracle in complex128 and complex64."""
    w = uccsd_energy(10, 4, seed=5, kind=kind)
    a = w.ansatz
    ans = q2.Ansatz.from_uccsd(a)
    ham = q2.Hamiltonian(10, w.ham.x, w.ham.z, w.ham.c)
    theta = np.random.default_rng(8).normal(0, 0.3, size=a.n_params)
    e_ref, gphi = c_oracle.energy_and_gradient(10, 4, a.x, a.z, a.angles(theta), w.ham.x, w.ham.z, w.ham.c)
    g_ref = sv.fold_to_theta(gphi, a.param, a.coef, a.n_params)
    for dtype, tol_g in (("complex128", 1e-9), ("complex64", 1e-4)):
        e, g, _ = q2.vqe_energy_grad(ans, ham, theta, dtype=dtype, want_grad=True)
        assert abs(e - e_ref) < TOL_E[dtype]
        assert np.max(np.abs(g - g_ref)) < tol_g


def test_autograd_function():
    w = uccsd_energy(8, 4, seed=3)
    ans = q2.Ansatz.from_uccsd(w.ansatz)
    ham = q2.Hamiltonian(8, w.ham.x, w.ham.z, w.ham.c)
    theta = torch.tensor(w.theta, dtype=torch.float64, requires_grad=True)
    e = q2.Energy.apply(theta, ans, ham, "complex128")
    (2.0 * e).backward()
    a = w.ansatz
    e_ref, gphi = c_oracle.energy_and_gradient(8, 4, a.x, a.z, a.angles(w.theta), w.ham.x, w.ham.z, w.ham.c)
    assert abs(e.item() - e_ref) < 1e-10
    assert np.max(np.abs(theta.grad.numpy() - 2 * sv.fold_to_theta(gphi, a.param, a.coef, a.n_params))) < 2e-9


def test_errors_are_loud():
    psi = q2.new_state(8, "complex64")
    with pytest.raises(q2.Q2Error):
        q2.apply_pauli_rotations(psi, 8, [1 << 8], [0], [0.1])
    with pytest.raises(q2.Q2Error):
        q2.state_init_hf(psi, 8, 9)


@pytest.mark.parametrize("dtype", ["complex128", "complex64"])
def test_pool_gradients_match_oracle(dtype):
    """Operator-pool screening: Im<H psi|P_k|psi> for a pool of UCCSD generator strings
    (a different excitation set than the ansatz) plus random strings, against the oracle."""
    from synth.uccsd import uccsd_rotations
    n, ne = 11, 5
    w = uccsd_energy(10, 4, seed=6)
    a = w.ansatz
    ans = q2.Ansatz(n, ne, a.x, a.z, a.param, a.coef, a.n_params)
    ham = q2.Hamiltonian(n, np.concatenate([w.ham.x, [1 << 10]]).astype(np.uint64),
                         np.concatenate([w.ham.z, [0]]).astype(np.uint64), np.concatenate([w.ham.c, [0.4]]))
    pool = uccsd_rotations(n, ne, "spin_conserving")
    rng = np.random.default_rng(21)
    px = np.concatenate([pool.x, rng.integers(0, 1 << n, size=40).astype(np.uint64), [0]]).astype(np.uint64)
    pz = np.concatenate([pool.z, rng.integers(0, 1 << n, size=40).astype(np.uint64), [5]]).astype(np.uint64)
    theta = rng.normal(0, 0.3, size=a.n_params)
    e, g, _ = q2.pool_gradients(ans, ham, theta, px, pz, dtype=dtype)
    hx = np.concatenate([w.ham.x, [1 << 10]]).astype(np.uint64)
    hz = np.concatenate([w.ham.z, [0]]).astype(np.uint64)
    hc = np.concatenate([w.ham.c, [0.4]])
    psi = sv.apply_rotations(sv.hf_state(n, ne), a.x, a.z, a.angles(theta))
    lam = sv.apply_hamiltonian(psi, hx, hz, hc)
    g_ref = np.array([np.imag(np.vdot(lam, sv.apply_pauli(psi, x, z))) for x, z in zip(px, pz)])
    assert abs(e - sv.expectation(psi, hx, hz, hc) / np.vdot(psi, psi).real) < TOL_E[dtype]
    assert np.max(np.abs(g - g_ref)) < (1e-10 if dtype == "complex128" else 1e-4)


def test_device_wait_gives_up_and_context_survives():
    """A bounded device wait on an mbarrier that nothing completes gives up, the call
    reports Q2_ERR_TIMEOUT, and the context stays usable for the next evaluation."""
    import ctypes
    L = q2.lib()
    L.q2_debug_wait_probe.argtypes = [ctypes.c_uint, ctypes.c_void_p]
    L.q2_debug_wait_probe.restype = ctypes.c_int
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert L.q2_debug_wait_probe(1000, stream) == q2.Q2_ERR_TIMEOUT
    assert L.q2_debug_wait_probe(0, stream) == q2.Q2_ERR_INVALID
    w = uccsd_energy(10, 4, seed=2)
    a = w.ansatz
    ans = q2.Ansatz.from_uccsd(a)
    ham = q2.Hamiltonian(10, w.ham.x, w.ham.z, w.ham.c)
    e, _, _ = q2.vqe_energy_grad(ans, ham, w.theta, dtype="complex64", want_grad=False)
    psi = sv.apply_rotations(sv.hf_state(10, 4), a.x, a.z, a.angles(w.theta))
    e_ref, _ = sv.energy(psi, w.ham.x, w.ham.z, w.ham.c)
    assert abs(e - e_ref) < TOL_E["complex64"]


def test_timeout_reported_only_by_the_call_that_timed_out():
    """Per-call fault words: a bounded wait that gives up in one call (the wait probe on
    one stream and host thread) is reported by that call alone; an evaluation running at
    the same time on another stream returns Q2_OK with the right energy, and so do the
    asynchronous calls' status and the next calls on the probe's stream."""
    import ctypes
    import threading
    L = q2.lib()
    L.q2_debug_wait_probe.argtypes = [ctypes.c_uint, ctypes.c_void_p]
    L.q2_debug_wait_probe.restype = ctypes.c_int
    w = uccsd_energy(14, 7, seed=3)
    a = w.ansatz
    ans = q2.Ansatz.from_uccsd(a)
    ham = q2.Hamiltonian(14, w.ham.x, w.ham.z, w.ham.c)
    ref = c_oracle.apply_rotations(c_oracle.hf_state(14, 7), 14, a.x, a.z, a.angles(w.theta))
    num, nrm = c_oracle.expectation(ref, 14, w.ham.x, w.ham.z, w.ham.c)
    e_ref = num / nrm
    s_probe, s_eval = torch.cuda.Stream(), torch.cuda.Stream()
    out = {}

    def probe():
        torch.cuda.set_device(0)
        out["probe"] = [L.q2_debug_wait_probe(1 << 20, ctypes.c_void_p(s_probe.cuda_stream)) for _ in range(3)]

    def evaluate():
        torch.cuda.set_device(0)
        res = []
        with torch.cuda.stream(s_eval):
            for _ in range(3):
                try:
                    res.append(q2.vqe_energy_grad(ans, ham, w.theta, dtype="complex64", want_grad=False)[0])
                except q2.Q2Error as exc:
                    res.append(exc)
        out["eval"] = res

    threads = [threading.Thread(target=probe), threading.Thread(target=evaluate)]
    for t in threads:
        t.start()
    for t in threads:
        t.join(timeout=300)
    assert out["probe"] == [q2.Q2_ERR_TIMEOUT] * 3
    for e in out["eval"]:
        assert not isinstance(e, Exception), e
        assert abs(e - e_ref) < TOL_E["complex64"]
    q2.async_status()          # the probe's give-ups are not the asynchronous calls' either


@pytest.mark.parametrize("dtype", ["complex128", "complex64"])
def test_hamiltonian_shards_sum_to_whole(dtype):
    """Term-group sharding (q2_ham_shard) on one GPU: the shards' energies and gradients, each
    evaluated through q2_vqe_energy_grad and q2_expectation, sum to the whole Hamiltonian's and
    to the oracle's; with more shards than passes some shards are empty and give exactly 0."""
    w = uccsd_energy(12, 6, seed=4)
    a = w.ansatz
    ans = q2.Ansatz.from_uccsd(a)
    ham = q2.Hamiltonian(12, w.ham.x, w.ham.z, w.ham.c)
    theta = np.random.default_rng(2).normal(0, 0.3, size=a.n_params)
    e_ref, gphi = c_oracle.energy_and_gradient(12, 6, a.x, a.z, a.angles(theta), w.ham.x, w.ham.z, w.ham.c)
    g_ref = sv.fold_to_theta(gphi, a.param, a.coef, a.n_params)
    e_all, g_all, ws = q2.vqe_energy_grad(ans, ham, theta, dtype=dtype, want_grad=True)
    psi = q2.new_state(12, dtype)
    q2.state_init_hf(psi, 12, 6)
    q2.apply_pauli_rotations(psi, 12, a.x, a.z, a.angles(theta))
    e_psi, _ = ham.expectation(psi)
    tol_g = 1e-9 if dtype == "complex128" else 1e-4
    n_all = len(ham.shard(0, 1).shard_terms(dtype))
    for k in (2, 3, 64):
        shards = [ham.shard(r, k) for r in range(k)]
        es, gs, ex = 0.0, np.zeros(a.n_params), 0.0
        empty = 0
        for sh in shards:
            e, g, ws = q2.vqe_energy_grad(ans, sh, theta, dtype=dtype, want_grad=True, workspace=ws)
            e0, _, ws = q2.vqe_energy_grad(ans, sh, theta, dtype=dtype, want_grad=False, workspace=ws)
            ee, nrm = sh.expectation(psi)
            assert abs(e - e0) < TOL_E[dtype] and abs(nrm - 1) < 1e-5
            if len(sh.shard_terms(dtype)) == 0:
                empty += 1
                assert e == 0.0 and e0 == 0.0 and ee == 0.0 and not np.any(g)
            es, gs, ex = es + e, gs + g, ex + ee
        assert abs(es - e_all) < TOL_E[dtype] and abs(es - e_ref) < TOL_E[dtype]
        assert abs(ex - e_psi) < TOL_E[dtype]
        assert np.max(np.abs(gs - g_all)) < tol_g and np.max(np.abs(gs - g_ref)) < tol_g
        if k == 64:
            assert empty > 0 and n_all == w.ham.n_terms


@pytest.mark.parametrize("n", [17, 20])
def test_sweep_fast_path_and_general_path_match_oracle(n):
    """Random-order UCCSD sweep (whole double excitations, 12-qubit tiles): nearly every pass
    is made of canonical 4-dimensional blocks and takes the fast path (k_sweep_c4); the same
    sweep with the fast path switched off takes the general block path.  Both match the
    oracle per amplitude, complex64."""
    import ctypes
    from synth.workloads import sweep_ansatz
    L = q2.lib()
    L.q2_debug_sweep_fast_path.argtypes = [ctypes.c_int]
    ans, theta = sweep_ansatz(n, n // 2, 600, n)
    phi = ans.angles(theta)
    rng = np.random.default_rng(n)
    psi0 = rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)
    psi0 /= np.linalg.norm(psi0)
    ref = c_oracle.apply_rotations(psi0, n, ans.x, ans.z, phi)
    out = {}
    try:
        for fast in (1, 0):
            L.q2_debug_sweep_fast_path(fast)
            psi = to_dev(psi0, "complex64")
            q2.apply_pauli_rotations(psi, n, ans.x, ans.z, phi)
            q2.async_status()
            out[fast] = to_host(psi)
    finally:
        L.q2_debug_sweep_fast_path(1)
    for fast in (1, 0):
        assert np.max(np.abs(out[fast] - ref)) < TOL_AMP["complex64"], fast


@pytest.mark.parametrize("n,seed", [(18, 0), (20, 1)])
def test_expectation_fast_path_and_general_path_match_oracle(n, seed):
    """The expectation's lean path (k_expect_fast: complex64 passes of REAL and DIAG groups in
    blocks of at most 3 dimensions, 13-qubit tiles) and the general path give the oracle's
    energy and norm on a random normalised state, for whole xmask groups of a UCCSD
    Hamiltonian (every group of a real-integral Hamiltonian is REAL or DIAG)."""
    import ctypes
    from synth.workloads import sweep32
    L = q2.lib()
    L.q2_debug_expect_fast_path.argtypes = [ctypes.c_int]
    w = sweep32(seed=seed, n=n, n_elec=n // 2, n_rot=16, min_terms=3000)
    rng = np.random.default_rng(seed)
    psi0 = rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)
    psi0 /= np.linalg.norm(psi0)
    num, nrm_ref = c_oracle.expectation(psi0, n, w.ham.x, w.ham.z, w.ham.c)
    psi = to_dev(psi0, "complex64")
    ham = q2.Hamiltonian(n, w.ham.x, w.ham.z, w.ham.c)
    try:
        for fast in (1, 0):
            L.q2_debug_expect_fast_path(fast)
            e, nrm = ham.expectation(psi)
            assert abs(e - num / nrm_ref) < TOL_E["complex64"], fast
            assert abs(nrm - nrm_ref) < 1e-5, fast
    finally:
        L.q2_debug_expect_fast_path(1)
