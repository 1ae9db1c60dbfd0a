"""Full-size parity of the CUDA path on the benchmark workloads.

* 8 qubits (4 electrons), complex128: energy and gradient vs the oracle.
* 20 qubits (10 electrons), 16,400 rotations, 14,251 terms: energy and the
  largest amplitudes vs stored oracle values (tests/golden/uccsd20_seed0.json,
  written by tests/golden/make_golden.py from oracle/ only), complex128 and
  complex64.
* 24 qubits (12 electrons), 35,136 rotations, energy + reverse-mode gradient:
  per-rotation gradients vs the exact parameter-shift rule on 32 sampled
  rotations and dE/dtheta vs central differences (h = 1e-4), both on the
  complex128 GPU path; complex64 vs complex128; stored oracle values when
  tests/golden/uccsd24_seed0.json exists.
* 32 qubits (16 electrons), the 50,000-rotation workload: the first two
  excitations applied to |HF> on the full 2^32 state vs the sparse-state
  oracle (amplitudes at bits 16..31, zeros elsewhere, energy with the
  ~30k-term Hamiltonian), and the theta = 0 energy, complex64 and complex128.
"""

import json
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2208_10978_gb300 as q2
from oracle import statevector as sv
from oracle import sparse, fock
from synth.workloads import uccsd_energy, sweep32

pytestmark = pytest.mark.gpu

GOLD = os.path.join(os.path.dirname(__file__), "golden")
TOL_E = {"complex128": 1e-10, "complex64": 1e-5}


def _check_fingerprint(w, rec):
    fp = rec["inputs"]
    assert fp["n_terms"] == w.ham.n_terms and fp["n_rot"] == w.ansatz.n_rot
    for key, val in (("h00", w.h[0, 0]), ("eri0000", w.eri[0, 0, 0, 0]), ("theta0", w.theta[0]),
                     ("theta_last", w.theta[-1]), ("c_sum", np.sum(w.ham.c))):
        assert abs(fp[key] - val) <= 1e-12 * max(1.0, abs(val)), f"input generator changed: {key}"


def test_uccsd8_seed0_energy_and_gradient():
    w = uccsd_energy(8, 4, seed=0)
    a = w.ansatz
    ans, ham = q2.Ansatz.from_uccsd(a), q2.Hamiltonian(8, w.ham.x, w.ham.z, w.ham.c)
    e_ref, gphi = sv.energy_and_gradient(8, 4, a.x, a.z, a.angles(w.theta), w.ham.x, w.ham.z, w.ham.c)
    g_ref = sv.fold_to_theta(gphi, a.param, a.coef, a.n_params)
    e, g, _ = q2.vqe_energy_grad(ans, ham, w.theta, dtype="complex128", want_grad=True)
    assert abs(e - e_ref) < 1e-10
    assert np.max(np.abs(g - g_ref)) < 1e-9
    e64, g64, _ = q2.vqe_energy_grad(ans, ham, w.theta, dtype="complex64", want_grad=True)
    assert abs(e64 - e_ref) < 1e-5
    assert np.max(np.abs(g64 - g_ref)) < 1e-4


@pytest.mark.parametrize("dtype", ["complex128", "complex64"])
def test_uccsd20_energy_vs_golden(dtype):
    rec = json.load(open(os.path.join(GOLD, "uccsd20_seed0.json")))
    w = uccsd_energy(20, 10, seed=0)
    _check_fingerprint(w, rec)
    ans, ham = q2.Ansatz.from_uccsd(w.ansatz), q2.Hamiltonian(20, w.ham.x, w.ham.z, w.ham.c)
    e, _, ws = q2.vqe_energy_grad(ans, ham, w.theta, dtype=dtype, want_grad=False)
    assert abs(e - rec["energy"]) < TOL_E[dtype]
    psi = q2.workspace_state(ws, 20, dtype)
    idx = torch.tensor([int(k) for k in rec["largest_amplitudes"]], device="cuda")
    got = psi[idx].to("cpu", torch.complex128).numpy()
    ref = np.array([complex(*v) for v in rec["largest_amplitudes"].values()])
    assert np.max(np.abs(got - ref)) < (1e-12 if dtype == "complex128" else 2e-6)


@pytest.fixture(scope="module")
def w24():
    return uccsd_energy(24, 12, seed=0)


def _per_rotation_ansatz(a, phi):
    """Ansatz whose parameters are the rotation angles themselves."""
    n_rot = a.n_rot
    return q2.Ansatz(a.n, a.n_elec, a.x, a.z, np.arange(n_rot, dtype=np.int32), np.ones(n_rot), n_rot), phi.copy()


def test_uccsd24_gradient_parameter_shift_and_fd(w24):
    a = w24.ansatz
    ham = q2.Hamiltonian(24, w24.ham.x, w24.ham.z, w24.ham.c)
    phi = a.angles(w24.theta)
    rot_ans, p = _per_rotation_ansatz(a, phi)
    e, gphi, ws = q2.vqe_energy_grad(rot_ans, ham, p, dtype="complex128", want_grad=True)
    rng = np.random.default_rng(24)
    sample = rng.choice(a.n_rot, size=32, replace=False)
    for k in sample:
        pp, pm = p.copy(), p.copy()
        pp[k] += np.pi / 2
        pm[k] -= np.pi / 2
        ep, _, ws = q2.vqe_energy_grad(rot_ans, ham, pp, dtype="complex128", want_grad=False, workspace=ws)
        em, _, ws = q2.vqe_energy_grad(rot_ans, ham, pm, dtype="complex128", want_grad=False, workspace=ws)
        assert abs(gphi[k] - 0.5 * (ep - em)) < 1e-9, k
    # dE/dtheta through the UCCSD parameters vs central differences
    ans = q2.Ansatz.from_uccsd(a)
    e_t, g_t, ws2 = q2.vqe_energy_grad(ans, ham, w24.theta, dtype="complex128", want_grad=True)
    assert abs(e_t - e) < 1e-10
    assert np.max(np.abs(g_t - sv.fold_to_theta(gphi, a.param, a.coef, a.n_params))) < 1e-12
    h = 1e-4
    for k in rng.choice(a.n_params, size=8, replace=False):
        tp, tm = w24.theta.copy(), w24.theta.copy()
        tp[k] += h
        tm[k] -= h
        ep, _, ws2 = q2.vqe_energy_grad(ans, ham, tp, dtype="complex128", want_grad=False, workspace=ws2)
        em, _, ws2 = q2.vqe_energy_grad(ans, ham, tm, dtype="complex128", want_grad=False, workspace=ws2)
        assert abs(g_t[k] - (ep - em) / (2 * h)) < 1e-6, k


def test_uccsd24_complex64_vs_complex128_and_golden(w24):
    a = w24.ansatz
    ans = q2.Ansatz.from_uccsd(a)
    ham = q2.Hamiltonian(24, w24.ham.x, w24.ham.z, w24.ham.c)
    e128, g128, _ = q2.vqe_energy_grad(ans, ham, w24.theta, dtype="complex128", want_grad=True)
    e64, g64, _ = q2.vqe_energy_grad(ans, ham, w24.theta, dtype="complex64", want_grad=True)
    assert abs(e64 - e128) < 1e-5
    assert np.max(np.abs(g64 - g128)) < 1e-4
    path = os.path.join(GOLD, "uccsd24_seed0.json")
    if os.path.exists(path):
        rec = json.load(open(path))
        _check_fingerprint(w24, rec)
        assert abs(e128 - rec["energy"]) < 1e-10
        assert np.max(np.abs(g128 - np.array(rec["grad_theta"]))) < 1e-9
    # the gradient at theta = 0 equals 2 s_k <HF|H|Phi_k> (Slater-Condon, no state vector)
    from synth import excitations
    z0 = np.zeros(a.n_params)
    _, g0, _ = q2.vqe_energy_grad(ans, ham, z0, dtype="complex128", want_grad=True)
    hf = (1 << 12) - 1
    exc = excitations(24, 12)
    for k in np.random.default_rng(5).choice(a.n_params, size=6, replace=False):
        s, phi_bits = fock.apply_ops(exc[k][0], hf)
        assert abs(g0[k] - 2 * s * fock.matrix_element(w24.h, w24.eri, 24, hf, phi_bits)) < 1e-10


@pytest.fixture(scope="module")
def w32():
    return sweep32(seed=0)


@pytest.mark.parametrize("dtype", ["complex64", "complex128"])
def test_sweep32_sparse_oracle(w32, dtype):
    """First two excitations (16 rotations) on the 2^32 state vs the sparse oracle."""
    a = w32.ansatz
    k = 16
    phi = a.angles(w32.theta)[:k]
    x, z = a.x[:k], a.z[:k]
    ref = sparse.rotations_apply({(1 << 16) - 1: 1.0 + 0j}, x, z, phi)
    ref = {i: v for i, v in ref.items() if abs(v) > 1e-15}
    assert any(i >> 24 for i in ref)              # amplitudes with index bits >= 24 are exercised
    # whole xmask groups of the 32-qubit Hamiltonian (x = 0 first); the full ~30k-term
    # energy is the benchmark's and costs minutes in complex128
    from synth.jw import group_starts
    st = group_starts(w32.ham.x)
    cut = st[min(300, len(st) - 1)]
    hx, hz, hc = w32.ham.x[:cut], w32.ham.z[:cut], w32.ham.c[:cut]
    ham = q2.Hamiltonian(32, hx, hz, hc)
    psi = q2.new_state(32, dtype)
    q2.state_init_hf(psi, 32, 16)
    e_hf, nrm = ham.expectation(psi)
    hf_ref = sparse.expectation({(1 << 16) - 1: 1.0 + 0j}, hx, hz, hc)
    assert abs(e_hf - hf_ref) < TOL_E[dtype]
    q2.apply_pauli_rotations(psi, 32, x, z, phi)
    keys = sorted(ref)
    got = psi[torch.tensor(keys, device="cuda")].to("cpu", torch.complex128).numpy()
    tol = 1e-12 if dtype == "complex128" else 1e-6
    assert np.max(np.abs(got - np.array([ref[i] for i in keys]))) < tol
    probe = np.random.default_rng(1).integers(0, 1 << 32, size=64, dtype=np.uint64)
    probe = [int(i) for i in probe if int(i) not in ref]
    zeros = psi[torch.tensor(probe, device="cuda")].abs().max().item()
    assert zeros == 0.0
    e, nrm = ham.expectation(psi)
    assert abs(nrm - 1.0) < (1e-13 if dtype == "complex128" else 1e-6)
    assert abs(e - sparse.expectation(ref, hx, hz, hc)) < TOL_E[dtype]
    del psi
    torch.cuda.empty_cache()
