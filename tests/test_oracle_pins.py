"""Pins of the oracle against what the paper and the mathematics fix.

Each check below is independent of the function it pins: dense matrix
exponentials of Kronecker-product Paulis, Algorithm 2's gate product, the
Hartree-Fock closed form, Fock-space FCI (no Pauli algebra), the
variational principle, Slater-Condon-style matrix elements of one
excitation, and the parameter-shift rule.  The planted-mistake tests at the
end show the pins fail for plausible slips in the oracle.
"""

import numpy as np
import pytest
import scipy.linalg
import scipy.sparse
import scipy.sparse.linalg

from synth import random_integrals, qubit_hamiltonian, uccsd_rotations, excitations
from synth.workloads import uccsd_energy
from oracle import statevector as sv
from oracle import fock, circuits, sparse
from oracle import c_oracle


def _rng(s):
    return np.random.default_rng(s)


# ---------------------------------------------------------------- Pauli action

@pytest.mark.parametrize("n", [1, 2, 3])
def test_pauli_and_rotation_exhaustive_small(n):
    """Every (x, z) at n <= 3: P psi and exp(-i phi/2 P) psi match dense expm."""
    rng = _rng(n)
    for x in range(1 << n):
        for z in range(1 << n):
            P = sv.dense_pauli(n, x, z)
            assert np.allclose(P, P.conj().T)
            psi = rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)
            assert np.allclose(sv.apply_pauli(psi, x, z), P @ psi, atol=1e-14)
            phi = rng.uniform(-4, 4)
            U = scipy.linalg.expm(-0.5j * phi * P)
            assert np.allclose(sv.apply_rotation(psi, x, z, phi), U @ psi, atol=1e-13)


@pytest.mark.parametrize("n", [5, 6])
def test_rotation_random_masks(n):
    rng = _rng(10 + n)
    for _ in range(12):
        x, z = int(rng.integers(1 << n)), int(rng.integers(1 << n))
        psi = rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)
        phi = rng.uniform(-4, 4)
        U = scipy.linalg.expm(-0.5j * phi * sv.dense_pauli(n, x, z))
        assert np.allclose(sv.apply_rotation(psi, x, z, phi), U @ psi, atol=1e-12)


@pytest.mark.parametrize("n", [3, 4, 5])
def test_algorithm2_circuit_equals_rotation(n):
    """Algorithm 2 gate product == exp(i theta P) == rotation with phi = -2 theta."""
    rng = _rng(20 + n)
    for _ in range(10):
        x, z = int(rng.integers(1, 1 << n)), int(rng.integers(1 << n))
        theta = rng.uniform(-2, 2)
        U = circuits.circuit_unitary(circuits.exp_pauli_circuit(n, x, z, theta), n)
        ref = scipy.linalg.expm(1j * theta * sv.dense_pauli(n, x, z))
        assert np.allclose(U, ref, atol=1e-12)
        psi = rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)
        assert np.allclose(sv.apply_rotation(psi, x, z, -2 * theta), U @ psi, atol=1e-12)


# ---------------------------------------------------------------- chemistry pins

@pytest.mark.parametrize("m,ne,seed", [(4, 4, 0), (4, 3, 1), (6, 6, 2)])
def test_theta_zero_is_hf_closed_form(m, ne, seed):
    h, eri = random_integrals(m, seed)
    x, z, c = qubit_hamiltonian(h, eri)
    psi = sv.hf_state(2 * m, ne)
    e = sv.expectation(psi, x, z, c)
    assert abs(e - fock.hf_energy(h, eri, ne)) < 1e-12


@pytest.mark.parametrize("m,ne", [(4, 4), (5, 5), (4, 3)])
def test_jw_spectrum_equals_fci(m, ne):
    """N-electron block of the JW Hamiltonian == Fock-space FCI matrix (same basis)."""
    h, eri = random_integrals(m, 5)
    x, z, c = qubit_hamiltonian(h, eri)
    n = 2 * m
    dets, Hf = fock.fci_matrix(h, eri, n, ne)
    Hj = np.zeros_like(Hf)
    for j, d in enumerate(dets):
        e = np.zeros(1 << n, dtype=np.complex128)
        e[d] = 1
        col = sv.apply_hamiltonian(e, x, z, c)
        Hj[:, j] = col[dets].real
        assert np.allclose(col[dets].imag, 0)
        outside = np.delete(col, dets)
        assert np.allclose(outside, 0)                 # particle number conserved
    assert np.allclose(Hj, Hf, atol=1e-12)
    assert np.allclose(np.linalg.eigvalsh(Hj), np.linalg.eigvalsh(Hf), atol=1e-10)


def test_fock_hf_closed_form():
    h, eri = random_integrals(5, 4)
    for ne in (2, 5, 7):
        hf = (1 << ne) - 1
        assert abs(fock.matrix_element(h, eri, 10, hf, hf) - fock.hf_energy(h, eri, ne)) < 1e-12


@pytest.mark.parametrize("seed", [0, 1])
def test_variational_bound_n8(seed):
    w = uccsd_energy(8, 4, seed=seed)
    dets, H = fock.fci_matrix(w.h, w.eri, 8, 4)
    lam = np.linalg.eigvalsh(H)[0]
    rng = _rng(seed)
    for scale in (0.05, 0.5, 2.0):
        th = rng.normal(0, scale, size=len(w.theta))
        psi = sv.apply_rotations(sv.hf_state(8, 4), w.ansatz.x, w.ansatz.z, w.ansatz.angles(th))
        e, nrm = sv.energy(psi, w.ham.x, w.ham.z, w.ham.c)
        assert abs(nrm - 1) < 1e-13
        assert e >= lam - 1e-12


def test_variational_bound_n12_sparse_eigsh():
    n, ne = 12, 6
    w = uccsd_energy(n, ne, seed=0)
    dets = fock.determinants(n, ne)
    rows, cols, vals = [], [], []
    pos = {d: k for k, d in enumerate(dets)}
    for j, d in enumerate(dets):
        for b, v in fock.hamiltonian_apply(w.h, w.eri, n, d).items():
            rows.append(pos[b]); cols.append(j); vals.append(v)
    H = scipy.sparse.csr_matrix((vals, (rows, cols)), shape=(len(dets), len(dets)))
    lam = scipy.sparse.linalg.eigsh(H, k=1, which="SA")[0][0]
    psi = c_oracle.apply_rotations(c_oracle.hf_state(n, ne), n, w.ansatz.x, w.ansatz.z, w.angles())
    e, nrm = c_oracle.expectation(psi, n, w.ham.x, w.ham.z, w.ham.c)
    assert abs(nrm - 1) < 1e-12
    assert e / nrm >= lam - 1e-10


@pytest.mark.parametrize("which", [0, 3, 17, 40, 51])
def test_single_excitation_closed_form(which):
    """Rotations of one excitation == cos|HF> + s sin|Phi>; energy closed form."""
    n, ne = 8, 4
    h, eri = random_integrals(4, 2)
    x, z, c = qubit_hamiltonian(h, eri)
    a = uccsd_rotations(n, ne)
    ops, _ = excitations(n, ne)[which]
    idx = a.param == which
    for theta in (0.3, -1.1):
        psi = sv.apply_rotations(sv.hf_state(n, ne), a.x[idx], a.z[idx], a.coef[idx] * theta)
        e_ref, s, phi_bits, _ = fock.single_excitation_energy(h, eri, n, ne, ops, theta)
        exp = np.zeros(1 << n, dtype=np.complex128)
        exp[(1 << ne) - 1] = np.cos(theta)
        exp[phi_bits] = s * np.sin(theta)
        assert np.allclose(psi, exp, atol=1e-14)
        assert abs(sv.expectation(psi, x, z, c) - e_ref) < 1e-12


def test_gradient_at_theta_zero_closed_form():
    """dE/dtheta_k at theta = 0 equals 2 s_k <HF|H|Phi_k> for every excitation."""
    w = uccsd_energy(8, 4, seed=3)
    a = w.ansatz
    e, g = sv.energy_and_gradient(8, 4, a.x, a.z, np.zeros(a.n_rot), w.ham.x, w.ham.z, w.ham.c)
    gt = sv.fold_to_theta(g, a.param, a.coef, a.n_params)
    hf = (1 << 4) - 1
    for k, (ops, _) in enumerate(excitations(8, 4)):
        s, phi = fock.apply_ops(ops, hf)
        assert abs(gt[k] - 2 * s * fock.matrix_element(w.h, w.eri, 8, hf, phi)) < 1e-12
    assert abs(e - fock.hf_energy(w.h, w.eri, 4)) < 1e-12


def test_adjoint_matches_parameter_shift_and_fd():
    w = uccsd_energy(6, 2, seed=4)
    a = w.ansatz
    th = _rng(9).normal(0, 0.4, size=a.n_params)
    phis = a.angles(th)
    args = (w.ham.x, w.ham.z, w.ham.c)
    e, g = sv.energy_and_gradient(6, 2, a.x, a.z, phis, *args)
    for k in range(0, a.n_rot, 3):
        ps = sv.parameter_shift(6, 2, a.x, a.z, phis, *args, k)
        assert abs(g[k] - ps) < 1e-12
    gt = sv.fold_to_theta(g, a.param, a.coef, a.n_params)
    h = 1e-4
    for p in range(0, a.n_params, 2):
        tp, tm = th.copy(), th.copy()
        tp[p] += h
        tm[p] -= h
        ep = sv.energy_of_angles(6, 2, a.x, a.z, a.angles(tp), *args)
        em = sv.energy_of_angles(6, 2, a.x, a.z, a.angles(tm), *args)
        assert abs(gt[p] - (ep - em) / (2 * h)) < 1e-7


def test_sparse_oracle_matches_dense():
    w = uccsd_energy(8, 4, seed=1)
    a = w.ansatz
    sel = slice(0, 40)
    phis = a.angles(_rng(1).normal(0, 0.5, size=a.n_params))[sel]
    psi = sv.apply_rotations(sv.hf_state(8, 4), a.x[sel], a.z[sel], phis)
    st = sparse.rotations_apply({15: 1.0 + 0j}, a.x[sel], a.z[sel], phis)
    dense = np.zeros(256, dtype=np.complex128)
    for k, v in st.items():
        dense[k] = v
    assert np.allclose(dense, psi, atol=1e-14)
    assert abs(sparse.expectation(st, w.ham.x, w.ham.z, w.ham.c)
               - sv.expectation(psi, w.ham.x, w.ham.z, w.ham.c)) < 1e-12


def test_sparse_oracle_high_bits_closed_form():
    """One 32-qubit double excitation from HF: amplitudes at bits >= 24."""
    n, ne = 32, 16
    ex = [(i, j, a, b) for (i, j, a, b) in [(3, 14, 25, 31), (0, 15, 16, 30)]]
    a_all = uccsd_rotations(n, ne, exc_list=[([(a, True), (b, True), (j, False), (i, False)], None)
                                            for (i, j, a, b) in ex])
    for k, (i, j, a, b) in enumerate(ex):
        idx = a_all.param == k
        theta = 0.37
        st = sparse.rotations_apply({(1 << ne) - 1: 1.0 + 0j}, a_all.x[idx], a_all.z[idx],
                                    a_all.coef[idx] * theta)
        s, phi = fock.apply_ops([(a, True), (b, True), (j, False), (i, False)], (1 << ne) - 1)
        st = {key: v for key, v in st.items() if abs(v) > 1e-15}
        assert set(st) == {(1 << ne) - 1, phi}
        assert abs(st[(1 << ne) - 1] - np.cos(theta)) < 1e-15
        assert abs(st[phi] - s * np.sin(theta)) < 1e-15


# ---------------------------------------------------------------- C oracle pins

def test_c_oracle_rotation_matches_expm():
    n = 4
    rng = _rng(31)
    xs = rng.integers(0, 1 << n, size=30).astype(np.uint64)
    zs = rng.integers(0, 1 << n, size=30).astype(np.uint64)
    ph = rng.uniform(-3, 3, size=30)
    psi0 = rng.normal(size=16) + 1j * rng.normal(size=16)
    ref = psi0.copy()
    for x, z, p in zip(xs, zs, ph):
        ref = scipy.linalg.expm(-0.5j * p * sv.dense_pauli(n, x, z)) @ ref
    got = c_oracle.apply_rotations(psi0, n, xs, zs, ph)
    assert np.allclose(got, ref, atol=1e-12)


def test_c_oracle_hf_closed_form_and_grad_at_zero():
    w = uccsd_energy(8, 4, seed=5)
    a = w.ansatz
    psi = c_oracle.hf_state(8, 4)
    e, nrm = c_oracle.expectation(psi, 8, w.ham.x, w.ham.z, w.ham.c)
    assert abs(e - fock.hf_energy(w.h, w.eri, 4)) < 1e-12 and nrm == 1.0
    e0, g = c_oracle.energy_and_gradient(8, 4, a.x, a.z, np.zeros(a.n_rot), w.ham.x, w.ham.z, w.ham.c)
    gt = sv.fold_to_theta(g, a.param, a.coef, a.n_params)
    hf = 15
    for k, (ops, _) in enumerate(excitations(8, 4)[::7]):
        kk = 7 * k
        s, phi = fock.apply_ops(ops, hf)
        assert abs(gt[kk] - 2 * s * fock.matrix_element(w.h, w.eri, 8, hf, phi)) < 1e-12


def test_c_oracle_grad_matches_parameter_shift():
    w = uccsd_energy(6, 2, seed=6)
    a = w.ansatz
    phis = a.angles(_rng(2).normal(0, 0.5, size=a.n_params))
    args = (w.ham.x, w.ham.z, w.ham.c)
    e, g = c_oracle.energy_and_gradient(6, 2, a.x, a.z, phis, *args)
    for k in range(0, a.n_rot, 5):
        assert abs(g[k] - sv.parameter_shift(6, 2, a.x, a.z, phis, *args, k)) < 1e-12
    lam = c_oracle.apply_hamiltonian(c_oracle.apply_rotations(c_oracle.hf_state(6, 2), 6, a.x, a.z, phis),
                                     6, *args)
    psi = sv.apply_rotations(sv.hf_state(6, 2), a.x, a.z, phis)
    assert np.allclose(lam, sv.dense_hamiltonian(6, *args) @ psi, atol=1e-12)


# ---------------------------------------------------------------- planted mistakes

def test_pins_catch_planted_sign_error(monkeypatch):
    """A wrong phase convention in the oracle's Pauli action fails the expm pin."""
    def bad_apply(psi, x, z):
        i = np.arange(len(psi), dtype=np.uint64)
        src = i ^ np.uint64(x)
        sign = 1.0 - 2.0 * (sv._popcount(i & np.uint64(z)) & 1)   # parity of i, not i^x
        ny = int(sv._popcount(np.array([np.uint64(x) & np.uint64(z)]))[0])
        return (1j ** ny) * sign * psi[src]
    n, x, z = 3, 0b011, 0b001
    P = sv.dense_pauli(n, x, z)
    psi = np.arange(8) + 1j
    assert np.allclose(sv.apply_pauli(psi, x, z), P @ psi)
    assert not np.allclose(bad_apply(psi, x, z), P @ psi)


def test_pins_catch_dropped_exchange_term():
    """Dropping the exchange term in the HF closed form breaks the theta = 0 pin."""
    h, eri = random_integrals(4, 0)
    x, z, c = qubit_hamiltonian(h, eri)
    e = sv.expectation(sv.hf_state(8, 4), x, z, c)
    no_k = sum(h[i // 2, i // 2] for i in range(4)) + 0.5 * sum(
        eri[i // 2, i // 2, j // 2, j // 2] for i in range(4) for j in range(4))
    assert abs(e - fock.hf_energy(h, eri, 4)) < 1e-12
    assert abs(e - no_k) > 1e-3


def test_pins_catch_transposed_gradient_order():
    """Reading g from the un-rotated psi (one step late) differs from parameter shift."""
    w = uccsd_energy(6, 2, seed=8)
    a = w.ansatz
    phis = a.angles(_rng(3).normal(0, 0.5, size=a.n_params))
    args = (w.ham.x, w.ham.z, w.ham.c)
    psi = sv.apply_rotations(sv.hf_state(6, 2), a.x, a.z, phis)
    lam = sv.apply_hamiltonian(psi, *args)
    k = a.n_rot - 1
    psi_late = sv.apply_rotation(psi, a.x[k], a.z[k], -phis[k])
    wrong = np.vdot(lam, sv.apply_pauli(psi_late, a.x[k], a.z[k])).imag
    right = sv.parameter_shift(6, 2, a.x, a.z, phis, *args, k)
    assert abs(np.vdot(lam, sv.apply_pauli(psi, a.x[k], a.z[k])).imag - right) < 1e-12
    assert abs(wrong - right) > 1e-6
