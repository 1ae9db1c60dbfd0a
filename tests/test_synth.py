"""Input generators: JW algebra, Hamiltonian tables, UCCSD rotation lists.

The JW mapping is pinned against the canonical anticommutation relations and
the occupation-number sign rule (oracle/fock.py), which share no Pauli code;
counts are pinned against closed-form combinatorics and Table 1.
"""

import os
from itertools import combinations
from math import comb

import numpy as np
import pytest

from synth import random_integrals, qubit_hamiltonian, uccsd_rotations, excitations
from synth.jw import fermion_operator_to_pauli, group_starts, popcount
from synth.workloads import uccsd_energy, sweep32, served_stream
from oracle import fock
from oracle.statevector import dense_pauli
from oracle.circuits import cnot_count

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _dense(n, x, z, c):
    m = np.zeros((1 << n, 1 << n), dtype=np.complex128)
    for xi, zi, ci in zip(x, z, c):
        m += ci * dense_pauli(n, xi, zi)
    return m


@pytest.mark.parametrize("n", [1, 3, 4])
def test_ladder_car(n):
    """{a_p, a_q^+} = delta_pq and {a_p, a_q} = 0 for the JW ladder operators."""
    a = [_dense(n, *fermion_operator_to_pauli([(1.0, [(q, False)])])) for q in range(n)]
    ad = [_dense(n, *fermion_operator_to_pauli([(1.0, [(q, True)])])) for q in range(n)]
    eye = np.eye(1 << n)
    for p in range(n):
        assert np.allclose(ad[p], a[p].conj().T)
        for q in range(n):
            assert np.allclose(a[p] @ ad[q] + ad[q] @ a[p], eye * (p == q))
            assert np.allclose(a[p] @ a[q] + a[q] @ a[p], 0)


def test_ladder_matches_occupation_sign_rule():
    """JW a_q^+ on |bits> equals the canonical Fock-space action (fock.apply_ops)."""
    n = 5
    for q in range(n):
        for dag in (True, False):
            m = _dense(n, *fermion_operator_to_pauli([(1.0, [(q, dag)])]))
            for bits in range(1 << n):
                col = m[:, bits]
                r = fock.apply_ops([(q, dag)], bits)
                exp = np.zeros(1 << n)
                if r is not None:
                    exp[r[1]] = r[0]
                assert np.allclose(col, exp), (q, dag, bits)


@pytest.mark.parametrize("m,terms,groups", [(4, 361, 51), (10, 14251, 2536)])
def test_hamiltonian_counts(m, terms, groups):
    """Term and xmask-group counts of the random-integral JW Hamiltonian.

    Groups: 1 + 2C(m,2) + C(m,2)^2 + 2C(m,4) distinct xmasks (x = 0; one-body
    and same-spin pairs; alpha-beta quadruples; same-spin quadruples).
    """
    h, eri = random_integrals(m, 0)
    x, z, c = qubit_hamiltonian(h, eri)
    assert len(c) == terms
    assert len(group_starts(x)) - 1 == groups
    assert groups == 1 + 2 * comb(m, 2) + comb(m, 2) ** 2 + 2 * comb(m, 4)


def test_hamiltonian_hermitian_real_even_y():
    h, eri = random_integrals(4, 3)
    x, z, c = qubit_hamiltonian(h, eri)
    assert c.dtype == np.float64
    assert np.all(popcount(x & z) % 2 == 0)          # even Y count <=> real Hermitian term
    H = _dense(8, x, z, c)
    assert np.allclose(H, H.conj().T)
    assert np.allclose(H.imag, 0)
    # sorted by (x, z) and unique
    key = x.astype(object) * (1 << 64) + z.astype(object)
    assert list(key) == sorted(set(key))


def test_integrals_symmetry():
    h, eri = random_integrals(5, 7)
    assert np.allclose(h, h.T)
    for perm in [(1, 0, 2, 3), (0, 1, 3, 2), (2, 3, 0, 1), (3, 2, 1, 0)]:
        assert np.array_equal(eri, eri.transpose(perm))


@pytest.mark.parametrize("n,ne", [(8, 4), (20, 10), (24, 12), (32, 16)])
def test_uccsd_counts(n, ne):
    """All-pairs set: C(ne,2) C(n-ne,2) doubles (8 strings) + ne(n-ne) singles (2 strings)."""
    nd = comb(ne, 2) * comb(n - ne, 2)
    ns = ne * (n - ne)
    assert len(excitations(n, ne)) == nd + ns
    if n <= 24:
        a = uccsd_rotations(n, ne)
        assert a.n_rot == 8 * nd + 2 * ns
        assert a.n_params == nd + ns
        assert set(np.round(np.abs(a.coef), 12)) == {1.0, 0.25}


def test_uccsd_strings_commute_within_excitation_and_are_imaginary():
    a = uccsd_rotations(8, 4)
    assert np.all(popcount(a.x & a.z) % 2 == 1)       # odd Y count: T - T^+ is real antisymmetric
    for k in range(a.n_params):
        idx = np.flatnonzero(a.param == k)
        assert len(set(a.x[idx])) == 1                  # one xmask per excitation
        for i, j in combinations(idx, 2):
            s = popcount(np.array([(a.x[i] & a.z[j]) ^ (a.z[i] & a.x[j])]))[0]
            assert s % 2 == 0


def test_uccsd_generator_is_t_minus_tdagger():
    """sum_j i c_j P_j equals T - T^+ as a dense matrix, T from the Fock sign rule."""
    n, ne = 6, 2
    a = uccsd_rotations(n, ne)
    for k, (ops, _) in enumerate(excitations(n, ne)):
        idx = a.param == k
        G = _dense(n, a.x[idx], a.z[idx], 1j * (-a.coef[idx] / 2))
        T = np.zeros((1 << n, 1 << n))
        for b in range(1 << n):
            r = fock.apply_ops(ops, b)
            if r is not None:
                T[r[1], b] = r[0]
        assert np.allclose(G, T - T.T), k


def _table1():
    rows = []
    with open(os.path.join(GOLD, "table1_uccsd_params.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            mol, q, e, p, exp = line.split()
            rows.append((mol, int(q), int(e), int(p), exp))
    return rows


@pytest.mark.parametrize("row", _table1(), ids=lambda r: r[0])
def test_table1_parameter_counts(row):
    mol, q, e, p, exp = row
    got = len(excitations(q, e, "paper_spin_adapted"))
    o, v = e // 2, q // 2 - e // 2
    assert got == o * v + o * v * (o * v + 1) // 2
    assert (got == p) == (exp == "match")


def test_table1_h2_cnot_count():
    with open(os.path.join(GOLD, "table1_h2_cnot.txt")) as f:
        mol, q, e, cn = [l for l in f if not l.startswith("#")][0].split()
    a = uccsd_rotations(int(q), int(e), "paper_spin_adapted")
    assert a.n_params == 2
    assert cnot_count(a.x, a.z) == int(cn)


def test_workloads_shapes():
    w = uccsd_energy(8, 4, seed=0)
    assert (w.ham.n_terms, w.ham.n_groups, w.ansatz.n_rot, len(w.theta)) == (361, 51, 320, 52)
    assert abs(np.std(uccsd_energy(20, 10, seed=1).theta) - 0.05) < 0.005
    reqs = served_stream(seed=0, n_requests=300)
    assert all(r.n in range(10, 27, 2) and r.n_elec == r.n // 2 for r in reqs)
    assert 0.3 < np.mean([r.want_grad for r in reqs]) < 0.5
    assert all(b.arrival_s > a.arrival_s for a, b in zip(reqs, reqs[1:]))


@pytest.mark.slow
def test_sweep32_shape():
    w = sweep32(seed=0)
    assert w.ansatz.n_rot == 50_000
    assert w.ham.n_terms >= 30_000
    assert w.ham.x[0] == 0
    assert int(np.max(w.ansatz.x | w.ansatz.z)) < (1 << 32)
