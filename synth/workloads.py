"""Seeded workloads shaped like the paper's UCCSD-VQE problems.

Each builder returns a ``Workload`` holding inputs only (integrals, the
qubit Hamiltonian table, the rotation list and theta).  Sizes:

  uccsd_energy(8, 4)      8 qubits, 320 rotations, 361 terms in 51 xmask groups
  uccsd_energy(20, 10)    20 qubits, 16,400 rotations, 14,251 terms / 2,536 groups
  uccsd_energy(24, 12)    24 qubits, 35,136 rotations over 4,500 parameters
  sweep32()               32 qubits, 50,000 rotations from randomly ordered
                          UCCSD excitations, ~30k-term Hamiltonian made of
                          whole xmask groups of the full 32-qubit Hamiltonian
  served_stream()         Poisson request stream over 10..26 qubits

Theta is drawn N(0, 0.05) (0.05 read as the standard deviation) from a
stream separate from the integrals.
"""

from dataclasses import dataclass

import numpy as np

from .integrals import random_integrals
from .jw import qubit_hamiltonian, group_starts, U64
from .uccsd import excitations, uccsd_rotations, UccsdAnsatz


@dataclass
class Hamiltonian:
    n: int
    x: np.ndarray   # uint64, sorted by (x, z)
    z: np.ndarray   # uint64
    c: np.ndarray   # float64

    @property
    def n_terms(self):
        return len(self.c)

    @property
    def n_groups(self):
        return len(group_starts(self.x)) - 1


@dataclass
class Workload:
    name: str
    n: int
    n_elec: int
    h: np.ndarray
    eri: np.ndarray
    ham: Hamiltonian
    ansatz: UccsdAnsatz
    theta: np.ndarray

    def angles(self):
        return self.ansatz.angles(self.theta)


def _theta(n_params, seed):
    return np.random.default_rng([seed, 0x7E7A]).normal(0.0, 0.05, size=n_params)


def hamiltonian_from_integrals(h, eri):
    x, z, c = qubit_hamiltonian(h, eri)
    return Hamiltonian(2 * h.shape[0], x, z, c)


def uccsd_energy(n, n_elec, seed=0, kind="all_pairs"):
    """Full UCCSD single Trotter step on n qubits from the HF determinant."""
    if n % 2:
        raise ValueError("n must be even (two spin-orbitals per spatial orbital)")
    h, eri = random_integrals(n // 2, seed)
    ham = hamiltonian_from_integrals(h, eri)
    ans = uccsd_rotations(n, n_elec, kind)
    return Workload(f"uccsd{n}", n, n_elec, h, eri, ham, ans, _theta(ans.n_params, seed))


def _subset_groups(ham, min_terms, rng):
    """Whole xmask groups in seeded random order (x = 0 first) until >= min_terms."""
    st = group_starts(ham.x)
    ng = len(st) - 1
    order = [g for g in rng.permutation(ng) if ham.x[st[g]] != 0]
    zero = [g for g in range(ng) if ham.x[st[g]] == 0]
    chosen, total = [], 0
    for g in zero + order:
        chosen.append(g)
        total += st[g + 1] - st[g]
        if total >= min_terms:
            break
    chosen.sort()
    idx = np.concatenate([np.arange(st[g], st[g + 1]) for g in chosen])
    return Hamiltonian(ham.n, ham.x[idx], ham.z[idx], ham.c[idx])


def sweep_ansatz(n, n_elec, n_rot, seed=0):
    """Random-order UCCSD rotation list: whole all-pairs excitations drawn
    without replacement in a seeded order, strings emitted consecutively,
    cut at n_rot rotations.  Returns (ansatz, theta)."""
    rng = np.random.default_rng([seed, 0x5EED32, n])
    pool = excitations(n, n_elec, "all_pairs")
    perm = rng.permutation(len(pool))
    chosen, count = [], 0
    for k in perm:
        ops, _ = pool[k]
        count += 2 if len(ops) == 2 else 8
        chosen.append(pool[k])
        if count >= n_rot:
            break
    ans = uccsd_rotations(n, n_elec, exc_list=chosen)
    if ans.n_rot > n_rot:
        keep = slice(0, n_rot)
        ans = UccsdAnsatz(n, n_elec, ans.x[keep], ans.z[keep], ans.param[keep],
                          ans.coef[keep], ans.n_params, ans.tags)
    return ans, _theta(ans.n_params, seed)


def sweep32(seed=0, n=32, n_elec=16, n_rot=50_000, min_terms=30_000):
    """32-qubit sweep workload.

    Rotations: whole all-pairs excitations drawn without replacement in a
    seeded random order, each excitation's strings emitted consecutively,
    stopping at n_rot rotations (the last excitation may be cut short).
    Hamiltonian: whole xmask groups of the full random-integral Hamiltonian,
    x = 0 group first then seeded random order, until >= min_terms terms.
    """
    rng = np.random.default_rng([seed, 0x5EED32])
    h, eri = random_integrals(n // 2, seed)
    full = hamiltonian_from_integrals(h, eri)
    ham = _subset_groups(full, min_terms, rng)
    ans, theta = sweep_ansatz(n, n_elec, n_rot, seed)
    return Workload(f"sweep{n}", n, n_elec, h, eri, ham, ans, theta)


@dataclass
class Request:
    rid: int
    arrival_s: float
    n: int
    n_elec: int
    want_grad: bool
    problem_seed: int     # selects integrals and theta (repeats share tables)


def served_stream(seed=0, n_requests=2000, rate_per_s=100.0, n_choices=(10, 12, 14, 16, 18, 20, 22, 24, 26),
                  p_grad=0.4, p_repeat=0.2, repeat_pool=16):
    """Poisson-arrival request stream.

    n uniform over n_choices, n_elec = n/2, want_grad ~ Bernoulli(p_grad);
    with probability p_repeat a request reuses one of ``repeat_pool`` earlier
    problem seeds (same integrals and theta, so resident tables can be reused).
    """
    rng = np.random.default_rng([seed, 0x5E7E])
    t = 0.0
    out = []
    pool = []
    for rid in range(n_requests):
        t += rng.exponential(1.0 / rate_per_s)
        if pool and rng.random() < p_repeat:
            n, ps = pool[rng.integers(len(pool))]
        else:
            n = int(rng.choice(n_choices))
            ps = int(rng.integers(1 << 30))
            if len(pool) < repeat_pool:
                pool.append((n, ps))
        out.append(Request(rid, t, n, n // 2, bool(rng.random() < p_grad), ps))
    return out
