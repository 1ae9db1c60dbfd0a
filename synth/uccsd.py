"""UCCSD excitations and their single-Trotter-step Pauli-rotation sequence.

Eq. ucc writes the UCC state as exp(T - T^dagger)|HF>; after the JW mapping
the paper applies a first-order Trotter product of one exponential per Pauli
string (the product formula following Eq. ucc).  For excitation k with
generator G_k = T_k - T_k^dagger the mapping gives G_k = sum_j i c_kj P_kj
with real c_kj, so

    exp(theta_k G_k) -> prod_j exp(i theta_k c_kj P_kj)
                      = prod_j exp(-i phi_kj / 2 P_kj),  phi_kj = -2 c_kj theta_k.

The rotation list therefore stores, per string, (x, z, param index k,
coef = -2 c_kj) and the angle is phi = coef * theta[param].

Excitation sets (the paper says "spin-adapted CCD0" operators; Table 1's
parameter counts equal ov + ov(ov+1)/2; the benchmark size "~16k Pauli
rotations at 20 qubits" equals the spin-orbital all-pairs set):
  * "all_pairs" (default): singles i in occ, a in virt; doubles i<j in occ,
    a<b in virt, all over spin-orbitals.  T = a+_a a_i, resp. a+_a a+_b a_j a_i.
  * "spin_conserving": the subset that conserves S_z.
  * "paper_spin_adapted": spatial singles E_ai = sum_s a+_{as} a_{is} and
    pair doubles E_ai E_bj for (i,a) <= (j,b) (ov + ov(ov+1)/2 parameters).
Order: singles then doubles, lexicographic; strings inside an excitation
sorted by (x, z).
"""

from dataclasses import dataclass, field
from itertools import combinations

import numpy as np

from .jw import _expand_products, U64


def excitations(n, n_elec, kind="all_pairs"):
    """List of excitations as (tuple of (q, dagger) ops, tag) in ansatz order.

    HF occupies spin-orbitals 0..n_elec-1 (qubit index = spin-orbital).
    """
    occ = list(range(n_elec))
    vir = list(range(n_elec, n))
    out = []
    if kind in ("all_pairs", "spin_conserving"):
        for i in occ:
            for a in vir:
                if kind == "spin_conserving" and (i % 2) != (a % 2):
                    continue
                out.append(([(a, True), (i, False)], ("s", i, a)))
        for i, j in combinations(occ, 2):
            for a, b in combinations(vir, 2):
                if kind == "spin_conserving" and sorted((i % 2, j % 2)) != sorted((a % 2, b % 2)):
                    continue
                out.append(([(a, True), (b, True), (j, False), (i, False)], ("d", i, j, a, b)))
        return out
    if kind == "paper_spin_adapted":
        if n % 2 or n_elec % 2:
            raise ValueError("spin-adapted set needs even n and n_elec")
        o = list(range(n_elec // 2))
        v = list(range(n_elec // 2, n // 2))
        ia = [(i, a) for i in o for a in v]
        for (i, a) in ia:
            ops = [[(2 * a + s, True), (2 * i + s, False)] for s in (0, 1)]
            out.append((ops, ("S", i, a)))
        for u in range(len(ia)):
            for w in range(u, len(ia)):
                (i, a), (j, b) = ia[u], ia[w]
                ops = [[(2 * a + s, True), (2 * i + s, False), (2 * b + t, True), (2 * j + t, False)]
                       for s in (0, 1) for t in (0, 1)]
                out.append((ops, ("D", i, a, j, b)))
        return out
    raise ValueError(f"unknown excitation set {kind!r}")


def _generator_strings(exc_list):
    """Pauli strings of G_k = T_k - T_k^dagger for every excitation.

    Returns arrays (k, x, z, c) with G_k = sum i c P, sorted by (k, x, z).
    """
    ks, xs, zs, res, ims = [], [], [], [], []
    # Bucket products by their dagger pattern so each bucket is vectorized.
    buckets = {}
    for k, (ops, _tag) in enumerate(exc_list):
        prods = ops if isinstance(ops[0], list) else [ops]
        for prod in prods:
            dag = tuple(d for _, d in prod)
            buckets.setdefault(dag, []).append((k, [q for q, _ in prod], 1.0))
            # T^dagger: reversed order with daggers flipped, weight -1
            rdag = tuple(not d for _, d in reversed(prod))
            buckets.setdefault(rdag, []).append((k, [q for q, _ in reversed(prod)], -1.0))
    for dag, items in buckets.items():
        kk = np.array([t[0] for t in items], dtype=np.int64)
        idx = np.array([t[1] for t in items], dtype=np.int64)
        w = np.array([t[2] for t in items])
        x, z, re, im = _expand_products(idx, dag, w)
        ks.append(np.tile(kk, 1 << len(dag)))
        xs.append(x)
        zs.append(z)
        res.append(re)
        ims.append(im)
    k = np.concatenate(ks)
    x = np.concatenate(xs)
    z = np.concatenate(zs)
    re = np.concatenate(res)
    im = np.concatenate(ims)
    order = np.lexsort((z, x, k))
    k, x, z, re, im = k[order], x[order], z[order], re[order], im[order]
    new = np.ones(len(k), dtype=bool)
    new[1:] = (k[1:] != k[:-1]) | (x[1:] != x[:-1]) | (z[1:] != z[:-1])
    st = np.flatnonzero(new)
    k, x, z = k[st], x[st], z[st]
    re = np.add.reduceat(re, st)
    im = np.add.reduceat(im, st)
    if len(re) and np.max(np.abs(re)) > 1e-12:
        raise AssertionError("T - T^dagger must map to i * (real) Pauli coefficients")
    keep = np.abs(im) > 1e-13
    return k[keep], x[keep], z[keep], im[keep]


@dataclass
class UccsdAnsatz:
    """Single-Trotter-step UCCSD rotation list (see module docstring)."""
    n: int
    n_elec: int
    x: np.ndarray          # uint64 per rotation
    z: np.ndarray          # uint64 per rotation
    param: np.ndarray      # int32 parameter index per rotation
    coef: np.ndarray       # float64, phi = coef * theta[param]
    n_params: int
    tags: list = field(default_factory=list)

    @property
    def n_rot(self):
        return len(self.x)

    def angles(self, theta):
        theta = np.asarray(theta, dtype=np.float64)
        return self.coef * theta[self.param]

    @property
    def hf_index(self):
        return (1 << self.n_elec) - 1


def uccsd_rotations(n, n_elec, kind="all_pairs", exc_list=None):
    """Build the UccsdAnsatz for n qubits and n_elec electrons."""
    if exc_list is None:
        exc_list = excitations(n, n_elec, kind)
    if len(exc_list) == 0:
        e = np.zeros(0, dtype=U64)
        return UccsdAnsatz(n, n_elec, e, e, np.zeros(0, np.int32), np.zeros(0), 0, [])
    k, x, z, c = _generator_strings(exc_list)
    return UccsdAnsatz(n, n_elec, x, z, k.astype(np.int32), -2.0 * c,
                       len(exc_list), [t for _, t in exc_list])
