"""Second-quantized Hamiltonian on occupation-number determinants.

Independent of any Pauli algebra: operators act on determinant bit strings
with the canonical sign rule (spin-orbitals ordered by index),

    a_q^dagger |n> = (-1)^{sum_{k<q} n_k} |n + e_q>   (0 if n_q = 1),
    a_q        |n> = (-1)^{sum_{k<q} n_k} |n - e_q>   (0 if n_q = 0),

which is what the Jordan-Wigner mapping has to reproduce.  The Hamiltonian is
the reading of Eq. ferm-ham used throughout (chemists' integrals, 1/2 in
front of the two-electron sum, spin-orbital q = 2*spatial + spin):

    H = sum_{PQ} h_PQ a+_P a_Q + 1/2 sum_{PQRS} (PQ|RS) a+_P a+_R a_S a_Q,
    h_PQ = h_pq delta(s_P, s_Q),  (PQ|RS) = (pq|rs) delta(s_P, s_Q) delta(s_R, s_S).

Pure-Python loops; meant for small cases and sampled matrix elements.
"""

from itertools import combinations

import numpy as np


def apply_ops(ops, bits):
    """Apply prod of ladder ops (list of (q, dagger), leftmost applied last).

    Returns (sign, new_bits) or None when the result vanishes.
    """
    sign = 1
    for q, dagger in reversed(ops):
        occ = (bits >> q) & 1
        if dagger == bool(occ):
            return None
        if bin(bits & ((1 << q) - 1)).count("1") & 1:
            sign = -sign
        bits ^= 1 << q
    return sign, bits


def _so_h(h, P, Q):
    return h[P // 2, Q // 2] if (P & 1) == (Q & 1) else 0.0


def _so_eri(eri, P, Q, R, S):
    if (P & 1) != (Q & 1) or (R & 1) != (S & 1):
        return 0.0
    return eri[P // 2, Q // 2, R // 2, S // 2]


def hamiltonian_apply(h, eri, n, bits):
    """H |bits> as a dict {bits': amplitude}."""
    out = {}
    occ = [q for q in range(n) if (bits >> q) & 1]
    for Q in occ:
        for P in range(n):
            v = _so_h(h, P, Q)
            if v == 0.0:
                continue
            r = apply_ops([(P, True), (Q, False)], bits)
            if r is not None:
                out[r[1]] = out.get(r[1], 0.0) + v * r[0]
    for Q in occ:
        for S in occ:
            if S == Q:
                continue
            for P in range(n):
                for R in range(n):
                    if P == R:
                        continue
                    v = _so_eri(eri, P, Q, R, S)
                    if v == 0.0:
                        continue
                    r = apply_ops([(P, True), (R, True), (S, False), (Q, False)], bits)
                    if r is not None:
                        out[r[1]] = out.get(r[1], 0.0) + 0.5 * v * r[0]
    return out


def determinants(n, n_elec):
    """All n_elec-electron determinants of n spin-orbitals, ascending."""
    return sorted(sum(1 << q for q in c) for c in combinations(range(n), n_elec))


def fci_matrix(h, eri, n, n_elec):
    """Hamiltonian matrix in the n_elec-electron determinant basis."""
    dets = determinants(n, n_elec)
    pos = {d: k for k, d in enumerate(dets)}
    H = np.zeros((len(dets), len(dets)))
    for j, d in enumerate(dets):
        for b, v in hamiltonian_apply(h, eri, n, d).items():
            H[pos[b], j] += v
    return dets, H


def matrix_element(h, eri, n, bra, ket):
    """<bra|H|ket> by the definition, summing only operators that can connect."""
    occ_k = [q for q in range(n) if (ket >> q) & 1]
    occ_b = [q for q in range(n) if (bra >> q) & 1]
    v = 0.0
    for Q in occ_k:
        for P in occ_b:
            hv = _so_h(h, P, Q)
            if hv == 0.0:
                continue
            r = apply_ops([(P, True), (Q, False)], ket)
            if r is not None and r[1] == bra:
                v += hv * r[0]
    for Q in occ_k:
        for S in occ_k:
            if S == Q:
                continue
            for P in occ_b:
                for R in occ_b:
                    if P == R:
                        continue
                    ev = _so_eri(eri, P, Q, R, S)
                    if ev == 0.0:
                        continue
                    r = apply_ops([(P, True), (R, True), (S, False), (Q, False)], ket)
                    if r is not None and r[1] == bra:
                        v += 0.5 * ev * r[0]
    return v


def hf_energy(h, eri, n_elec):
    """Closed form E_HF = sum_i h_ii + 1/2 sum_ij [(ii|jj) - delta_s (ij|ji)].

    Sums over occupied spin-orbitals 0..n_elec-1 (open shells included).
    """
    occ = range(n_elec)
    e = sum(h[i // 2, i // 2] for i in occ)
    for i in occ:
        for j in occ:
            p, q = i // 2, j // 2
            e += 0.5 * eri[p, p, q, q]
            if (i & 1) == (j & 1):
                e -= 0.5 * eri[p, q, q, p]
    return float(e)


def determinant_energy(h, eri, occ_list):
    """Diagonal element <D|H|D> for the determinant with the given occupied list."""
    e = sum(h[i // 2, i // 2] for i in occ_list)
    for i in occ_list:
        for j in occ_list:
            p, q = i // 2, j // 2
            e += 0.5 * eri[p, p, q, q]
            if (i & 1) == (j & 1):
                e -= 0.5 * eri[p, q, q, p]
    return float(e)


def single_excitation_energy(h, eri, n, n_elec, ops, theta):
    """E(theta) for exp(theta (T - T^dagger))|HF> with T one excitation.

    T|HF> = s |Phi> and T^dagger |HF> = 0, so the state is
    cos(theta)|HF> + s sin(theta)|Phi> and
    E = cos^2 E_HF + sin^2 E_Phi + s sin(2 theta) <HF|H|Phi>.
    Returns (E, s, phi_bits, coupling <HF|H|Phi>).
    """
    hf = (1 << n_elec) - 1
    s, phi = apply_ops(ops, hf)
    e_hf = hf_energy(h, eri, n_elec)
    e_phi = determinant_energy(h, eri, [q for q in range(n) if (phi >> q) & 1])
    v = matrix_element(h, eri, n, hf, phi)
    c, sn = np.cos(theta), np.sin(theta)
    return c * c * e_hf + sn * sn * e_phi + s * np.sin(2 * theta) * v, s, phi, v
