"""Plain complex128 state-vector definitions (test infrastructure only).

Every function is the textbook definition, vectorised over the amplitude
index with NumPy and nothing else: no blocking, fusion or reordering.

Conventions: qubit q is bit q of the index; a Pauli string (x, z) is
P = i^{|x&z|} X^x Z^z; a rotation (x, z, phi) is exp(-i phi/2 P).
"""

import numpy as np


def _popcount(a):
    a = np.asarray(a, dtype=np.uint64)
    if hasattr(np, "bitwise_count"):
        return np.bitwise_count(a).astype(np.int64)
    out = np.zeros(a.shape, dtype=np.int64)
    b = a.copy()
    for _ in range(64):
        out += (b & np.uint64(1)).astype(np.int64)
        b >>= np.uint64(1)
    return out


def hf_state(n, n_elec):
    """|HF> of Eq. jw-wfn-map: qubits 0..n_elec-1 in |1>, index 2^n_elec - 1."""
    psi = np.zeros(1 << n, dtype=np.complex128)
    psi[(1 << n_elec) - 1] = 1.0
    return psi


def apply_pauli(psi, x, z):
    """(P psi)[i] = i^{|x&z|} (-1)^{|(i^x) & z|} psi[i ^ x]."""
    x = np.uint64(x)
    z = np.uint64(z)
    i = np.arange(len(psi), dtype=np.uint64)
    src = i ^ x
    ny = int(_popcount(np.array([x & z]))[0])
    sign = 1.0 - 2.0 * (_popcount(src & z) & 1)
    return (1j ** ny) * sign * psi[src]


def apply_rotation(psi, x, z, phi):
    """exp(-i phi/2 P) psi = cos(phi/2) psi - i sin(phi/2) P psi  (P^2 = 1)."""
    return np.cos(phi / 2) * psi - 1j * np.sin(phi / 2) * apply_pauli(psi, x, z)


def apply_rotations(psi, xs, zs, phis):
    """Apply rotations k = 0, 1, ... in order (product formula after Eq. ucc)."""
    for x, z, phi in zip(xs, zs, phis):
        psi = apply_rotation(psi, x, z, phi)
    return psi


def pauli_expectations(psi, xs, zs):
    """<psi|P_t|psi> for every string (real parts; P_t is Hermitian)."""
    return np.array([np.vdot(psi, apply_pauli(psi, x, z)).real for x, z in zip(xs, zs)])


def expectation(psi, xs, zs, cs):
    """E = sum_t c_t <psi|P_t|psi>  (Eq. qubit-ham-detail), unnormalised."""
    return float(np.dot(np.asarray(cs, dtype=np.float64), pauli_expectations(psi, xs, zs)))


def energy(psi, xs, zs, cs):
    """Normalised energy <psi|H|psi> / <psi|psi> and the norm <psi|psi>."""
    nrm = float(np.vdot(psi, psi).real)
    return expectation(psi, xs, zs, cs) / nrm, nrm


def apply_hamiltonian(psi, xs, zs, cs):
    """lambda = H psi = sum_t c_t P_t psi."""
    lam = np.zeros_like(psi)
    for x, z, c in zip(xs, zs, cs):
        lam += c * apply_pauli(psi, x, z)
    return lam


def energy_and_gradient(n, n_elec, rot_x, rot_z, phis, ham_x, ham_z, ham_c):
    """Reverse-mode gradient (Algorithm 1) with respect to each rotation angle.

    Forward: psi = U_N ... U_1 |HF>.  Then lambda = H psi.  Reverse over
    k = N .. 1:  g[k] = dE/dphi_k = Im <lambda|P_k|psi>, then
    psi <- U_k^dagger psi, lambda <- U_k^dagger lambda.

    The reading of Algorithm 1: it un-rotates psi before evaluating its
    dU/dtheta term; taking the derivative with both vectors at the same
    point before the un-rotation is the same quantity, because
    dU_k/dphi_k = -(i/2) P_k U_k, so dE/dphi_k = 2 Re <lambda_k|(-i/2) P_k psi_k>
    = Im <lambda_k|P_k|psi_k>.  Returns (E, g) with E = <psi|H|psi>.
    """
    psi = apply_rotations(hf_state(n, n_elec), rot_x, rot_z, phis)
    lam = apply_hamiltonian(psi, ham_x, ham_z, ham_c)
    e = float(np.vdot(psi, lam).real)
    g = np.zeros(len(phis))
    for k in range(len(phis) - 1, -1, -1):
        g[k] = np.vdot(lam, apply_pauli(psi, rot_x[k], rot_z[k])).imag
        psi = apply_rotation(psi, rot_x[k], rot_z[k], -phis[k])
        lam = apply_rotation(lam, rot_x[k], rot_z[k], -phis[k])
    return e, g


def fold_to_theta(g_phi, param, coef, n_params):
    """dE/dtheta_p = sum_{j: param_j = p} coef_j dE/dphi_j  (phi_j = coef_j theta_p)."""
    out = np.zeros(n_params)
    np.add.at(out, np.asarray(param), np.asarray(coef) * np.asarray(g_phi))
    return out


def energy_of_angles(n, n_elec, rot_x, rot_z, phis, ham_x, ham_z, ham_c):
    psi = apply_rotations(hf_state(n, n_elec), rot_x, rot_z, phis)
    return expectation(psi, ham_x, ham_z, ham_c)


def parameter_shift(n, n_elec, rot_x, rot_z, phis, ham_x, ham_z, ham_c, k):
    """dE/dphi_k = [E(phi_k + pi/2) - E(phi_k - pi/2)] / 2 (P_k has eigenvalues +-1)."""
    p = np.array(phis, dtype=np.float64)
    p[k] += np.pi / 2
    ep = energy_of_angles(n, n_elec, rot_x, rot_z, p, ham_x, ham_z, ham_c)
    p[k] -= np.pi
    em = energy_of_angles(n, n_elec, rot_x, rot_z, p, ham_x, ham_z, ham_c)
    return 0.5 * (ep - em)


# ---- dense-matrix restatements used only to pin the above on small registers

_PAULI = {
    (0, 0): np.eye(2, dtype=np.complex128),
    (1, 0): np.array([[0, 1], [1, 0]], dtype=np.complex128),
    (0, 1): np.array([[1, 0], [0, -1]], dtype=np.complex128),
    (1, 1): np.array([[0, -1j], [1j, 0]], dtype=np.complex128),
}


def dense_pauli(n, x, z):
    """Kronecker product of single-qubit I/X/Y/Z; qubit 0 is the fastest index."""
    m = np.eye(1, dtype=np.complex128)
    for q in range(n - 1, -1, -1):
        m = np.kron(m, _PAULI[((int(x) >> q) & 1, (int(z) >> q) & 1)])
    return m


def dense_hamiltonian(n, xs, zs, cs):
    h = np.zeros((1 << n, 1 << n), dtype=np.complex128)
    for x, z, c in zip(xs, zs, cs):
        h += c * dense_pauli(n, x, z)
    return h
