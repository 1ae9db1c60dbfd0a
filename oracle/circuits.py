"""Algorithm 2 (exp(i theta P) -> gates) as dense matrices on small registers.

Algorithm 2 changes the basis of every X qubit with H and every Y qubit with
HY = (Z + Y)/sqrt(2), collects the parity of the string onto one qubit with
a CNOT ladder, applies RZ(-2 theta) = exp(i theta Z) there, and undoes the
ladder and the basis change.  As printed, its ladder runs over all qubits
while RZ sits on the last qubit regardless of the support; the reading used
here runs the ladder over the string's support only (identity qubits take
no gates), CNOT(control s_k, target s_{k+1}) for consecutive support qubits,
RZ on the last support qubit, and the reverse ladder afterwards.  The gate
count of this reading is 2(|support| - 1) CNOTs per string.
"""

import numpy as np

_I2 = np.eye(2, dtype=np.complex128)
_H = np.array([[1, 1], [1, -1]], dtype=np.complex128) / np.sqrt(2)
_Y = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
_Z = np.array([[1, 0], [0, -1]], dtype=np.complex128)
_HY = (_Z + _Y) / np.sqrt(2)


def _one_qubit(n, q, g):
    m = np.eye(1, dtype=np.complex128)
    for k in range(n - 1, -1, -1):
        m = np.kron(m, g if k == q else _I2)
    return m


def _cnot(n, c, t):
    dim = 1 << n
    m = np.zeros((dim, dim), dtype=np.complex128)
    for i in range(dim):
        j = i ^ (1 << t) if (i >> c) & 1 else i
        m[j, i] = 1.0
    return m


def _rz(n, q, angle):
    # RZ(angle) = exp(-i angle/2 Z)
    g = np.diag([np.exp(-0.5j * angle), np.exp(0.5j * angle)])
    return _one_qubit(n, q, g)


def exp_pauli_circuit(n, x, z, theta):
    """Gate list for exp(i theta P), P = (x, z); returns list of dense matrices."""
    sup = [q for q in range(n) if ((x | z) >> q) & 1]
    gates = []
    basis = []
    for q in sup:
        xq, zq = (x >> q) & 1, (z >> q) & 1
        if xq and not zq:
            basis.append(_one_qubit(n, q, _H))
        elif xq and zq:
            basis.append(_one_qubit(n, q, _HY))
    gates += basis
    ladder = [_cnot(n, sup[k], sup[k + 1]) for k in range(len(sup) - 1)]
    gates += ladder
    if sup:
        gates.append(_rz(n, sup[-1], -2.0 * theta))
    gates += ladder[::-1]
    gates += basis[::-1]
    return gates


def circuit_unitary(gates, n):
    u = np.eye(1 << n, dtype=np.complex128)
    for g in gates:
        u = g @ u
    return u


def cnot_count(xs, zs):
    """CNOTs of the support-only reading: sum 2(|supp| - 1) over strings."""
    return int(sum(2 * (bin(int(x) | int(z)).count("1") - 1) for x, z in zip(xs, zs)))
