"""Seeded synthetic inputs shared by the oracle tests and the CUDA path.

This package produces *inputs only*: random one- and two-electron integrals,
the Jordan-Wigner qubit Hamiltonian H = sum_i c_i P_i built from them
(Sec. "Hamiltonian", Eq. qubit-ham and Eq. ferm-ham), the UCCSD excitation
list and its single-Trotter-step Pauli-rotation sequence (Sec. "Variational
quantum circuit ansatz", Eq. ucc and the product formula after it), and the
workload builders for the benchmark configurations.

None of the state-vector arithmetic (rotation sweep, expectation, adjoint
gradient) lives here; that is implemented independently by ``oracle/`` (the
reference used by the tests) and by the CUDA library.

Conventions (readings of the paper, which leaves them open):
  * qubit q is bit q of the amplitude index (little endian);
  * spin-orbital q = 2*p + sigma for spatial orbital p (sigma=0 alpha, 1 beta);
  * |1> on qubit q means spin-orbital q is occupied (Eq. jw-wfn-map);
  * a Pauli string (x, z) is P = i^{popcount(x & z)} X^x Z^z, so qubit q
    carries I, X, Z or Y for (x_q, z_q) = (0,0), (1,0), (0,1), (1,1);
  * a rotation (x, z, phi) is exp(-i phi/2 P).
"""

from .integrals import random_integrals
from .jw import qubit_hamiltonian, fermion_operator_to_pauli
from .uccsd import (
    excitations,
    uccsd_rotations,
    UccsdAnsatz,
)

__all__ = [
    "random_integrals",
    "qubit_hamiltonian",
    "fermion_operator_to_pauli",
    "excitations",
    "uccsd_rotations",
    "UccsdAnsatz",
]
