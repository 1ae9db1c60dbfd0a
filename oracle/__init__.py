"""CPU oracle for the state-vector UCCSD-VQE hot path (test infrastructure).

This package is test infrastructure: only the tests, ``__graft_entry__.smoke``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import
or run it.  The library's compute path never routes through it.

It restates what the paper defines, plainly and in complex128:

  statevector.py   Eq. sv state, Eq. jw-wfn-map HF determinant, Pauli-string
                   action, exp(-i phi/2 P) rotations (product formula after
                   Eq. ucc), Eq. qubit-ham-detail expectation, H|psi>, and the
                   reverse-mode gradient of Algorithm 1.
  fock.py          Eq. ferm-ham acting on occupation-number determinants
                   (no Pauli algebra), FCI matrices, the Hartree-Fock energy
                   closed form and single-excitation matrix elements.
  circuits.py      Algorithm 2 (exp(i theta P) as basis change + CNOT ladder
                   + RZ), as dense gate products on small registers.
  sparse.py        dict-of-amplitudes state for a few rotations on up to
                   64 qubits (checks high index bits without a 2^n vector).
  c/q2_oracle.c    the same state-vector definitions as plain C loops in
                   double precision (OpenMP over amplitudes), used for the
                   larger goldens and as the timed CPU baseline.

It shares no code with the CUDA library.
"""
