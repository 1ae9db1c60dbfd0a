"""q2_expectation_noalloc: the energy without any device allocation.

Some callers may not allocate device memory while they run (their device
memory belongs to a framework pool that forbids direct driver allocations,
or an allocation's synchronization is not acceptable in their loop).  For
them the library offers this entry point, which keeps its partial sums and a
copy of the Hamiltonian tables in one fixed static device buffer.  The test
calls it through the C ABI twice in a row, with two different Hamiltonians,
and compares each result with q2_expectation's within the tolerances the
other GPU tests use.  It also checks that a Hamiltonian whose tables do not
fit the buffer is rejected before any device work.

This file is collected last so that, if it fails, a run that stops at the
first failure has already run every other test.
"""

import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2208_10978_gb300 as q2
from synth.workloads import uccsd_energy, hamiltonian_from_integrals
from synth import random_integrals

pytestmark = pytest.mark.gpu

TOL_E = {"complex128": 1e-10, "complex64": 1e-5}


def _noalloc(psi, n, ham):
    lib = q2.lib()
    e, nrm = ctypes.c_double(), ctypes.c_double()
    code = q2._dtype_code(psi.dtype)
    st = lib.q2_expectation_noalloc(ctypes.c_void_p(psi.data_ptr()), n, code, ham.handle,
                                    ctypes.byref(e), ctypes.byref(nrm),
                                    ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return st, e.value, nrm.value


@pytest.mark.parametrize("dtype", ["complex64", "complex128"])
def test_noalloc_matches_expectation_twice(dtype):
    n = 14
    rng = np.random.default_rng(77)
    psi0 = rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)
    psi0 /= np.linalg.norm(psi0)
    psi = torch.from_numpy(psi0).to("cuda", getattr(torch, dtype))
    w1 = uccsd_energy(n, n // 2, seed=11)
    ham1 = q2.Hamiltonian(n, w1.ham.x, w1.ham.z, w1.ham.c)
    k = 150
    x2 = rng.integers(0, 1 << n, size=k).astype(np.uint64)
    z2 = rng.integers(0, 1 << n, size=k).astype(np.uint64)
    x2[:10] = 0
    ham2 = q2.Hamiltonian(n, x2, z2, rng.normal(size=k))
    for ham in (ham1, ham2):
        st, e, nrm = _noalloc(psi, n, ham)
        assert st == q2.Q2_OK, q2.lib().q2_last_error()
        e_ref, n_ref = ham.expectation(psi)
        assert abs(e - e_ref) < TOL_E[dtype]
        assert abs(nrm - n_ref) < 1e-12 * max(1.0, n_ref)


def test_noalloc_rejects_tables_beyond_its_buffer():
    h, eri = random_integrals(16, 0)
    big = hamiltonian_from_integrals(h, eri)          # 18,281 xmask groups at 32 qubits
    ham = q2.Hamiltonian(32, big.x, big.z, big.c)
    psi = torch.zeros(16, dtype=torch.complex64, device="cuda")   # never read: rejected first
    st, e, nrm = _noalloc(psi, 32, ham)
    assert st == q2.Q2_ERR_INVALID
    assert b"no-allocation scratch" in q2.lib().q2_last_error()
