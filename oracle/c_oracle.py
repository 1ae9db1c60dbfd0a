"""ctypes loader for the plain-C oracle (test infrastructure only).

``build()`` compiles ``c/q2_oracle.c`` with gcc (OpenMP) into
``c/_build/libq2oracle.so``; the functions below wrap its entry points with
NumPy arrays.  The state is a complex128 NumPy array (interleaved re, im).
"""

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "c", "q2_oracle.c")
_OUT_DIR = os.path.join(_HERE, "c", "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "libq2oracle.so")
_lock = threading.Lock()
_lib = None


def build(force=False):
    """Compile the C oracle; returns the path of the shared library."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-o", tmp,
                        _SRC, "-lm"], check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB_PATH)
            P = ctypes.c_void_p
            I64 = ctypes.c_int64
            L.q2o_apply_rotations.argtypes = [ctypes.c_int, P, I64, P, P, P]
            L.q2o_expectation.argtypes = [ctypes.c_int, P, I64, P, P, P, P, P]
            L.q2o_apply_hamiltonian.argtypes = [ctypes.c_int, P, P, I64, P, P, P]
            L.q2o_energy_grad.argtypes = [ctypes.c_int, ctypes.c_int, I64, P, P, P, I64, P, P, P, P, P]
            L.q2o_hf_state.argtypes = [ctypes.c_int, ctypes.c_int, P]
            L.q2o_max_threads.restype = ctypes.c_int
            L.q2o_set_threads.argtypes = [ctypes.c_int]
            _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _u64(a):
    return np.ascontiguousarray(a, dtype=np.uint64)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def threads():
    return lib().q2o_max_threads()


def set_threads(t):
    lib().q2o_set_threads(int(t))


def hf_state(n, n_elec):
    psi = np.empty(1 << n, dtype=np.complex128)
    lib().q2o_hf_state(n, n_elec, _p(psi))
    return psi


def apply_rotations(psi, n, xs, zs, phis):
    psi = np.ascontiguousarray(psi, dtype=np.complex128).copy()
    xs, zs, phis = _u64(xs), _u64(zs), _f64(phis)
    if lib().q2o_apply_rotations(n, _p(psi), len(phis), _p(xs), _p(zs), _p(phis)) != 0:
        raise MemoryError("C oracle: allocation failed")
    return psi


def expectation(psi, n, xs, zs, cs):
    """Returns (sum_t c_t <P_t>, <psi|psi>)."""
    psi = np.ascontiguousarray(psi, dtype=np.complex128)
    xs, zs, cs = _u64(xs), _u64(zs), _f64(cs)
    e = np.zeros(1)
    nrm = np.zeros(1)
    lib().q2o_expectation(n, _p(psi), len(cs), _p(xs), _p(zs), _p(cs), _p(e), _p(nrm))
    return float(e[0]), float(nrm[0])


def apply_hamiltonian(psi, n, xs, zs, cs):
    psi = np.ascontiguousarray(psi, dtype=np.complex128)
    lam = np.empty_like(psi)
    xs, zs, cs = _u64(xs), _u64(zs), _f64(cs)
    lib().q2o_apply_hamiltonian(n, _p(psi), _p(lam), len(cs), _p(xs), _p(zs), _p(cs))
    return lam


def energy_and_gradient(n, n_elec, rx, rz, phis, hx, hz, hc):
    rx, rz, phis = _u64(rx), _u64(rz), _f64(phis)
    hx, hz, hc = _u64(hx), _u64(hz), _f64(hc)
    e = np.zeros(1)
    g = np.zeros(len(phis))
    if lib().q2o_energy_grad(n, n_elec, len(phis), _p(rx), _p(rz), _p(phis), len(hc), _p(hx),
                             _p(hz), _p(hc), _p(e), _p(g)) != 0:
        raise MemoryError("C oracle: allocation failed")
    return float(e[0]), g
