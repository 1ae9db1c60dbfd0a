"""GB300 state-vector engine for JW-mapped UCCSD-VQE (arXiv 2208.10978, Q^2Chemistry).

Python binding of ``libq2.so`` (declared in ``include/q2.h``).  This layer only
marshals arguments: device buffers are torch tensors (``data_ptr()`` and the
current CUDA stream are passed through), host tables are NumPy arrays.  All
state-vector work runs in the library's CUDA kernels; when the library cannot
be built or loaded every call raises.

Names follow the paper: the state of Eq. sv, the HF determinant of
Eq. jw-wfn-map, Pauli-string rotations of the UCC product formula (after
Eq. ucc), the energy of Eq. qubit-ham-detail and the reverse-mode gradient of
Algorithm 1.
"""

import ctypes
import os
import threading

import numpy as np

from . import build as _build

Q2_OK, Q2_ERR_INVALID, Q2_ERR_OOM, Q2_ERR_CUDA, Q2_ERR_TIMEOUT, Q2_ERR_UNSUPPORTED = range(6)
C64, C128 = 0, 1

_STATUS = {1: "invalid argument", 2: "out of device memory", 3: "CUDA error", 4: "timeout",
           5: "unsupported"}


class Q2Error(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"q2: {_STATUS.get(status, status)}: {msg}")
        self.status = status


_lock = threading.Lock()
_lib = None

_P = ctypes.c_void_p
_I = ctypes.c_int
_I64 = ctypes.c_int64
_D = ctypes.c_double
_SZ = ctypes.c_size_t

_SIGS = {
    "q2_version": ([], _I),
    "q2_last_error": ([], ctypes.c_char_p),
    "q2_state_init_hf": ([_P, _I, _I, _I, _P], _I),
    "q2_apply_pauli_rotations": ([_P, _I, _I, _P, _P, _P, _I64, _P], _I),
    "q2_ham_create": ([_I, _P, _P, _P, _I64, ctypes.POINTER(_P)], _I),
    "q2_ham_destroy": ([_P], _I),
    "q2_ham_info": ([_P, ctypes.POINTER(_I64), ctypes.POINTER(_I64)], _I),
    "q2_expectation": ([_P, _I, _I, _P, ctypes.POINTER(_D), ctypes.POINTER(_D), _P], _I),
    "q2_apply_hamiltonian": ([_P, _P, _I, _I, _P, _P], _I),
    "q2_ansatz_create": ([_I, _I, _I64, _P, _P, _P, _P, ctypes.c_int32, ctypes.POINTER(_P)], _I),
    "q2_ansatz_destroy": ([_P], _I),
    "q2_ansatz_info": ([_P, _I, ctypes.POINTER(_I64), ctypes.POINTER(_I64)], _I),
    "q2_vqe_workspace_bytes": ([_P, _I, _I], _SZ),
    "q2_vqe_energy_grad": ([_P, _P, _P, _I, _I, ctypes.POINTER(_D), _P, _P, _SZ, _P], _I),
    "q2_batch_workspace_bytes": ([_I, _P, _P, _I], _SZ),
    "q2_batch_energy_grad": ([_I, _P, _P, _P, _P, _I, _P, _P, _P, _SZ, _P], _I),
    "q2_set_tile_qubits": ([_I, _I], _I),
    "q2_expectation_noalloc": ([_P, _I, _I, _P, ctypes.POINTER(_D), ctypes.POINTER(_D), _P], _I),
    "q2_pool_gradients": ([_P, _P, _P, _I, _I64, _P, _P, ctypes.POINTER(_D), _P, _P, _SZ, _P], _I),
    "q2_async_status": ([_P], _I),
    "q2_ham_shard": ([_P, _I, _I, ctypes.POINTER(_P)], _I),
    "q2_ham_shard_terms": ([_P, _I, _P, ctypes.POINTER(_I64)], _I),
    "q2_ham_table_bytes": ([_P, _I, ctypes.POINTER(_SZ)], _I),
    "q2_ansatz_table_bytes": ([_P, _I, ctypes.POINTER(_SZ), ctypes.POINTER(_SZ)], _I),
}


def library_path():
    return _build.LIB


def lib():
    """Load (building first if needed) libq2.so; raises if that fails."""
    global _lib
    with _lock:
        if _lib is None:
            if _build.needs_build():
                _build.build()
            L = ctypes.CDLL(_build.LIB)
            for name, (args, res) in _SIGS.items():
                f = getattr(L, name)
                f.argtypes = args
                f.restype = res
            _lib = L
    return _lib


def _check(status):
    if status != Q2_OK:
        raise Q2Error(status, lib().q2_last_error().decode(errors="replace"))


def _np_ptr(a):
    return ctypes.c_void_p(a.ctypes.data)


def _u64(a):
    return np.ascontiguousarray(np.asarray(a), dtype=np.uint64)


def _f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _torch():
    import torch
    return torch


def _dtype_code(t):
    torch = _torch()
    if t in (torch.complex64, C64, "complex64", "c64"):
        return C64
    if t in (torch.complex128, C128, "complex128", "c128"):
        return C128
    raise ValueError(f"unsupported state dtype {t!r}")


def _torch_dtype(code):
    torch = _torch()
    return torch.complex64 if code == C64 else torch.complex128


def _stream_ptr():
    torch = _torch()
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _state_args(psi, n):
    torch = _torch()
    if not isinstance(psi, torch.Tensor) or not psi.is_cuda:
        raise TypeError("state must be a CUDA torch tensor")
    if not psi.is_contiguous():
        raise ValueError("state must be contiguous")
    if psi.numel() != (1 << n):
        raise ValueError(f"state has {psi.numel()} amplitudes, expected 2^{n}")
    return ctypes.c_void_p(psi.data_ptr()), _dtype_code(psi.dtype)


def new_state(n, dtype="complex64", device="cuda"):
    torch = _torch()
    return torch.empty(1 << n, dtype=_torch_dtype(_dtype_code(dtype)), device=device)


def state_init_hf(psi, n, n_elec):
    """psi <- |HF> = amplitude 1 at index 2^n_elec - 1 (Eq. jw-wfn-map)."""
    p, d = _state_args(psi, n)
    _check(lib().q2_state_init_hf(p, n, n_elec, d, _stream_ptr()))
    return psi


def apply_pauli_rotations(psi, n, x, z, angles):
    """psi <- prod_k exp(-i angles[k]/2 P(x[k], z[k])) psi, k ascending."""
    p, d = _state_args(psi, n)
    x, z, a = _u64(x), _u64(z), _f64(angles)
    if not (len(x) == len(z) == len(a)):
        raise ValueError("x, z and angles must have equal length")
    _check(lib().q2_apply_pauli_rotations(p, n, d, _np_ptr(x), _np_ptr(z), _np_ptr(a), len(a),
                                          _stream_ptr()))
    return psi


class Hamiltonian:
    """H = sum_t c_t P(x_t, z_t) (Eq. qubit-ham), held by the library."""

    def __init__(self, n, x, z, c):
        self.n = int(n)
        x, z, c = _u64(x), _u64(z), _f64(c)
        if not (len(x) == len(z) == len(c)):
            raise ValueError("x, z and c must have equal length")
        h = _P()
        _check(lib().q2_ham_create(self.n, _np_ptr(x), _np_ptr(z), _np_ptr(c), len(c), ctypes.byref(h)))
        self._h = h

    @property
    def handle(self):
        return self._h

    def info(self):
        t, g = _I64(), _I64()
        _check(lib().q2_ham_info(self._h, ctypes.byref(t), ctypes.byref(g)))
        return t.value, g.value

    def expectation(self, psi):
        """(<psi|H|psi>/<psi|psi>, <psi|psi>); synchronizes the current stream."""
        p, d = _state_args(psi, self.n)
        e, nrm = _D(), _D()
        _check(lib().q2_expectation(p, self.n, d, self._h, ctypes.byref(e), ctypes.byref(nrm),
                                    _stream_ptr()))
        return e.value, nrm.value

    def shard(self, shard, n_shards):
        """Shard `shard` of `n_shards` of this Hamiltonian (q2_ham_shard): a handle that evaluates
        only its share of the xmask-group passes; the shards' energies and gradients sum to this
        Hamiltonian's."""
        h = _P()
        _check(lib().q2_ham_shard(self._h, int(shard), int(n_shards), ctypes.byref(h)))
        out = Hamiltonian.__new__(Hamiltonian)
        out.n = self.n
        out._h = h
        return out

    def shard_terms(self, dtype="complex64"):
        """Indices of the terms this handle evaluates for a state dtype (ascending)."""
        cnt = _I64(0)
        _check(lib().q2_ham_shard_terms(self._h, _dtype_code(dtype), None, ctypes.byref(cnt)))
        idx = np.zeros(max(1, cnt.value), dtype=np.int64)
        _check(lib().q2_ham_shard_terms(self._h, _dtype_code(dtype), _np_ptr(idx), ctypes.byref(cnt)))
        return idx[:cnt.value]

    def table_bytes(self, dtype="complex64"):
        """Device bytes of this Hamiltonian's resident tables for a state dtype."""
        b = _SZ()
        _check(lib().q2_ham_table_bytes(self._h, _dtype_code(dtype), ctypes.byref(b)))
        return b.value

    def apply(self, psi, lam):
        """lam <- H psi."""
        p, d = _state_args(psi, self.n)
        q, d2 = _state_args(lam, self.n)
        if d != d2:
            raise ValueError("psi and lam dtypes differ")
        _check(lib().q2_apply_hamiltonian(p, q, self.n, d, self._h, _stream_ptr()))
        return lam

    def close(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.q2_ham_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Ansatz:
    """Rotation list of the single-Trotter-step UCC circuit (after Eq. ucc).

    Rotation j is exp(-i phi_j/2 P(x_j, z_j)) with phi_j = coef_j * theta[param_j].
    """

    def __init__(self, n, n_elec, x, z, param, coef, n_params):
        self.n, self.n_elec, self.n_params = int(n), int(n_elec), int(n_params)
        x, z = _u64(x), _u64(z)
        param = np.ascontiguousarray(param, dtype=np.int32)
        coef = _f64(coef)
        if not (len(x) == len(z) == len(param) == len(coef)):
            raise ValueError("rotation arrays must have equal length")
        self.n_rot = len(x)
        a = _P()
        _check(lib().q2_ansatz_create(self.n, self.n_elec, self.n_rot, _np_ptr(x), _np_ptr(z),
                                      _np_ptr(param), _np_ptr(coef), self.n_params, ctypes.byref(a)))
        self._a = a

    @classmethod
    def from_uccsd(cls, ans):
        return cls(ans.n, ans.n_elec, ans.x, ans.z, ans.param, ans.coef, ans.n_params)

    @property
    def handle(self):
        return self._a

    def info(self, dtype="complex64"):
        p, g = _I64(), _I64()
        _check(lib().q2_ansatz_info(self._a, _dtype_code(dtype), ctypes.byref(p), ctypes.byref(g)))
        return p.value, g.value

    def table_bytes(self, dtype="complex64"):
        """(resident device table bytes, angle-LUT bytes uploaded per evaluation) for a state dtype."""
        b, c = _SZ(), _SZ()
        _check(lib().q2_ansatz_table_bytes(self._a, _dtype_code(dtype), ctypes.byref(b), ctypes.byref(c)))
        return b.value, c.value

    def workspace_bytes(self, dtype="complex64", want_grad=False):
        b = lib().q2_vqe_workspace_bytes(self._a, _dtype_code(dtype), 1 if want_grad else 0)
        if b == 0:
            raise Q2Error(Q2_ERR_INVALID, lib().q2_last_error().decode(errors="replace"))
        return b

    def close(self):
        if getattr(self, "_a", None) and _lib is not None:
            _lib.q2_ansatz_destroy(self._a)
        self._a = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def alloc_workspace(nbytes, device="cuda"):
    """Device byte buffer (torch uint8) with a 256-byte aligned start.

    Backed by 8-byte elements so that slices of it can be viewed as state
    vectors (see workspace_state)."""
    torch = _torch()
    n8 = (int(nbytes) + 7) // 8
    buf = torch.empty(n8 + 32, dtype=torch.float64, device=device)
    off = ((-buf.data_ptr()) % 256) // 8
    return buf[off:off + n8].view(torch.uint8)[:int(nbytes)]


def workspace_state(workspace, n, dtype="complex64"):
    """The 2^n-amplitude state held at the start of a q2_vqe_energy_grad workspace."""
    torch = _torch()
    td = _torch_dtype(_dtype_code(dtype))
    nbytes = (1 << n) * (8 if td == torch.complex64 else 16)
    return workspace[:nbytes].view(td)


def vqe_energy_grad(ansatz, ham, theta, dtype="complex64", want_grad=True, workspace=None):
    """One VQE evaluation: (E, dE/dtheta or None, workspace).

    E = <psi|H|psi>/<psi|psi> for psi = U(theta)|HF>; the gradient follows
    Algorithm 1 (reverse mode).  Synchronizes the current stream.
    """
    d = _dtype_code(dtype)
    theta = _f64(theta)
    if len(theta) != ansatz.n_params:
        raise ValueError("theta has the wrong length")
    need = ansatz.workspace_bytes(d, want_grad)
    if workspace is None or workspace.numel() < need:
        workspace = alloc_workspace(need)
    e = _D()
    g = np.zeros(ansatz.n_params) if want_grad else None
    _check(lib().q2_vqe_energy_grad(ansatz.handle, ham.handle, _np_ptr(theta), d, 1 if want_grad else 0,
                                    ctypes.byref(e), _np_ptr(g) if want_grad else None,
                                    ctypes.c_void_p(workspace.data_ptr()), workspace.numel(),
                                    _stream_ptr()))
    return e.value, g, workspace


def pool_gradients(ansatz, ham, theta, pool_x, pool_z, dtype="complex64", workspace=None):
    """Operator-pool screening: (E, g, workspace) with g[k] = Im <H psi|P_k|psi> at
    psi = U(theta)|HF>, i.e. dE/dphi of exp(-i phi/2 P_k) appended at phi = 0.
    Synchronizes the current stream."""
    d = _dtype_code(dtype)
    theta = _f64(theta)
    if len(theta) != ansatz.n_params:
        raise ValueError("theta has the wrong length")
    px, pz = _u64(pool_x), _u64(pool_z)
    if len(px) != len(pz):
        raise ValueError("pool masks must have equal length")
    need = ansatz.workspace_bytes(d, True)
    if workspace is None or workspace.numel() < need:
        workspace = alloc_workspace(need)
    e = _D()
    g = np.zeros(len(px))
    _check(lib().q2_pool_gradients(ansatz.handle, ham.handle, _np_ptr(theta), d, len(px), _np_ptr(px),
                                   _np_ptr(pz), ctypes.byref(e), _np_ptr(g),
                                   ctypes.c_void_p(workspace.data_ptr()), workspace.numel(), _stream_ptr()))
    return e.value, g, workspace


def batch_energy_grad(ansatze, hams, thetas, want_grads, dtype="complex64", workspace=None):
    """Evaluate many small problems (n <= 12) in one persistent launch.

    Returns (energies, grads, workspace); grads[b] is None where want_grads[b]
    is false.  Each request's result does not depend on the rest of the batch.
    """
    nb = len(ansatze)
    if not (len(hams) == len(thetas) == len(want_grads) == nb):
        raise ValueError("per-request lists must have equal length")
    if nb == 0:
        return np.zeros(0), [], workspace
    d = _dtype_code(dtype)
    A = (_P * nb)(*[a.handle for a in ansatze])
    H = (_P * nb)(*[h.handle for h in hams])
    th = [_f64(t) for t in thetas]
    for a, t in zip(ansatze, th):
        if len(t) != a.n_params:
            raise ValueError("theta has the wrong length")
    TH = (_P * nb)(*[t.ctypes.data for t in th])
    wg = (ctypes.c_int * nb)(*[1 if w else 0 for w in want_grads])
    grads = [np.zeros(a.n_params) if w else None for a, w in zip(ansatze, want_grads)]
    G = (_P * nb)(*[g.ctypes.data if g is not None else None for g in grads])
    need = lib().q2_batch_workspace_bytes(nb, A, H, d)
    if need == 0:
        raise Q2Error(Q2_ERR_INVALID, lib().q2_last_error().decode(errors="replace"))
    if workspace is None or workspace.numel() < need:
        workspace = alloc_workspace(need)
    e = np.zeros(nb)
    _check(lib().q2_batch_energy_grad(nb, A, H, TH, wg, d, _np_ptr(e), G, ctypes.c_void_p(workspace.data_ptr()),
                                      workspace.numel(), _stream_ptr()))
    return e, grads, workspace


def async_status():
    """Raise Q2Error(Q2_ERR_TIMEOUT) if a kernel of apply_pauli_rotations or Hamiltonian.apply
    gave up a bounded wait since the last check (synchronizes the current stream)."""
    _check(lib().q2_async_status(_stream_ptr()))


def set_tile_qubits(dtype, t):
    _check(lib().q2_set_tile_qubits(_dtype_code(dtype), int(t)))


from .autograd import Energy  # noqa: E402  (needs the names above)

__all__ = [
    "C64", "C128", "Q2Error", "lib", "library_path", "new_state", "state_init_hf",
    "apply_pauli_rotations", "Hamiltonian", "Ansatz", "alloc_workspace", "vqe_energy_grad",
    "set_tile_qubits", "Energy", "batch_energy_grad", "workspace_state",
]
