"""Continuous-batching request loop for VQE energy (+ gradient) evaluations.

Requests are (Hamiltonian, ansatz, theta, want_grad) solves on 10..26 qubits.
The loop keeps every problem's Pauli tables resident on the device (one
library handle pair per distinct problem), admits requests by device-memory
footprint through the C++ admission core (include/q2_serve.h) -- running
workspaces plus the resident tables, with unused problems released least
recently used first when room is needed -- and runs them while others are
still on the GPU:

* small states (n <= 12) are gathered for a short window and evaluated
  together in one persistent launch (q2_batch_energy_grad), each CTA holding
  one request's state in shared memory;
* larger states run q2_vqe_energy_grad on a pool of CUDA streams, one worker
  thread per stream (the library call releases the GIL), so their kernels
  overlap on the device.

Each request's arithmetic is independent of its neighbours (fixed reduction
trees, per-request launches or per-request CTAs), so a result is the same
whether it was evaluated alone or in the mix.  This module only orchestrates:
every evaluation runs in the library's CUDA kernels.
"""

import ctypes
import queue
import threading
import time
from concurrent.futures import Future
from dataclasses import dataclass, field

import numpy as np

from . import (Ansatz, Hamiltonian, Q2Error, Q2_ERR_INVALID, Q2_ERR_TIMEOUT, Q2_OK, _dtype_code, alloc_workspace,
               batch_energy_grad, lib, vqe_energy_grad)

SMALL_MAX_QUBITS = 12


@dataclass
class Problem:
    """Pauli tables of one problem (what a client sends)."""
    key: object
    n: int
    n_elec: int
    ham_x: np.ndarray
    ham_z: np.ndarray
    ham_c: np.ndarray
    rot_x: np.ndarray
    rot_z: np.ndarray
    rot_param: np.ndarray
    rot_coef: np.ndarray
    n_params: int


@dataclass
class Result:
    rid: int
    status: int
    energy: float = float("nan")
    grad: object = None
    path: str = ""
    t_submit: float = 0.0
    t_done: float = 0.0
    error: str = ""

    @property
    def latency(self):
        return self.t_done - self.t_submit


@dataclass
class _Job:
    rid: int
    problem: Problem
    theta: np.ndarray
    want_grad: bool
    future: Future
    t_submit: float
    handles: tuple = field(default=None)


def _setup_core():
    L = lib()
    P, I, I64, D, SZ = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double, ctypes.c_size_t
    L.q2_server_create.argtypes = [SZ, I, D, ctypes.POINTER(P)]
    L.q2_server_destroy.argtypes = [P]
    L.q2_server_submit.argtypes = [P, I64, SZ, I64, SZ, D]
    L.q2_server_admit.argtypes = [P, D, ctypes.POINTER(I64), I]
    L.q2_server_admit.restype = I
    L.q2_server_expire.argtypes = [P, D, ctypes.POINTER(I64), I]
    L.q2_server_expire.restype = I
    L.q2_server_complete.argtypes = [P, I64, D]
    L.q2_server_take_evicted.argtypes = [P, ctypes.POINTER(I64), I]
    L.q2_server_take_evicted.restype = I
    L.q2_server_stats.argtypes = [P, ctypes.POINTER(D)]
    return L


class Server:
    """Request loop over the library; see the module docstring."""

    def __init__(self, dtype="complex64", budget_bytes=150 * 10**9, max_slots=64, n_streams=4,
                 batch_window_s=0.002, max_batch=256, queue_timeout_s=300.0, device="cuda"):
        import torch
        self._torch = torch
        self.dtype = dtype
        self.device = self._device_index(device)
        self.budget = int(budget_bytes)
        self.batch_window_s = batch_window_s
        self.max_batch = max_batch
        self._L = _setup_core()
        h = ctypes.c_void_p()
        st = self._L.q2_server_create(self.budget, int(max_slots), float(queue_timeout_s), ctypes.byref(h))
        if st != Q2_OK:
            raise Q2Error(st, "server core creation failed")
        self._core = h
        self._t0 = time.perf_counter()
        self._lock = threading.Lock()
        self._wake = threading.Condition(self._lock)
        self._jobs = {}
        self._tables = {}          # problem key -> (Ansatz, Hamiltonian) handles
        self._table_ids = {}       # problem key -> int64 id in the admission core
        self._table_keys = {}      # id -> problem key
        self._table_lock = threading.Lock()
        self._closed = False
        self._large = queue.Queue()
        self._small = []
        self._small_cv = threading.Condition()
        self._stop = False
        self._broken = ""          # set when a loop died: new requests fail at once
        self._threads = [threading.Thread(target=self._admit_loop, daemon=True),
                         threading.Thread(target=self._batch_loop, daemon=True)]
        self._threads += [threading.Thread(target=self._worker_loop, daemon=True) for _ in range(n_streams)]
        for t in self._threads:
            t.start()

    # ------------------------------------------------------------------ client side

    def now(self):
        return time.perf_counter() - self._t0

    def footprint(self, problem, want_grad, handles=None):
        """Device bytes a request needs while it runs (state vectors and per-call tables)."""
        a, h = handles if handles else self._handles(problem)
        if problem.n <= SMALL_MAX_QUBITS:
            A = (ctypes.c_void_p * 1)(a.handle)
            H = (ctypes.c_void_p * 1)(h.handle)
            return int(lib().q2_batch_workspace_bytes(1, A, H, _dtype_code(self.dtype)))
        return int(a.workspace_bytes(self.dtype, want_grad))

    def table_bytes(self, handles):
        """Device bytes of a problem's resident tables (Hamiltonian and ansatz handles)."""
        a, h = handles
        return int(a.table_bytes(self.dtype)[0] + h.table_bytes(self.dtype))

    def submit(self, rid, problem, theta, want_grad):
        """Queue one request; returns a Future resolving to a Result."""
        fut = Future()
        job = _Job(int(rid), problem, np.asarray(theta, dtype=np.float64), bool(want_grad), fut, self.now())
        job.handles = self._handles(problem)
        nbytes = self.footprint(problem, want_grad, job.handles)
        tbytes = self.table_bytes(job.handles)
        pid = self._table_ids[problem.key]
        with self._lock:
            if self._closed:
                raise RuntimeError("server is closed")
            if self._broken:
                fut.set_result(Result(job.rid, Q2_ERR_INVALID, t_submit=job.t_submit, t_done=self.now(),
                                      error="server loop stopped: " + self._broken))
                return fut
            self._jobs[job.rid] = job
            st = self._L.q2_server_submit(self._core, job.rid, nbytes, pid, tbytes, job.t_submit)
            if st != Q2_OK:
                del self._jobs[job.rid]
                fut.set_result(Result(job.rid, st, t_submit=job.t_submit, t_done=self.now()))
                return fut
            self._wake.notify_all()
        return fut

    def stats(self):
        out = (ctypes.c_double * 14)()
        self._L.q2_server_stats(self._core, out)
        keys = ["submitted", "admitted", "completed", "expired", "queued", "running", "bytes_in_use",
                "high_water_bytes", "p50_s", "p99_s", "mean_s", "table_bytes", "resident_problems",
                "evictions"]
        return dict(zip(keys, list(out)))

    def close(self, timeout_s=600.0):
        """Stop the loops and release the admission core and the resident tables.

        Waits for every worker to return (each is at most inside one library call,
        whose device waits are bounded).  If one is still alive after timeout_s the
        core and the tables are kept (a worker may still use them) and RuntimeError
        is raised."""
        with self._lock:
            if self._closed:
                return
            self._stop = True
            self._wake.notify_all()
        with self._small_cv:
            self._small_cv.notify_all()
        for _ in self._threads:
            self._large.put(None)
        deadline = time.perf_counter() + timeout_s
        for t in self._threads:
            t.join(timeout=max(0.0, deadline - time.perf_counter()))
        alive = [t for t in self._threads if t.is_alive()]
        if alive:
            raise RuntimeError(f"{len(alive)} serving threads still running after {timeout_s} s; "
                               "the admission core and the resident tables are kept")
        self._fail_all(Q2_ERR_INVALID, "server closed before the request ran")
        with self._lock:
            self._closed = True
        self._L.q2_server_destroy(self._core)
        self._core = None
        with self._table_lock:
            self._tables.clear()

    # ------------------------------------------------------------------ resident tables

    def _handles(self, problem):
        with self._table_lock:
            h = self._tables.get(problem.key)
            if h is None:
                h = (Ansatz(problem.n, problem.n_elec, problem.rot_x, problem.rot_z, problem.rot_param,
                            problem.rot_coef, problem.n_params),
                     Hamiltonian(problem.n, problem.ham_x, problem.ham_z, problem.ham_c))
                self._tables[problem.key] = h
            if problem.key not in self._table_ids:
                pid = len(self._table_ids) + 1
                self._table_ids[problem.key] = pid
                self._table_keys[pid] = problem.key
            return h

    def _release_evicted(self):
        """Drop the handles of problems the core released.  A request that already holds
        them keeps them alive until it finishes; the next request re-creates them."""
        ids = (ctypes.c_int64 * 64)()
        while True:
            k = self._L.q2_server_take_evicted(self._core, ids, 64)
            if k <= 0:
                return
            with self._table_lock:
                for i in range(k):
                    self._tables.pop(self._table_keys.get(ids[i]), None)

    # ------------------------------------------------------------------ loops

    def _finish(self, job, status, energy=float("nan"), grad=None, path="", error=""):
        t = self.now()
        self._L.q2_server_complete(self._core, job.rid, t)     # releases its bytes and slot
        with self._lock:
            self._jobs.pop(job.rid, None)
            self._wake.notify_all()
        if not job.future.done():
            job.future.set_result(Result(job.rid, status, energy, grad, path, job.t_submit, t, error))

    def _admit_loop(self):
        ids = (ctypes.c_int64 * 256)()
        while True:
            with self._lock:
                if self._stop:
                    return
                t = self.now()
                k = self._L.q2_server_expire(self._core, t, ids, 256)
                expired = [self._jobs[ids[i]] for i in range(max(k, 0))]
                k = self._L.q2_server_admit(self._core, t, ids, 256)
                admitted = [self._jobs[ids[i]] for i in range(max(k, 0))]
                if not expired and not admitted:
                    self._wake.wait(timeout=0.002)
            self._release_evicted()
            for job in expired:
                if not job.future.done():
                    job.future.set_result(Result(job.rid, Q2_ERR_TIMEOUT, t_submit=job.t_submit, t_done=self.now()))
                with self._lock:
                    self._jobs.pop(job.rid, None)
            for job in admitted:
                if job.problem.n <= SMALL_MAX_QUBITS:
                    with self._small_cv:
                        self._small.append(job)
                        self._small_cv.notify_all()
                else:
                    self._large.put(job)

    def _fail_all(self, status, error):
        with self._lock:
            if not self._broken and status != Q2_OK and "server closed" not in error:
                self._broken = error
            jobs = list(self._jobs.values())
        for j in jobs:
            if not j.future.done():
                j.future.set_result(Result(j.rid, status, t_submit=j.t_submit, t_done=self.now(), error=error))

    def _batch_loop(self):
        try:
            self._batch_loop_body()
        except Exception as exc:                           # never leave futures unresolved
            self._fail_all(Q2_ERR_INVALID, "batch loop: " + repr(exc))
            raise

    def _worker_loop(self):
        try:
            self._worker_loop_body()
        except Exception as exc:
            self._fail_all(Q2_ERR_INVALID, "stream worker: " + repr(exc))
            raise

    # ------------------------------------------------------------------ device work (overridable)

    def _device_index(self, device):
        dev = self._torch.device(device)
        return dev.index if dev.index is not None else self._torch.cuda.current_device()

    def _make_stream(self):
        """A CUDA stream of this loop's device, made current for the calling thread's device."""
        self._torch.cuda.set_device(self.device)
        return self._torch.cuda.Stream(device=self.device)

    def _run_batch(self, batch, stream, ws):
        with self._torch.cuda.stream(stream):
            return batch_energy_grad([j.handles[0] for j in batch], [j.handles[1] for j in batch],
                                     [j.theta for j in batch], [j.want_grad for j in batch],
                                     dtype=self.dtype, workspace=ws)

    def _run_large(self, job, stream, ws):
        with self._torch.cuda.stream(stream):
            return vqe_energy_grad(job.handles[0], job.handles[1], job.theta, dtype=self.dtype,
                                   want_grad=job.want_grad, workspace=ws)

    # ------------------------------------------------------------------ loop bodies

    def _batch_loop_body(self):
        stream = self._make_stream()
        ws = None
        while True:
            with self._small_cv:
                while not self._small and not self._stop:
                    self._small_cv.wait(timeout=0.05)
                if self._stop and not self._small:
                    return
            time.sleep(self.batch_window_s)                 # let a batch gather
            with self._small_cv:
                batch, self._small = self._small[:self.max_batch], self._small[self.max_batch:]
            try:
                e, g, ws = self._run_batch(batch, stream, ws)
                for j, ej, gj in zip(batch, e, g):
                    self._finish(j, Q2_OK, float(ej), gj, "batch")
            except Q2Error as exc:
                for j in batch:
                    self._finish(j, exc.status, path="batch", error=str(exc))
            except Exception as exc:
                for j in batch:
                    self._finish(j, Q2_ERR_INVALID, path="batch", error=repr(exc))
                raise

    def _worker_loop_body(self):
        stream = self._make_stream()
        ws = None
        while True:
            job = self._large.get()
            if job is None:
                return
            try:
                e, g, ws = self._run_large(job, stream, ws)
                self._finish(job, Q2_OK, e, g, "stream")
            except Q2Error as exc:
                self._finish(job, exc.status, path="stream", error=str(exc))
            except Exception as exc:
                self._finish(job, Q2_ERR_INVALID, path="stream", error=repr(exc))
                raise


def evaluate_alone(problem, theta, want_grad, dtype="complex64", handles=None):
    """The same evaluation outside the loop, on the path the loop would use for it."""
    a, h = handles if handles else (
        Ansatz(problem.n, problem.n_elec, problem.rot_x, problem.rot_z, problem.rot_param, problem.rot_coef,
               problem.n_params),
        Hamiltonian(problem.n, problem.ham_x, problem.ham_z, problem.ham_c))
    if problem.n <= SMALL_MAX_QUBITS:
        e, g, _ = batch_energy_grad([a], [h], [theta], [want_grad], dtype=dtype)
        return float(e[0]), g[0]
    e, g, _ = vqe_energy_grad(a, h, theta, dtype=dtype, want_grad=want_grad)
    return e, g


def problem_from_workload(w, key):
    a = w.ansatz
    return Problem(key, w.n, w.n_elec, w.ham.x, w.ham.z, w.ham.c, a.x, a.z, a.param, a.coef, a.n_params)


def serve_stream(server, requests, problems, thetas, speed=1.0, wait_s=900.0):
    """Submit requests at their arrival times (seconds, scaled by 1/speed); wait for all.

    Returns (results by rid, wall seconds from the first arrival to the last completion).
    Raises concurrent.futures.TimeoutError if a result takes longer than wait_s.
    """
    futs = {}
    t_start = time.perf_counter()
    for r in requests:
        delay = r.arrival_s / speed - (time.perf_counter() - t_start)
        if delay > 0:
            time.sleep(delay)
        futs[r.rid] = server.submit(r.rid, problems[r.problem_seed], thetas[r.problem_seed], r.want_grad)
    deadline = time.perf_counter() + wait_s
    results = {rid: f.result(timeout=max(0.0, deadline - time.perf_counter())) for rid, f in futs.items()}
    wall = time.perf_counter() - t_start
    return results, wall
