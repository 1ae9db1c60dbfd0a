#!/usr/bin/env python3
"""Benchmark: UCCSD Pauli-rotation sweep + grouped energy on one GB300.

Workload (default "sweep32"): 32 qubits, complex64 state (32 GiB), the HF
determinant of 16 electrons, 50,000 Pauli rotations from randomly ordered
all-pairs UCCSD excitations, then the energy of a ~30,000-term Hamiltonian
made of whole xmask groups of the 32-qubit random-integral JW Hamiltonian.
One step = one q2_vqe_energy_grad call (energy only): HF init, angle
expansion and LUT upload, every sweep pass, every expectation pass, the
fixed-order reductions and the read-back of the energy.

metric: amplitude updates per second (rotations x 2^n per step / step time).
The state (32 GiB) is larger than L2 (129 MB), so no flush is needed.

Besides the timed steps the line carries: the roofline of the sweep and of
the expectation kernel (measured live with CUDA events), the same step with
the complex128 state as the FP64 reference on the same GPU (|dE| and the
FP64-ALU roofline of its sweep), the 8- and 20-qubit configurations, the
24-qubit energy + gradient, a short served stream, the end-to-end rate from
host arrays through the public API, and the oracle timed on the host cores.

Flags: --gpus N --steps K --warmup W [--impl ours|reference] [--workload ...]
       [--config5]: the served-stream configuration alone (2,000 Poisson
       requests at 0.5, 0.8 and 1.0 x the measured serial capacity).
Under torchrun (N > 1) every rank runs an independent replica (the sweep
does not shard); value = all ranks' units / max-over-ranks time.
"""

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

WORKLOADS = {
    # name: (n, n_elec, n_rot, min_terms)
    "sweep32": (32, 16, 50_000, 30_000),
    "sweep30": (30, 15, 20_000, 10_000),
    "sweep28": (28, 14, 10_000, 5_000),
}

# The oracle's bounded sample (both arms): the first ORACLE_ROTATIONS rotations of
# the random-order UCCSD sweep at ORACLE_QUBITS qubits, complex128.
ORACLE_QUBITS = 28
ORACLE_ROTATIONS = 48


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(x, dist, device="cpu"):
    """Largest value of x over all ranks (x itself without a process group)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world, steps, units_per_step, max_ms):
    """Units all replicas processed per second of the slowest rank's time."""
    return world * steps * units_per_step / (max_ms / 1000.0)


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks/throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.gpu_id = gpu_id
        self.lines = []
        self.proc = None

    def start(self):
        try:
            cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                   "-lms", "200"]
            if self.gpu_id is not None:
                cmd += ["-i", str(self.gpu_id)]
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def gpu_smi_id(torch, dev):
    try:
        u = str(torch.cuda.get_device_properties(dev).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        vis = os.environ.get("CUDA_VISIBLE_DEVICES")
        return vis.split(",")[dev] if vis else dev


def kernels_sha():
    import hashlib
    src = os.path.join(ROOT, "paper_2208_10978_gb300", "csrc", "kernels.cu")
    return hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]


def traffic_record(kernel, workload):
    """DRAM bytes per launch from a committed ncu summary, if it matches the current kernel source."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f)
        r = rec[kernel]
        if r.get("kernels_cu_sha") != kernels_sha():
            return None
        return r["bytes_per_launch"].get(workload)
    except Exception:
        return None


def cpu_oracle_sample(n=ORACLE_QUBITS, k=ORACLE_ROTATIONS, seed=0):
    """Time the plain-C oracle (all host threads) on the first k rotations of the
    random-order UCCSD sweep at n qubits; returns (amp-updates/s, threads, k)."""
    from oracle import c_oracle
    from synth.workloads import sweep_ansatz
    ans, theta = sweep_ansatz(n, n // 2, max(k, 64), seed)
    phi = ans.angles(theta)
    psi = c_oracle.hf_state(n, n // 2)
    t = time.perf_counter()
    c_oracle.apply_rotations(psi, n, ans.x[:k], ans.z[:k], phi[:k])
    dt = time.perf_counter() - t
    return k * (1 << n) / dt, c_oracle.threads(), k


def oracle_sample_text(k):
    return (f"first {k} rotations of the random-order UCCSD sweep at {ORACLE_QUBITS} qubits "
            f"({ORACLE_QUBITS // 2} electrons), complex128 state, plain C oracle")


def workload_config(name, dtype, ws, w):
    """The `config` object of both arms' JSON lines."""
    n, ne = w.n, w.n_elec
    return {"workload": f"{name}: {n} qubits, {ne} electrons, {w.ansatz.n_rot} UCCSD rotations (random "
                        f"excitation order), {w.ham.n_terms}-term JW Hamiltonian energy",
            "state": f"{dtype} (f32 pairs, f64 reductions)" if dtype == "complex64" else f"{dtype} (f64)",
            "parallelism": f"replicas x{ws}", "l2": "state (2^n amplitudes) larger than L2"}


def run_reference(args, ws, rank):
    """--impl reference: the oracle (plain C, host cores) on a bounded sample."""
    if rank != 0:
        return 0
    from synth.workloads import sweep32
    n_w, ne_w, n_rot, min_terms = WORKLOADS[args.workload]
    config = workload_config(args.workload, args.dtype, ws,
                             sweep32(seed=0, n=n_w, n_elec=ne_w, n_rot=n_rot, min_terms=min_terms))
    for _ in range(args.warmup):
        cpu_oracle_sample(k=4)
    vals = []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        v, cores, k = cpu_oracle_sample()
        vals.append(v)
    wall = time.perf_counter() - t0
    value = float(np.mean(vals))
    line = {
        "impl": "reference", "metric": "amp_updates_per_s", "value": value, "unit": "amp-updates/s",
        "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000.0 * wall / max(1, args.steps), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config,
        "cpu_baseline": {"value": value, "unit": "amp-updates/s", "cores": cores, "kind": "oracle",
                         "sample": oracle_sample_text(k)},
        "e2e": {"value": value, "unit": "amp-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def roofline_entry(kernel, alg_bytes, launches, total_ms, peak, peak_kind, workload):
    avg_s = total_ms / 1000.0 / max(1.0, launches)
    achieved = alg_bytes / avg_s / 1e9
    return {"kernel": kernel, "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "peak_source": peak_kind, "traffic": traffic_record(kernel, workload),
            "algorithmic_bytes_per_launch": alg_bytes, "launches_per_step": launches,
            "avg_launch_ms": avg_s * 1000.0}


def table_h2d_bytes(ans, ham, dtype):
    """Host->device bytes of one public-API evaluation from host arrays: both handles'
    resident tables plus the per-call angle LUT (reported by the library)."""
    res, per_call = ans.table_bytes(dtype)
    return int(res + per_call + ham.table_bytes(dtype))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="sweep32", choices=sorted(WORKLOADS))
    ap.add_argument("--dtype", default="complex64", choices=["complex64", "complex128"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-grad", action="store_true", help="skip the 24-qubit energy+gradient phase")
    ap.add_argument("--no-configs", action="store_true", help="skip the 8- and 20-qubit configurations")
    ap.add_argument("--no-fp64-check", action="store_true",
                    help="skip the same step with the complex128 state (|dE| and the FP64 roofline)")
    ap.add_argument("--served", type=int, default=48, help="requests in the short served phase (0: skip)")
    ap.add_argument("--served-rate", type=float, default=2.0, help="Poisson arrival rate (requests/s)")
    ap.add_argument("--config5", action="store_true",
                    help="only the served-stream configuration: 2,000 requests at 0.5/0.8/1.0 x capacity")
    ap.add_argument("--config5-requests", type=int, default=2000)
    ap.add_argument("--served-child", nargs=2, default=None, help=argparse.SUPPRESS)
    args = ap.parse_args()
    if args.served_child:
        return served_child(*args.served_child)
    ws, rank, local = dist_env()

    if args.impl == "reference":
        return run_reference(args, ws, rank)
    if args.config5:
        return config5(args, local) if rank == 0 else 0

    import torch
    import paper_2208_10978_gb300 as q2
    from synth.workloads import sweep32

    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    n, ne, n_rot, min_terms = WORKLOADS[args.workload]
    t0 = time.perf_counter()
    w = sweep32(seed=0, n=n, n_elec=ne, n_rot=n_rot, min_terms=min_terms)
    log(f"[bench] workload {args.workload}: {w.ansatz.n_rot} rotations, {w.ham.n_terms} terms "
        f"({w.ham.n_groups} groups), built in {time.perf_counter() - t0:.1f}s")
    ans = q2.Ansatz.from_uccsd(w.ansatz)
    ham = q2.Hamiltonian(n, w.ham.x, w.ham.z, w.ham.c)
    theta = w.theta
    lib = q2.lib()
    import ctypes
    lib.q2_debug_enable_timing.argtypes = [ctypes.c_int]
    lib.q2_debug_last_timing.argtypes = [ctypes.c_void_p]
    lib.q2_debug_fp64_rate.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    lib.q2_debug_enable_timing(1)
    wsb = ans.workspace_bytes(args.dtype, False)
    work = q2.alloc_workspace(wsb)
    tim = np.zeros(8)

    def step(aa=ans, hh=ham, dtype=args.dtype, wk=None):
        e, _, _ = q2.vqe_energy_grad(aa, hh, theta, dtype=dtype, want_grad=False, workspace=wk if wk is not None
                                     else work)
        lib.q2_debug_last_timing(ctypes.c_void_p(tim.ctypes.data))
        return e, tim.copy()

    for i in range(args.warmup):
        t = time.perf_counter()
        e, tt = step()
        log(f"[bench] warmup {i}: E = {e:.9f}, {time.perf_counter() - t:.2f}s "
            f"(sweep {tt[0]:.1f} ms / {int(tt[3])} kernels, energy {tt[1]:.1f} ms / {int(tt[4])} kernels)")

    sampler = ClockSampler(gpu_smi_id(torch, local)) if rank == 0 else None
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    if sampler:
        sampler.start()
    stream = torch.cuda.current_stream()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    per = []
    for _ in range(args.steps):
        e, tt = step()
        per.append(tt)
    ev1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = sampler.stop() if sampler else None
    ms = max_over_ranks(ev0.elapsed_time(ev1), dist, "cuda")
    per = np.array(per)
    units_per_step = float(w.ansatz.n_rot) * float(1 << n)
    value = whole_job_rate(ws, args.steps, units_per_step, ms)

    # per-kernel rooflines from the per-phase CUDA events of the timed steps:
    # k_sweep reads and writes the state once per launch, k_expect reads it once
    state_bytes = float(per[0, 7])
    peak, peak_kind = measured_peaks()
    sweep_ms = float(per[:, 0].mean())
    sweep_launches = float(per[0, 3])
    expect_ms = float(per[:, 1].mean())
    expect_launches = float(per[0, 4] - 1)          # the expectation passes; the last launch is the reduction
    r_sweep = roofline_entry("k_sweep", 2.0 * state_bytes, sweep_launches, sweep_ms, peak, peak_kind, args.workload)
    r_expect = roofline_entry("k_expect", state_bytes, expect_launches, expect_ms, peak, peak_kind, args.workload)
    roofline = r_sweep if sweep_ms >= expect_ms else r_expect       # the kernel with the larger share
    gpu_launches = int(per[:, 6].sum())

    e2e = None
    if not args.no_e2e:
        # public API from host arrays, every step: both handles built from host tables (schedules,
        # table uploads), the angle LUT upload, all kernels and the energy read-back
        torch.cuda.synchronize()
        t = time.perf_counter()
        for _ in range(args.steps):
            hh = q2.Hamiltonian(n, w.ham.x, w.ham.z, w.ham.c)
            aa = q2.Ansatz.from_uccsd(w.ansatz)
            q2.vqe_energy_grad(aa, hh, theta, dtype=args.dtype, want_grad=False, workspace=work)
            h2d = table_h2d_bytes(aa, hh, args.dtype)
            hh.close()
            aa.close()
        torch.cuda.synchronize()
        wall = max_over_ranks(time.perf_counter() - t, dist, "cuda")
        e2e = {"value": whole_job_rate(ws, args.steps, units_per_step, 1000.0 * wall), "unit": "amp-updates/s",
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": 32, "steps": args.steps,
               "includes": "Hamiltonian and ansatz handles from host arrays (schedules, table uploads), "
                           "angle LUT upload, all kernels, energy read-back"}

    fp64_check = None
    if not args.no_fp64_check and rank == 0 and args.dtype == "complex64":
        # the complex128 state (64 GiB at 32 qubits) fits beside the complex64 workspace
        fp64_check = fp64_phase(q2, torch, lib, ctypes, ans, ham, theta, e, n, tim)

    configs = None if args.no_configs or rank != 0 else small_configs(q2, torch, lib, ctypes)
    grad = None if args.no_grad or rank != 0 else grad_phase(q2, torch)
    served = None if args.served <= 0 or rank != 0 else served_isolated(args.served, args.served_rate, local)

    cpu = None
    if rank == 0 and not args.no_cpu_baseline and ws == 1:
        v, cores, k = cpu_oracle_sample()
        cpu = {"value": v, "unit": "amp-updates/s", "cores": cores, "kind": "oracle",
               "sample": oracle_sample_text(k)}

    if rank == 0:
        line = {
            "metric": "amp_updates_per_s", "value": value, "unit": "amp-updates/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if args.dtype == "complex64" else "f64", "data": "synthetic",
            "config": workload_config(args.workload, args.dtype, ws, w),
            "energy": e,
            "sweep": {"ms_per_step": sweep_ms, "kernels_per_step": int(sweep_launches),
                      "amp_updates_per_s": units_per_step / (sweep_ms / 1000.0), "hbm_gbs": r_sweep["achieved"]},
            "expectation": {"ms_per_step": expect_ms, "kernels_per_step": int(expect_launches),
                            "hbm_gbs_read": r_expect["achieved"]},
            "roofline": roofline,
            "rooflines": [r_sweep, r_expect],
            "kernels_cu_sha": kernels_sha(),
            "fp64_check": fp64_check,
            "configs": configs,
            "grad": grad,
            "served": served,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": gpu_launches,
            "clocks": clocks,
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def fp64_phase(q2, torch, lib, ctypes, ans, ham, theta, e64, n, tim):
    """The same step with the complex128 state (FP64 amplitudes, 2^n x 16 bytes) as the GPU
    reference: |dE| against complex64, and the FP64-ALU roofline of its sweep.  Each rotation
    group updates every amplitude once per pass with 6 FP64 flops (a real 2x2 rotation of a
    complex pair: 4 outputs of one multiply and one fused multiply-add each)."""
    rate = ctypes.c_double()
    st = lib.q2_debug_fp64_rate(ctypes.byref(rate), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    t = time.perf_counter()
    e128, _, w128 = q2.vqe_energy_grad(ans, ham, theta, dtype="complex128", want_grad=False)
    lib.q2_debug_last_timing(ctypes.c_void_p(tim.ctypes.data))
    wall = time.perf_counter() - t
    del w128
    torch.cuda.empty_cache()
    passes, groups = ans.info("complex128")
    flops = 6.0 * float(1 << n) * groups
    achieved = flops / (tim[0] / 1000.0) / 1e12
    peak = rate.value / 1e12 if st == 0 else 1.25
    return {"energy_complex128": e128, "energy_complex64": e64, "abs_dE": abs(e64 - e128),
            "complex128_step_s": wall, "state_bytes_complex128": 16 * (1 << n),
            "sweep_ms": float(tim[0]), "expectation_ms": float(tim[1]),
            "roofline": {"kernel": "k_sweep<double>", "bound": "alu", "achieved": achieved, "peak": peak,
                         "unit": "TFLOP/s", "frac": achieved / peak,
                         "peak_source": "measured FP64 FMA rate (q2_debug_fp64_rate)" if st == 0
                         else "nominal FP64 1.25 TFLOP/s",
                         "flops_per_launch": flops / passes, "launches": int(passes)}}


def small_configs(q2, torch, lib, ctypes):
    """8 qubits (complex128, us per energy) and 20 qubits (both dtypes, amp-updates/s);
    both states stay in L2 (4 KiB and 8/16 MiB), which is these configurations' own bound."""
    from synth.workloads import uccsd_energy
    out = {}
    w = uccsd_energy(8, 4, seed=0)
    a8, h8 = q2.Ansatz.from_uccsd(w.ansatz), q2.Hamiltonian(8, w.ham.x, w.ham.z, w.ham.c)
    for dtype in ("complex128", "complex64"):
        e, _, wk = q2.vqe_energy_grad(a8, h8, w.theta, dtype=dtype, want_grad=False)
        for _ in range(20):
            q2.vqe_energy_grad(a8, h8, w.theta, dtype=dtype, want_grad=False, workspace=wk)
        k = 300
        t = time.perf_counter()
        for _ in range(k):
            e, _, _ = q2.vqe_energy_grad(a8, h8, w.theta, dtype=dtype, want_grad=False, workspace=wk)
        out[f"n8_{dtype}"] = {"us_per_energy": 1e6 * (time.perf_counter() - t) / k, "energy": e,
                              "rotations": w.ansatz.n_rot, "terms": w.ham.n_terms}
    golden = None
    try:
        with open(os.path.join(ROOT, "tests", "golden", "uccsd20_seed0.json")) as f:
            golden = json.load(f)["energy"]
    except Exception:
        pass
    w = uccsd_energy(20, 10, seed=0)
    a20, h20 = q2.Ansatz.from_uccsd(w.ansatz), q2.Hamiltonian(20, w.ham.x, w.ham.z, w.ham.c)
    tim = np.zeros(8)
    for dtype in ("complex128", "complex64"):
        e, _, wk = q2.vqe_energy_grad(a20, h20, w.theta, dtype=dtype, want_grad=False)
        q2.vqe_energy_grad(a20, h20, w.theta, dtype=dtype, want_grad=False, workspace=wk)
        k = 5
        sw = []
        t = time.perf_counter()
        for _ in range(k):
            e, _, _ = q2.vqe_energy_grad(a20, h20, w.theta, dtype=dtype, want_grad=False, workspace=wk)
            lib.q2_debug_last_timing(ctypes.c_void_p(tim.ctypes.data))
            sw.append(tim[0])
        dt = (time.perf_counter() - t) / k
        upd = w.ansatz.n_rot * float(1 << 20)
        out[f"n20_{dtype}"] = {"amp_updates_per_s": upd / dt, "sweep_amp_updates_per_s": upd / (np.mean(sw) / 1e3),
                               "ms_per_energy": 1e3 * dt, "energy": e,
                               "abs_dE_vs_golden": abs(e - golden) if golden is not None else None,
                               "rotations": w.ansatz.n_rot, "terms": w.ham.n_terms}
    return out


def grad_phase(q2, torch, steps=3):
    """24 qubits, 12 electrons, 35,136 rotations: complex64 energy + reverse-mode gradient per second."""
    from synth.workloads import uccsd_energy
    w = uccsd_energy(24, 12, seed=0)
    ans = q2.Ansatz.from_uccsd(w.ansatz)
    ham = q2.Hamiltonian(24, w.ham.x, w.ham.z, w.ham.c)
    e, g, ws = q2.vqe_energy_grad(ans, ham, w.theta, dtype="complex64", want_grad=True)
    torch.cuda.synchronize()
    t = time.perf_counter()
    for _ in range(steps):
        e, g, ws = q2.vqe_energy_grad(ans, ham, w.theta, dtype="complex64", want_grad=True, workspace=ws)
    dt = (time.perf_counter() - t) / steps
    e128, g128, _ = q2.vqe_energy_grad(ans, ham, w.theta, dtype="complex128", want_grad=True)
    return {"workload": "24 qubits, 12 electrons, 35136 rotations over 4500 parameters, energy + dE/dtheta",
            "evals_per_s": 1.0 / dt, "ms_per_eval": 1000.0 * dt, "energy": e,
            "abs_dE_vs_complex128": abs(e - e128), "max_abs_dgrad_vs_complex128": float(np.max(np.abs(g - g128)))}


def _problem_for(args):
    """(problem seed, n, n_elec) -> serve.Problem and theta (runs in a spawned worker process)."""
    seed, n, ne = args
    from paper_2208_10978_gb300 import serve
    from synth.workloads import uccsd_energy
    w = uccsd_energy(n, ne, seed=seed % 100000)
    return seed, serve.problem_from_workload(w, key=seed), w.theta


def build_problems(reqs, processes=None):
    """Every distinct problem of a request stream, built in a spawned process pool
    (started before this process makes any CUDA call)."""
    import multiprocessing as mp
    todo = {}
    for r in reqs:
        todo.setdefault(r.problem_seed, (r.problem_seed, r.n, r.n_elec))
    problems, thetas = {}, {}
    ctx = mp.get_context("spawn")
    with ctx.Pool(processes or max(1, (os.cpu_count() or 2) - 1)) as pool:
        for seed, p, th in pool.imap_unordered(_problem_for, list(todo.values()), chunksize=8):
            problems[seed], thetas[seed] = p, th
    return problems, thetas


def served_phase(q2, n_requests, rate, problems=None, thetas=None, reqs=None, max_slots=64, n_streams=4):
    """Poisson stream through the serving loop (10..26 qubits, 40% with gradient, 150 GB budget)."""
    from paper_2208_10978_gb300 import serve
    from synth.workloads import served_stream
    if reqs is None:
        reqs = served_stream(seed=0, n_requests=n_requests, rate_per_s=rate)
    gen_s = 0.0
    if problems is None:
        t = time.perf_counter()
        problems, thetas = {}, {}
        for seed, p, th in map(_problem_for, [(r.problem_seed, r.n, r.n_elec) for r in reqs]):
            problems[seed], thetas[seed] = p, th
        gen_s = time.perf_counter() - t
    srv = serve.Server(dtype="complex64", budget_bytes=150 * 10**9, max_slots=max_slots, n_streams=n_streams)
    try:
        results, wall = serve.serve_stream(srv, reqs, problems, thetas, wait_s=1800)
        st = srv.stats()
    finally:
        srv.close()
    ok = [r for r in results.values() if r.status == 0]
    grad_ok = [r for r in ok if r.grad is not None]
    return {"requests": len(reqs), "completed": len(ok), "with_grad": len(grad_ok),
            "arrival_rate_per_s": rate, "evals_per_s": len(ok) / wall, "wall_s": wall,
            "p50_latency_s": st["p50_s"], "p99_latency_s": st["p99_s"], "mean_latency_s": st["mean_s"],
            "hbm_high_water_bytes": st["high_water_bytes"], "budget_bytes": 150 * 10**9,
            "resident_table_bytes": st["table_bytes"], "evictions": st["evictions"],
            "dtype": "c64 state, f64 reductions", "problem_generation_s_excluded": gen_s}


def served_isolated(n_requests, rate, local, timeout_s=900):
    """served_phase in a fresh interpreter with its own CUDA context, so that a failure
    there cannot reach the step measurement; returns its dict or {"error": ...}."""
    cmd = [sys.executable, os.path.abspath(__file__), "--served-child", str(n_requests), str(rate)]
    env = dict(os.environ, LOCAL_RANK=str(local), WORLD_SIZE="1", RANK="0")
    try:
        r = subprocess.run(cmd, capture_output=True, text=True, timeout=timeout_s, env=env)
    except subprocess.TimeoutExpired:
        return {"error": f"served phase did not finish within {timeout_s} s"}
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    if r.returncode != 0 or not lines:
        tail = (r.stderr.strip().splitlines() or ["no output"])[-1]
        return {"error": f"served phase exited {r.returncode}: {tail[:300]}"}
    try:
        return json.loads(lines[-1])
    except ValueError as exc:
        return {"error": f"served phase printed no result: {exc}"}


def served_child(n_requests, rate):
    import torch
    import paper_2208_10978_gb300 as q2
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    print(json.dumps(served_phase(q2, int(n_requests), float(rate))), flush=True)
    return 0


def config5(args, local):
    """The served configuration: a stream of Poisson-arrival requests over 10..26 qubits
    (n_elec = n/2, 40% with gradient, 20% repeating one of 16 earlier problems), complex64
    with FP64 reductions, admitted under a 150 GB budget.  The serial capacity is measured
    first (requests evaluated one at a time on the path the loop would use); the stream is
    then offered at 0.5, 0.8 and 1.0 x that capacity, each to a fresh server."""
    from synth.workloads import served_stream
    base = served_stream(seed=0, n_requests=args.config5_requests, rate_per_s=1.0)
    t = time.perf_counter()
    problems, thetas = build_problems(base)            # before the first CUDA call (spawned pool)
    gen_s = time.perf_counter() - t
    log(f"[config5] {len(problems)} distinct problems built in {gen_s:.1f}s")
    import torch
    import paper_2208_10978_gb300 as q2
    from paper_2208_10978_gb300 import serve
    torch.cuda.set_device(local)
    # serial capacity on the first requests of the stream (fresh handles, as a new problem would have)
    sample = base[:min(len(base), 200)]
    t = time.perf_counter()
    for r in sample:
        serve.evaluate_alone(problems[r.problem_seed], thetas[r.problem_seed], r.want_grad)
    cap = len(sample) / (time.perf_counter() - t)
    log(f"[config5] serial capacity {cap:.2f} evals/s on {len(sample)} requests")
    rates = []
    for frac in (0.5, 0.8, 1.0):
        rate = frac * cap
        reqs = [serve_request_at(r, rate) for r in base]
        t = time.perf_counter()
        res = served_phase(q2, len(reqs), rate, problems, thetas, reqs)
        res["offered_fraction_of_capacity"] = frac
        log(f"[config5] {frac:.1f} x capacity: {res['completed']}/{res['requests']} in {res['wall_s']:.1f}s, "
            f"{res['evals_per_s']:.2f} evals/s, p50 {res['p50_latency_s']:.3f}s p99 {res['p99_latency_s']:.3f}s")
        log("[config5] " + json.dumps(res))
        rates.append(res)
    line = {"metric": "served_evals_per_s", "value": rates[-1]["evals_per_s"], "unit": "evals/s",
            "n_gpus": 1, "higher_is_better": True, "data": "synthetic", "dtype": "f32",
            "config": {"workload": f"served stream: {len(base)} Poisson-arrival UCCSD requests, 10..26 qubits, "
                                   "40% energy+gradient, 150 GB HBM budget"},
            "serial_capacity_evals_per_s": cap, "serial_sample": len(sample),
            "problem_generation_s": gen_s, "distinct_problems": len(problems), "rates": rates}
    print(json.dumps(line), flush=True)
    return 0


def serve_request_at(r, rate):
    """The request r of a rate-1 stream, with its arrival time rescaled to `rate`."""
    from dataclasses import replace
    return replace(r, arrival_s=r.arrival_s / rate)


if __name__ == "__main__":
    sys.exit(main())
