"""Host logic of the library, without a GPU.

* libq2.so loads and exports every function declared in include/*.h;
* argument checks reject bad input before any device work;
* the pass/group/LUT tables built by the schedulers, walked on the CPU the
  way the tile kernels index memory (tests/plan_emulator.py), reproduce the
  oracle's rotations, energies, H|psi> and reverse-mode gradients.
"""

import ctypes
import os
import re

import numpy as np
import pytest

import paper_2208_10978_gb300 as q2
from oracle import statevector as sv
from synth import uccsd_rotations
from synth.workloads import uccsd_energy
from tests import plan_emulator as emu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    return q2.lib()


def _declared():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            txt = re.sub(r"//[^\n]*", "", txt)
            names |= set(re.findall(r"^\s*(?:[\w\s\*]+?)\b(q2_\w+)\s*\(", txt, flags=re.M))
    return names


def test_exports_every_declared_symbol(lib):
    names = _declared()
    assert len(names) >= 18
    for nm in sorted(names):
        assert hasattr(lib, nm), nm


def test_version_and_error_text(lib):
    assert lib.q2_version() >= 100
    assert isinstance(lib.q2_last_error(), bytes)


def _status(f, *args):
    return f(*args)


def test_argument_checks_without_device_work(lib):
    x = np.array([1 << 9], dtype=np.uint64)
    z = np.zeros(1, dtype=np.uint64)
    a = np.array([0.1])
    P = ctypes.c_void_p
    dummy = P(256)
    f = lib.q2_apply_pauli_rotations
    assert f(dummy, 8, 0, P(x.ctypes.data), P(z.ctypes.data), P(a.ctypes.data), 1, None) == q2.Q2_ERR_INVALID
    assert b"mask bit" in lib.q2_last_error()
    assert f(dummy, 0, 0, P(x.ctypes.data), P(z.ctypes.data), P(a.ctypes.data), 1, None) == q2.Q2_ERR_INVALID
    assert f(dummy, 35, 0, P(x.ctypes.data), P(z.ctypes.data), P(a.ctypes.data), 1, None) == q2.Q2_ERR_INVALID
    assert f(dummy, 34, 1, P(x.ctypes.data), P(z.ctypes.data), P(a.ctypes.data), 1, None) == q2.Q2_ERR_INVALID
    bad = np.array([np.nan])
    xs = np.array([1], dtype=np.uint64)
    assert f(dummy, 8, 0, P(xs.ctypes.data), P(z.ctypes.data), P(bad.ctypes.data), 1, None) == q2.Q2_ERR_INVALID
    assert f(P(257), 8, 0, P(xs.ctypes.data), P(z.ctypes.data), P(a.ctypes.data), 1, None) == q2.Q2_ERR_INVALID
    assert lib.q2_state_init_hf(dummy, 8, 9, 0, None) == q2.Q2_ERR_INVALID
    assert lib.q2_set_tile_qubits(0, 20) == q2.Q2_ERR_INVALID
    h = P()
    c = np.array([np.inf])
    assert lib.q2_ham_create(8, P(xs.ctypes.data), P(z.ctypes.data), P(c.ctypes.data), 1,
                             ctypes.byref(h)) == q2.Q2_ERR_INVALID
    p = np.array([3], dtype=np.int32)
    one = np.array([1.0])
    assert lib.q2_ansatz_create(8, 4, 1, P(xs.ctypes.data), P(z.ctypes.data), P(p.ctypes.data),
                                P(one.ctypes.data), 2, ctypes.byref(h)) == q2.Q2_ERR_INVALID


def test_handles_info_without_gpu(lib):
    w = uccsd_energy(8, 4, seed=0)
    ham = q2.Hamiltonian(8, w.ham.x, w.ham.z, w.ham.c)
    assert ham.info() == (361, 51)
    ans = q2.Ansatz.from_uccsd(w.ansatz)
    npass, ngroup = ans.info("complex64")
    assert ngroup == w.ansatz.n_params        # one group per excitation (8 or 2 commuting strings)
    assert npass >= 1
    assert ans.workspace_bytes("complex128", True) > 2 * 256 * 16


def _random_rotations(rng, n, k, p_zero=0.1):
    x = rng.integers(0, 1 << n, size=k).astype(np.uint64)
    x[rng.random(k) < p_zero] = 0
    z = rng.integers(0, 1 << n, size=k).astype(np.uint64)
    # runs of equal x to exercise grouping
    for i in range(1, k):
        if rng.random() < 0.5:
            x[i] = x[i - 1]
    phi = rng.uniform(-3, 3, size=k)
    return x, z, phi


@pytest.mark.parametrize("n,T,C", [(6, 4, 2), (9, 5, 2), (10, 8, 3), (12, 8, 4), (11, 11, 4), (13, 9, 4)])
def test_tiles_partition_the_state(lib, n, T, C):
    rng = np.random.default_rng(n)
    x, z, phi = _random_rotations(rng, n, 60)
    passes, groups, blocks, lut, sm = emu.rot_plan(lib, n, x, z, phi, T, C)
    for pd in passes:
        idx = emu.tile_index(n, pd)
        assert np.array_equal(np.sort(idx.ravel()), np.arange(1 << n, dtype=np.uint64))
        for b in range(int(pd["C"])):
            assert int(pd["w"][b]) == 1 << b


@pytest.mark.parametrize("n,T,C,seed", [(6, 4, 2, 0), (9, 5, 2, 1), (10, 8, 3, 2), (12, 8, 4, 3),
                                        (11, 11, 4, 4), (13, 9, 4, 5), (7, 7, 4, 6)])
def test_schedule_sweep_matches_oracle(lib, n, T, C, seed):
    rng = np.random.default_rng(100 + seed)
    x, z, phi = _random_rotations(rng, n, 120)
    passes, groups, blocks, lut, sm = emu.rot_plan(lib, n, x, z, phi, T, C)
    psi0 = rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)
    psi0 /= np.linalg.norm(psi0)
    ref = sv.apply_rotations(psi0, x, z, phi)
    got = emu.sweep(psi0, n, passes, groups, blocks, lut, lib.q2_debug_threads_per_cta())
    assert np.max(np.abs(got - ref)) < 1e-12
    back = emu.sweep(got, n, passes, groups, blocks, lut, lib.q2_debug_threads_per_cta(), inverse=True)
    assert np.max(np.abs(back - psi0)) < 1e-12


@pytest.mark.parametrize("n,ne,T,C", [(8, 4, 6, 2), (12, 6, 9, 3), (12, 6, 12, 4)])
def test_schedule_uccsd_matches_oracle(lib, n, ne, T, C):
    w = uccsd_energy(n, ne, seed=1)
    a = w.ansatz
    phi = a.angles(np.random.default_rng(3).normal(0, 0.3, size=a.n_params))
    passes, groups, blocks, lut, sm = emu.rot_plan(lib, n, a.x, a.z, phi, T, C)
    ref = sv.apply_rotations(sv.hf_state(n, ne), a.x, a.z, phi)
    got = emu.sweep(sv.hf_state(n, ne), n, passes, groups, blocks, lut, lib.q2_debug_threads_per_cta())
    assert np.max(np.abs(got - ref)) < 1e-12


@pytest.mark.parametrize("n,T,C,seed", [(8, 5, 2, 0), (10, 7, 3, 1), (12, 8, 4, 2), (10, 10, 4, 3)])
def test_schedule_expectation_and_happly(lib, n, T, C, seed):
    rng = np.random.default_rng(200 + seed)
    k = 80
    x = rng.integers(0, 1 << n, size=k).astype(np.uint64)
    x[:10] = 0
    z = rng.integers(0, 1 << n, size=k).astype(np.uint64)
    c = rng.normal(size=k)
    x[k // 2:k // 2 + 10] = x[k // 2]            # a group with many terms
    passes, groups, blocks, lut = emu.ham_plan(lib, n, x, z, c, T, C)
    psi = rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)
    e, nrm = emu.expectation(psi, n, passes, groups, blocks, lut, lib.q2_debug_threads_per_cta())
    assert abs(e - sv.expectation(psi, x, z, c)) < 1e-9 * max(1.0, abs(e))
    lam = emu.happly(psi, n, passes, groups, lut, lib.q2_debug_threads_per_cta())
    assert np.max(np.abs(lam - sv.apply_hamiltonian(psi, x, z, c))) < 1e-11


def test_schedule_chemistry_hamiltonian(lib):
    w = uccsd_energy(10, 5, seed=2)
    passes, groups, blocks, lut = emu.ham_plan(lib, 10, w.ham.x, w.ham.z, w.ham.c, 8, 4)
    psi = sv.apply_rotations(sv.hf_state(10, 5), w.ansatz.x, w.ansatz.z, w.angles())
    e, nrm = emu.expectation(psi, 10, passes, groups, blocks, lut, lib.q2_debug_threads_per_cta())
    assert abs(e - sv.expectation(psi, w.ham.x, w.ham.z, w.ham.c)) < 1e-11


def test_lut_tables_aligned(lib):
    """Every group's LUT starts at a multiple of its 2^r entries and every pass's
    LUT at a multiple of the largest table (XOR addressing of the entries)."""
    w = uccsd_energy(10, 5, seed=2)
    a = w.ansatz
    rp, rg, rb, rl, sm = emu.rot_plan(lib, 10, a.x, a.z, a.angles(w.theta), 8, 4)
    hp, hg, hb, hl = emu.ham_plan(lib, 10, w.ham.x, w.ham.z, w.ham.c, 8, 4)
    for groups, passes, rmax in ((rg, rp, 6), (hg, hp, 8)):
        assert np.all(groups["lut"] % (1 << groups["r"].astype(np.int64)) == 0)
        assert np.all(passes["lut_begin"] % (1 << rmax) == 0)
        assert np.all(passes["lut_count"] <= 1024)


def test_real_coefficient_groups(lib):
    """Groups whose members all have an even Y count are marked real and have Q = 0;
    a group with an odd-Y member keeps the general kind."""
    w = uccsd_energy(10, 5, seed=2)
    passes, groups, blocks, lut = emu.ham_plan(lib, 10, w.ham.x, w.ham.z, w.ham.c, 8, 4)
    off = groups[groups["kind"] != emu.DIAG]
    assert len(off) > 0 and np.all(off["kind"] == emu.REAL)
    for g in off:
        assert np.all(lut[int(g["lut"]):int(g["lut"]) + (1 << int(g["r"])), 1] == 0.0)
    x = np.array([3, 3, 5], dtype=np.uint64)
    z = np.array([1, 0, 4], dtype=np.uint64)      # (X Y), (X X): one odd-Y member; (X Z Y) alone
    passes, groups, blocks, lut = emu.ham_plan(lib, 4, x, z, np.array([0.5, 0.25, 1.0]), 4, 1)
    kinds = {int(g["xl"]): int(g["kind"]) for g in groups}
    assert sorted(kinds.values()) == [emu.PAIR, emu.PAIR]
    psi = np.random.default_rng(1).normal(size=16) + 1j * np.random.default_rng(2).normal(size=16)
    e, _ = emu.expectation(psi, 4, passes, groups, blocks, lut, lib.q2_debug_threads_per_cta())
    assert abs(e - sv.expectation(psi, x, z, [0.5, 0.25, 1.0])) < 1e-12


@pytest.mark.parametrize("n,ne,T,C", [(8, 4, 6, 2), (10, 4, 7, 3)])
def test_schedule_reverse_gradient(lib, n, ne, T, C):
    w = uccsd_energy(n, ne, seed=4)
    a = w.ansatz
    rng = np.random.default_rng(5)
    phi = a.angles(rng.normal(0, 0.4, size=a.n_params))
    # add generic rotations (x = 0 groups and even-Y strings) to the tail
    x2, z2, p2 = _random_rotations(rng, n, 30)
    X = np.concatenate([a.x, x2])
    Z = np.concatenate([a.z, z2])
    PH = np.concatenate([phi, p2])
    e_ref, g_ref = sv.energy_and_gradient(n, ne, X, Z, PH, w.ham.x, w.ham.z, w.ham.c)
    NT = lib.q2_debug_threads_per_cta()
    passes, groups, blocks, lut, sm = emu.rot_plan(lib, n, X, Z, PH, T, C)
    hp, hg, hb, hl = emu.ham_plan(lib, n, w.ham.x, w.ham.z, w.ham.c, T, C)
    psi = emu.sweep(sv.hf_state(n, ne), n, passes, groups, blocks, lut, NT)
    lam = emu.happly(psi, n, hp, hg, hl, NT)
    assert abs(np.vdot(psi, lam).real - e_ref) < 1e-11
    psi_b, lam_b, g = emu.reverse(psi, lam, n, passes, groups, lut, sm, NT)
    assert np.max(np.abs(g - g_ref)) < 1e-11
    assert np.max(np.abs(psi_b - sv.hf_state(n, ne))) < 1e-12


@pytest.mark.parametrize("n,ne,T,C", [(8, 4, 6, 2), (10, 5, 8, 3)])
def test_gradient_weights_match_oracle(lib, n, ne, T, C):
    """Gradient tables of the kernels (one-parameter group weights, fold factors):
    the reverse sweep emulated with them gives the oracle's dE/dtheta for an ansatz
    that mixes runs sharing one parameter with per-rotation parameters, over every
    group kind (x = 0, odd and even Y counts)."""
    rng = np.random.default_rng(40 + n)
    w = uccsd_energy(n, ne, seed=7)
    x, z, _ = _random_rotations(rng, n, 70)
    run = np.cumsum(np.concatenate([[0], (x[1:] != x[:-1]).astype(np.int64)]))
    shared = rng.random(run.max() + 1) < 0.5            # half the runs share one parameter
    param = np.where(shared[run], run, run.max() + 1 + np.arange(len(x)))
    _, param = np.unique(param, return_inverse=True)
    param = param.astype(np.int32)
    n_params = int(param.max()) + 1
    coef = rng.choice([-1.0, -0.25, 0.5, 1.0], size=len(x))
    theta = rng.normal(0, 0.5, size=n_params)
    phi = coef * theta[param]
    e_ref, gphi = sv.energy_and_gradient(n, ne, x, z, phi, w.ham.x, w.ham.z, w.ham.c)
    g_ref = sv.fold_to_theta(gphi, param, coef, n_params)
    NT = lib.q2_debug_threads_per_cta()
    passes, groups, blocks, lut, sm = emu.rot_plan(lib, n, x, z, phi, T, C)
    wgroups, wl, fold = emu.rot_weights(lib, n, x, z, param, coef, T, C, len(groups))
    assert np.any(wgroups["one_param"] == 1) and np.any(wgroups["one_param"] == 0)
    hp, hg, hb, hl = emu.ham_plan(lib, n, w.ham.x, w.ham.z, w.ham.c, T, C)
    psi = emu.sweep(sv.hf_state(n, ne), n, passes, groups, blocks, lut, NT)
    lam = emu.happly(psi, n, hp, hg, hl, NT)
    _, _, g_rot = emu.reverse_weighted(psi, lam, n, passes, wgroups, lut, sm, wl, NT)
    g = np.zeros(n_params)
    np.add.at(g, param, fold[:len(x)] * g_rot)
    assert np.max(np.abs(g - g_ref)) < 1e-11


def test_canonical_blocks(lib):
    """A block marked canonical has its first d groups pairing along bits 0..d-1, REAL."""
    from synth.workloads import sweep32
    w = sweep32(0, n=20, n_elec=10, n_rot=3000, min_terms=2000)
    a = w.ansatz
    for plan in (emu.rot_plan(lib, 20, a.x, a.z, a.angles(w.theta), 12, 4),
                 emu.ham_plan(lib, 20, w.ham.x, w.ham.z, w.ham.c, 13, 4)):
        passes, groups, blocks = plan[0], plan[1], plan[2]
        assert np.mean(blocks["canon"] == blocks["d"]) > 0.5
        for pd in passes:
            for b in blocks[pd["b_begin"]:pd["b_end"]]:
                for k in range(int(b["canon"])):
                    g = groups[pd["g_begin"] + int(b["g_begin"]) + k]
                    assert int(g["a"]) == 1 << k and int(g["kind"]) == emu.REAL


def test_schedule_fusion_depth_32_qubits(lib):
    """On the 32-qubit random-order workload, one pass holds many excitations."""
    from synth import excitations
    rng = np.random.default_rng(0)
    pool = excitations(32, 16)
    chosen = [pool[k] for k in rng.permutation(len(pool))[:200]]
    a = uccsd_rotations(32, 16, exc_list=chosen)
    passes, groups, blocks, lut, sm = emu.rot_plan(lib, 32, a.x, a.z, np.zeros(a.n_rot), 12, 4)
    rots_per_pass = a.n_rot / len(passes)
    assert len(groups) == 200
    assert rots_per_pass > 40          # one tile dimension per excitation


def test_tile_walk_masked_add():
    """Persistent CTAs walk tile bases by one masked add per step: the deposit of
    t + g equals ((deposit(t) | ~mask) + deposit(g)) & mask while t + g < 2^popcount(mask)."""
    def deposit(v, m):
        out, k = 0, 0
        while m:
            low = m & -m
            if (v >> k) & 1:
                out |= low
            k += 1
            m &= m - 1
        return out
    full = (1 << 64) - 1
    rng = np.random.default_rng(12)
    for _ in range(300):
        n = int(rng.integers(9, 35))
        T = int(rng.integers(8, min(13, n) + 1))
        m = 0
        for b in rng.choice(n, size=n - T, replace=False):
            m |= 1 << int(b)
        ntiles = 1 << (n - T)
        g = int(rng.integers(1, 1200))
        t = int(rng.integers(0, g))
        base, step = deposit(t, m), deposit(g, m)
        for _ in range(64):                     # the first steps and, below, the last ones
            if t >= ntiles:
                break
            assert base == deposit(t, m)
            base = ((base | (~m & full)) + step) & m
            t += g
        k = max(0, (ntiles - 1 - t) // g - 8)   # jump close to the end and walk out of the range
        t += k * g
        base = deposit(t, m)
        while t < ntiles:
            assert base == deposit(t, m)
            base = ((base | (~m & full)) + step) & m
            t += g


@pytest.mark.parametrize("n,T,seed", [(17, 12, 2), (17, 12, 5)])
def test_sweep_fast_path_walk_matches_oracle(lib, n, T, seed):
    """The canonical 4-dimensional fast path of the sweep (k_sweep_c4): its Gray-code
    walks over amplitude byte offsets and LUT byte addresses, on the real schedule of a
    random-order UCCSD sweep (whole double excitations, as in the 32-qubit workload),
    reproduce the oracle's state; most passes qualify for the fast path."""
    from synth.workloads import sweep_ansatz
    ans, theta = sweep_ansatz(n, n // 2, 500, seed)
    phi = ans.angles(theta)
    passes, groups, blocks, lut, sm = emu.rot_plan(lib, n, ans.x, ans.z, phi, T, 4)
    c4 = [emu.pass_is_canon4(pd, blocks) for pd in passes]
    assert sum(c4) >= 0.8 * len(passes)
    rng = np.random.default_rng(seed)
    psi0 = rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)
    psi0 /= np.linalg.norm(psi0)
    ref = sv.apply_rotations(psi0, ans.x, ans.z, phi)
    got = emu.sweep_c4(psi0, n, passes, groups, blocks, lut, lib.q2_debug_threads_per_cta())
    assert np.max(np.abs(got - ref)) < 1e-12


@pytest.mark.parametrize("n,T,C", [(14, 13, 4), (15, 12, 4), (13, 11, 4)])
def test_expectation_chunk_shapes_and_lean_walk_match_oracle(lib, n, T, C):
    """The general expectation kernel takes each block's cosets in chunks; every chunk size
    the template admits for every block dimension (d = 1, 2, 3; chunks of 1, 2, 4, ... cosets
    up to J) walks bjcode[j0 + j] the same way and gives the oracle's energy, so the chunk
    indexing is not a source of error.  The lean path's Gray-code address walks give it too."""
    from synth.workloads import sweep32
    w = sweep32(seed=n, n=n, n_elec=n // 2, n_rot=8, min_terms=900)
    passes, groups, blocks, lut = emu.ham_plan(lib, n, w.ham.x, w.ham.z, w.ham.c, T, C)
    rng = np.random.default_rng(n)
    psi = rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)
    psi /= np.linalg.norm(psi)
    e_ref = sv.expectation(psi, w.ham.x, w.ham.z, w.ham.c)
    NT = lib.q2_debug_threads_per_cta()
    dims = {int(b["d"]) for b in blocks}
    assert {1, 3} <= dims
    J_min = min((1 << (T - int(b["d"]))) // NT for b in blocks)
    for jc in [1, 2, 4, 8, 16]:
        if jc > J_min and jc > 1:
            break
        e, nrm = emu.expectation_chunked(psi, n, passes, groups, blocks, lut, NT, jc)
        assert abs(e - e_ref) < 1e-10, jc
        assert abs(nrm - 1) < 1e-12
    if all(int(g["kind"]) in (emu.DIAG, emu.REAL) for g in groups) and all(int(b["d"]) <= 3 for b in blocks):
        e, _ = emu.expectation_lean(psi, n, passes, groups, blocks, lut, NT)
        assert abs(e - e_ref) < 1e-10


@pytest.mark.parametrize("n,T,C,amps", [(14, 12, 4, 2), (16, 13, 4, 2), (14, 12, 3, 1), (16, 13, 3, 1)])
def test_tile_pieces_are_aligned_and_contiguous(lib, n, T, C, amps):
    """The per-thread tile copies move 16-byte pieces (2 complex64 or 1 complex128 amplitudes):
    piece v of a tile is local indices v*amps .. v*amps + amps - 1, copied to shared offset 16 v.
    On real sweep and Hamiltonian plans every piece must start 16-byte aligned in the state and be
    contiguous there, which holds because tile bases and chunk offsets have their low C bits clear."""
    w = uccsd_energy(n, n // 2, seed=n)
    a = w.ansatz
    rot = emu.rot_plan(lib, n, a.x, a.z, a.angles(w.theta), T, C)[0]
    ham = emu.ham_plan(lib, n, w.ham.x, w.ham.z, w.ham.c, T, C)[0]
    checked = 0
    for pd in list(rot) + list(ham):
        Cp = int(pd["C"])
        if int(pd["T"]) < 9:
            continue   # tiles below 2^9 amplitudes take the guarded plain-load kernels
        low = (1 << Cp) - 1
        assert int(pd["umask"]) & low == 0
        assert all(int(pd["w"][b]) & low == 0 for b in range(Cp, int(pd["T"])))
        idx = emu.tile_index(n, pd).astype(np.int64)
        start = idx[:, ::amps]
        assert np.all(start % amps == 0)
        for k in range(1, amps):
            assert np.array_equal(idx[:, k::amps], start + k)
        checked += 1
    assert checked > 0
