"""Host-side walk of the library's pass/group tables (test helper).

Reads the schedules exported by include/q2_debug.h and applies them to a
NumPy state exactly the way the tile kernels index memory: tile t, local
index l -> amplitude deposit(t, umask) ^ XOR_b(l_b w_b); thread tid handles
pair q = tid + NT * j with code = code(tile, tid) ^ jcode[j].  Comparing the
result with the oracle checks the schedulers (tiling bases, codes, LUTs,
sign masks) on the CPU; the CUDA kernels themselves are checked on the GPU.
"""

import ctypes

import numpy as np

PASS_DT = np.dtype([("w", "<u8", 13), ("umask", "<u8"), ("T", "<i4"), ("C", "<i4"),
                    ("g_begin", "<i4"), ("g_end", "<i4"), ("rot_begin", "<i4"), ("rot_end", "<i4"),
                    ("lut_begin", "<i4"), ("lut_count", "<i4")])
GROUP_DT = np.dtype([("bp", "<u8", 8), ("xl", "<u4"), ("lut", "<u4"), ("rot0", "<u4"), ("kind", "u1"),
                     ("pivot", "u1"), ("r", "u1"), ("m", "u1"), ("jcode", "u1", 32)])
assert PASS_DT.itemsize == 144 and GROUP_DT.itemsize == 112

DIAG, REAL, XROT, PAIR = 0, 1, 2, 3


def _p(a):
    return ctypes.c_void_p(a.ctypes.data) if a is not None else None


def rot_plan(lib, n, x, z, phi, T, C):
    x = np.ascontiguousarray(x, dtype=np.uint64)
    z = np.ascontiguousarray(z, dtype=np.uint64)
    phi = np.ascontiguousarray(phi, dtype=np.float64)
    counts = np.zeros(3, dtype=np.int64)
    f = lib.q2_debug_rot_plan
    f.argtypes = [ctypes.c_int, ctypes.c_int64] + [ctypes.c_void_p] * 3 + [ctypes.c_int] * 2 + [ctypes.c_void_p] * 5
    f.restype = ctypes.c_int
    assert f(n, len(x), _p(x), _p(z), _p(phi), T, C, _p(counts), None, None, None, None) == 0
    passes = np.zeros(counts[0], dtype=PASS_DT)
    groups = np.zeros(counts[1], dtype=GROUP_DT)
    lut = np.zeros(2 * max(1, counts[2]))
    sm = np.zeros(max(1, len(x)), dtype=np.uint64)
    assert f(n, len(x), _p(x), _p(z), _p(phi), T, C, _p(counts), _p(passes), _p(groups), _p(lut), _p(sm)) == 0
    return passes, groups, lut.reshape(-1, 2), sm


def ham_plan(lib, n, x, z, c, T, C):
    x = np.ascontiguousarray(x, dtype=np.uint64)
    z = np.ascontiguousarray(z, dtype=np.uint64)
    c = np.ascontiguousarray(c, dtype=np.float64)
    counts = np.zeros(3, dtype=np.int64)
    f = lib.q2_debug_ham_plan
    f.argtypes = [ctypes.c_int, ctypes.c_int64] + [ctypes.c_void_p] * 3 + [ctypes.c_int] * 2 + [ctypes.c_void_p] * 4
    f.restype = ctypes.c_int
    assert f(n, len(x), _p(x), _p(z), _p(c), T, C, _p(counts), None, None, None) == 0
    passes = np.zeros(counts[0], dtype=PASS_DT)
    groups = np.zeros(counts[1], dtype=GROUP_DT)
    lut = np.zeros(2 * max(1, counts[2]))
    assert f(n, len(x), _p(x), _p(z), _p(c), T, C, _p(counts), _p(passes), _p(groups), _p(lut)) == 0
    return passes, groups, lut.reshape(-1, 2)


def _par(a):
    return (np.bitwise_count(np.asarray(a, dtype=np.uint64)) & 1).astype(np.int64)


def _deposit(v, mask):
    v = np.asarray(v, dtype=np.uint64)
    out = np.zeros_like(v)
    k = 0
    for q in range(64):
        if (int(mask) >> q) & 1:
            out |= ((v >> np.uint64(k)) & np.uint64(1)) << np.uint64(q)
            k += 1
    return out


def _insert0(q, p):
    q = np.asarray(q, dtype=np.uint64)
    lo = q & np.uint64((1 << p) - 1)
    return ((q >> np.uint64(p)) << np.uint64(p + 1)) | lo


def tile_index(n, pd):
    """(ntiles, 2^T) array of amplitude indices of every tile of a pass."""
    T, C = int(pd["T"]), int(pd["C"])
    t = np.arange(1 << (n - T), dtype=np.uint64)
    base = _deposit(t, int(pd["umask"]))
    h = np.arange(1 << (T - C), dtype=np.uint64)
    off = np.zeros_like(h)
    for b in range(T - C):
        off ^= np.where((h >> np.uint64(b)) & np.uint64(1), np.uint64(pd["w"][C + b]), np.uint64(0))
    l = np.arange(1 << T, dtype=np.uint64)
    return (base[:, None] ^ off[l >> np.uint64(C)][None, :]) | (l & np.uint64((1 << C) - 1))[None, :]


def _codes(g, T, ntiles, nt, pair):
    """code[t, tid, j] as the kernels form it."""
    tid = np.arange(nt, dtype=np.uint64)
    lt = _insert0(tid, int(g["pivot"])) if pair else tid
    packed = (np.arange(ntiles, dtype=np.uint64)[:, None] << np.uint64(T)) | lt[None, :]
    code0 = np.zeros(packed.shape, dtype=np.int64)
    for l in range(int(g["r"])):
        code0 |= _par(packed & np.uint64(g["bp"][l])) << l
    return code0


def _layout(g, T, NT, pair):
    per = 1 << (T - 1) if pair else 1 << T
    P = max(1, per // NT)
    nt = min(NT, per)
    tid = np.arange(nt, dtype=np.uint64)
    j = np.arange(P, dtype=np.uint64)
    q = tid[:, None] + np.uint64(NT) * j[None, :]
    li = _insert0(q, int(g["pivot"])) if pair else q
    return P, nt, li.astype(np.int64)


def sweep(psi, n, passes, groups, lut, NT, inverse=False):
    psi = psi.copy()
    order = range(len(passes) - 1, -1, -1) if inverse else range(len(passes))
    sgn = -1.0 if inverse else 1.0
    for pi in order:
        pd = passes[pi]
        T = int(pd["T"])
        idx = tile_index(n, pd)
        tile = psi[idx]
        gr = range(pd["g_end"] - 1, pd["g_begin"] - 1, -1) if inverse else range(pd["g_begin"], pd["g_end"])
        for gi in gr:
            g = groups[gi]
            kind = int(g["kind"])
            pair = kind != DIAG
            P, nt, li = _layout(g, T, NT, pair)
            code = _codes(g, T, tile.shape[0], nt, pair)[:, :, None] ^ g["jcode"][:P].astype(np.int64)[None, None, :]
            cs = lut[int(g["lut"]) + code]
            c, s = cs[..., 0], sgn * cs[..., 1]
            if not pair:
                a = tile[:, li]
                tile[:, li] = (c - 1j * s) * a
                continue
            lj = li ^ int(g["xl"])
            a, b = tile[:, li], tile[:, lj]
            if kind == REAL:
                tile[:, li], tile[:, lj] = c * a - s * b, s * a + c * b
            else:
                tile[:, li], tile[:, lj] = c * a - 1j * s * b, c * b - 1j * s * a
        psi[idx] = tile
    return psi


def expectation(psi, n, passes, groups, lut, NT):
    """(sum_t c_t <P_t>, <psi|psi>) walking the Hamiltonian schedule."""
    e = 0.0
    for pd in passes:
        T = int(pd["T"])
        idx = tile_index(n, pd)
        tile = psi[idx]
        for gi in range(pd["g_begin"], pd["g_end"]):
            g = groups[gi]
            pair = int(g["kind"]) != DIAG
            P, nt, li = _layout(g, T, NT, pair)
            code = _codes(g, T, tile.shape[0], nt, pair)[:, :, None] ^ g["jcode"][:P].astype(np.int64)[None, None, :]
            rq = lut[int(g["lut"]) + code]
            if not pair:
                e += float(np.sum(rq[..., 0] * np.abs(tile[:, li]) ** 2))
            else:
                w = np.conj(tile[:, li]) * tile[:, li ^ int(g["xl"])]
                e += float(np.sum(2 * (rq[..., 0] * w.real + rq[..., 1] * w.imag)))
    return e, float(np.vdot(psi, psi).real)


def happly(psi, n, passes, groups, lut, NT):
    lam = np.zeros_like(psi)
    for pd in passes:
        T = int(pd["T"])
        idx = tile_index(n, pd)
        tp = psi[idx]
        tl = lam[idx]
        for gi in range(pd["g_begin"], pd["g_end"]):
            g = groups[gi]
            pair = int(g["kind"]) != DIAG
            P, nt, li = _layout(g, T, NT, pair)
            code = _codes(g, T, tp.shape[0], nt, pair)[:, :, None] ^ g["jcode"][:P].astype(np.int64)[None, None, :]
            rq = lut[int(g["lut"]) + code]
            if not pair:
                tl[:, li] += rq[..., 0] * tp[:, li]
            else:
                lj = li ^ int(g["xl"])
                R, Q = rq[..., 0], rq[..., 1]
                tl[:, li] += (R - 1j * Q) * tp[:, lj]
                tl[:, lj] += (R + 1j * Q) * tp[:, li]
        lam[idx] = tl
    return lam


def reverse(psi, lam, n, passes, groups, lut, signmask, NT):
    """Reverse sweep with per-rotation gradients g[k] = Im <lam|P_k|psi>."""
    psi, lam = psi.copy(), lam.copy()
    g_out = np.zeros(int(passes["rot_end"].max()) if len(passes) else 0)
    for pi in range(len(passes) - 1, -1, -1):
        pd = passes[pi]
        T = int(pd["T"])
        idx = tile_index(n, pd)
        tp, tl = psi[idx], lam[idx]
        for gi in range(pd["g_end"] - 1, pd["g_begin"] - 1, -1):
            g = groups[gi]
            kind = int(g["kind"])
            pair = kind != DIAG
            P, nt, li = _layout(g, T, NT, pair)
            code = _codes(g, T, tp.shape[0], nt, pair)[:, :, None] ^ g["jcode"][:P].astype(np.int64)[None, None, :]
            cs = lut[int(g["lut"]) + code]
            c, s = cs[..., 0], -cs[..., 1]
            k0 = int(pd["rot_begin"]) + int(g["rot0"])
            if not pair:
                a, b = tp[:, li], tl[:, li]
                val = (np.conj(b) * a).imag
            else:
                lj = li ^ int(g["xl"])
                pa, pb, la, lb = tp[:, li], tp[:, lj], tl[:, li], tl[:, lj]
                if kind == REAL:
                    val = (np.conj(lb) * pa - np.conj(la) * pb).real
                else:
                    val = (np.conj(la) * pb + np.conj(lb) * pa).imag
            for k in range(int(g["m"])):
                sign = 1.0 - 2.0 * ((signmask[k0 + k].astype(np.uint64) >> code.astype(np.uint64)) & np.uint64(1)).astype(np.float64)
                g_out[k0 + k] += float(np.sum(sign * val))
            if not pair:
                tp[:, li] = (c - 1j * s) * a
                tl[:, li] = (c - 1j * s) * b
            elif kind == REAL:
                tp[:, li], tp[:, lj] = c * pa - s * pb, s * pa + c * pb
                tl[:, li], tl[:, lj] = c * la - s * lb, s * la + c * lb
            else:
                tp[:, li], tp[:, lj] = c * pa - 1j * s * pb, c * pb - 1j * s * pa
                tl[:, li], tl[:, lj] = c * la - 1j * s * lb, c * lb - 1j * s * la
        psi[idx] = tp
        lam[idx] = tl
    return psi, lam, g_out
