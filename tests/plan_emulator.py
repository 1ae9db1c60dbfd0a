"""Host-side walk of the library's pass/group/block tables (test helper).

Reads the schedules exported by include/q2_debug.h and applies them to a
NumPy state exactly the way the tile kernels index memory:

* tile t, local index l -> amplitude deposit(t, umask) ^ XOR_b(l_b w_b);
* sweep and expectation walk register blocks: thread tid, coset j holds the
  local indices base(tid) ^ uj[j] ^ comb[c]; a group pairs combo c with c ^ a;
  code = tilecode ^ blane[lane] ^ bwarp[warp] ^ bjcode[j] ^ bccode[c];
* H apply and the reverse sweep walk groups one at a time: pair j of thread
  tid is insert_zero(tid, pivot) | pu[j] (diagonal: tid + NT*j);
  code = tilecode ^ plane[lane] ^ pwarp[warp] ^ pjcode[j].

Comparing the result with the oracle checks the schedulers (tiling bases,
blocks, codes, LUTs, sign masks) on the CPU; the CUDA kernels themselves are
checked on the GPU.
"""

import ctypes

import numpy as np

PASS_DT = np.dtype([("w", "<u8", 13), ("umask", "<u8"), ("T", "<i4"), ("C", "<i4"),
                    ("g_begin", "<i4"), ("g_end", "<i4"), ("rot_begin", "<i4"), ("rot_end", "<i4"),
                    ("lut_begin", "<i4"), ("lut_count", "<i4"), ("b_begin", "<i4"), ("b_end", "<i4")])
GROUP_DT = np.dtype([("bp", "<u8", 8), ("xl", "<u4"), ("lut", "<u4"), ("rot0", "<u4"), ("kind", "u1"),
                     ("r", "u1"), ("m", "u1"), ("a", "u1"), ("bjcode", "u1", 16), ("bccode", "u1", 16),
                     ("blane", "u1", 32), ("bwarp", "u1", 8), ("pivot", "u1"), ("one_param", "u1"), ("pad0", "u1", 2),
                     ("wlut", "<u4"),
                     ("pjcode", "u1", 32), ("plane", "u1", 32), ("pwarp", "u1", 8), ("pu", "<u2", 16),
                     ("pad1", "u1", 8)])
BLOCK_DT = np.dtype([("comb", "<u2", 16), ("uj", "<u2", 16), ("d", "u1"), ("piv", "u1", 4), ("canon", "u1"), ("pad0", "u1", 2),
                     ("g_begin", "<u2"), ("g_end", "<u2"), ("pad1", "u1", 4)])
assert PASS_DT.itemsize == 152 and GROUP_DT.itemsize == 272 and BLOCK_DT.itemsize == 80

DIAG, REAL, XROT, PAIR = 0, 1, 2, 3


def _p(a):
    return ctypes.c_void_p(a.ctypes.data) if a is not None else None


def rot_plan(lib, n, x, z, phi, T, C):
    x = np.ascontiguousarray(x, dtype=np.uint64)
    z = np.ascontiguousarray(z, dtype=np.uint64)
    phi = np.ascontiguousarray(phi, dtype=np.float64)
    counts = np.zeros(4, dtype=np.int64)
    f = lib.q2_debug_rot_plan
    f.argtypes = [ctypes.c_int, ctypes.c_int64] + [ctypes.c_void_p] * 3 + [ctypes.c_int] * 2 + [ctypes.c_void_p] * 6
    f.restype = ctypes.c_int
    assert f(n, len(x), _p(x), _p(z), _p(phi), T, C, _p(counts), None, None, None, None, None) == 0
    passes = np.zeros(counts[0], dtype=PASS_DT)
    groups = np.zeros(counts[1], dtype=GROUP_DT)
    blocks = np.zeros(counts[3], dtype=BLOCK_DT)
    lut = np.zeros(2 * max(1, counts[2]))
    sm = np.zeros(max(1, len(x)), dtype=np.uint64)
    assert f(n, len(x), _p(x), _p(z), _p(phi), T, C, _p(counts), _p(passes), _p(groups), _p(blocks),
             _p(lut), _p(sm)) == 0
    return passes, groups, blocks, lut.reshape(-1, 2), sm


def ham_plan(lib, n, x, z, c, T, C):
    x = np.ascontiguousarray(x, dtype=np.uint64)
    z = np.ascontiguousarray(z, dtype=np.uint64)
    c = np.ascontiguousarray(c, dtype=np.float64)
    counts = np.zeros(4, dtype=np.int64)
    f = lib.q2_debug_ham_plan
    f.argtypes = [ctypes.c_int, ctypes.c_int64] + [ctypes.c_void_p] * 3 + [ctypes.c_int] * 2 + [ctypes.c_void_p] * 5
    f.restype = ctypes.c_int
    assert f(n, len(x), _p(x), _p(z), _p(c), T, C, _p(counts), None, None, None, None) == 0
    passes = np.zeros(counts[0], dtype=PASS_DT)
    groups = np.zeros(counts[1], dtype=GROUP_DT)
    blocks = np.zeros(counts[3], dtype=BLOCK_DT)
    lut = np.zeros(2 * max(1, counts[2]))
    assert f(n, len(x), _p(x), _p(z), _p(c), T, C, _p(counts), _p(passes), _p(groups), _p(blocks),
             _p(lut)) == 0
    return passes, groups, blocks, lut.reshape(-1, 2)


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


def _tilecode(g, T, ntiles):
    t = np.arange(ntiles, dtype=np.uint64) << np.uint64(T)
    c = np.zeros(ntiles, dtype=np.int64)
    for k in range(int(g["r"])):
        c |= _par(t & np.uint64(g["bp"][k])) << k
    return c


def _block_layout(b, T, NT):
    """Local indices [nthr, J, 2^d] of every thread's cosets and their (lane, warp)."""
    d = int(b["d"])
    ncos = 1 << (T - d)
    J = max(1, ncos // NT)
    nthr = min(NT, ncos)
    tid = np.arange(nthr, dtype=np.uint64)
    base = tid.copy()
    for i in range(d):
        base = _insert0(base, int(b["piv"][i]))
    l = (base[:, None, None] ^ b["uj"][:J].astype(np.uint64)[None, :, None]
         ^ b["comb"][:1 << d].astype(np.uint64)[None, None, :])
    return d, J, nthr, l.astype(np.int64), (tid % 32).astype(np.int64), (tid // 32).astype(np.int64)


def _block_codes(g, d, J, lane, warp, tcode):
    """code[t, tid, j, c]."""
    th = (g["blane"][lane].astype(np.int64) ^ g["bwarp"][warp].astype(np.int64))
    return (tcode[:, None, None, None] ^ th[None, :, None, None]
            ^ g["bjcode"][:J].astype(np.int64)[None, None, :, None]
            ^ g["bccode"][:1 << d].astype(np.int64)[None, None, None, :])


def _pair_combos(a, d):
    """Combos c with the highest set bit of a clear, and their partners c ^ a."""
    hb = a.bit_length() - 1
    cs = np.array([c for c in range(1 << d) if not (c >> hb) & 1], dtype=np.int64)
    return cs, cs ^ a


def sweep(psi, n, passes, groups, blocks, lut, NT, inverse=False):
    psi = psi.copy()
    order = range(len(passes) - 1, -1, -1) if inverse else range(len(passes))
    sgn = -1.0 if inverse else 1.0
    for pi in order:
        pd = passes[pi]
        T = int(pd["T"])
        idx = tile_index(n, pd)
        tile = psi[idx]
        ntiles = tile.shape[0]
        g0 = int(pd["g_begin"])
        bb_, be_ = int(pd["b_begin"]), int(pd["b_end"])
        brange = range(be_ - 1, bb_ - 1, -1) if inverse else range(bb_, be_)
        for bi in brange:
            b = blocks[bi]
            d, J, nthr, l, lane, warp = _block_layout(b, T, NT)
            amps = tile[:, l]                      # [t, tid, j, c]
            gb_, ge_ = int(b["g_begin"]), int(b["g_end"])
            grange = range(ge_ - 1, gb_ - 1, -1) if inverse else range(gb_, ge_)
            for gk in grange:
                g = groups[g0 + gk]
                code = _block_codes(g, d, J, lane, warp, _tilecode(g, T, ntiles))
                cs = lut[int(g["lut"]) + code]
                c, s = cs[..., 0], sgn * cs[..., 1]
                kind = int(g["kind"])
                if kind == DIAG:
                    amps = (c - 1j * s) * amps
                    continue
                ci, cj = _pair_combos(int(g["a"]), d)
                x, y = amps[..., ci], amps[..., cj]
                cc, ss = c[..., ci], s[..., ci]
                if kind == REAL:
                    amps[..., ci], amps[..., cj] = cc * x - ss * y, ss * x + cc * y
                else:
                    amps[..., ci], amps[..., cj] = cc * x - 1j * ss * y, cc * y - 1j * ss * x
            tile[:, l] = amps
        psi[idx] = tile
    return psi


def expectation(psi, n, passes, groups, blocks, lut, NT):
    """(sum_t c_t <P_t>, <psi|psi>) walking the Hamiltonian schedule."""
    e = 0.0
    for pd in passes:
        T = int(pd["T"])
        idx = tile_index(n, pd)
        tile = psi[idx]
        ntiles = tile.shape[0]
        g0 = int(pd["g_begin"])
        for bi in range(pd["b_begin"], pd["b_end"]):
            b = blocks[bi]
            d, J, nthr, l, lane, warp = _block_layout(b, T, NT)
            amps = tile[:, l]
            for gk in range(int(b["g_begin"]), int(b["g_end"])):
                g = groups[g0 + gk]
                code = _block_codes(g, d, J, lane, warp, _tilecode(g, T, ntiles))
                rq = lut[int(g["lut"]) + code]
                if int(g["kind"]) == DIAG:
                    e += float(np.sum(rq[..., 0] * np.abs(amps) ** 2))
                    continue
                ci, cj = _pair_combos(int(g["a"]), d)
                w = np.conj(amps[..., ci]) * amps[..., cj]
                e += float(np.sum(2 * (rq[..., ci, 0] * w.real + rq[..., ci, 1] * w.imag)))
    return e, float(np.vdot(psi, psi).real)


def _pair_layout(g, T, NT):
    pair = int(g["kind"]) != DIAG
    per = 1 << (T - 1) if pair else 1 << T
    P = max(1, per // NT)
    nthr = min(NT, per)
    tid = np.arange(nthr, dtype=np.uint64)
    if pair:
        li = _insert0(tid, int(g["pivot"]))[:, None] | g["pu"][:P].astype(np.uint64)[None, :]
    else:
        li = tid[:, None] + np.uint64(NT) * np.arange(P, dtype=np.uint64)[None, :]
    lane, warp = (tid % 32).astype(np.int64), (tid // 32).astype(np.int64)
    return P, li.astype(np.int64), lane, warp


def _pair_codes(g, P, lane, warp, tcode):
    th = g["plane"][lane].astype(np.int64) ^ g["pwarp"][warp].astype(np.int64)
    return tcode[:, None, None] ^ th[None, :, None] ^ g["pjcode"][:P].astype(np.int64)[None, None, :]


def happly(psi, n, passes, groups, lut, NT):
    lam = np.zeros_like(psi)
    for pd in passes:
        T = int(pd["T"])
        idx = tile_index(n, pd)
        tp = psi[idx]
        tl = lam[idx]
        for gi in range(pd["g_begin"], pd["g_end"]):
            g = groups[gi]
            P, li, lane, warp = _pair_layout(g, T, NT)
            code = _pair_codes(g, P, lane, warp, _tilecode(g, T, tp.shape[0]))
            rq = lut[int(g["lut"]) + code]
            if int(g["kind"]) == DIAG:
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
            P, li, lane, warp = _pair_layout(g, T, NT)
            code = _pair_codes(g, P, lane, warp, _tilecode(g, T, tp.shape[0]))
            cs = lut[int(g["lut"]) + code]
            c, s = cs[..., 0], -cs[..., 1]
            k0 = int(pd["rot_begin"]) + int(g["rot0"])
            if kind == DIAG:
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
                sign = 1.0 - 2.0 * ((signmask[k0 + k].astype(np.uint64) >> code.astype(np.uint64))
                                    & np.uint64(1)).astype(np.float64)
                g_out[k0 + k] += float(np.sum(sign * val))
            if kind == DIAG:
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


def rot_weights(lib, n, x, z, param, coef, T, C, n_groups):
    """Gradient tables of an ansatz schedule: (groups with one_param/wlut, weights, fold)."""
    x = np.ascontiguousarray(x, dtype=np.uint64)
    z = np.ascontiguousarray(z, dtype=np.uint64)
    param = np.ascontiguousarray(param, dtype=np.int32)
    coef = np.ascontiguousarray(coef, dtype=np.float64)
    f = lib.q2_debug_rot_weights
    f.argtypes = [ctypes.c_int, ctypes.c_int64] + [ctypes.c_void_p] * 4 + [ctypes.c_int] * 2 + [ctypes.c_void_p] * 4
    f.restype = ctypes.c_int
    nw = np.zeros(1, dtype=np.int64)
    assert f(n, len(x), _p(x), _p(z), _p(param), _p(coef), T, C, _p(nw), None, None, None) == 0
    groups = np.zeros(n_groups, dtype=GROUP_DT)
    wl = np.zeros(max(1, int(nw[0])))
    fold = np.zeros(max(1, len(x)))
    assert f(n, len(x), _p(x), _p(z), _p(param), _p(coef), T, C, _p(nw), _p(groups), _p(wl), _p(fold)) == 0
    return groups, wl, fold


def reverse_weighted(psi, lam, n, passes, groups, lut, signmask, wlut, NT):
    """Reverse sweep as the kernels run it with gradient weights: a one-parameter
    group adds sum_pairs w(code) val at its first rotation, other groups per rotation."""
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
            P, li, lane, warp = _pair_layout(g, T, NT)
            code = _pair_codes(g, P, lane, warp, _tilecode(g, T, tp.shape[0]))
            cs = lut[int(g["lut"]) + code]
            c, s = cs[..., 0], -cs[..., 1]
            k0 = int(pd["rot_begin"]) + int(g["rot0"])
            if kind == DIAG:
                a, b = tp[:, li], tl[:, li]
                val = (np.conj(b) * a).imag
            else:
                lj = li ^ int(g["xl"])
                pa, pb, la, lb = tp[:, li], tp[:, lj], tl[:, li], tl[:, lj]
                if kind == REAL:
                    val = (np.conj(lb) * pa - np.conj(la) * pb).real
                else:
                    val = (np.conj(la) * pb + np.conj(lb) * pa).imag
            if int(g["one_param"]):
                g_out[k0] += float(np.sum(wlut[int(g["wlut"]) + code] * val))
            else:
                for k in range(int(g["m"])):
                    sign = 1.0 - 2.0 * ((signmask[k0 + k].astype(np.uint64) >> code.astype(np.uint64))
                                        & np.uint64(1)).astype(np.float64)
                    g_out[k0 + k] += float(np.sum(sign * val))
            if kind == DIAG:
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


def _gray(t):
    return t ^ (t >> 1)


def _ctz(v):
    return (v & -v).bit_length() - 1


def pass_is_canon4(pd, blocks):
    """The sweep fast path's condition: every block canonical, 4-dimensional, exactly 4 groups."""
    if pd["g_end"] - pd["g_begin"] > 16 or pd["b_end"] <= pd["b_begin"]:
        return False
    for b in blocks[int(pd["b_begin"]):int(pd["b_end"])]:
        if not (int(b["d"]) == 4 and int(b["canon"]) == 4 and int(b["g_end"]) - int(b["g_begin"]) == 4):
            return False
    return True


def sweep_c4(psi, n, passes, groups, blocks, lut, NT, lut_base=5 * 1024):
    """The sweep's canonical 4-dimensional fast path, with its exact address arithmetic:
    byte offsets of amplitudes (8 bytes) walked in Gray-code order over the block's four
    combo generators W_i = comb[1 << i] << 3 from the coset base (base(tid) ^ uj[j]) << 3;
    per group K, the LUT byte address A = lutoff | (code << 4) with
    code = tilecode ^ (blane[lane] ^ bwarp[warp]) ^ bjcode[j], walked in Gray-code order
    over the three pair generators bccode[1 << i] << 4 (i != K).  lutoff is the group's
    LUT offset (16-byte entries) from a 1 KiB-aligned staged LUT start `lut_base`.
    Passes that do not qualify take the general walk."""
    psi = psi.copy()
    for pd in passes:
        if not pass_is_canon4(pd, blocks):
            psi = sweep(psi, n, pd[None], groups, blocks, lut, NT)
            continue
        T = int(pd["T"])
        idx = tile_index(n, pd)
        tile = psi[idx]
        ntiles = tile.shape[0]
        g0 = int(pd["g_begin"])
        tid = np.arange(NT, dtype=np.int64)
        lane, warp = tid % 32, tid // 32
        J = (1 << (T - 4)) // NT
        for bi in range(int(pd["b_begin"]), int(pd["b_end"])):
            b = blocks[bi]
            bt = tid.astype(np.uint64)
            for i in range(4):
                bt = _insert0(bt, int(b["piv"][i]))
            bt = bt.astype(np.int64)
            W = [int(b["comb"][1 << i]) << 3 for i in range(4)]
            for j in range(J):
                o = (bt ^ int(b["uj"][j])) << 3
                addr = {}
                for t in range(16):
                    addr[_gray(t)] = o.copy()
                    if t < 15:
                        o = o ^ W[_ctz(t + 1)]
                assert all(np.all(a % 8 == 0) for a in addr.values())
                v = {c: tile[:, addr[c] >> 3] for c in range(16)}          # [t, tid]
                for k in range(4):
                    g = groups[g0 + int(b["g_begin"]) + k]
                    lutoff = lut_base + (int(g["lut"]) - int(pd["lut_begin"])) * 16
                    thr = g["blane"][lane].astype(np.int64) ^ g["bwarp"][warp].astype(np.int64)
                    cb = _tilecode(g, T, ntiles)[:, None] ^ thr[None, :] ^ int(g["bjcode"][j])
                    A = lutoff | (cb << 4)
                    dims = [d for d in range(4) if d != k]
                    G = [int(g["bccode"][1 << d]) << 4 for d in dims]
                    a = A.copy()
                    for t in range(8):
                        p = _gray(t)
                        c = sum(((p >> i) & 1) << dims[i] for i in range(3))
                        e = (a - lut_base) // 16 + int(pd["lut_begin"])
                        cc, ss = lut[e, 0], lut[e, 1]
                        x, y = v[c], v[c | (1 << k)]
                        v[c], v[c | (1 << k)] = cc * x - ss * y, ss * x + cc * y
                        if t < 7:
                            a = a ^ G[_ctz(t + 1)]
                for c in range(16):
                    tile[:, addr[c] >> 3] = v[c]
        psi[idx] = tile
    return psi


def expectation_chunked(psi, n, passes, groups, blocks, lut, NT, jc):
    """(sum_t c_t <P_t>, <psi|psi>) walking the Hamiltonian schedule as the general
    expectation kernel does: a thread's J cosets of a block are taken in chunks of jc
    (jc * 2^d amplitudes in registers); within a chunk, coset j0 + j uses code
    tilecode ^ blane ^ bwarp ^ bjcode[j0 + j] ^ bccode[c]; every group of the block is
    walked once per chunk.  Any jc in 1..J that divides J gives the same sum."""
    e = 0.0
    for pd in passes:
        T = int(pd["T"])
        idx = tile_index(n, pd)
        tile = psi[idx]
        ntiles = tile.shape[0]
        g0 = int(pd["g_begin"])
        for bi in range(int(pd["b_begin"]), int(pd["b_end"])):
            b = blocks[bi]
            d, J, nthr, l, lane, warp = _block_layout(b, T, NT)
            step = min(jc, J)
            assert J % step == 0
            for j0 in range(0, J, step):
                amps = tile[:, l[:, j0:j0 + step, :]]           # [t, tid, j, c]
                for gk in range(int(b["g_begin"]), int(b["g_end"])):
                    g = groups[g0 + gk]
                    th = g["blane"][lane].astype(np.int64) ^ g["bwarp"][warp].astype(np.int64)
                    cb = _tilecode(g, T, ntiles)[:, None, None] ^ th[None, :, None]
                    cj = cb ^ g["bjcode"][j0:j0 + step].astype(np.int64)[None, None, :]
                    code = cj[..., None] ^ g["bccode"][:1 << d].astype(np.int64)[None, None, None, :]
                    rq = lut[int(g["lut"]) + code]
                    if int(g["kind"]) == DIAG:
                        e += float(np.sum(rq[..., 0] * np.abs(amps) ** 2))
                        continue
                    ci, cjp = _pair_combos(int(g["a"]), d)
                    w = np.conj(amps[..., ci]) * amps[..., cjp]
                    e += float(np.sum(2 * (rq[..., ci, 0] * w.real + rq[..., ci, 1] * w.imag)))
    return e, float(np.vdot(psi, psi).real)


def expectation_lean(psi, n, passes, groups, blocks, lut, NT, lut_base=7 * 2048):
    """The lean expectation path's exact address arithmetic (REAL and DIAG groups, blocks of
    d <= 3): amplitude byte offsets (8 bytes) walked in Gray-code order from
    (base(tid) ^ uj[j]) << 3 over W_i = comb[1 << i] << 3; per group the LUT byte address
    A = lutaddr | (tilecode ^ blane ^ bwarp) << 3, per coset A ^ bjcode[j] << 3, then a Gray
    walk over the pair (or, for DIAG, combo) bits with generators bccode[1 << i] << 3;
    the group's LUT starts at a multiple of its size from a 2 KiB-aligned `lut_base`."""
    e = 0.0
    for pd in passes:
        T = int(pd["T"])
        idx = tile_index(n, pd)
        tile = psi[idx]
        ntiles = tile.shape[0]
        g0 = int(pd["g_begin"])
        tid = np.arange(NT, dtype=np.int64)
        lane, warp = tid % 32, tid // 32
        for bi in range(int(pd["b_begin"]), int(pd["b_end"])):
            b = blocks[bi]
            d = int(b["d"])
            assert d <= 3
            N, J = 1 << d, (1 << (T - d)) // NT
            bt = tid.astype(np.uint64)
            for i in range(d):
                bt = _insert0(bt, int(b["piv"][i]))
            bt = bt.astype(np.int64)
            W = [int(b["comb"][1 << i]) << 3 for i in range(d)]
            v = {}
            for j in range(J):
                o = (bt ^ int(b["uj"][j])) << 3
                for t in range(N):
                    v[j, _gray(t)] = tile[:, o >> 3]
                    if t + 1 < N:
                        o = o ^ W[_ctz(t + 1)]
            for gk in range(int(b["g_begin"]), int(b["g_end"])):
                g = groups[g0 + gk]
                kind = int(g["kind"])
                assert kind in (DIAG, REAL)
                lutaddr = lut_base + (int(g["lut"]) - int(pd["lut_begin"])) * 8
                assert lutaddr % (8 << int(g["r"])) == 0
                th = g["blane"][lane].astype(np.int64) ^ g["bwarp"][warp].astype(np.int64)
                A = lutaddr | ((_tilecode(g, T, ntiles)[:, None] ^ th[None, :]) << 3)
                gens = [int(g["bccode"][1 << i]) << 3 for i in range(d)]
                s = 0.0
                for j in range(J):
                    a = A ^ (int(g["bjcode"][j]) << 3)
                    if kind == DIAG:
                        for t in range(N):
                            r = lut[(a - lut_base) // 8 + int(pd["lut_begin"]), 0]
                            s += float(np.sum(r * np.abs(v[j, _gray(t)]) ** 2))
                            if t + 1 < N:
                                a = a ^ gens[_ctz(t + 1)]
                    else:
                        x = int(g["a"])
                        hb = x.bit_length() - 1
                        free = [i for i in range(d) if i != hb]
                        for t in range(N // 2):
                            p = _gray(t)
                            c = sum(((p >> i) & 1) << free[i] for i in range(d - 1))
                            r = lut[(a - lut_base) // 8 + int(pd["lut_begin"]), 0]
                            w = np.conj(v[j, c]) * v[j, c ^ x]
                            s += 2 * float(np.sum(r * w.real))
                            if t + 1 < N // 2:
                                a = a ^ gens[free[_ctz(t + 1)]]
                e += s
    return e, float(np.vdot(psi, psi).real)
