"""Jordan-Wigner mapping of fermionic operators to Pauli strings.

The paper maps the second-quantized Hamiltonian (Eq. ferm-ham) to the qubit
form H = sum_i c_i P_i (Eq. qubit-ham) with a Jordan-Wigner transformation
(Sec. "Hamiltonian"); the cluster operators of Eq. ucc go through the same
mapping.  The convention is not printed; the one used here is

    a_q^dagger = Z_0 ... Z_{q-1} (X_q - i Y_q) / 2,
    a_q        = Z_0 ... Z_{q-1} (X_q + i Y_q) / 2,

so |1> on qubit q is an occupied spin-orbital (Eq. jw-wfn-map).

Arithmetic is carried in "XZ form": a term is  coef * X^x Z^z  (the matrix
product of all X factors, then all Z factors).  Two identities make this
exact with integer phase bookkeeping:

    (X^x1 Z^z1)(X^x2 Z^z2) = (-1)^{|z1 & x2|} X^{x1^x2} Z^{z1^z2},
    X^x Z^z = i^{-|x & z|} P(x, z),   P(x, z) = i^{|x & z|} X^x Z^z (Hermitian).

With Y = i X Z on one qubit: X - iY = X + XZ and X + iY = X - XZ, so each
ladder operator is a sum of two XZ-form strings with real weights +-1/2.
"""

import numpy as np

U64 = np.uint64


def popcount(a):
    """Bit count of each element of a uint64 array."""
    a = np.asarray(a, dtype=U64)
    if hasattr(np, "bitwise_count"):
        return np.bitwise_count(a).astype(np.int64)
    a = a - ((a >> U64(1)) & U64(0x5555555555555555))
    a = (a & U64(0x3333333333333333)) + ((a >> U64(2)) & U64(0x3333333333333333))
    a = (a + (a >> U64(4))) & U64(0x0F0F0F0F0F0F0F0F)
    return ((a * U64(0x0101010101010101)) >> U64(56)).astype(np.int64)


def _ladder_factor(q, dagger, choice):
    """XZ-form pieces of a_q^(dagger): returns (x, z, weight) arrays.

    choice 0 -> the X_q Z_{<q} piece (weight +1/2);
    choice 1 -> the X_q Z_q Z_{<q} piece (weight +1/2 for a^dagger, -1/2 for a).
    """
    q = np.asarray(q, dtype=U64)
    e = U64(1) << q
    chain = e - U64(1)
    x = e
    z = chain | (e if choice else U64(0))
    w = 0.5 if (choice == 0 or dagger) else -0.5
    return x, z, w


def _expand_products(idx, dag, coef):
    """Expand sum_k coef[k] * prod_l a_{idx[k,l]}^{(dag[l])} into XZ-form terms.

    idx: (K, L) integer qubit indices; dag: length-L sequence of bools, one
    pattern shared by every product; coef: (K,) real.  Returns (x, z, re, im)
    arrays of length K * 2**L with the Hermitian-basis coefficient split into
    real and imaginary parts (still with repeated (x, z) keys).
    """
    idx = np.asarray(idx, dtype=np.int64)
    K, L = idx.shape
    coef = np.asarray(coef, dtype=np.float64)
    xs, zs, res, ims = [], [], [], []
    for combo in range(1 << L):
        x = np.zeros(K, dtype=U64)
        z = np.zeros(K, dtype=U64)
        sign = np.zeros(K, dtype=np.int64)  # number of -1 factors
        w = coef.copy()
        for l in range(L):
            fx, fz, fw = _ladder_factor(idx[:, l], bool(dag[l]), (combo >> l) & 1)
            sign += popcount(z & fx)
            x ^= fx
            z ^= fz
            w = w * fw
        # coefficient of P(x, z) is  w * (-1)^sign * i^{-|x&z|}
        k = (2 * (sign & 1) - popcount(x & z)) % 4
        re = np.where(k == 0, w, np.where(k == 2, -w, 0.0))
        im = np.where(k == 1, w, np.where(k == 3, -w, 0.0))
        xs.append(x)
        zs.append(z)
        res.append(re)
        ims.append(im)
    return (np.concatenate(xs), np.concatenate(zs), np.concatenate(res),
            np.concatenate(ims))


def _combine(x, z, re, im):
    """Sum coefficients of equal (x, z); return keys sorted by (x, z)."""
    if len(x) == 0:
        e = np.zeros(0, dtype=U64)
        return e, e, np.zeros(0), np.zeros(0)
    order = np.lexsort((z, x))
    x, z, re, im = x[order], z[order], re[order], im[order]
    new = np.ones(len(x), dtype=bool)
    new[1:] = (x[1:] != x[:-1]) | (z[1:] != z[:-1])
    starts = np.flatnonzero(new)
    return x[starts], z[starts], np.add.reduceat(re, starts), np.add.reduceat(im, starts)


def fermion_operator_to_pauli(products, tol=1e-13):
    """Map a fermionic operator to Hermitian-basis Pauli strings.

    products: iterable of (coef, [(q, dagger), ...]) with complex coef.
    Returns (x, z, c) with complex c, sorted by (x, z), |c| > tol.
    """
    groups = {}
    for coef, ops in products:
        key = tuple(bool(d) for _, d in ops)
        groups.setdefault(key, []).append((complex(coef), [q for q, _ in ops]))
    xs, zs, res, ims = [], [], [], []
    for dag, items in groups.items():
        idx = np.array([q for _, q in items], dtype=np.int64).reshape(len(items), len(dag))
        cre = np.array([c.real for c, _ in items])
        cim = np.array([c.imag for c, _ in items])
        x, z, re, im = _expand_products(idx, dag, np.ones(len(items)))
        reps = 1 << len(dag)
        cr = np.tile(cre, reps)
        ci = np.tile(cim, reps)
        # (re + i im)(cr + i ci)
        xs.append(x)
        zs.append(z)
        res.append(re * cr - im * ci)
        ims.append(re * ci + im * cr)
    x, z, re, im = _combine(np.concatenate(xs), np.concatenate(zs),
                            np.concatenate(res), np.concatenate(ims))
    c = re + 1j * im
    keep = np.abs(c) > tol
    return x[keep], z[keep], c[keep]


def qubit_hamiltonian(h, eri, tol=1e-13):
    """JW qubit Hamiltonian of the spin-orbital electronic Hamiltonian.

    Reading of Eq. ferm-ham (the paper prints g^{pq}_{rs} a+_p a+_q a_r a_s
    with no factor and no index map): the standard chemists' form

      H = sum_{pq,s} h_pq a+_{ps} a_{qs}
          + 1/2 sum_{pqrs,s,t} (pq|rs) a+_{ps} a+_{rt} a_{st} a_{qs},

    with spin-orbital q = 2 * spatial + spin.  No constant (nuclear) term is
    added; the identity string arises from the algebra and is kept as
    x = z = 0.  Returns (x, z, c) with real c, sorted by (x, z), so terms
    sharing an xmask are contiguous.
    """
    h = np.asarray(h, dtype=np.float64)
    eri = np.asarray(eri, dtype=np.float64)
    m = h.shape[0]
    n = 2 * m
    so = np.arange(n)
    sp, sg = so // 2, so % 2

    # one-body: a+_P a_Q with equal spins
    P, Q = np.meshgrid(so, so, indexing="ij")
    P, Q = P.ravel(), Q.ravel()
    ok = sg[P] == sg[Q]
    P, Q = P[ok], Q[ok]
    x1, z1, r1, i1 = _expand_products(np.stack([P, Q], 1), (True, False), h[sp[P], sp[Q]])

    # two-body: 1/2 (PQ|RS) a+_P a+_R a_S a_Q, sigma_P = sigma_Q, sigma_R = sigma_S
    P, Q, R, S = np.meshgrid(so, so, so, so, indexing="ij")
    P, Q, R, S = P.ravel(), Q.ravel(), R.ravel(), S.ravel()
    ok = (sg[P] == sg[Q]) & (sg[R] == sg[S]) & (P != R) & (Q != S)
    P, Q, R, S = P[ok], Q[ok], R[ok], S[ok]
    w = 0.5 * eri[sp[P], sp[Q], sp[R], sp[S]]
    x2, z2, r2, i2 = _expand_products(np.stack([P, R, S, Q], 1),
                                      (True, True, False, False), w)

    x, z, re, im = _combine(np.concatenate([x1, x2]), np.concatenate([z1, z2]),
                            np.concatenate([r1, r2]), np.concatenate([i1, i2]))
    scale = max(1.0, float(np.max(np.abs(re))) if len(re) else 1.0)
    if len(im) and np.max(np.abs(im)) > 1e-12 * scale:
        raise AssertionError("JW Hamiltonian has non-real coefficients")
    keep = np.abs(re) > tol
    return x[keep], z[keep], re[keep]


def group_starts(x):
    """Start offsets of runs of equal x (x sorted); final entry = len(x)."""
    x = np.asarray(x)
    if len(x) == 0:
        return np.zeros(1, dtype=np.int64)
    new = np.ones(len(x), dtype=bool)
    new[1:] = x[1:] != x[:-1]
    return np.concatenate([np.flatnonzero(new), [len(x)]]).astype(np.int64)
