"""Seeded random molecular-integral stand-ins.

The paper obtains h_pq and the two-electron integrals from PySCF
(Sec. "Hamiltonian", Eq. ferm-ham).  No chemistry package or molecule data
is used here: both are drawn from one ``numpy.random.default_rng(seed)``
stream with the symmetries real integrals have.

  * h: symmetric, h_pq ~ N(0, 1) * exp(-|p - q|), drawn for p <= q
    (row-major upper triangle, diagonal included) and mirrored.
  * (pq|rs): chemists' notation with the 8-fold permutational symmetry
    (pq|rs) = (qp|rs) = (pq|sr) = (rs|pq) = ...; one N(0, 0.1) draw (0.1 is
    read as the standard deviation) per symmetry class, classes enumerated
    over compound indices pq = p*(p+1)/2 + q (p >= q), rs likewise, pq >= rs,
    in increasing (pq, rs) order.
"""

import numpy as np


def random_integrals(m, seed):
    """Return (h, eri) for m spatial orbitals; eri[p, q, r, s] = (pq|rs)."""
    if m < 1:
        raise ValueError("need at least one spatial orbital")
    rng = np.random.default_rng(seed)
    h = np.zeros((m, m))
    iu = np.triu_indices(m)
    vals = rng.standard_normal(len(iu[0])) * np.exp(-np.abs(iu[0] - iu[1]))
    h[iu] = vals
    h = h + np.triu(h, 1).T

    npair = m * (m + 1) // 2
    pairs = [(p, q) for p in range(m) for q in range(p + 1)]  # index = p(p+1)/2+q
    ncls = npair * (npair + 1) // 2
    draws = rng.normal(0.0, 0.1, size=ncls)
    eri = np.zeros((m, m, m, m))
    k = 0
    for a in range(npair):
        p, q = pairs[a]
        for b in range(a + 1):
            r, s = pairs[b]
            v = draws[k]
            k += 1
            for (i, j) in ((p, q), (q, p)):
                for (u, w) in ((r, s), (s, r)):
                    eri[i, j, u, w] = v
                    eri[u, w, i, j] = v
    return h, eri
