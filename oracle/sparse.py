"""Dict-of-amplitudes state for a few rotations on large registers.

A state with few nonzero amplitudes is kept as {index: complex}.  The
definitions are those of ``statevector``: (P psi)[i] = i^{|x&z|}
(-1)^{|(i^x)&z|} psi[i^x], i.e. P|j> = i^{|x&z|} (-1)^{|j&z|} |j^x>, and a
rotation is cos(phi/2) psi - i sin(phi/2) P psi.  Used to check the CUDA
path at 32 qubits, where a dense complex128 copy would take 64 GiB.
"""

def _pc(v):
    return bin(v).count("1")


def pauli_apply(state, x, z):
    x, z = int(x), int(z)
    ph = 1j ** _pc(x & z)
    out = {}
    for j, a in state.items():
        s = -1.0 if _pc(j & z) & 1 else 1.0
        k = j ^ x
        out[k] = out.get(k, 0.0) + ph * s * a
    return out


def rotation_apply(state, x, z, phi):
    import math
    c, s = math.cos(phi / 2), math.sin(phi / 2)
    p = pauli_apply(state, x, z)
    out = {j: c * a for j, a in state.items()}
    for j, a in p.items():
        out[j] = out.get(j, 0.0) - 1j * s * a
    return out


def rotations_apply(state, xs, zs, phis):
    for x, z, phi in zip(xs, zs, phis):
        state = rotation_apply(state, x, z, phi)
    return state


def expectation(state, xs, zs, cs):
    """sum_t c_t <psi|P_t|psi> for a sparse psi."""
    e = 0.0
    for x, z, c in zip(xs, zs, cs):
        p = pauli_apply(state, x, z)
        e += c * sum((state.get(j, 0.0).conjugate() * a) for j, a in p.items()).real
    return float(e)


def norm2(state):
    return float(sum(abs(a) ** 2 for a in state.values()))
