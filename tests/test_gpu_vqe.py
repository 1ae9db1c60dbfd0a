"""VQE outer loop on the GPU path (L-BFGS-B on the adjoint gradient).

* the energy goes down from the HF point and never below the lowest
  eigenvalue of H in the N-electron sector (variational bound, dense eigh);
* the returned energy equals the oracle's energy at the returned theta;
* the returned gradient equals the oracle's (Algorithm 1) gradient there.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2208_10978_gb300 as q2
from paper_2208_10978_gb300 import vqe
from oracle import statevector as sv
from synth.workloads import uccsd_energy

pytestmark = pytest.mark.gpu


def _sector_min(n, ne, ham):
    Hd = sv.dense_hamiltonian(n, ham.x, ham.z, ham.c)
    idx = [i for i in range(1 << n) if bin(i).count("1") == ne]
    return float(np.linalg.eigvalsh(Hd[np.ix_(idx, idx)]).min())


@pytest.mark.parametrize("n,ne,seed", [(8, 4, 0), (8, 3, 1)])
def test_vqe_descends_within_variational_bound(n, ne, seed):
    w = uccsd_energy(n, ne, seed=seed)
    ans = q2.Ansatz.from_uccsd(w.ansatz)
    ham = q2.Hamiltonian(n, w.ham.x, w.ham.z, w.ham.c)
    th0 = np.zeros(w.ansatz.n_params)
    e_hf, _, _ = q2.vqe_energy_grad(ans, ham, th0, dtype="complex128", want_grad=False)
    res = vqe.minimize(ans, ham, th0, dtype="complex128", maxiter=300, gtol=1e-8)
    lam = _sector_min(n, ne, w.ham)
    assert res.energy < e_hf - 1e-3
    assert res.energy >= lam - 1e-9
    assert res.energy <= res.history[0]
    a = w.ansatz
    e_ref, gphi = sv.energy_and_gradient(n, ne, a.x, a.z, a.angles(res.theta), w.ham.x, w.ham.z, w.ham.c)
    assert abs(res.energy - e_ref) < 1e-10
    g_ref = sv.fold_to_theta(gphi, a.param, a.coef, a.n_params)
    assert abs(res.grad_norm - np.linalg.norm(g_ref)) < 1e-9
