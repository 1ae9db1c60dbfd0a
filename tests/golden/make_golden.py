#!/usr/bin/env python3
"""Write the stored expected values of the full-size parity tests.

Every value comes from the oracle (oracle/c_oracle: plain C, double
precision) on inputs from synth/ (seeded generators); nothing here touches
the CUDA library.  Usage:

    python tests/golden/make_golden.py uccsd20   # 20 qubits, energy (~1 min on 8 cores)
    python tests/golden/make_golden.py uccsd24   # 24 qubits, energy + dE/dtheta (~2 h)

Each output file records the generator seed, the sizes, a few input values
(to detect a changed random stream) and the oracle results.
"""

import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

from oracle import c_oracle  # noqa: E402
from oracle.statevector import fold_to_theta  # noqa: E402
from synth.workloads import uccsd_energy  # noqa: E402


def fingerprint(w):
    return {"h00": float(w.h[0, 0]), "eri0000": float(w.eri[0, 0, 0, 0]), "theta0": float(w.theta[0]),
            "theta_last": float(w.theta[-1]), "c_sum": float(np.sum(w.ham.c)),
            "n_terms": int(w.ham.n_terms), "n_rot": int(w.ansatz.n_rot), "n_params": int(w.ansatz.n_params)}


def uccsd20():
    w = uccsd_energy(20, 10, seed=0)
    t = time.time()
    psi = c_oracle.apply_rotations(c_oracle.hf_state(20, 10), 20, w.ansatz.x, w.ansatz.z, w.angles())
    e, nrm = c_oracle.expectation(psi, 20, w.ham.x, w.ham.z, w.ham.c)
    amps = {str(i): [float(psi[i].real), float(psi[i].imag)] for i in
            sorted(np.argsort(-np.abs(psi))[:16].tolist())}
    out = {"workload": "uccsd_energy(20, 10, seed=0)", "oracle": "c_oracle (double)",
           "threads": c_oracle.threads(), "seconds": time.time() - t, "inputs": fingerprint(w),
           "energy": e / nrm, "norm": nrm, "largest_amplitudes": amps}
    with open(os.path.join(HERE, "uccsd20_seed0.json"), "w") as f:
        json.dump(out, f, indent=1)
    print("uccsd20", out["energy"], out["seconds"])


def uccsd24():
    w = uccsd_energy(24, 12, seed=0)
    a = w.ansatz
    t = time.time()
    e, gphi = c_oracle.energy_and_gradient(24, 12, a.x, a.z, a.angles(w.theta), w.ham.x, w.ham.z, w.ham.c)
    g = fold_to_theta(gphi, a.param, a.coef, a.n_params)
    out = {"workload": "uccsd_energy(24, 12, seed=0)", "oracle": "c_oracle (double), reverse mode",
           "threads": c_oracle.threads(), "seconds": time.time() - t, "inputs": fingerprint(w),
           "energy": e, "grad_theta": [float(v) for v in g]}
    with open(os.path.join(HERE, "uccsd24_seed0.json"), "w") as f:
        json.dump(out, f)
    print("uccsd24", e, out["seconds"])


if __name__ == "__main__":
    for name in sys.argv[1:]:
        {"uccsd20": uccsd20, "uccsd24": uccsd24}[name]()
