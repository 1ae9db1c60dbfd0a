"""VQE outer loop: minimise E(theta) with the library's energy and adjoint gradient.

The paper's workflow (Fig. 1b, Sec. "Variational quantum circuit ansatz")
alternates circuit evaluations with a classical optimiser.  Here each
evaluation is one q2_vqe_energy_grad call on resident tables (Hamiltonian and
ansatz handles, one reused workspace), so an iteration costs one forward
sweep, one H-apply and one reverse sweep; the optimiser is scipy's L-BFGS-B
on the host.
"""

from dataclasses import dataclass, field

import numpy as np

from . import vqe_energy_grad


@dataclass
class VqeResult:
    theta: np.ndarray
    energy: float
    grad_norm: float
    evaluations: int
    converged: bool
    history: list = field(default_factory=list)   # energy after every evaluation


def minimize(ansatz, ham, theta0, dtype="complex64", maxiter=200, gtol=1e-6):
    """L-BFGS-B from theta0; returns the best parameters and their energy."""
    from scipy.optimize import minimize as _minimize

    state = {"ws": None, "n": 0}
    hist = []

    def fun(theta):
        e, g, state["ws"] = vqe_energy_grad(ansatz, ham, theta, dtype=dtype, want_grad=True,
                                            workspace=state["ws"])
        state["n"] += 1
        hist.append(e)
        return e, np.asarray(g, dtype=np.float64)

    res = _minimize(fun, np.asarray(theta0, dtype=np.float64), jac=True, method="L-BFGS-B",
                    options={"maxiter": maxiter, "gtol": gtol})
    e, g = fun(res.x)
    return VqeResult(theta=res.x, energy=float(e), grad_norm=float(np.linalg.norm(g)),
                     evaluations=state["n"], converged=bool(res.success), history=hist)
