"""Term-group parallelism over ranks (Sec. "Parallel evaluation of an expectation value", Fig. 4).

The paper splits the Pauli strings of the Hamiltonian over processes, each
evaluating its share of the energy, and sums the shares.  Here every rank
holds a replica of the state (it runs the whole rotation sweep on its own
GPU) and evaluates a disjoint, balanced share of the Hamiltonian's
xmask-group passes (``Hamiltonian.shard``, q2_ham_shard).  The only exchange
is one FP64 all-reduce (sum) per evaluation:

* energy only: the rank's share of <psi|H|psi>/<psi|psi> (one double);
* with the gradient: that share and the rank's dE/dtheta.  The reverse sweep
  of Algorithm 1 is linear in lambda = H psi, so each rank runs it with its
  own lambda_r = H_r psi and the gradients add; lambda itself (2^n
  amplitudes) is never exchanged, only the n_params components.

The state sweep is replicated, so this shortens the expectation (and the
H-apply) by the number of ranks, not the sweep.  Host-side logic only: all
device work is the library's.
"""

import numpy as np

from . import vqe_energy_grad


class ShardedEnergy:
    """E(theta) (and dE/dtheta) of `ham` with its passes split over the ranks of `group`.

    `evaluate(shard, theta, want_grad) -> (energy, grad or None)` computes one
    rank's share; by default it is this rank's q2_vqe_energy_grad on its GPU.
    """

    def __init__(self, ansatz, ham, dtype="complex64", group=None, evaluate=None):
        import torch.distributed as dist
        self._dist = dist
        self.group = group
        self.rank = dist.get_rank(group)
        self.world = dist.get_world_size(group)
        self.ansatz = ansatz
        self.dtype = dtype
        self.shard = ham.shard(self.rank, self.world)
        self._evaluate = evaluate or self._on_gpu
        self._ws = None

    def _on_gpu(self, shard, theta, want_grad):
        e, g, self._ws = vqe_energy_grad(self.ansatz, shard, theta, dtype=self.dtype, want_grad=want_grad,
                                         workspace=self._ws)
        return e, g

    def _device(self):
        import torch
        backend = self._dist.get_backend(self.group)
        return torch.device("cuda", torch.cuda.current_device()) if backend == "nccl" else torch.device("cpu")

    def __call__(self, theta, want_grad=True):
        """(E, dE/dtheta or None), the same on every rank."""
        import torch
        e, g = self._evaluate(self.shard, np.asarray(theta, dtype=np.float64), want_grad)
        vals = np.concatenate([[e], np.asarray(g, dtype=np.float64)]) if want_grad else np.array([e])
        buf = torch.from_numpy(vals).to(self._device())
        self._dist.all_reduce(buf, op=self._dist.ReduceOp.SUM, group=self.group)
        out = buf.cpu().numpy()
        return float(out[0]), (out[1:].copy() if want_grad else None)

    def close(self):
        self.shard.close()
