"""Term-group sharding of the energy and gradient across ranks, on CPU (gloo, world size 2).

Each rank builds the Hamiltonian handle, takes its shard (q2_ham_shard, the
library's host-side pass assignment) and runs paper_2208_10978_gb300.sharding
.ShardedEnergy, whose per-rank evaluation is replaced here by the C oracle on
the shard's terms (q2_ham_shard_terms); the all-reduce is real.  Checks:

* the shards' term sets are disjoint and together are all terms, for both dtypes;
* the all-reduced energy and dE/dtheta equal the oracle's unsharded ones
  (energy to 1e-12, gradient to 1e-11: the same FP64 sums in another order);
* the energy-only call returns the same energy and no gradient.
"""

import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _workload():
    from synth.workloads import uccsd_energy
    return uccsd_energy(10, 4, seed=7)


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import paper_2208_10978_gb300 as q2
    from paper_2208_10978_gb300.sharding import ShardedEnergy
    from oracle import c_oracle, statevector as sv
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w = _workload()
        a = w.ansatz
        ans = q2.Ansatz.from_uccsd(a)
        ham = q2.Hamiltonian(w.n, w.ham.x, w.ham.z, w.ham.c)

        def oracle_share(shard, theta, want_grad):
            idx = shard.shard_terms("complex128")
            e, gphi = c_oracle.energy_and_gradient(w.n, w.n_elec, a.x, a.z, a.angles(theta), w.ham.x[idx],
                                                   w.ham.z[idx], w.ham.c[idx])
            return e, (sv.fold_to_theta(gphi, a.param, a.coef, a.n_params) if want_grad else None)

        se = ShardedEnergy(ans, ham, dtype="complex128", evaluate=oracle_share)
        theta = np.random.default_rng(5).normal(0, 0.3, size=a.n_params)
        e, g = se(theta, want_grad=True)
        e0, g0 = se(theta, want_grad=False)
        terms = {d: se.shard.shard_terms(d).tolist() for d in ("complex128", "complex64")}
        out[rank] = (e, g.tolist(), e0, g0, terms, theta.tolist())
        dist.barrier()
        se.close()
    finally:
        dist.destroy_process_group()


def test_sharded_energy_and_gradient_match_unsharded_oracle():
    sys.path.insert(0, ROOT)
    from oracle import c_oracle, statevector as sv
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    w = _workload()
    a = w.ansatz
    theta = np.array(res[0][5])
    e_ref, gphi = c_oracle.energy_and_gradient(w.n, w.n_elec, a.x, a.z, a.angles(theta), w.ham.x, w.ham.z, w.ham.c)
    g_ref = sv.fold_to_theta(gphi, a.param, a.coef, a.n_params)
    for d in ("complex128", "complex64"):
        sets = [set(res[r][4][d]) for r in range(world)]
        assert all(len(s) > 0 for s in sets)
        assert not (sets[0] & sets[1])
        assert sets[0] | sets[1] == set(range(w.ham.n_terms))
    for r in range(world):
        e, g, e0, g0, _, _ = res[r]
        assert abs(e - e_ref) < 1e-12
        assert np.max(np.abs(np.array(g) - g_ref)) < 1e-11
        assert abs(e0 - e_ref) < 1e-12 and g0 is None
