"""torch.autograd.Function for the VQE energy with the reverse-mode gradient.

forward(theta) runs one library evaluation with the gradient (Algorithm 1:
lambda = H psi, then psi and lambda are un-rotated together) and keeps
dE/dtheta; backward returns grad_output * dE/dtheta.  theta is a CPU double
tensor of the ansatz's parameters; the energy comes back as a CPU double
scalar tensor.
"""

import numpy as np
import torch


class Energy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta, ansatz, ham, dtype="complex64"):
        from . import vqe_energy_grad
        th = theta.detach().to("cpu", torch.float64).numpy()
        need_grad = bool(theta.requires_grad)
        e, g, _ = vqe_energy_grad(ansatz, ham, th, dtype=dtype, want_grad=need_grad)
        if need_grad:
            ctx.save_for_backward(torch.from_numpy(np.asarray(g)).to(theta.dtype))
        return torch.tensor(e, dtype=theta.dtype)

    @staticmethod
    def backward(ctx, grad_out):
        (g,) = ctx.saved_tensors
        return grad_out * g, None, None, None
