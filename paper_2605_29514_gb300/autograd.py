"""torch.autograd wrapper of the adjoint log-likelihood (stn_logprob_grad).

`RecordLogLikelihood.apply(theta, sim, records, shot_offset)` returns
sum_r log P(record r | theta) as a 0-d tensor; its backward multiplies the
incoming gradient by the adjoint gradient the library computed on the GPU
in the same call (the paper's rotation exp(-i theta P), Eq. 4, differentiated
through the stabilizer tensor network of Eq. 7).  theta is the K per-pair
angles, on any device (the library reads a host copy).  Only argument
marshalling happens here.
"""

import numpy as np
import torch


class RecordLogLikelihood(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta, sim, records, shot_offset=0):
        th = theta.detach().to("cpu", torch.float64).numpy()
        logp, grad = sim.logprob_grad(records, th, shot_offset)
        ctx.save_for_backward(torch.as_tensor(grad, dtype=theta.dtype, device=theta.device))
        return torch.as_tensor(float(np.sum(logp)), dtype=theta.dtype, device=theta.device)

    @staticmethod
    def backward(ctx, grad_out):
        (grad,) = ctx.saved_tensors
        return grad_out * grad, None, None, None


def record_log_likelihood(theta, sim, records, shot_offset=0, chunk=None):
    """sum_r log P(record r | theta) over records [n][rec_bytes] of global
    shots shot_offset.., in chunks of at most `chunk` records (default: the
    simulator's max_shots), differentiable in theta."""
    chunk = chunk or sim.max_shots
    total = None
    for lo in range(0, len(records), chunk):
        part = RecordLogLikelihood.apply(theta, sim, records[lo:lo + chunk], shot_offset + lo)
        total = part if total is None else total + part
    return total
