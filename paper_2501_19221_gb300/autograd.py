"""torch.autograd.Function over the library's adjoint of the unrolled step.

BSBRelaxedEnergy.apply(dt, kappa, knots, ctx, replicas, steps, seed, ckpt_every)
returns L = mean over replicas of the relaxed energy after `steps` steps
(the QUBO energy identity under x = (1 + s)/2 evaluated at the continuous
state). The forward pass calls veloxq_grad, which runs the checkpointed
forward and the hand-written reverse sweep on the GPU and returns the
gradient w.r.t. dt, kappa and the a(t) knots; backward scales it by the
incoming gradient. dt, kappa: 0-d float64 tensors; knots: 1-d float64 tensor.
"""
from __future__ import annotations

import torch

from . import binding as B


class BSBRelaxedEnergy(torch.autograd.Function):
    @staticmethod
    def forward(fctx, dt, kappa, knots, handle, replicas: int, steps: int, seed: int, ckpt_every: int):
        sched = B.make_schedule(dt=float(dt), kappa=float(kappa), knots=[float(v) for v in knots.tolist()],
                                readout_every=0)
        g = B.veloxq_grad(handle, replicas, steps, sched, seed, ckpt_every)
        fctx.save_for_backward(torch.tensor(g["d_dt"], dtype=torch.float64),
                               torch.tensor(g["d_kappa"], dtype=torch.float64),
                               torch.as_tensor(g["d_knots"], dtype=torch.float64))
        return torch.tensor(g["loss"], dtype=torch.float64)

    @staticmethod
    def backward(fctx, grad_out):
        d_dt, d_kappa, d_knots = fctx.saved_tensors
        return grad_out * d_dt, grad_out * d_kappa, grad_out * d_knots, None, None, None, None, None
