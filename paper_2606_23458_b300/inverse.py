"""Differentiable fracture run and fracture-toughness inversion (Sec. 4.1).

`FractureRun` is a torch.autograd.Function whose forward runs the staggered
explicit solver on the GPU with segment checkpoints (pff_run_ckpt) and
returns the final damage field; its backward calls the hand-written adjoint
(pff_backward: implicit differentiation of every damage solve, Sec. 4.2)
and returns dL/dGc.  `recover_gc` minimises the nodewise MSE of Eq.
(inversion_loss) over log Gc with L-BFGS and a strong-Wolfe line search, as
in Sec. 4.1.  All arithmetic of the method runs in libpff's kernels.
"""
from __future__ import annotations

import math

import torch

from . import Checkpoint, Mesh, options


class FractureRun(torch.autograd.Function):
    @staticmethod
    def forward(ctx, gc, mesh: Mesh, material: dict, nsteps: int, every: int, opts):
        mat = dict(material, Gc=float(gc.item()))
        mesh.set_material(mat, mesh.cfl)
        st = mesh.new_state()
        ckpt = Checkpoint(mesh, nsteps, every)
        mesh.run_ckpt(st, ckpt, opts=opts)
        ctx.mesh, ctx.ckpt, ctx.opts = mesh, ckpt, opts
        return st["d"].clone()

    @staticmethod
    def backward(ctx, grad_d):
        g = ctx.mesh.backward(ctx.ckpt, grad_d.contiguous().to(ctx.mesh.dtype), opts=ctx.opts)
        ctx.ckpt.close()
        return torch.tensor(g, dtype=torch.float64), None, None, None, None, None


def final_damage(gc, mesh, material, nsteps, every=25, opts=None):
    """Final damage field d_T(Gc), differentiable in the scalar tensor gc."""
    return FractureRun.apply(gc, mesh, material, nsteps, every, opts or options())


def mse_loss(d, dstar):
    """Eq. (inversion_loss): (1/N) sum_i (d_T,i - d*_i)^2."""
    return torch.mean((d.double() - dstar.double()) ** 2)


def recover_gc(mesh, material, nsteps, dstar, gc0, every=25, opts=None, max_states=10, history_size=10):
    """L-BFGS with a strong-Wolfe line search on log Gc (Sec. 4.1; the
    logarithm keeps Gc positive), driven one accepted state at a time so
    that each state's Gc is recorded.  Each closure evaluation reruns the
    differentiable forward run and the adjoint.  Stops after max_states
    accepted states, or earlier when the gradient or the step vanishes.
    Returns (Gc, dict(states=[Gc after each accepted state],
    evals=[(Gc, loss, dL/dlogGc) per closure evaluation, line-search probes
    included]))."""
    logg = torch.tensor(math.log(float(gc0)), dtype=torch.float64, requires_grad=True)
    opt = torch.optim.LBFGS([logg], lr=1.0, max_iter=1, history_size=history_size,
                            line_search_fn="strong_wolfe", tolerance_grad=1e-14, tolerance_change=1e-16)
    evals, states = [], []

    def closure():
        opt.zero_grad()
        gc = torch.exp(logg)
        d = final_damage(gc, mesh, material, nsteps, every, opts)
        loss = mse_loss(d, dstar)
        loss.backward()
        evals.append((float(gc.item()), float(loss.item()), float(logg.grad.item())))
        return loss

    for _ in range(max_states):
        before = float(logg.item())
        opt.step(closure)
        states.append(float(torch.exp(logg).item()))
        if float(logg.item()) == before:   # no step taken: converged
            break
    return states[-1], dict(states=states, evals=evals)
