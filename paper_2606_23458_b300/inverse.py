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
    that each state's Gc is recorded; each closure evaluation reruns the
    differentiable forward run and the adjoint.

    Scaling (the minimiser is unchanged): the objective is Eq.
    (inversion_loss) divided by its value L0 at gc0, and the variable is
    z = log(Gc) / sigma with sigma = 2 L0 / |dL/dlog Gc| at gc0 (clamped to
    [1e-3, 1]), the step a quadratic model of the loss predicts.  L-BFGS's
    first step has no curvature information and moves z by one unit, so it
    moves log Gc by sigma; its fixed thresholds (curvature test y.s > 1e-10)
    then do not depend on the MSE's scale, which is tiny on fine meshes
    whose damage lies in thin bands.  The line search may use up to 25
    evaluations per accepted state.  Stops after max_states accepted
    states, or earlier when the step vanishes.
    Returns (Gc, dict(states=[Gc after each accepted state],
    evals=[(Gc, MSE, dMSE/dlogGc) per closure evaluation, line-search probes
    and the initial scaling evaluation included], scale=L0, sigma))."""
    evals = []

    def mse_and_grad(gc_value):
        gc = torch.tensor(float(gc_value), dtype=torch.float64, requires_grad=True)
        mse = mse_loss(final_damage(gc, mesh, material, nsteps, every, opts), dstar)
        mse.backward()
        m, g = float(mse.detach()), float(gc.grad) * float(gc_value)  # d/dlog Gc
        evals.append((float(gc_value), m, g))
        return m, g

    L0, g0 = mse_and_grad(gc0)
    if L0 <= 0.0 or g0 == 0.0:  # already at the target
        return float(gc0), dict(states=[float(gc0)], evals=evals, scale=L0, sigma=1.0)
    sigma = min(1.0, max(1e-3, 2.0 * L0 / abs(g0)))
    z = torch.tensor(math.log(float(gc0)) / sigma, dtype=torch.float64, requires_grad=True)
    opt = torch.optim.LBFGS([z], lr=1.0, max_iter=1, max_eval=25, history_size=history_size,
                            line_search_fn="strong_wolfe", tolerance_grad=1e-14, tolerance_change=1e-16)
    states = []

    def closure():
        opt.zero_grad()
        m, g = mse_and_grad(math.exp(sigma * float(z.detach())))
        z.grad = torch.tensor(g * sigma / L0, dtype=torch.float64)
        return torch.tensor(m / L0, dtype=torch.float64)

    for _ in range(max_states):
        before = float(z.detach())
        opt.step(closure)
        states.append(math.exp(sigma * float(z.detach())))
        if float(z.detach()) == before:   # no step taken: converged
            break
    return states[-1], dict(states=states, evals=evals, scale=L0, sigma=sigma)
