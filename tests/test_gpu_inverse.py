"""Fracture-toughness inversion (Sec. 4.1, Eq. inversion_loss): the
differentiable run (torch.autograd.Function over the C ABI's checkpointed
run and adjoint) gives dL/dGc that matches a central finite difference of
the GPU forward, and L-BFGS on log Gc recovers the toughness that made the
target damage field from a start at two thirds of it, to a relative error
below 1e-3 within a few accepted states (the paper reports three)."""
import math

import numpy as np
import pytest

import pff_synth as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pff():
    import paper_2606_23458_b300 as pff
    return pff


def _setup(pff, prec="fp64"):
    import torch
    from paper_2606_23458_b300 import inverse
    p = S.plate(40, 16)
    mat = S.material(2 * p["h"])
    mesh = pff.Mesh.from_plate(p, precision=prec)
    mesh.set_material(mat, 0.5)
    opts = pff.options(cg_tol=1e-12)
    nsteps = 60
    dstar = inverse.final_damage(torch.tensor(3.0, dtype=torch.float64), mesh, mat, nsteps, 0, opts).detach()
    return mesh, mat, opts, nsteps, dstar


def test_gradient_matches_central_difference(pff):
    """dL/dlog Gc through autograd against a central difference of the loss
    in log Gc (delta = 1e-4), both on the GPU in FP64."""
    import torch
    from paper_2606_23458_b300 import inverse
    mesh, mat, opts, nsteps, dstar = _setup(pff)
    for gc0 in (2.0, 2.5, 3.5):
        lg = torch.tensor(math.log(gc0), dtype=torch.float64, requires_grad=True)
        loss = inverse.mse_loss(inverse.final_damage(torch.exp(lg), mesh, mat, nsteps, 0, opts), dstar)
        loss.backward()
        h = 1e-4
        lp = float(inverse.mse_loss(inverse.final_damage(torch.tensor(math.exp(math.log(gc0) + h), dtype=torch.float64),
                                                         mesh, mat, nsteps, 0, opts), dstar))
        lm = float(inverse.mse_loss(inverse.final_damage(torch.tensor(math.exp(math.log(gc0) - h), dtype=torch.float64),
                                                         mesh, mat, nsteps, 0, opts), dstar))
        fd = (lp - lm) / (2 * h)
        print(f"Gc {gc0}: dL/dlogGc autograd {lg.grad.item():.8e}, central FD {fd:.8e}")
        assert abs(lg.grad.item() - fd) <= 1e-5 * abs(fd), (gc0, lg.grad.item(), fd)
        assert (lg.grad.item() < 0) == (gc0 < 3.0)   # the misfit falls toward Gc* = 3


def test_lbfgs_recovers_gc(pff):
    from paper_2606_23458_b300 import inverse
    mesh, mat, opts, nsteps, dstar = _setup(pff)
    gc, hist = inverse.recover_gc(mesh, mat, nsteps, dstar, 2.0, every=0, opts=opts, max_states=8)
    errs = [abs(g - 3.0) / 3.0 for g in hist["states"]]
    print(f"accepted states {hist['states']}, closure evaluations {len(hist['evals'])}")
    first = next((k + 1 for k, e in enumerate(errs) if e < 1e-3), None)
    assert first is not None and first <= 5, errs
    assert abs(gc - 3.0) / 3.0 < 1e-6, gc


def test_lbfgs_recovers_gc_fp32_checkpointed(pff):
    """The same recovery with FP32 kernels and segment checkpoints (every 20
    steps): the FP32 gradient carries its solver floor, the recovered
    toughness still meets 1e-3."""
    from paper_2606_23458_b300 import inverse
    mesh, mat, opts, nsteps, dstar = _setup(pff, "fp32")
    gc, hist = inverse.recover_gc(mesh, mat, nsteps, dstar, 2.0, every=20,
                                  opts=pff.options(cg_tol=1e-8), max_states=8)
    print(f"fp32 accepted states {hist['states']}")
    assert abs(gc - 3.0) / 3.0 < 1e-3, hist["states"]
