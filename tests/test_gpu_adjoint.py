"""GPU adjoint (checkpointed recompute + reverse sweep, Sec. 4.2) against the
oracle's discrete adjoint and central finite differences of dL/dGc."""
import numpy as np
import pytest

import pff_synth as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pff():
    import paper_2606_23458_b300 as pff
    return pff


def _problem(nx=20, ny=8):
    p = S.plate(nx, ny)
    mat = S.material(2 * p["h"])
    return p, mat


def _gpu_grad(pff, p, mat, Gc, nsteps, dstar, prec, every, tol, policy="recompute"):
    import torch
    mesh = pff.Mesh.from_plate(p, precision=prec)
    mesh.set_material(dict(mat, Gc=Gc), 0.5)
    opts = pff.options(cg_tol=tol)
    st = mesh.new_state()
    ck = pff.Checkpoint(mesh, nsteps, every, policy)
    mesh.run_ckpt(st, ck, opts=opts)
    d = st["d"].double()
    ds = torch.tensor(dstar, device="cuda")
    loss = float(torch.mean((d - ds) ** 2))
    g = (2.0 * (d - ds) / mesh.N).to(mesh.dtype).contiguous()
    return loss, mesh.backward(ck, g, opts=opts), st


def test_fp64_adjoint_matches_oracle(orc, pff):
    p, mat = _problem()
    om = orc.Mesh.from_plate(p)
    dt = om.stable_dt(mat, 0.5)
    nsteps = 40
    st = om.new_state()
    om.run(dict(mat, Gc=3.0), st, nsteps, dt, tol=1e-13)
    dstar = st["d"].copy()
    for Gc, every in ((2.0, 10), (3.5, 0)):
        L, g, status = om.adjoint_gc(dict(mat, Gc=Gc), nsteps, dt, dstar, tol=1e-13)
        gL, gg, _ = _gpu_grad(pff, p, mat, Gc, nsteps, dstar, "fp64", every, 1e-13)
        assert abs(gL - L) <= 1e-10 * L
        assert abs(gg - g) <= 1e-7 * abs(g), (gg, g)


def test_checkpoint_segmentation_is_exact(orc, pff):
    """Recompute is bit-identical, so the gradient does not depend on the
    checkpoint spacing or on the checkpoint policy (full recompute, or the
    mechanics alone with the damage solutions taped), and a full tape
    (every = 0, no recompute) gives the same gradient; the taped run equals
    a plain run."""
    import torch
    p, mat = _problem()
    nsteps = 30
    dstar = np.zeros(p["xy"].shape[0])
    grads = []
    for every in (1, 7, 30, 0):
        L, g, st = _gpu_grad(pff, p, mat, 2.5, nsteps, dstar, "fp32", every, 1e-8)
        grads.append(g)
    assert grads[0] == grads[1] == grads[2] == grads[3]
    # the damage-tape policy (each step's unclamped solution taped, the
    # mechanics alone recomputed) reverses the same trajectory bit for bit
    for every in (1, 7, 30):
        grads.append(_gpu_grad(pff, p, mat, 2.5, nsteps, dstar, "fp32", every, 1e-8, "damage_tape")[1])
    assert all(g == grads[0] for g in grads), grads
    mesh = pff.Mesh.from_plate(p, precision="fp32")
    mesh.set_material(dict(mat, Gc=2.5), 0.5)
    s2 = mesh.new_state()
    mesh.run(s2, nsteps)
    torch.cuda.synchronize()
    for k in ("u", "v", "a", "d", "H"):
        assert torch.equal(s2[k], st[k]), k


def test_fp32_adjoint_vs_fd_and_oracle(orc, pff):
    p, mat = _problem(40, 16)
    om = orc.Mesh.from_plate(p)
    dt = om.stable_dt(mat, 0.5)
    nsteps = 60
    st = om.new_state()
    om.run(dict(mat, Gc=3.0), st, nsteps, dt, tol=1e-12)
    dstar = st["d"].copy()
    Gc = 2.5
    L, g_or, _ = om.adjoint_gc(dict(mat, Gc=Gc), nsteps, dt, dstar, tol=1e-12)
    _, g32, _ = _gpu_grad(pff, p, mat, Gc, nsteps, dstar, "fp32", 25, 1e-8)
    h = 1e-4 * Gc
    Lp, _, _ = _gpu_grad(pff, p, mat, Gc + h, nsteps, dstar, "fp64", 25, 1e-13)
    Lm, _, _ = _gpu_grad(pff, p, mat, Gc - h, nsteps, dstar, "fp64", 25, 1e-13)
    fd = (Lp - Lm) / (2 * h)
    print(f"dL/dGc: oracle {g_or:.6e}, gpu fp32 {g32:.6e}, gpu fp64 central FD {fd:.6e}")
    assert abs(fd - g_or) <= 1e-4 * abs(g_or)
    assert abs(g32 - g_or) <= 2e-3 * abs(g_or)


def test_autograd_function(pff):
    import torch
    from paper_2606_23458_b300 import inverse
    p, mat = _problem()
    mesh = pff.Mesh.from_plate(p, precision="fp64")
    mesh.set_material(mat, 0.5)
    nsteps = 20
    gc_t = torch.tensor(3.0, dtype=torch.float64)
    dstar = inverse.final_damage(gc_t, mesh, mat, nsteps, every=5).detach()
    gc = torch.tensor(2.0, dtype=torch.float64, requires_grad=True)
    loss = inverse.mse_loss(inverse.final_damage(gc, mesh, mat, nsteps, every=5), dstar)
    loss.backward()
    _, g, _ = _gpu_grad(pff, p, mat, 2.0, nsteps, dstar.cpu().numpy(), "fp64", 5, 1e-8)
    assert abs(gc.grad.item() - g) <= 1e-12 * abs(g)
    assert gc.grad.item() < 0  # Gc below the target: increasing it reduces the misfit


def test_plane_stress_adjoint_matches_oracle(orc, pff):
    """dL/dGc in plane stress with the volumetric-deviatoric split (its
    tangent carries the out-of-plane strain) against the oracle's discrete
    adjoint, FP64."""
    p, mat = _problem()
    mat = dict(mat, split="amor", plane="stress")
    om = orc.Mesh.from_plate(p)
    dt = om.stable_dt(mat, 0.5)
    nsteps = 40
    st = om.new_state()
    om.run(dict(mat, Gc=3.0), st, nsteps, dt, tol=1e-13)
    dstar = st["d"].copy()
    L, g, status = om.adjoint_gc(dict(mat, Gc=2.0), nsteps, dt, dstar, tol=1e-13)
    gL, gg, _ = _gpu_grad(pff, p, mat, 2.0, nsteps, dstar, "fp64", 0, 1e-13)
    assert abs(gL - L) <= 1e-10 * L
    assert abs(gg - g) <= 1e-7 * abs(g), (gg, g)



@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_damage_tape_policy_matches_oracle(orc, pff, prec):
    """The damage-tape checkpoint policy against the oracle's discrete
    adjoint (FP64 1e-7, FP32 2e-3), segments of 9 steps over 40 (a ragged
    last segment)."""
    p, mat = _problem()
    om = orc.Mesh.from_plate(p)
    dt = om.stable_dt(mat, 0.5)
    nsteps = 40
    st = om.new_state()
    om.run(dict(mat, Gc=3.0), st, nsteps, dt, tol=1e-13)
    dstar = st["d"].copy()
    L, g, status = om.adjoint_gc(dict(mat, Gc=2.0), nsteps, dt, dstar, tol=1e-13)
    gL, gg, _ = _gpu_grad(pff, p, mat, 2.0, nsteps, dstar, prec, 9, 1e-13 if prec == "fp64" else 1e-8,
                          "damage_tape")
    tol = 1e-7 if prec == "fp64" else 2e-3
    assert abs(gg - g) <= tol * abs(g), (gg, g)
