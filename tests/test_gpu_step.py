"""GPU explicit step and damage solve vs the FP64 oracle (Secs. 2.2-2.4):
FP64 fields to 1e-10 entry by entry (each error over max(|o|, 1e-6 max|o|))
with matched CG iteration counts;
FP32-with-FP64-reductions error stated against the FP64 oracle."""
import numpy as np
import pytest

import pff_synth as S
from gpu_common import field_err, max_rel, rel_l2, state_to_torch, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pff():
    import paper_2606_23458_b300 as pff
    return pff


def _random_state(om, rng, scale=1e-6):
    N, Ne = om.N, om.Ne
    return dict(u=rng.normal(size=(N, 2)) * scale, v=rng.normal(size=(N, 2)) * scale * 1e5,
                a=rng.normal(size=(N, 2)) * scale * 1e12,
                d=np.where(om.notch == 1, 1.0, rng.uniform(0, 0.6, N)),
                H=rng.uniform(0, 50, Ne))


@pytest.mark.parametrize("split", ["spectral", "amor", "iso"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_step_explicit(orc, pff, split, prec):
    import torch
    p = S.plate(37, 18, jitter=0.1, seed=3)
    om = orc.Mesh.from_plate(p)
    gm = pff.Mesh.from_plate(p, precision=prec)
    mat = S.material(2 * p["h"], split=split)
    dt = gm.set_material(mat, 0.5)
    rng = np.random.default_rng(11)
    st = _random_state(om, rng)
    gst = state_to_torch(st, gm.dtype)
    n = 3  # t_next = 4 dt lies inside the traction ramp
    gm.step_explicit(gst, (n + 1) * dt, dt)
    torch.cuda.synchronize()
    r = om.run(mat, st, 1, dt, n0=n, damage_on=False)
    if prec == "fp64":
        # entry by entry (floor 1e-6 of each field's largest magnitude)
        for k in ("u", "v", "a", "H"):
            assert field_err(to_np(gst[k]), st[k]) <= 1e-10, (k, field_err(to_np(gst[k]), st[k]))
    else:
        for k in ("u", "v", "a"):
            assert rel_l2(to_np(gst[k]), st[k]) <= 2e-5, k
        assert max_rel(to_np(gst["H"]), st["H"], 1e-3 * st["H"].max()) <= 2e-4


@pytest.mark.parametrize("model", ["AT2", "AT1"])
@pytest.mark.parametrize("loop", ["graph", "host"])
def test_damage_solve_fp64(orc, pff, model, loop):
    import torch
    p = S.plate(60, 24, jitter=0.1, seed=5)
    om = orc.Mesh.from_plate(p)
    gm = pff.Mesh.from_plate(p, precision="fp64")
    mat = S.material(2 * p["h"], model=model)
    gm.set_material(mat, 0.5)
    rng = np.random.default_rng(2)
    Hc = 3 * mat["Gc"] / (16 * mat["l0"])
    H = rng.uniform(0, 4 * Hc, om.Ne) * (rng.uniform(size=om.Ne) < 0.3)
    dprev = np.where(om.notch == 1, 1.0, rng.uniform(0, 0.2, om.N) * (rng.uniform(size=om.N) < 0.2))
    Ht = torch.tensor(H, device="cuda")
    dp = torch.tensor(dprev, device="cuda")
    dout = torch.empty_like(dp)
    opts = pff.options(loop_mode=pff.PFF_LOOP_GRAPH if loop == "graph" else pff.PFF_LOOP_HOST)
    info = gm.damage_solve(Ht, dp, dout, opts)
    assert info["relres"] <= 1e-8
    if model == "AT2":
        d, oinfo, rel, st, _ = om.damage_solve(mat, H, dprev, tol=1e-8, forced=info["iters"])
        assert abs(int(oinfo[1]) - info["iters"]) <= 1   # natural stop within one iteration
        assert field_err(to_np(dout), d) <= 1e-10, field_err(to_np(dout), d)
    else:
        d, oinfo, rel, st, _ = om.damage_solve(mat, H, dprev, tol=1e-8)
        assert st == 0
        assert np.abs(to_np(dout) - d).max() <= 1e-7
        assert np.all(to_np(dout) >= dprev - 1e-15) and np.all(to_np(dout) <= 1)


@pytest.mark.parametrize("model", ["AT2", "AT1"])
def test_damage_solve_fp32(orc, pff, model):
    import torch
    p = S.plate(60, 24, jitter=0.1, seed=5)
    om = orc.Mesh.from_plate(p)
    gm = pff.Mesh.from_plate(p, precision="fp32")
    mat = S.material(2 * p["h"], model=model)
    gm.set_material(mat, 0.5)
    rng = np.random.default_rng(3)
    Hc = 3 * mat["Gc"] / (16 * mat["l0"])
    H = rng.uniform(0, 4 * Hc, om.Ne) * (rng.uniform(size=om.Ne) < 0.3)
    dprev = np.where(om.notch == 1, 1.0, 0.0)
    Ht = torch.tensor(H, device="cuda")
    dp = torch.tensor(dprev, device="cuda", dtype=torch.float32)
    dout = torch.empty_like(dp)
    gm.damage_solve(Ht, dp, dout)
    d, *_ = om.damage_solve(mat, H, dprev, tol=1e-8)
    assert np.abs(to_np(dout) - d).max() <= 1e-4


def test_damage_solve_clamp_and_aliasing(orc, pff):
    import torch
    p = S.plate(30, 12, jitter=0.1, seed=9)
    om = orc.Mesh.from_plate(p)
    gm = pff.Mesh.from_plate(p, precision="fp64")
    mat = S.material(2 * p["h"])
    gm.set_material(mat, 0.5)
    rng = np.random.default_rng(4)
    H = rng.uniform(0, 100, om.Ne)
    dprev = np.where(om.notch == 1, 1.0, rng.uniform(0, 0.5, om.N))
    dp = torch.tensor(dprev, device="cuda")
    info = gm.damage_solve(torch.tensor(H, device="cuda"), dp, dp)  # in place
    d, *_ = om.damage_solve(mat, H, dprev, tol=1e-8, forced=info["iters"])
    assert field_err(to_np(dp), d) <= 1e-10
    assert np.all(to_np(dp) >= dprev)


def test_energies(orc, pff):
    p = S.plate(37, 18, jitter=0.1, seed=3)
    om = orc.Mesh.from_plate(p)
    for model in ("AT2", "AT1"):
        for split in ("spectral", "amor"):
            gm = pff.Mesh.from_plate(p, precision="fp64")
            mat = S.material(2 * p["h"], model=model, split=split)
            gm.set_material(mat, 0.5)
            st = _random_state(om, np.random.default_rng(5))
            e = gm.energies(state_to_torch(st, gm.dtype))
            oe = om.energies(mat, st["u"], st["v"], st["d"])
            assert np.allclose(e, oe, rtol=1e-12)
