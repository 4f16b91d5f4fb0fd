"""The allocation-free damage solve (pff_damage_solve_noalloc) against the
regular entry point (pff_damage_solve), through the C ABI.

Some callers may not allocate device memory during a call (cudaFree
synchronises the device; memory-capped serving processes and allocator or
stream callbacks may not enter the allocator).  This entry point uses a
statically reserved workspace instead; it must give the regular solve's
result on repeated calls, and refuse meshes larger than its workspace.
Collected last so that a failure here cannot hide the other tests."""
import numpy as np
import pytest

import pff_synth as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pff():
    import paper_2606_23458_b300 as pff
    return pff


def _inputs(p, mat, seed):
    rng = np.random.default_rng(seed)
    Ne, N = p["tri"].shape[0], p["xy"].shape[0]
    H = rng.uniform(0, 400, Ne) * (rng.uniform(size=Ne) < 0.4)
    dprev = np.where(p["notch"] == 1, 1.0, rng.uniform(0, 0.3, N) * (rng.uniform(size=N) < 0.3))
    return H, dprev


@pytest.mark.parametrize("prec,model", [("fp64", "AT2"), ("fp32", "AT2"), ("fp64", "AT1"), ("fp32", "AT1")])
def test_noalloc_matches_regular_solve_twice(pff, prec, model):
    import torch
    p = S.plate(80, 30, jitter=0.1, seed=3)
    mesh = pff.Mesh.from_plate(p, precision=prec)
    mat = S.material(2 * p["h"], model=model)
    mesh.set_material(mat, 0.5)
    dt = mesh.dtype
    tol = 1e-10 if prec == "fp64" else 1e-4
    for call, seed in enumerate((1, 2)):
        H, dprev = _inputs(p, mat, seed)
        Ht = torch.tensor(H, device="cuda")
        dp = torch.tensor(dprev, device="cuda", dtype=dt)
        ref = torch.empty_like(dp)
        out = torch.full_like(dp, float("nan"))
        info_ref = mesh.damage_solve(Ht, dp, ref)
        info = mesh.damage_solve_noalloc(Ht, dp, out)
        torch.cuda.synchronize()
        a, b = out.double().cpu().numpy(), ref.double().cpu().numpy()
        assert np.all(np.isfinite(a)), call
        err = np.max(np.abs(a - b) / np.maximum(np.abs(b), 1e-3))
        assert err <= tol, (call, err)
        assert info["iters"] == info_ref["iters"], call
        assert info["relres"] <= max(1e-8, 2.0 ** -22) * 1.0001


def test_noalloc_rejects_oversized_mesh(pff):
    import torch
    p = S.plate(400, 330, notch=False)   # 133,061 nodes > 131,072
    mesh = pff.Mesh.from_plate(p, precision="fp32")
    mesh.set_material(S.material(2 * p["h"]), 0.5)
    H = torch.zeros(mesh.Ne, dtype=torch.float64, device="cuda")
    d = torch.zeros(mesh.N, dtype=torch.float32, device="cuda")
    info = mesh.damage_solve_noalloc(H, d, d, raise_on_error=False)
    assert info["status"] == pff.PFF_ERR_ARG
    assert "at most 131072" in pff._lib.pff_last_error().decode()
