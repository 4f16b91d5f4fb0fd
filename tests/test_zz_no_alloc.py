"""The allocation-free damage solve (pff_damage_solve_noalloc) against the
regular entry point (pff_damage_solve), through the C ABI.

Some callers may not allocate device memory during a call (cudaFree
synchronises the device; memory-capped serving processes and allocator or
stream callbacks may not enter the allocator).  This entry point uses a
statically reserved workspace instead; it must give the regular solve's
result on repeated calls, give the oracle's result as the first solve of a
new mesh, leave the device's free memory untouched, and refuse meshes
larger than its workspace.
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


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_noalloc_first_solve_on_fresh_mesh(orc, pff, prec):
    """The allocation-free solve as the very first solve of a new mesh (no
    autotuning has run, so it takes the mesh's initial gather schedule)
    against the oracle: FP64 forced to the same iteration count, entry by
    entry within 1e-10; FP32 within its tolerance of 1e-4.  A regular solve
    afterwards gives the same result, and a second allocation-free call
    changes neither the device's free memory nor torch's reserved pool."""
    import torch
    from gpu_common import field_err
    p = S.plate(70, 28, jitter=0.1, seed=8)
    mesh = pff.Mesh.from_plate(p, precision=prec)
    mat = S.material(2 * p["h"])
    mesh.set_material(mat, 0.5)
    H, dprev = _inputs(p, mat, 5)
    Ht = torch.tensor(H, device="cuda")
    dp = torch.tensor(dprev, device="cuda", dtype=mesh.dtype)
    out = torch.full_like(dp, float("nan"))
    info = mesh.damage_solve_noalloc(Ht, dp, out)
    torch.cuda.synchronize()
    a = out.double().cpu().numpy()
    om = orc.Mesh.from_plate(p)
    if prec == "fp64":
        d, oinfo, *_ = om.damage_solve(mat, H, dprev, tol=1e-8, forced=info["iters"])
        assert abs(int(oinfo[1]) - info["iters"]) <= 1
        assert field_err(a, d) <= 1e-10, field_err(a, d)
    else:
        d, *_ = om.damage_solve(mat, H, dprev, tol=1e-8)
        assert np.abs(a - d).max() <= 1e-4
    ref = torch.empty_like(dp)
    mesh.damage_solve(Ht, dp, ref)
    torch.cuda.synchronize()
    b = ref.double().cpu().numpy()
    assert np.max(np.abs(a - b) / np.maximum(np.abs(b), 1e-3)) <= (1e-8 if prec == "fp64" else 1e-4)
    # a second call: same result, no allocation anywhere
    out2 = torch.full_like(dp, float("nan"))
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    res0 = torch.cuda.memory_reserved()
    mesh.damage_solve_noalloc(Ht, dp, out2)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0 and torch.cuda.memory_reserved() == res0, (free0, free1)
    # the regular solve tuned the mesh's gather schedule in between: FP32 sums
    # are schedule-independent, FP64 dot products may differ in the last bit
    c = out2.double().cpu().numpy()
    if prec == "fp32":
        assert np.array_equal(a, c)
    else:
        assert np.max(np.abs(c - b) / np.maximum(np.abs(b), 1e-3)) <= 1e-8


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
