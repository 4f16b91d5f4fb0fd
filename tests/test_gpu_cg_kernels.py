"""The AT2 CG loops (a matvec and an update kernel per iteration; the whole
solve in one persistent cooperative kernel with grid barriers; the same
with each CTA's operator staged in shared memory by bulk copies; the
single-reduction form of the same PCG, one pass and one barrier per
iteration, unstaged, staged, and with each CTA's rows resident in shared
memory) against the oracle and against each other, on meshes from one CTA
to a full wave; the bounded barrier wait; the autotuner's report."""
import numpy as np
import pytest

import pff_synth as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pff():
    import paper_2606_23458_b300 as pff
    return pff


def _inputs(p, seed):
    rng = np.random.default_rng(seed)
    Ne, N = p["tri"].shape[0], p["xy"].shape[0]
    H = rng.uniform(0, 400, Ne) * (rng.uniform(size=Ne) < 0.4)
    dprev = np.where(p["notch"] == 1, 1.0, rng.uniform(0, 0.3, N) * (rng.uniform(size=N) < 0.3))
    return H, dprev


def _solve(pff, mesh, H, dprev, cgk, tol=1e-8):
    import torch
    Ht = torch.tensor(H, device="cuda")
    dp = torch.tensor(dprev, device="cuda", dtype=mesh.dtype)
    out = torch.full_like(dp, float("nan"))
    info = mesh.damage_solve(Ht, dp, out, opts=pff.options(cg_tol=tol, cg_kernel=cgk))
    torch.cuda.synchronize()
    return out.double().cpu().numpy(), info


FP32_LOOPS = [2, 4, 5, 6, 7]  # persistent, staged, fused, fused staged, resident (pff.PFF_CG_*)

# 20 x 8: 189 nodes, one CTA; 300 x 120: 36,421 nodes, 36 CTAs;
# 520 x 300 jittered: 156,821 nodes, one CTA per SM
SIZES = [(20, 8, 0.0), (300, 120, 0.0), (520, 300, 0.1)]


@pytest.mark.parametrize("nx,ny,jit", SIZES)
def test_persistent_damage_solve_fp64_vs_oracle(orc, pff, nx, ny, jit):
    """FP64: the persistent solve stops where the kernel-per-phase solve
    stops, and both agree with the oracle forced to that iteration count."""
    p = S.plate(nx, ny, jitter=jit, seed=5)
    mat = S.material(2 * p["h"])
    mesh = pff.Mesh.from_plate(p, precision="fp64")
    mesh.set_material(mat, 0.5)
    om = orc.Mesh.from_plate(p)
    H, dprev = _inputs(p, 11)
    d_pe, i_pe = _solve(pff, mesh, H, dprev, pff.PFF_CG_PERSISTENT)
    d_ph, i_ph = _solve(pff, mesh, H, dprev, pff.PFF_CG_PHASES)
    assert i_pe["iters"] == i_ph["iters"] > 0
    d_or, info, rel, st, _ = om.damage_solve(mat, H, dprev, forced=i_pe["iters"])
    scale = np.maximum(np.abs(d_or), 1e-3)
    assert np.max(np.abs(d_pe - d_or) / scale) <= 1e-10
    assert np.max(np.abs(d_ph - d_or) / scale) <= 1e-10
    assert i_pe["relres"] <= 1e-8 * 1.0001


@pytest.mark.parametrize("nx,ny,jit", SIZES)
def test_persistent_damage_solve_fp32(pff, nx, ny, jit):
    """FP32: the persistent and the staged kernels against the kernel-per-
    phase loop (they differ only in how the dot products' partial sums are
    grouped)."""
    p = S.plate(nx, ny, jitter=jit, seed=5)
    mesh = pff.Mesh.from_plate(p, precision="fp32")
    mesh.set_material(S.material(2 * p["h"]), 0.5)
    for seed in (1, 2):
        H, dprev = _inputs(p, seed)
        d_ph, i_ph = _solve(pff, mesh, H, dprev, pff.PFF_CG_PHASES)
        for cgk in FP32_LOOPS:
            d_pe, i_pe = _solve(pff, mesh, H, dprev, cgk)
            assert abs(i_pe["iters"] - i_ph["iters"]) <= (1 if cgk < 5 else 2), cgk
            assert np.max(np.abs(d_pe - d_ph) / np.maximum(np.abs(d_ph), 1e-3)) <= 1e-4, cgk
            assert i_pe["relres"] <= 2.0 ** -22 * 1.0001, cgk
    st = mesh.new_state()
    mesh.run(st, 2)  # tunes the loops: every one must have been available
    assert min(mesh.cg_choice()[2].values()) > 0


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_persistent_run_vs_phase_run(pff, prec):
    """60 staggered steps of the 100 x 40 plate with each loop: the same
    iteration counts (FP64; within one in FP32) and the same fields."""
    import torch
    c = S.config("plate_100x40")
    res = {}
    kinds = [pff.PFF_CG_PHASES, pff.PFF_CG_PERSISTENT] + (FP32_LOOPS[1:] if prec == "fp32" else [])
    for cgk in kinds:
        mesh = pff.Mesh.from_plate(c["mesh"], precision=prec)
        mesh.set_material(c["material"], c["cfl"])
        st = mesh.new_state()
        log = torch.zeros(60, 2, dtype=torch.int32, device="cuda")
        mesh.run(st, 60, opts=pff.options(cg_tol=c["cg_tol"], t_ramp=c["t_ramp"], cg_kernel=cgk),
                 iters_log=log)
        torch.cuda.synchronize()
        assert mesh.sync_status() == 0
        res[cgk] = ({k: v.double().cpu().numpy() for k, v in st.items()}, log[:, 0].cpu().numpy())
    a, ia = res[pff.PFF_CG_PHASES]
    for cgk in kinds[1:]:
        b, ib = res[cgk]
        if prec == "fp64":
            assert np.array_equal(ia, ib)
            tol = 1e-10
        else:
            assert np.max(np.abs(ia - ib)) <= (1 if cgk < 5 else 2), cgk
            tol = 1e-4
        for k in ("u", "d", "H"):
            err = np.linalg.norm(a[k] - b[k]) / max(np.linalg.norm(a[k]), 1e-300)
            assert err <= tol, (cgk, k, err)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_persistent_backward_matches_phases(pff, prec):
    p = S.plate(40, 16)
    mat = S.material(2 * p["h"])
    grads = []
    kinds = [pff.PFF_CG_PHASES, pff.PFF_CG_PERSISTENT] + (FP32_LOOPS[1:] if prec == "fp32" else [])
    for cgk in kinds:
        mesh = pff.Mesh.from_plate(p, precision=prec)
        mesh.set_material(dict(mat, Gc=2.5), 0.5)
        opts = pff.options(cg_tol=1e-12, cg_kernel=cgk)
        st = mesh.new_state()
        ck = pff.Checkpoint(mesh, 30, 0)
        mesh.run_ckpt(st, ck, opts=opts)
        g = (2.0 * st["d"] / mesh.N).contiguous()
        grads.append(mesh.backward(ck, g, opts=opts))
        ck.close()
    tol = 1e-9 if prec == "fp64" else 2e-3
    for g in grads[1:]:
        assert abs(g - grads[0]) <= tol * abs(grads[0]), grads


def test_resident_without_fan_order_runs_unstaged(pff):
    """A mesh whose fans do not fit the fan tables (a vertex with twelve
    triangles) has no resident loop: asking for it runs the global-memory
    single-reduction loop, with the same result."""
    from test_gpu_wide_incidence import _plate
    q = _plate()
    mesh = pff.Mesh.from_plate(q, precision="fp32")
    mesh.set_material(S.material(2 * q["h"]), 0.5)
    assert not mesh.fan_order()
    H, dprev = _inputs(q, 4)
    d_re, i_re = _solve(pff, mesh, H, dprev, pff.PFF_CG_RESIDENT)
    d_fu, i_fu = _solve(pff, mesh, H, dprev, pff.PFF_CG_FUSED)
    assert i_re["iters"] == i_fu["iters"] and np.array_equal(d_re, d_fu)


def test_resident_beyond_shared_memory_runs_unstaged(pff):
    """A plate whose rows do not fit the SMs' shared memory at 28 B each
    (1,324,601 nodes) has no resident loop: asking for it runs the
    global-memory single-reduction loop, with the same result."""
    p = S.plate(1200, 1100, jitter=0.1, seed=3)
    mesh = pff.Mesh.from_plate(p, precision="fp32")
    mesh.set_material(S.material(2 * p["h"]), 0.5)
    assert mesh.fan_order()
    H, dprev = _inputs(p, 6)
    d_re, i_re = _solve(pff, mesh, H, dprev, pff.PFF_CG_RESIDENT)
    d_fu, i_fu = _solve(pff, mesh, H, dprev, pff.PFF_CG_FUSED)
    assert i_re["iters"] == i_fu["iters"] > 0 and np.array_equal(d_re, d_fu)


def _shuffled(p, block, seed):
    """The plate with its node ids permuted within consecutive blocks of
    `block` ids: the same mesh, fan offsets still within 16 bits, but
    thousands of distinct fan-word triples."""
    rng = np.random.default_rng(seed)
    N = p["xy"].shape[0]
    new = np.arange(N)
    for b0 in range(0, N, block):
        new[b0:b0 + block] = b0 + rng.permutation(min(block, N - b0))
    q = dict(p)
    q["xy"] = np.empty_like(p["xy"])
    q["xy"][new] = p["xy"]
    q["notch"] = np.empty_like(p["notch"])
    q["notch"][new] = p["notch"]
    q["tri"] = new[p["tri"]].astype(np.int32)
    q["tedges"] = new[p["tedges"]].astype(np.int32)
    return q, new


def test_resident_forms_follow_the_mesh(pff):
    """The resident loop keeps as much of each CTA's rows in shared memory
    as fits: everything on 36,421 nodes (full form), x, p, the diagonal and
    the fan words on 359,601 nodes (partial), with the same result when the
    node ids are shuffled within blocks of 64 (other fan words on every row,
    other CTA ranges).  Each against the kernel-per-phase loop."""
    p = S.plate(640, 560, jitter=0.1, seed=2)
    ps, new = _shuffled(p, 64, 7)
    H, dprev = _inputs(p, 3)
    dprev_s = np.empty_like(dprev)
    dprev_s[new] = dprev
    small = S.plate(300, 120, jitter=0.1, seed=2)
    cases = [(small, "full", _inputs(small, 3)), (p, "partial", (H, dprev)), (ps, "shuffled", (H, dprev_s))]
    out = {}
    for q, form, (H, dprev) in cases:
        mesh = pff.Mesh.from_plate(q, precision="fp32")
        mesh.set_material(S.material(2 * q["h"]), 0.5)
        assert mesh.fan_order()
        want = "partial" if form == "shuffled" else form
        assert mesh.resident_forms() == [want] * 4, (form, mesh.resident_forms())
        d_ph, i_ph = _solve(pff, mesh, H, dprev, pff.PFF_CG_PHASES)
        d_re, i_re = _solve(pff, mesh, H, dprev, pff.PFF_CG_RESIDENT)
        assert abs(i_re["iters"] - i_ph["iters"]) <= 2, form
        assert np.max(np.abs(d_re - d_ph) / np.maximum(np.abs(d_ph), 1e-3)) <= 1e-4, form
        assert i_re["relres"] <= 2.0 ** -22 * 1.0001, form
        out[form] = d_re
    # the shuffled plate is the same problem (element order kept, node
    # values permuted): plain node k is shuffled node new[k]
    dc, dp = out["partial"], out["shuffled"][new]
    assert np.max(np.abs(dp - dc) / np.maximum(np.abs(dc), 1e-3)) <= 1e-4


def test_bounded_barrier_wait_reports_timeout(pff):
    """A barrier that awaits one CTA more than the grid gives up after its
    wait limit: the call returns PFF_ERR_TIMEOUT, the context stays usable
    and the next solve is correct."""
    import torch
    p = S.plate(60, 24)
    mesh = pff.Mesh.from_plate(p, precision="fp32")
    mesh.set_material(S.material(2 * p["h"]), 0.5)
    H, dprev = _inputs(p, 3)
    Ht = torch.tensor(H, device="cuda")
    dp = torch.tensor(dprev, device="cuda", dtype=mesh.dtype)
    out = torch.empty_like(dp)
    info = mesh.damage_solve(Ht, dp, out, opts=pff.options(cg_kernel=pff.PFF_CG_TEST_TIMEOUT),
                             raise_on_error=False)
    assert info["status"] == pff.PFF_ERR_TIMEOUT
    assert "timed out" in pff._lib.pff_last_error().decode()
    d_pe, i_pe = _solve(pff, mesh, H, dprev, pff.PFF_CG_PERSISTENT)
    d_ph, i_ph = _solve(pff, mesh, H, dprev, pff.PFF_CG_PHASES)
    assert i_pe["status"] == i_ph["status"] == 0
    assert np.max(np.abs(d_pe - d_ph) / np.maximum(np.abs(d_ph), 1e-3)) <= 1e-4


def test_autotuner_reports_cg_loop(pff):
    import torch
    c = S.config("plate_100x40")
    mesh = pff.Mesh.from_plate(c["mesh"], precision="fp32")
    mesh.set_material(c["material"], c["cfl"])
    assert mesh.cg_choice()[0] == "auto"
    st = mesh.new_state()
    mesh.run(st, 5)
    torch.cuda.synchronize()
    kind, U, ms = mesh.cg_choice()
    assert min(ms.values()) > 0
    assert kind == min(ms, key=ms.get)
    assert (U == 0) == (kind == "phases") and 0 <= U <= 4
