"""Batched plates (one graph launch per step for all plates, per-plate CG
convergence) against single-plate runs and the oracle."""
import numpy as np
import pytest

import pff_synth as S
from gpu_common import rel_l2, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pff():
    import paper_2606_23458_b300 as pff
    return pff


def _plates():
    out = []
    for nx, ny, Gc, t in ((20, 8, 3.0, 1e6), (37, 14, 1.5, 2e6), (26, 10, 4.2, 0.7e6), (1, 2, 2.0, 1e6)):
        p = S.plate(nx, ny, jitter=0.1 if nx > 1 else 0.0, seed=nx, traction=t)
        out.append((p, S.material(2 * p["h"], Gc=Gc)))
    return out


def test_batch_layout(pff):
    plates = _plates()
    b = pff.Batch(plates, precision="fp32")
    assert b.nplates == 4
    for k, (p, mat) in enumerate(plates):
        inf = b.info[k]
        assert inf["node0"] % 256 == 0 and inf["N"] == p["xy"].shape[0]
        assert inf["Ne"] == p["tri"].shape[0]
        if k:
            prev = b.info[k - 1]
            assert inf["node0"] >= prev["node0"] + prev["N"]
            assert inf["elem0"] == prev["elem0"] + prev["Ne"]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_batch_matches_single_plate_runs(pff, prec):
    import torch
    plates = _plates()
    nsteps = 40
    b = pff.Batch(plates, precision=prec)
    st = b.new_state()
    log = torch.zeros(nsteps, len(plates), dtype=torch.int32, device="cuda")
    b.run(st, nsteps, iters_log=log)
    torch.cuda.synchronize()
    tol_u = 1e-9 if prec == "fp64" else 2e-5
    tol_d = 1e-9 if prec == "fp64" else 1e-4
    for k, (p, mat) in enumerate(plates):
        m = pff.Mesh.from_plate(p, precision=prec)
        dt = m.set_material(mat, 0.5)
        assert abs(dt - b.info[k]["dt"]) <= 1e-14 * dt
        s1 = m.new_state()
        l1 = torch.zeros(nsteps, 2, dtype=torch.int32, device="cuda")
        m.run(s1, nsteps, iters_log=l1)
        torch.cuda.synchronize()
        v = b.plate(st, k)
        if np.abs(to_np(s1["u"])).max() > 0:
            assert rel_l2(to_np(v["u"]), to_np(s1["u"])) <= tol_u, k
        assert np.abs(to_np(v["d"]) - to_np(s1["d"])).max() <= tol_d, k
        assert np.abs(log[:, k].cpu().numpy() - l1[:, 0].cpu().numpy()).max() <= 1, k


def test_batch_fp32_vs_oracle(orc, pff):
    import torch
    plates = _plates()[:3]
    nsteps = 60
    b = pff.Batch(plates, precision="fp32")
    st = b.new_state()
    b.run(st, nsteps)
    torch.cuda.synchronize()
    for k, (p, mat) in enumerate(plates):
        om = orc.Mesh.from_plate(p)
        ost = om.new_state()
        om.run(mat, ost, nsteps, b.info[k]["dt"])
        v = b.plate(st, k)
        assert rel_l2(to_np(v["u"]), ost["u"]) <= 1e-4, k
        assert np.abs(to_np(v["d"]) - ost["d"]).max() <= 1e-3, k


@pytest.mark.parametrize("prec,loop", [("fp64", "persistent"), ("fp32", "persistent"), ("fp32", "resident")])
def test_batch_persistent_loop_matches_phases(pff, prec, loop):
    """The per-plate persistent CG (one cooperative launch, a CTA group per
    plate iterating to its own stop), and the per-plate resident CG (the
    single-reduction loop with each CTA's rows in shared memory, in waves
    of plates), against the kernel-per-phase batch loop: the same Jacobi
    PCG per plate, the dot products' partial sums grouped differently (and
    for the resident loop the single-reduction recurrences), so iteration
    counts within one (two) and fields within the rounding of the solve."""
    import torch
    plates = _plates()
    nsteps = 40
    out = {}
    kind = pff.PFF_CG_PERSISTENT if loop == "persistent" else pff.PFF_CG_RESIDENT
    for k in (pff.PFF_CG_PHASES, kind):
        b = pff.Batch(plates, precision=prec)
        st = b.new_state()
        log = torch.zeros(nsteps, len(plates), dtype=torch.int32, device="cuda")
        b.run(st, nsteps, opts=pff.options(cg_kernel=k), iters_log=log)
        torch.cuda.synchronize()
        assert b.tuning()["persistent_ctas"] >= len(plates)
        if loop == "resident":  # the autotuner timed the resident loop: it is available
            assert max(b.tuning()["ms"]["cg_resident"]) > 0
        out[k] = ({n: to_np(v) for n, v in st.items()}, log.cpu().numpy())
    (a, la), (c, lc) = out[pff.PFF_CG_PHASES], out[kind]
    assert np.abs(la - lc).max() <= (1 if loop == "persistent" else 2)
    tol = 1e-9 if prec == "fp64" else 2e-5
    assert rel_l2(c["u"], a["u"]) <= tol
    assert np.abs(c["d"] - a["d"]).max() <= (1e-9 if prec == "fp64" else 1e-4)


def test_batch_autotuner_report(pff):
    import torch
    plates = _plates()
    b = pff.Batch(plates, precision="fp32")
    assert not b.tuning()["tuned"]
    st = b.new_state()
    b.run(st, 3)
    torch.cuda.synchronize()
    t = b.tuning()
    assert t["tuned"] and t["cg"] in ("phases", "persistent", "resident")
    assert 1 <= t["force_U"] <= 4 and 1 <= t["rhs_U"] <= 4 and 1 <= t["cg_U"] <= 4
    assert min(t["ms"]["force"]) > 0 and min(t["ms"]["rhs"]) > 0 and min(t["ms"]["cg_phases"]) > 0
    if t["persistent_ctas"]:
        assert min(t["ms"]["cg_persistent"]) > 0
    assert max(t["ms"]["cg_resident"]) > 0
    best = min(t["ms"]["cg_phases"] + [x for x in t["ms"]["cg_persistent"] + t["ms"]["cg_resident"] if x > 0])
    chosen = (t["ms"]["cg_phases"][t["cg_U"] - 1] if t["cg"] == "phases"
              else t["ms"]["cg_persistent"][t["cg_U"] - 2] if t["cg"] == "persistent"
              else t["ms"]["cg_resident"][t["cg_U"] - 1])
    assert chosen == best
