"""Full staggered runs on the GPU vs the oracle on the 100 x 40 plate
(4,141 nodes, 8,000 triangles, glass, AT2, 200 steps)."""
import numpy as np
import pytest

import pff_synth as S
from gpu_common import merge_worst, rel_l2, state_errs, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pff():
    import paper_2606_23458_b300 as pff
    return pff


def _setup(pff, orc, name="plate_100x40", split="spectral", model="AT2", prec="fp64"):
    c = S.config(name, split=split, model=model)
    om = orc.Mesh.from_plate(c["mesh"])
    gm = pff.Mesh.from_plate(c["mesh"], precision=prec)
    dt = gm.set_material(c["material"], c["cfl"])
    return c, om, gm, dt


@pytest.mark.parametrize("split", ["spectral", "amor"])
def test_fp64_per_step_parity(orc, pff, split):
    """FP64 fields agree with the oracle to 1e-10 after every step, entry by
    entry (|g - o| / max(|o|, floor), floors per field from gpu_common:
    1e-4, 1e-3, 1e-2 of the field's maximum for u, v, a, 1e-6 for d and H);
    the oracle is forced to the GPU's CG iteration count, whose own stop
    decision must be within one iteration."""
    import torch
    c, om, gm, dt = _setup(pff, orc, split=split)
    mat = c["material"]
    nsteps = 200
    gst = gm.new_state()
    ost = om.new_state()
    log = torch.zeros(nsteps, 2, dtype=torch.int32, device="cuda")
    worst = {}
    for n in range(nsteps):
        gm.run(gst, 1, step0=n, iters_log=log[n:n + 1])
        torch.cuda.synchronize()
        it = int(log[n, 0])
        r = om.run(mat, ost, 1, dt, n0=n, forced=[it])
        merge_worst(worst, state_errs(gst, ost))
        assert max(worst.values()) <= 1e-10, (n, worst)
    print(f"fp64 {split} 200 steps, element-wise worst per field: {worst}")
    assert gm.sync_status() == 0


def test_fp64_natural_stop_matches(orc, pff):
    import torch
    c, om, gm, dt = _setup(pff, orc)
    nsteps = 200
    gst = gm.new_state()
    log = torch.zeros(nsteps, 2, dtype=torch.int32, device="cuda")
    gm.run(gst, nsteps, iters_log=log)
    ost = om.new_state()
    r = om.run(c["material"], ost, nsteps, dt)
    gi = log[:, 0].cpu().numpy()
    assert np.abs(gi - r["iters"][:, 0]).max() <= 1
    assert rel_l2(to_np(gst["u"]), ost["u"]) <= 1e-8
    assert np.abs(to_np(gst["d"]) - ost["d"]).max() <= 1e-7


@pytest.mark.parametrize("split", ["spectral", "amor"])
def test_fp32_error_vs_fp64_oracle(orc, pff, split):
    """FP32 kernels with FP64 reductions over the 200-step window: relative
    L2 error of u <= 1e-4 and max |d - d_oracle| <= 1e-3."""
    import torch
    c, om, gm, dt = _setup(pff, orc, split=split, prec="fp32")
    nsteps = 200
    gst = gm.new_state()
    gm.run(gst, nsteps)
    torch.cuda.synchronize()
    ost = om.new_state()
    om.run(c["material"], ost, nsteps, dt)
    eu = rel_l2(to_np(gst["u"]), ost["u"])
    ed = np.abs(to_np(gst["d"]) - ost["d"]).max()
    print(f"fp32 {split}: u rel L2 {eu:.3e}, max|dd| {ed:.3e}")
    assert eu <= 1e-4 and ed <= 1e-3


def test_at1_run(orc, pff):
    import torch
    c, om, gm, dt = _setup(pff, orc, split="amor", model="AT1")
    nsteps = 100
    gst = gm.new_state()
    gm.run(gst, nsteps)
    torch.cuda.synchronize()
    assert gm.sync_status() == 0
    ost = om.new_state()
    r = om.run(c["material"], ost, nsteps, dt)
    assert r["status"] == 0
    assert rel_l2(to_np(gst["u"]), ost["u"]) <= 1e-7
    assert np.abs(to_np(gst["d"]) - ost["d"]).max() <= 1e-6


def test_energy_log_and_determinism(orc, pff):
    import torch
    c, om, gm, dt = _setup(pff, orc)
    nsteps = 60
    runs = []
    for rep in range(2):
        gst = gm.new_state()
        en = torch.full((nsteps, 4), float("nan"), dtype=torch.float64, device="cuda")
        gm.run(gst, nsteps, opts=pff.options(energy_every=10), energy_log=en)
        torch.cuda.synchronize()
        runs.append((gst, en.cpu().numpy()))
    for k in ("u", "v", "a", "d", "H"):
        assert torch.equal(runs[0][0][k], runs[1][0][k]), k
    ost = om.new_state()
    r = om.run(c["material"], ost, nsteps, dt, energy_every=10)
    rows = np.arange(9, nsteps, 10)
    assert np.allclose(runs[0][1][rows], r["energies"][rows], rtol=1e-8)
    assert np.all(np.isnan(runs[0][1][0]))


@pytest.mark.parametrize("prec,mech_only", [("fp32", False), ("fp64", True)])
def test_schedules_bit_identical(orc, pff, prec, mech_only):
    """Every gather schedule (entry-parallel / element pass + node gather,
    node-centric with 1..4 gathers in flight) sums each row in the same
    order: identical bits after 30 steps.  FP32 includes the damage solve
    (its dot products accumulate in double-word arithmetic, which rounds
    the same in any order here); the FP64 dot products are plain FP64 sums
    in schedule order, so FP64 is compared on the mechanics, and the full
    FP64 step to within a few ulp of the damage."""
    import torch
    outs, full = [], []
    for var in range(1, 6):
        c, om, gm, dt = _setup(pff, orc, prec=prec)
        st = gm.new_state()
        gm.run(st, 30, opts=pff.options(variant=var, damage_every=1000 if mech_only else 0))
        torch.cuda.synchronize()
        outs.append(st)
        if mech_only:
            s2 = gm.new_state()
            gm.run(s2, 30, opts=pff.options(variant=var))
            torch.cuda.synchronize()
            full.append(s2)
    for st in outs[1:]:
        for k in ("u", "v", "a", "d", "H"):
            assert torch.equal(st[k], outs[0][k]), k
    for st in full[1:]:
        assert float((st["d"] - full[0]["d"]).abs().max()) <= 1e-14
        assert rel_l2(to_np(st["u"]), to_np(full[0]["u"])) <= 1e-12


def test_autotuner_choice_reported(orc, pff):
    import torch
    c, om, gm, dt = _setup(pff, orc, prec="fp32")
    st = gm.new_state()
    gm.run(st, 2)
    torch.cuda.synchronize()
    var, ms = gm.schedule()
    for k in ("force", "rhs", "matvec"):
        assert 1 <= var[k] <= 5
        assert ms[k][var[k] - 1] == min(ms[k]) > 0


@pytest.mark.parametrize("n_sub", [2, 3])
def test_subcycled_run_per_step_parity(orc, pff, n_sub):
    """Damage subcycling (Sec. 2.4): FP64 fields within 1e-10 of the oracle,
    entry by entry, after every step of a 60-step window (oracle forced to
    the GPU's iteration counts); skipped steps log zero iterations and keep
    d."""
    import torch
    c, om, gm, dt = _setup(pff, orc)
    mat = c["material"]
    nsteps = 60
    opts = pff.options(damage_every=n_sub)
    gst = gm.new_state()
    ost = om.new_state()
    log = torch.zeros(nsteps, 2, dtype=torch.int32, device="cuda")
    worst = {}
    for n in range(nsteps):
        d_before = to_np(gst["d"]).copy()
        gm.run(gst, 1, step0=n, opts=opts, iters_log=log[n:n + 1])
        torch.cuda.synchronize()
        it = int(log[n, 0])
        om.run(mat, ost, 1, dt, n0=n, forced=[it], n_sub=n_sub)
        if (n + 1) % n_sub:
            assert it == 0 and np.array_equal(to_np(gst["d"]), d_before), n
        merge_worst(worst, state_errs(gst, ost))
        assert max(worst.values()) <= 1e-10, (n, worst)
    assert gm.sync_status() == 0


def test_subcycled_fp32_run_in_one_call(orc, pff):
    """FP32, one pff_run call of 120 steps at N_sub = N_max of the material
    against the FP64 oracle; a whole-run call gives the same fields as the
    same steps split over several calls."""
    import torch
    c, om, gm, dt = _setup(pff, orc, prec="fp32")
    mat = c["material"]
    n_sub = max(2, pff.subcycling_limit(mat)[1])
    opts = pff.options(damage_every=n_sub)
    a = gm.new_state()
    la = torch.zeros(120, 2, dtype=torch.int32, device="cuda")
    gm.run(a, 120, opts=opts, iters_log=la)
    b = gm.new_state()
    for k0 in range(0, 120, 7):
        gm.run(b, min(7, 120 - k0), step0=k0, opts=opts)
    torch.cuda.synchronize()
    for k in ("u", "v", "a", "d", "H"):
        assert torch.equal(a[k], b[k]), k
    li = la[:, 0].cpu().numpy()
    assert np.all(li[np.arange(120) % n_sub != n_sub - 1] == 0)
    ost = om.new_state()
    om.run(mat, ost, 120, dt, n_sub=n_sub)
    eu = rel_l2(to_np(a["u"]), ost["u"])
    ed = np.abs(to_np(a["d"]) - ost["d"]).max()
    assert eu <= 1e-4 and ed <= 1e-3, (eu, ed)


@pytest.mark.parametrize("split", ["amor", "spectral", "iso"])
def test_plane_stress_per_step_parity(orc, pff, split):
    """Plane stress (Sec. 2.1 plane assumptions): FP64 fields within 1e-10
    of the oracle, entry by entry, after each of 60 steps (oracle forced to
    the GPU's iteration counts)."""
    import torch
    c = S.config("plate_100x40", split=split)
    mat = dict(c["material"], plane="stress")
    om = orc.Mesh.from_plate(c["mesh"])
    gm = pff.Mesh.from_plate(c["mesh"], precision="fp64")
    dt = gm.set_material(mat, c["cfl"])
    assert abs(dt - om.stable_dt(mat, c["cfl"])) <= 1e-15 * dt
    nsteps = 60
    gst = gm.new_state()
    ost = om.new_state()
    log = torch.zeros(nsteps, 2, dtype=torch.int32, device="cuda")
    worst = {}
    for n in range(nsteps):
        gm.run(gst, 1, step0=n, iters_log=log[n:n + 1])
        torch.cuda.synchronize()
        om.run(mat, ost, 1, dt, n0=n, forced=[int(log[n, 0])])
        merge_worst(worst, state_errs(gst, ost))
        assert max(worst.values()) <= 1e-10, (n, worst)
    assert np.abs(to_np(gst["d"])).max() > 0  # the damage field moved
    # the plane matters: a plane-strain run differs
    om2 = orc.Mesh.from_plate(c["mesh"])
    st2 = om2.new_state()
    om2.run(c["material"], st2, nsteps, om2.stable_dt(c["material"], c["cfl"]))
    assert rel_l2(ost["u"], st2["u"]) > 1e-3


def test_plane_stress_fp32_vs_fp64_oracle(orc, pff):
    import torch
    c = S.config("plate_100x40", split="amor")
    mat = dict(c["material"], plane="stress")
    om = orc.Mesh.from_plate(c["mesh"])
    gm = pff.Mesh.from_plate(c["mesh"], precision="fp32")
    dt = gm.set_material(mat, c["cfl"])
    gst = gm.new_state()
    gm.run(gst, 200)
    torch.cuda.synchronize()
    ost = om.new_state()
    om.run(mat, ost, 200, dt)
    eu = rel_l2(to_np(gst["u"]), ost["u"])
    ed = np.abs(to_np(gst["d"]) - ost["d"]).max()
    assert eu <= 1e-4 and ed <= 1e-3, (eu, ed)


@pytest.mark.parametrize("prec,model", [("fp32", "AT2"), ("fp64", "AT2"), ("fp32", "AT1"), ("fp64", "AT1")])
def test_fused_force_rhs_matches_separate(orc, pff, prec, model):
    """The step's internal force and damage right-hand side in one kernel
    (pff_options.fuse = 2) against the two kernels (fuse = 1): FP32 fields
    bit-identical after 30 steps (per-element arithmetic identical, the
    set-up's double-word sums round alike); FP64 mechanics identical to the
    last bits of the damage, whose dot products sum in the kernel's own
    block order."""
    import torch
    c, om, gm, dt = _setup(pff, orc, prec=prec, split="amor" if model == "AT1" else "spectral", model=model)
    out = []
    for fuse in (1, 2):
        st = gm.new_state()
        log = torch.zeros(30, 2, dtype=torch.int32, device="cuda")
        gm.run(st, 30, opts=pff.options(fuse=fuse), iters_log=log)
        torch.cuda.synchronize()
        assert gm.sync_status() == 0
        out.append((st, log.cpu().numpy()))
    (a, la), (b, lb) = out
    if prec == "fp32":
        for k in ("u", "v", "a", "d", "H"):
            assert torch.equal(a[k], b[k]), k
        assert np.array_equal(la, lb)
    else:
        assert np.abs(la - lb).max() <= 1
        assert float((a["d"] - b["d"]).abs().max()) <= 1e-12
        assert rel_l2(to_np(a["u"]), to_np(b["u"])) <= 1e-12


def test_fused_force_rhs_fp64_per_step_parity(orc, pff):
    """60 FP64 steps with the fused kernel forced, every entry of every
    field against the oracle (per-field floors, 1e-10)."""
    import torch
    c, om, gm, dt = _setup(pff, orc)
    mat = c["material"]
    gst, ost = gm.new_state(), om.new_state()
    log = torch.zeros(60, 2, dtype=torch.int32, device="cuda")
    worst = {}
    for n in range(60):
        gm.run(gst, 1, step0=n, opts=pff.options(fuse=2), iters_log=log[n:n + 1])
        torch.cuda.synchronize()
        om.run(mat, ost, 1, dt, n0=n, forced=[int(log[n, 0])])
        merge_worst(worst, state_errs(gst, ost))
        assert max(worst.values()) <= 1e-10, (n, worst)
    assert gm.sync_status() == 0


@pytest.mark.parametrize("prec,loop,model", [("fp32", "graph", "AT2"), ("fp64", "graph", "AT2"),
                                              ("fp32", "host", "AT2"), ("fp32", "graph", "AT1")])
def test_run_host_matches_device_run(orc, pff, prec, loop, model):
    """pff_run_host (the state in pinned host memory, copied in and out every
    step, the copies back overlapping the damage solve) gives the bits of
    pff_run on the device state, step by step (AT1: its kernel-per-phase
    loop, one graph per step)."""
    import torch
    c, om, gm, dt = _setup(pff, orc, prec=prec, model=model, split="amor" if model == "AT1" else "spectral")
    opts = pff.options(cg_tol=c["cg_tol"], t_ramp=c["t_ramp"],
                       loop_mode=pff.PFF_LOOP_HOST if loop == "host" else pff.PFF_LOOP_GRAPH)
    ref = gm.new_state()
    work = gm.new_state()
    host = {k: torch.zeros(v.shape, dtype=v.dtype, pin_memory=True) for k, v in ref.items()}
    nsteps = 12
    for n in range(nsteps):
        gm.run(ref, 1, step0=n, opts=opts)
        gm.run_host(host, work, 1, step0=n, opts=opts)
        torch.cuda.synchronize()
        for k in ("u", "v", "a", "d", "H"):
            assert torch.equal(host[k], ref[k].cpu()), (n, k)
    # several steps in one call: 5 (one graph per step) and 21 (two
    # pipelined chunks of 8 steps in one graph each, then single steps)
    n0 = nsteps
    for k_steps in (5, 21):
        gm.run(ref, k_steps, step0=n0, opts=opts)
        gm.run_host(host, work, k_steps, step0=n0, opts=opts)
        torch.cuda.synchronize()
        for k in ("u", "v", "a", "d", "H"):
            assert torch.equal(host[k], ref[k].cpu()), (k_steps, k)
        n0 += k_steps
    assert gm.sync_status() == 0


@pytest.mark.parametrize("name,split,model,field", [("plate_100x40", "spectral", "AT2", False),
                                                     ("plate_100x40", "amor", "AT1", False),
                                                     ("plate_100x40", "spectral", "AT2", True),
                                                     ("plate_500x500", "spectral", "AT2", False)])
def test_fused_variants_bit_identical(orc, pff, name, split, model, field):
    """Every variant of the fused force and right-hand side (1..5: one to
    four entries in flight) against the two separate kernels: identical bits
    in every field and the same CG counts after FP32 steps.  The element
    arithmetic spells out every multiply-add, so kernels of different shape
    round alike; the 251k-node plate has more rows than the grid has
    threads (grid-stride rows), and the toughness field varies from element
    to element."""
    import torch
    c = S.config(name, split=split, model=model)
    gm = pff.Mesh.from_plate(c["mesh"], precision="fp32")
    gm.set_material(c["material"], c["cfl"])
    if field:
        cx = c["mesh"]["xy"][c["mesh"]["tri"]].mean(axis=1)[:, 0]
        gm.set_gc_field(c["material"]["Gc"] * (1.0 + 0.3 * np.sin(60.0 * cx)))
    nsteps = 30 if name == "plate_100x40" else 8
    out = []
    for var, fuse in [(0, 1), (1, 2), (2, 2), (3, 2), (4, 2), (5, 2)]:
        st = gm.new_state()
        log = torch.zeros(nsteps, 2, dtype=torch.int32, device="cuda")
        gm.run(st, nsteps, opts=pff.options(variant=var, fuse=fuse), iters_log=log)
        torch.cuda.synchronize()
        assert gm.sync_status() == 0
        if var > 0:
            assert gm.fused_schedule()[0] == var
        out.append((st, log.cpu().numpy()))
    assert float(out[0][0]["d"].max()) > 0.5
    for st, lg in out[1:]:
        for k in ("u", "v", "a", "d", "H"):
            assert torch.equal(st[k], out[0][0][k]), k
        assert np.array_equal(lg, out[0][1])
