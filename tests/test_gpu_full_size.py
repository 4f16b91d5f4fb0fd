"""Parity at the benchmark sizes, in the configurations the bench times.

* The 1M-node plate (1000 x 1000 cells, jittered): the first 8 steps in FP64
  against the oracle with the oracle forced to the GPU's CG iteration
  counts, every entry of every field within 1e-10 (spectral and
  volumetric-deviatoric AT2), 6 steps with plane stress (spectral and
  isotropic splits), 8 steps with the damage solved every 2nd step, 6
  steps with a per-element toughness field; 3
  steps of AT1 with the volumetric-deviatoric
  split and the projected CG at natural stops; FP32_MIXED with the bench's
  options against the same oracle state (u relative L2 <= 1e-4, max |d -
  d_oracle| <= 1e-3), and so for the volumetric-deviatoric split and AT1
  with it against the oracle at natural stops.
* The differentiation plate (500 x 500 cells): dL/dGc of a short window in
  FP32 against the oracle's discrete adjoint.
* The 700 x 700 SENT: one load increment with the tangent CG in FP32 against
  the same increment with it in FP64 (the oracle cannot run this size in a
  test's time; both GPU runs converge the FP64 Newton residual to 1e-8).
* The 64-plate batch: plates against their single-plate runs.
"""
import numpy as np
import pytest

import pff_synth as S
from gpu_common import FIELD_FLOOR, field_err, merge_worst, rel_l2, state_errs, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pff():
    import paper_2606_23458_b300 as pff
    return pff


def _fp64_window(orc, pff, c, nsteps, forced_counts=True, mat=None, n_sub=1, gc=None):
    """GPU FP64 and the oracle over the first nsteps steps of a plate, step
    by step: with forced_counts the oracle runs each step's CG for the GPU's
    iteration count (AT2), else to its own stop; mat replaces the plate's
    material, n_sub > 1 solves damage every n_sub-th step on both sides, gc
    (per element) is a toughness field set on both sides.
    Returns the worst element-wise error per field over the window, the
    last states and the GPU's iteration counts."""
    import torch
    mat = c["material"] if mat is None else mat
    gm = pff.Mesh.from_plate(c["mesh"], precision="fp64")
    dt = gm.set_material(mat, c["cfl"])
    opts = pff.options(cg_tol=c["cg_tol"], t_ramp=c["t_ramp"], damage_every=n_sub)
    if gc is not None:
        gm.set_gc_field(gc)
    gst = gm.new_state()
    om = orc.Mesh.from_plate(c["mesh"])
    if gc is not None:
        om.set_gc_field(gc)
    ost = om.new_state()
    log = torch.zeros(nsteps, 2, dtype=torch.int32, device="cuda")
    worst, oiters = {}, []
    for n in range(nsteps):
        gm.run(gst, 1, step0=n, opts=opts, iters_log=log[n:n + 1])
        torch.cuda.synchronize()
        forced = [int(log[n, 0])] if forced_counts else None
        r = om.run(mat, ost, 1, dt, n0=n, t_ramp=c["t_ramp"], forced=forced, n_sub=n_sub)
        oiters.append(int(r["iters"][0, 0]))
        merge_worst(worst, state_errs(gst, ost, floors=FIELD_FLOOR))  # 1e-6 on every field
    assert gm.sync_status() == 0
    return dict(c=c, dt=dt, nsteps=nsteps, ost=ost, g64={k: to_np(v) for k, v in gst.items()},
                worst=worst, iters=[int(v) for v in log[:, 0].cpu().numpy()], oracle_iters=oiters)


@pytest.fixture(scope="module")
def plate_1m(orc, pff):
    """The bench plate (spectral AT2) over its first 8 steps in FP64."""
    return _fp64_window(orc, pff, S.config("plate_1000x1000"), 8)


def test_fp64_1m_plate_matches_oracle(plate_1m):
    """Every entry of u, v, a, d and H within 1e-10 of the oracle after each
    of the first 8 steps (|g - o| / max(|o|, 1e-6 max|o|))."""
    w = plate_1m["worst"]
    print(f"1M plate, spectral FP64, 8 steps: element-wise worst {w}, CG iterations {plate_1m['iters']}")
    assert max(w.values()) <= 1e-10, w
    g = plate_1m["g64"]
    assert np.abs(g["u"]).max() > 0 and max(plate_1m["iters"]) > 0  # the window moved and solved
    assert np.abs(g["H"]).max() > 0


def test_fp64_1m_plate_amor_matches_oracle(orc, pff):
    """The volumetric-deviatoric split (Eq. amor_split) on the 1M-node plate:
    8 steps in FP64, every entry within 1e-10 of the oracle per step."""
    r = _fp64_window(orc, pff, S.config("plate_1000x1000", split="amor"), 8)
    print(f"1M plate, Amor FP64, 8 steps: element-wise worst {r['worst']}, CG iterations {r['iters']}")
    assert max(r["worst"].values()) <= 1e-10, r["worst"]
    assert np.abs(r["g64"]["H"]).max() > 0


@pytest.mark.parametrize("split", ["spectral", "iso"])
def test_fp64_1m_plate_plane_stress_matches_oracle(orc, pff, split):
    """Plane stress (Sec. 2.1 plane assumptions) on the 1M-node plate with
    the spectral and the isotropic split: 6 steps in FP64, every entry
    within 1e-10 of the oracle per step."""
    c = S.config("plate_1000x1000", split=split)
    r = _fp64_window(orc, pff, c, 6, mat=dict(c["material"], plane="stress"))
    print(f"1M plate, plane stress {split} FP64, 6 steps: element-wise worst {r['worst']}, CG iterations {r['iters']}")
    assert max(r["worst"].values()) <= 1e-10, r["worst"]
    assert np.abs(r["g64"]["H"]).max() > 0 and max(r["iters"]) > 0


def test_fp64_1m_plate_subcycled_matches_oracle(orc, pff):
    """Damage subcycling (Sec. 2.4) on the 1M-node plate: the damage solved
    every 2nd step (the glass plate's limit), H every step; 8 steps in FP64,
    every entry within 1e-10 of the oracle per step, and no solve on the
    skipped steps."""
    r = _fp64_window(orc, pff, S.config("plate_1000x1000"), 8, n_sub=2)
    print(f"1M plate, subcycled FP64, 8 steps: element-wise worst {r['worst']}, CG iterations {r['iters']}")
    assert max(r["worst"].values()) <= 1e-10, r["worst"]
    assert all(r["iters"][n] == 0 for n in range(0, 8, 2)) and max(r["iters"]) > 0


def test_fp64_1m_plate_toughness_field_matches_oracle(orc, pff):
    """A per-element toughness field Gc_e = Gc (1 + 0.3 sin(60 x_e / m))
    (Sec. 4.2's field-valued parameter) on the 1M-node plate: 6 steps in
    FP64, every entry within 1e-10 of the oracle per step."""
    c = S.config("plate_1000x1000")
    m = c["mesh"]
    cx = np.asarray(m["xy"])[np.asarray(m["tri"])].mean(axis=1)[:, 0]
    gc = c["material"]["Gc"] * (1.0 + 0.3 * np.sin(60.0 * cx))
    r = _fp64_window(orc, pff, c, 6, gc=gc)
    print(f"1M plate, toughness field FP64, 6 steps: element-wise worst {r['worst']}, CG iterations {r['iters']}")
    assert max(r["worst"].values()) <= 1e-10, r["worst"]
    assert max(r["iters"]) > 0


def test_fp64_1m_plate_at1_amor_matches_oracle(orc, pff):
    """AT1 with the volumetric-deviatoric split and the bound-projected CG
    (Sec. 2.4) on the 1M-node plate: 3 steps in FP64, GPU and oracle each to
    its own stop (projected CG restarts are decisions taken on the iterate,
    so counts are not forced).  Tolerances of the AT1 runs: u within 1e-7
    relative L2 and entry by entry 1e-7, d within 1e-6 absolute; the first
    solve builds the damage band around the notch."""
    r = _fp64_window(orc, pff, S.config("plate_1000x1000", split="amor", model="AT1"), 3,
                     forced_counts=False)
    g, o = r["g64"], r["ost"]
    print(f"1M plate, AT1 + Amor FP64, 3 steps: element-wise worst {r['worst']}, "
          f"GPU iterations {r['iters']}, oracle {r['oracle_iters']}")
    assert rel_l2(g["u"], o["u"]) <= 1e-7
    for k in ("u", "v", "a", "H"):
        assert r["worst"][k] <= 1e-7, (k, r["worst"])
    assert np.abs(g["d"] - o["d"]).max() <= 1e-6
    band = (o["d"] > 0) & (np.asarray(r["c"]["mesh"]["notch"]) == 0)
    assert band.sum() > 0  # the projected CG built the band around the notch
    assert np.all(g["d"] >= -1e-15) and np.all(g["d"] <= 1.0)


@pytest.mark.parametrize("cgk", ["auto", "resident", "fused"])
def test_fp32_1m_plate_bench_configuration(pff, plate_1m, cgk):
    """FP32 with the bench's options (graph loop, the default element-wise
    damage operator; the autotuned CG family, or the resident loop, whose
    rows at this size keep only x, p, the diagonal and the fan tables in
    shared memory, or the global-memory single-reduction loop) against the
    FP64 oracle state at the end of the window: u relative L2 <= 1e-4, max
    |d - d_oracle| <= 1e-3."""
    import torch
    c = plate_1m["c"]
    gm = pff.Mesh.from_plate(c["mesh"], precision="fp32")
    gm.set_material(c["material"], c["cfl"])
    gst = gm.new_state()
    kind = {v: k for k, v in pff.CG_KINDS.items()}[cgk]
    gm.run(gst, plate_1m["nsteps"], opts=pff.options(cg_tol=c["cg_tol"], t_ramp=c["t_ramp"], cg_kernel=kind))
    torch.cuda.synchronize()
    assert gm.sync_status() == 0
    o = plate_1m["ost"]
    assert rel_l2(to_np(gst["u"]), o["u"]) <= 1e-4
    assert np.abs(to_np(gst["d"]) - o["d"]).max() <= 1e-3


@pytest.mark.parametrize("split,model,nsteps,plane,field,n_sub", [("amor", "AT2", 8, "strain", False, 1),
                                                                  ("amor", "AT1", 3, "strain", False, 1),
                                                                  ("iso", "AT2", 6, "stress", False, 1),
                                                                  ("spectral", "AT2", 6, "strain", True, 1),
                                                                  ("spectral", "AT2", 8, "strain", False, 2)])
def test_fp32_1m_plate_variants_vs_oracle(orc, pff, split, model, nsteps, plane, field, n_sub):
    """FP32_MIXED with the bench's options on the 1M-node plate for the
    volumetric-deviatoric split (AT2), AT1 with it (bound-projected CG),
    plane stress with the isotropic split, a per-element toughness field,
    and the damage solved every 2nd step (both sides), against the FP64
    oracle at its natural stops: u relative L2
    <= 1e-4 and max |d - d_oracle| <= 1e-3, the FP32 bounds."""
    import torch
    c = S.config("plate_1000x1000", split=split, model=model)
    mat = dict(c["material"], plane=plane)
    gm = pff.Mesh.from_plate(c["mesh"], precision="fp32")
    dt = gm.set_material(mat, c["cfl"])
    om = orc.Mesh.from_plate(c["mesh"])
    if field:
        m = c["mesh"]
        cx = np.asarray(m["xy"])[np.asarray(m["tri"])].mean(axis=1)[:, 0]
        gc = mat["Gc"] * (1.0 + 0.3 * np.sin(60.0 * cx))
        gm.set_gc_field(gc)
        om.set_gc_field(gc)
    gst = gm.new_state()
    gm.run(gst, nsteps, opts=pff.options(cg_tol=c["cg_tol"], t_ramp=c["t_ramp"], damage_every=n_sub))
    torch.cuda.synchronize()
    assert gm.sync_status() == 0
    ost = om.new_state()
    om.run(mat, ost, nsteps, dt, t_ramp=c["t_ramp"], n_sub=n_sub)
    eu = rel_l2(to_np(gst["u"]), ost["u"])
    ed = float(np.abs(to_np(gst["d"]) - ost["d"]).max())
    print(f"1M plate, {model} {split} plane {plane}{' field' if field else ''} n_sub {n_sub} FP32 vs FP64 oracle, {nsteps} steps: "
          f"u rel L2 {eu:.2e}, max |dd| {ed:.2e}")
    assert eu <= 1e-4 and ed <= 1e-3, (eu, ed)
    band = (ost["d"] > 0) & (np.asarray(c["mesh"]["notch"]) == 0)
    assert np.abs(ost["u"]).max() > 0 and band.sum() > 0  # the window loaded the plate and grew damage


def test_differentiation_plate_gradient(orc, pff):
    import torch
    c = S.config("plate_500x500")
    mat = c["material"]
    nsteps = 6
    om = orc.Mesh.from_plate(c["mesh"])
    dt = om.stable_dt(mat, c["cfl"])
    st = om.new_state()
    om.run(dict(mat, Gc=3.0), st, nsteps, dt, t_ramp=c["t_ramp"], tol=1e-12)
    dstar = st["d"].copy()
    L, g, status = om.adjoint_gc(dict(mat, Gc=2.0), nsteps, dt, dstar, t_ramp=c["t_ramp"], tol=1e-12)
    assert status == 0 and g != 0.0
    gm = pff.Mesh.from_plate(c["mesh"], precision="fp32")
    gm.set_material(dict(mat, Gc=2.0), c["cfl"])
    opts = pff.options(cg_tol=1e-12, t_ramp=c["t_ramp"])
    s = gm.new_state()
    ck = pff.Checkpoint(gm, nsteps, 0)
    gm.run_ckpt(s, ck, opts=opts)
    up = (2.0 * (s["d"].double() - torch.tensor(dstar, device="cuda")) / gm.N).float().contiguous()
    gg = gm.backward(ck, up, opts=opts)
    ck.close()
    assert abs(gg - g) <= 2e-3 * abs(g), (gg, g)


def test_sent_full_size_increment(pff):
    import torch
    c = S.sent(700)
    out = []
    for krylov in ("fp32", "mesh"):
        m = pff.Mesh.from_plate(c["mesh"], precision="fp64")
        m.set_material(c["material"], 0.5)
        st = m.new_state()
        r = m.qs_run(st, c["bc"], 1, c["du"], newton_tol=c["newton_tol"], krylov=krylov,
                     opts=pff.options(cg_tol=c["cg_tol"], cg_max_it=100000))
        torch.cuda.synchronize()
        out.append((r["reaction"][0], to_np(st["d"])))
    assert abs(out[0][0] - out[1][0]) <= 1e-7 * abs(out[1][0]), (out[0][0], out[1][0])
    assert np.abs(out[0][1] - out[1][1]).max() <= 1e-6


def test_sent_full_size_increment_vs_oracle(orc, pff):
    """The 700 x 700 SENT's first increment (FP64 state, FP32 tangent CG)
    checked by the oracle where it can be checked at this size: the
    mechanics' equilibrium (the oracle's f_int at the GPU's u and the
    increment's starting damage meets the Newton stop test on the free dofs,
    and gives the GPU's reaction), the history (the oracle's psi+ at that u,
    element by element), and the damage (the oracle's own solve with the
    GPU's history from the same starting damage, entry by entry)."""
    import torch
    c = S.sent(700)
    mat = c["material"]
    m = pff.Mesh.from_plate(c["mesh"], precision="fp64")
    m.set_material(mat, 0.5)
    st = m.new_state()
    d0, H0 = to_np(st["d"]).copy(), to_np(st["H"]).copy()
    r = m.qs_run(st, c["bc"], 1, c["du"], newton_tol=c["newton_tol"], krylov="fp32",
                 opts=pff.options(cg_tol=c["cg_tol"], cg_max_it=100000))
    torch.cuda.synchronize()
    u, d, H = to_np(st["u"]).reshape(-1, 2), to_np(st["d"]), to_np(st["H"])
    om = orc.Mesh.from_plate(c["mesh"])
    f, psip = om.internal_force(mat, u, d0)
    bc = c["bc"]
    free = np.stack([(bc & 1) == 0, (bc & 6) == 0], axis=1)
    rfree = np.linalg.norm(f[free])
    assert rfree <= 1.01 * c["newton_tol"] * np.linalg.norm(f), (rfree, np.linalg.norm(f))
    reac = f[(bc & 4) != 0, 1].sum()
    assert abs(r["reaction"][0] - reac) <= 1e-9 * abs(reac), (r["reaction"][0], reac)
    Hor = np.maximum(H0, psip)
    assert field_err(H, Hor) <= 1e-10, field_err(H, Hor)
    dor, info, rel, status, _ = om.damage_solve(mat, H, d0, tol=c["cg_tol"], max_it=100000)
    assert status == 0 and np.abs(d - dor).max() <= 1e-6, np.abs(d - dor).max()


@pytest.fixture(scope="module", params=["auto", "resident"])
def batch64(pff, request):
    """The bench's 64-plate batch (5.24M nodes, FP32) after 6 steps, with
    the autotuned CG loop and with the per-plate resident loop (in waves of
    plates that fit the SMs' shared memory together)."""
    import torch
    plates = []
    for dr in S.batch_draws(64, seed=1):
        p = S.plate(dr["nx"], dr["ny"], jitter=0.1, seed=1, traction=dr["traction"])
        plates.append((p, S.material(2 * p["h"], Gc=dr["Gc"])))
    nsteps = 6
    b = pff.Batch(plates, precision="fp32")
    st = b.new_state()
    log = torch.zeros(nsteps, b.nplates, dtype=torch.int32, device="cuda")
    cgk = pff.PFF_CG_RESIDENT if request.param == "resident" else pff.PFF_CG_AUTO
    b.run(st, nsteps, opts=pff.options(cg_kernel=cgk), iters_log=log)
    torch.cuda.synchronize()
    assert max(b.tuning()["ms"]["cg_resident"]) > 0  # available on this batch
    sizes = [p["xy"].shape[0] for p, _ in plates]
    picks = sorted({0, int(np.argmin(sizes)), int(np.argmax(sizes))})
    return dict(plates=plates, b=b, st=st, log=log.cpu().numpy(), nsteps=nsteps, picks=picks)


def test_batch_workload_matches_single_plates(pff, batch64):
    """The first, smallest and largest plates of the batch agree with their
    single-plate runs."""
    import torch
    b, st, nsteps = batch64["b"], batch64["st"], batch64["nsteps"]
    for k in batch64["picks"]:
        p, mat = batch64["plates"][k]
        m = pff.Mesh.from_plate(p, precision="fp32")
        m.set_material(mat, 0.5)
        s1 = m.new_state()
        l1 = torch.zeros(nsteps, 2, dtype=torch.int32, device="cuda")
        m.run(s1, nsteps, iters_log=l1)
        torch.cuda.synchronize()
        v = b.plate(st, k)
        assert rel_l2(to_np(v["u"]), to_np(s1["u"])) <= 2e-5, k
        assert np.abs(to_np(v["d"]) - to_np(s1["d"])).max() <= 1e-4, k
        assert np.abs(batch64["log"][:, k] - l1[:, 0].cpu().numpy()).max() <= 1, k


def test_batch_workload_matches_oracle(orc, batch64):
    """The first, smallest and largest plates of the batch (FP32 kernels,
    FP64-class reductions) against the FP64 oracle run of the same plate,
    its own Gc, traction and time step: u relative L2 <= 1e-4 and max |d -
    d_oracle| <= 1e-3 (the FP32 tolerances)."""
    b, st, nsteps = batch64["b"], batch64["st"], batch64["nsteps"]
    for k in batch64["picks"]:
        p, mat = batch64["plates"][k]
        om = orc.Mesh.from_plate(p)
        dt = om.stable_dt(mat, 0.5)
        assert abs(dt - b.info[k]["dt"]) <= 1e-12 * dt, k
        ost = om.new_state()
        r = om.run(mat, ost, nsteps, dt)
        v = b.plate(st, k)
        eu = rel_l2(to_np(v["u"]), ost["u"])
        ed = np.abs(to_np(v["d"]) - ost["d"]).max()
        print(f"batch plate {k} ({om.N} nodes) vs oracle: u rel L2 {eu:.2e}, max|dd| {ed:.2e}")
        assert eu <= 1e-4 and ed <= 1e-3, (k, eu, ed)
        assert r["status"] == 0 and batch64["log"][-1, k] > 0, k
