"""Parity at the benchmark sizes, in the configurations the bench times.

* The 1M-node plate (1000 x 1000 cells, jittered, spectral AT2): the first
  steps in FP64 against the oracle with the oracle forced to the GPU's CG
  iteration counts (1e-10 relative on every field), and in FP32_MIXED with
  the bench's options (graph loop, autotuned CG family) against the same
  oracle state (u relative L2 <= 1e-4, max |d - d_oracle| <= 1e-3).
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
from gpu_common import max_rel, rel_l2, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pff():
    import paper_2606_23458_b300 as pff
    return pff


@pytest.fixture(scope="module")
def plate_1m(orc, pff):
    """GPU FP64 and the forced-count oracle over the first steps of the
    1M-node plate; returns the config, dt, oracle state and GPU states."""
    import torch
    c = S.config("plate_1000x1000")
    nsteps = 4
    gm = pff.Mesh.from_plate(c["mesh"], precision="fp64")
    dt = gm.set_material(c["material"], c["cfl"])
    gst = gm.new_state()
    log = torch.zeros(nsteps, 2, dtype=torch.int32, device="cuda")
    opts = pff.options(cg_tol=c["cg_tol"], t_ramp=c["t_ramp"])
    gm.run(gst, nsteps, opts=opts, iters_log=log)
    torch.cuda.synchronize()
    assert gm.sync_status() == 0
    forced = [int(v) for v in log[:, 0].cpu().numpy()]
    om = orc.Mesh.from_plate(c["mesh"])
    ost = om.new_state()
    om.run(c["material"], ost, nsteps, dt, t_ramp=c["t_ramp"], forced=forced)
    return dict(c=c, dt=dt, nsteps=nsteps, ost=ost, g64={k: to_np(v) for k, v in gst.items()}, forced=forced)


def test_fp64_1m_plate_matches_oracle(plate_1m):
    g, o = plate_1m["g64"], plate_1m["ost"]
    for k in ("u", "v", "a", "H"):
        assert rel_l2(g[k], o[k]) <= 1e-10, k
    assert max_rel(g["d"], o["d"], 1e-3) <= 1e-10
    assert np.abs(g["u"]).max() > 0 and max(plate_1m["forced"]) > 0  # the window moved and solved


def test_fp32_1m_plate_bench_configuration(pff, plate_1m):
    import torch
    c = plate_1m["c"]
    gm = pff.Mesh.from_plate(c["mesh"], precision="fp32")
    gm.set_material(c["material"], c["cfl"])
    gst = gm.new_state()
    gm.run(gst, plate_1m["nsteps"], opts=pff.options(cg_tol=c["cg_tol"], t_ramp=c["t_ramp"]))
    torch.cuda.synchronize()
    assert gm.sync_status() == 0
    o = plate_1m["ost"]
    assert rel_l2(to_np(gst["u"]), o["u"]) <= 1e-4
    assert np.abs(to_np(gst["d"]) - o["d"]).max() <= 1e-3


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


def test_batch_workload_matches_single_plates(pff):
    """The bench's 64-plate batch (5.24M nodes): after a few steps the
    first, smallest and largest plates agree with their single-plate runs."""
    import torch
    plates = []
    for dr in S.batch_draws(64, seed=1):
        p = S.plate(dr["nx"], dr["ny"], jitter=0.1, seed=1, traction=dr["traction"])
        plates.append((p, S.material(2 * p["h"], Gc=dr["Gc"])))
    nsteps = 6
    b = pff.Batch(plates, precision="fp32")
    st = b.new_state()
    log = torch.zeros(nsteps, b.nplates, dtype=torch.int32, device="cuda")
    b.run(st, nsteps, iters_log=log)
    torch.cuda.synchronize()
    sizes = [p["xy"].shape[0] for p, _ in plates]
    for k in sorted({0, int(np.argmin(sizes)), int(np.argmax(sizes))}):
        p, mat = plates[k]
        m = pff.Mesh.from_plate(p, precision="fp32")
        m.set_material(mat, 0.5)
        s1 = m.new_state()
        l1 = torch.zeros(nsteps, 2, dtype=torch.int32, device="cuda")
        m.run(s1, nsteps, iters_log=l1)
        torch.cuda.synchronize()
        v = b.plate(st, k)
        assert rel_l2(to_np(v["u"]), to_np(s1["u"])) <= 2e-5, k
        assert np.abs(to_np(v["d"]) - to_np(s1["d"])).max() <= 1e-4, k
        assert np.abs(log[:, k].cpu().numpy() - l1[:, 0].cpu().numpy()).max() <= 1, k
