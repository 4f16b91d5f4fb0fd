"""Toughness field on the GPU (Secs. 4.2 and 7, the field-valued inverse):
per-step parity with the oracle under a non-uniform field, a uniform field
identical to the scalar toughness, and the per-element gradient of the
discrete adjoint against the oracle's."""
import numpy as np
import pytest

import pff_synth as S
from gpu_common import field_err, merge_worst, rel_l2, state_errs, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pff():
    import paper_2606_23458_b300 as pff
    return pff


def _field(p, base):
    cx = p["xy"][p["tri"]].mean(axis=1)[:, 0]
    return base * (1.0 + 0.3 * np.sin(60.0 * cx))


def test_field_per_step_parity(orc, pff):
    import torch
    c = S.config("plate_100x40")
    mat = c["material"]
    gc = _field(c["mesh"], mat["Gc"])
    om = orc.Mesh.from_plate(c["mesh"])
    om.set_gc_field(gc)
    gm = pff.Mesh.from_plate(c["mesh"], precision="fp64")
    dt = gm.set_material(mat, c["cfl"])
    gm.set_gc_field(gc)
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
    assert gm.sync_status() == 0


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_uniform_field_is_bit_identical(pff, prec):
    import torch
    c = S.config("plate_100x40")
    out = []
    for field in (False, True):
        gm = pff.Mesh.from_plate(c["mesh"], precision=prec)
        gm.set_material(c["material"], c["cfl"])
        if field:
            gm.set_gc_field(np.full(gm.Ne, c["material"]["Gc"]))
        st = gm.new_state()
        gm.run(st, 40, opts=pff.options(cg_kernel=pff.PFF_CG_PERSISTENT))
        torch.cuda.synchronize()
        out.append(st)
    for k in ("u", "d", "H"):
        assert torch.equal(out[0][k], out[1][k]), k


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-7), ("fp32", 5e-3)])
def test_field_gradient_matches_oracle(orc, pff, prec, tol):
    import torch
    p = S.plate(20, 8)
    mat = S.material(2 * p["h"])
    om = orc.Mesh.from_plate(p)
    dt = om.stable_dt(mat, 0.5)
    nsteps = 30
    st = om.new_state()
    om.run(dict(mat, Gc=3.0), st, nsteps, dt, tol=1e-13)
    dstar = st["d"].copy()
    gc = _field(p, 2.5)
    om.set_gc_field(gc)
    L, g, status, ge = om.adjoint_gc(dict(mat, Gc=2.5), nsteps, dt, dstar, tol=1e-13, field=True)
    gm = pff.Mesh.from_plate(p, precision=prec)
    gm.set_material(dict(mat, Gc=2.5), 0.5)
    gm.set_gc_field(gc)
    opts = pff.options(cg_tol=1e-13)
    s = gm.new_state()
    ck = pff.Checkpoint(gm, nsteps, 0)
    gm.run_ckpt(s, ck, opts=opts)
    d = s["d"].double()
    up = (2.0 * (d - torch.tensor(dstar, device="cuda")) / gm.N).to(gm.dtype).contiguous()
    gg, gfield = gm.backward_field(ck, up, opts=opts)
    gfield = gfield.cpu().numpy()
    ck.close()
    assert abs(gg - g) <= tol * abs(g), (gg, g)
    # per element: each dL/dGc_e against the oracle's, its error over
    # max(|o_e|, 1e-3 max|o|) (the adjoint solves stop at 1e-13, so entries
    # far below the field's scale carry that absolute error)
    assert field_err(gfield, ge, 1e-3) <= tol, field_err(gfield, ge, 1e-3)
    print(f"{prec}: dL/dGc_e element-wise error (floor 1e-3 max) {field_err(gfield, ge, 1e-3):.2e}, "
          f"(floor 1e-6 max) {field_err(gfield, ge):.2e}, rel L2 {rel_l2(gfield, ge):.2e}")
    assert abs(gfield.sum() - gg) <= 1e-9 * abs(gg) + 1e-6 * np.abs(gfield).sum() * (prec == "fp32")
