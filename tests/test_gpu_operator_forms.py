"""The damage operator's two forms (pff_mesh_set_operator, Sec. 2.4 with Eq.
matrix_free_fe_operator): the element-wise matrix-free form, the default,
in which every CG product applies each element's own coefficients, and the
merged rows, in which a right-hand side sums the two elements' coefficients
of each edge (the solve's operator assembled per solve).  Each form against
the oracle (FP64 with forced iteration counts, entry by entry 1e-10) and
the two against each other (FP32), the switch's bookkeeping, and a mesh on
which merged rows do not exist."""
import numpy as np
import pytest

import pff_synth as S
from gpu_common import field_err, merge_worst, rel_l2, state_errs, to_np

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


def test_default_form_is_element_wise(pff):
    for prec in ("fp32", "fp64"):
        m = pff.Mesh.from_plate(S.plate(40, 16), precision=prec)
        assert m.operator() == ("element", True)
        m.set_operator("merged")
        assert m.operator() == ("merged", True)
        m.set_operator("element")
        assert m.operator()[0] == "element"


@pytest.mark.parametrize("form", ["element", "merged"])
@pytest.mark.parametrize("kind", ["phases", "persistent"])
def test_fp64_solve_each_form_vs_oracle(orc, pff, form, kind):
    import torch
    p = S.plate(60, 24, jitter=0.1, seed=5)
    mat = S.material(2 * p["h"])
    m = pff.Mesh.from_plate(p, precision="fp64")
    m.set_material(mat, 0.5)
    m.set_operator(form)
    H, dprev = _inputs(p, 4)
    Ht = torch.tensor(H, device="cuda")
    dp = torch.tensor(dprev, device="cuda")
    out = torch.empty_like(dp)
    cgk = {"phases": pff.PFF_CG_PHASES, "persistent": pff.PFF_CG_PERSISTENT}[kind]
    info = m.damage_solve(Ht, dp, out, pff.options(cg_kernel=cgk))
    om = orc.Mesh.from_plate(p)
    d, oinfo, *_ = om.damage_solve(mat, H, dprev, tol=1e-8, forced=info["iters"])
    assert abs(int(oinfo[1]) - info["iters"]) <= 1
    assert field_err(to_np(out), d) <= 1e-10, field_err(to_np(out), d)


@pytest.mark.parametrize("form", ["element", "merged"])
def test_fp64_run_each_form_per_step(orc, pff, form):
    """40 staggered steps of the 100 x 40 plate in FP64 with the form fixed:
    every entry of u, v, a, d, H within 1e-10 of the oracle after each step
    (oracle forced to the GPU's iteration counts)."""
    import torch
    c = S.config("plate_100x40")
    mat = c["material"]
    gm = pff.Mesh.from_plate(c["mesh"], precision="fp64")
    dt = gm.set_material(mat, c["cfl"])
    gm.set_operator(form)
    om = orc.Mesh.from_plate(c["mesh"])
    gst, ost = gm.new_state(), om.new_state()
    log = torch.zeros(40, 2, dtype=torch.int32, device="cuda")
    worst = {}
    for n in range(40):
        gm.run(gst, 1, step0=n, iters_log=log[n:n + 1])
        torch.cuda.synchronize()
        om.run(mat, ost, 1, dt, n0=n, forced=[int(log[n, 0])])
        merge_worst(worst, state_errs(gst, ost))
    print(f"fp64 {form}: element-wise worst {worst}")
    assert max(worst.values()) <= 1e-10, worst
    assert gm.sync_status() == 0


@pytest.mark.parametrize("kind", ["phases", "persistent", "fused"])
def test_fp32_forms_agree(orc, pff, kind):
    """FP32 runs of the 300 x 120 plate with each form and CG family: the
    forms differ only in where the two elements' coefficients of an edge are
    added (FP32 rounding), so they agree closely; both meet the FP32
    tolerances against the FP64 oracle."""
    import torch
    p = S.plate(300, 120, jitter=0.1, seed=2)
    mat = S.material(2 * p["h"])
    cgk = {"phases": pff.PFF_CG_PHASES, "persistent": pff.PFF_CG_PERSISTENT, "fused": pff.PFF_CG_FUSED}[kind]
    res = {}
    nsteps = 40
    for form in ("element", "merged"):
        m = pff.Mesh.from_plate(p, precision="fp32")
        m.set_material(mat, 0.5)
        m.set_operator(form)
        st = m.new_state()
        log = torch.zeros(nsteps, 2, dtype=torch.int32, device="cuda")
        m.run(st, nsteps, opts=pff.options(cg_kernel=cgk), iters_log=log)
        torch.cuda.synchronize()
        assert m.sync_status() == 0
        res[form] = ({k: to_np(st[k]) for k in ("u", "d")}, log[:, 0].cpu().numpy())
    (a, ia), (b, ib) = res["element"], res["merged"]
    assert np.abs(ia - ib).max() <= 2, (ia, ib)
    assert rel_l2(a["u"], b["u"]) <= 1e-5
    assert np.abs(a["d"] - b["d"]).max() <= 1e-4
    om = orc.Mesh.from_plate(p)
    ost = om.new_state()
    om.run(mat, ost, nsteps, om.stable_dt(mat, 0.5))
    for form, (f, _) in res.items():
        assert rel_l2(f["u"], ost["u"]) <= 1e-4, form
        assert np.abs(f["d"] - ost["d"]).max() <= 1e-3, form


def test_switch_drops_tuning_and_graphs(pff):
    import torch
    c = S.config("plate_100x40")
    m = pff.Mesh.from_plate(c["mesh"], precision="fp32")
    m.set_material(c["material"], c["cfl"])
    st = m.new_state()
    m.run(st, 3)
    torch.cuda.synchronize()
    assert m.cg_choice()[0] != "auto"
    m.set_operator("merged")
    assert m.cg_choice()[0] == "auto"   # re-timed on the next solve
    m.run(st, 3, step0=3)
    torch.cuda.synchronize()
    assert m.cg_choice()[0] != "auto" and m.sync_status() == 0
    m.set_operator("merged")            # same form: nothing dropped
    assert m.cg_choice()[0] != "auto"


def test_merged_unavailable_on_wide_mesh(pff):
    """A node meeting twelve triangles has more distinct neighbours than a
    merged row holds: the mesh keeps the element-wise form only."""
    from test_gpu_wide_incidence import _plate
    q = _plate()
    for prec in ("fp32", "fp64"):
        m = pff.Mesh.from_plate(q, precision=prec)
        assert m.operator() == ("element", False)
        with pytest.raises(pff.PffError) as e:
            m.set_operator("merged")
        assert e.value.status == pff.PFF_ERR_ARG


def test_fan_order_where_the_fans_fit(pff):
    """Plates (every vertex fan at most six triangles) store the element-wise
    entries in fan order; a vertex with twelve triangles keeps incidence
    order.  Both are checked against the oracle by the other tests."""
    from test_gpu_wide_incidence import _plate
    for prec in ("fp32", "fp64"):
        assert pff.Mesh.from_plate(S.plate(40, 16, jitter=0.1, seed=1), precision=prec).fan_order()
        assert not pff.Mesh.from_plate(_plate(), precision=prec).fan_order()
