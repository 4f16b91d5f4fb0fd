"""Meshes whose rows are too wide for merged rows keep the per-slot entry
records (compact 16-bit offsets): a plate whose six triangles around one
interior node are each split at their centroid, so that node meets twelve
triangles (incidence width 12, more than the eight a merged row holds).
The explicit step (every CG loop family) and the quasi-static mode against
the oracle."""
import numpy as np
import pytest

import pff_synth as S
from gpu_common import rel_l2, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pff():
    import paper_2606_23458_b300 as pff
    return pff


def _split_star(p, node):
    """Splits every triangle that holds `node` at its centroid (new nodes
    appended): the node then meets twice as many triangles."""
    xy = [*p["xy"]]
    tri = []
    for t in p["tri"]:
        if node in t:
            c = len(xy)
            xy.append(p["xy"][t].mean(axis=0))
            a, b, d = (int(v) for v in t)
            tri += [(a, b, c), (b, d, c), (d, a, c)]
        else:
            tri.append(tuple(int(v) for v in t))
    q = dict(p)
    q["xy"] = np.ascontiguousarray(np.array(xy, dtype=np.float64))
    q["tri"] = np.ascontiguousarray(np.array(tri, dtype=np.int32))
    q["notch"] = np.concatenate([p["notch"], np.zeros(len(xy) - len(p["xy"]), dtype=p["notch"].dtype)])
    return q


def _plate():
    p = S.plate(40, 16)
    nx = p["nx"]
    node = 8 * (nx + 1) + 20  # an interior node in the middle of the plate
    q = _split_star(p, node)
    assert np.bincount(q["tri"].ravel()).max() == 12
    return q


@pytest.mark.parametrize("kind", ["phases", "persistent", "fused"])
def test_wide_incidence_explicit_step(orc, pff, kind):
    import torch
    p = _plate()
    mat = S.material(2 * p["h"])
    cgk = {"phases": pff.PFF_CG_PHASES, "persistent": pff.PFF_CG_PERSISTENT, "fused": pff.PFF_CG_FUSED}[kind]
    m = pff.Mesh.from_plate(p, precision="fp32")
    m.set_material(mat, 0.5)
    st = m.new_state()
    m.run(st, 40, opts=pff.options(cg_tol=1e-8, cg_kernel=cgk))
    torch.cuda.synchronize()
    assert m.sync_status() == 0
    om = orc.Mesh.from_plate(p)
    dt = om.stable_dt(mat, 0.5)
    ost = om.new_state()
    om.run(mat, ost, 40, dt)
    assert rel_l2(to_np(st["u"]), ost["u"]) <= 1e-4
    assert np.abs(to_np(st["d"]) - ost["d"]).max() <= 1e-3


def test_wide_incidence_quasistatic(orc, pff):
    p = S.plate(16, 16, Lx=1e-3, Ly=1e-3, notch=True)
    nx = p["nx"]
    q = _split_star(p, 12 * (nx + 1) + 8)
    assert np.bincount(q["tri"].ravel()).max() == 12
    N = q["xy"].shape[0]
    y = q["xy"][:, 1]
    bc = np.zeros(N, np.uint8)
    bc[np.isclose(y, y.min())] = 3
    bc[np.isclose(y, y.max())] = 1 | 4
    mat = dict(S.material(2 * q["h"], split="amor"), E=210e9, nu=0.3, Gc=2700.0)
    om = orc.Mesh.from_plate(q)
    ost = om.new_state()
    ro = om.qs_run(mat, ost, bc, 6, 5e-7, tol=1e-10)
    m = pff.Mesh.from_plate(q, precision="fp64")
    m.set_material(mat, 0.5)
    st = m.new_state()
    r = m.qs_run(st, bc, 6, 5e-7, qopts=pff.qs_options(newton_tol=1e-10, krylov="fp32"),
                 opts=pff.options(cg_tol=1e-12))
    assert np.allclose(r["reaction"], ro["reaction"], rtol=1e-7), (r["reaction"], ro["reaction"])
    assert np.abs(to_np(st["d"]) - ost["d"]).max() <= 1e-6
