"""The damage CG's per-solve entry records in both layouts: a plate whose
nodes are numbered so that some element spans 2^15 or more node ids gets
the 16-byte records (explicit neighbour ids), the same plate in its natural
numbering the compact ones (16-bit offsets).  Renumbering nodes does not
change the physics, so both runs must agree after mapping the nodes back,
for every CG family that reads the records and for the adjoint; and a mesh
whose nodes meet up to eight triangles (wider than the six-slot fast path)
against the oracle."""
import numpy as np
import pytest

import pff_synth as S
from gpu_common import rel_l2, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pff():
    import paper_2606_23458_b300 as pff
    return pff


def _renumbered(p, seed=7):
    rng = np.random.default_rng(seed)
    N = p["xy"].shape[0]
    perm = rng.permutation(N)  # new id of old node i
    inv = np.argsort(perm)     # old id of new node j
    q = dict(p)
    q["xy"] = np.ascontiguousarray(p["xy"][inv])
    q["tri"] = np.ascontiguousarray(perm[p["tri"]].astype(np.int32))
    q["notch"] = np.ascontiguousarray(p["notch"][inv])
    q["tedges"] = np.ascontiguousarray(perm[p["tedges"]].astype(np.int32))
    return q, perm


def _span(p):
    t = p["tri"].astype(np.int64)
    return int((t.max(axis=1) - t.min(axis=1)).max())


def _run(pff, p, mat, cgk, nsteps=40):
    import torch
    m = pff.Mesh.from_plate(p, precision="fp32")
    m.set_material(mat, 0.5)
    st = m.new_state()
    log = torch.zeros(nsteps, 2, dtype=torch.int32, device="cuda")
    m.run(st, nsteps, opts=pff.options(cg_tol=1e-8, cg_kernel=cgk), iters_log=log)
    torch.cuda.synchronize()
    assert m.sync_status() == 0
    return {k: to_np(st[k]) for k in ("u", "d")}, log[:, 0].cpu().numpy()


@pytest.fixture(scope="module")
def plates():
    p = S.plate(250, 150)
    q, perm = _renumbered(p)
    assert _span(p) < 2 ** 15 <= _span(q)
    return p, q, perm


@pytest.mark.parametrize("kind", ["phases", "persistent", "fused"])
def test_wide_records_match_compact(pff, plates, kind):
    p, q, perm = plates
    mat = S.material(2 * p["h"])
    cgk = {"phases": pff.PFF_CG_PHASES, "persistent": pff.PFF_CG_PERSISTENT, "fused": pff.PFF_CG_FUSED}[kind]
    a, ia = _run(pff, p, mat, pff.PFF_CG_PERSISTENT)
    b, ib = _run(pff, q, mat, cgk)
    assert np.max(np.abs(ia - ib)) <= 2, (ia, ib)
    assert rel_l2(b["u"][perm], a["u"]) <= 1e-4
    assert np.max(np.abs(b["d"][perm] - a["d"])) <= 1e-4


def test_wide_records_adjoint(pff, plates):
    import torch
    p, q, perm = plates
    mat = dict(S.material(2 * p["h"]), Gc=2.5)
    grads = []
    for pl in (p, q):
        m = pff.Mesh.from_plate(pl, precision="fp32")
        m.set_material(mat, 0.5)
        opts = pff.options(cg_tol=1e-8)
        st = m.new_state()
        ck = pff.Checkpoint(m, 20, 0)
        m.run_ckpt(st, ck, opts=opts)
        g = (2.0 * st["d"] / m.N).contiguous()
        grads.append(m.backward(ck, g, opts=opts))
        ck.close()
        torch.cuda.synchronize()
    assert abs(grads[1] - grads[0]) <= 2e-3 * abs(grads[0]), grads


def _union_jack(nx, ny):
    """A plate whose quads are split along alternating diagonals, so that
    nodes meet up to eight triangles (incidence width 8)."""
    p = S.plate(nx, ny)
    tri = []
    for j in range(ny):
        for i in range(nx):
            n00 = j * (nx + 1) + i
            n10, n01, n11 = n00 + 1, n00 + nx + 1, n00 + nx + 2
            if (i + j) % 2 == 0:
                tri += [(n00, n10, n11), (n00, n11, n01)]
            else:
                tri += [(n00, n10, n01), (n10, n11, n01)]
    q = dict(p)
    q["tri"] = np.ascontiguousarray(np.array(tri, dtype=np.int32))
    return q


@pytest.mark.parametrize("kind", ["phases", "persistent", "fused"])
def test_incidence_wider_than_six(orc, pff, kind):
    import torch
    p = _union_jack(60, 24)
    counts = np.bincount(p["tri"].ravel())
    assert counts.max() == 8
    mat = S.material(2 * p["h"])
    cgk = {"phases": pff.PFF_CG_PHASES, "persistent": pff.PFF_CG_PERSISTENT, "fused": pff.PFF_CG_FUSED}[kind]
    b, _ = _run(pff, p, mat, cgk)
    om = orc.Mesh.from_plate(p)
    dt = om.stable_dt(mat, 0.5)
    ost = om.new_state()
    om.run(mat, ost, 40, dt)
    assert rel_l2(b["u"], ost["u"]) <= 1e-4
    assert np.abs(b["d"] - ost["d"]).max() <= 1e-3
