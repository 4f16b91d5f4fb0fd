"""Quasi-static staggered mode on the GPU (Sec. 3.5; the matrix-free
tangent of Sec. 2.3) against the oracle: the uniaxial bar's closed-form
reactions and a small single-edge-notched tension run increment by
increment (reactions, damage)."""
import numpy as np
import pytest

import pff_synth as S
from gpu_common import to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pff():
    import paper_2606_23458_b300 as pff
    return pff


def _sent(nx, ny, notch=True, rollers=False):
    p = S.plate(nx, ny, Lx=1e-3, Ly=1e-3 if notch else 2e-3, notch=notch)
    N = p["xy"].shape[0]
    j = np.arange(N) // (nx + 1)
    bc = np.zeros(N, np.uint8)
    if rollers:
        bc[j == 0] = 2
        bc[0] |= 1
        bc[j == ny] = 4
    else:
        bc[j == 0] = 3       # bottom edge clamped
        bc[j == ny] = 1 | 4  # top edge: u_x = 0, u_y = U
    return p, bc


@pytest.mark.parametrize("prec,krylov", [("fp64", "fp32"), ("fp64", "mesh"), ("fp32", "fp32")])
def test_uniaxial_bar_reaction(pff, prec, krylov):
    p, bc = _sent(6, 10, notch=False, rollers=True)
    mat = dict(S.material(2 * p["h"], split="amor"), E=210e9, nu=0.3, Gc=1e15)
    m = pff.Mesh.from_plate(p, precision=prec)
    m.set_material(mat, 0.5)
    st = m.new_state()
    du = 1e-7
    r = m.qs_run(st, bc, 3, du, newton_tol=1e-10 if prec == "fp64" else 1e-5, krylov=krylov)
    eps = du * np.arange(1, 4) / 2e-3
    want = (1 + mat["eta"]) * mat["E"] / (1 - mat["nu"] ** 2) * eps * 1e-3
    tol = 1e-9 if prec == "fp64" else 1e-5
    assert np.allclose(r["reaction"], want, rtol=tol), (r["reaction"], want)


@pytest.mark.parametrize("prec,krylov,tol", [("fp64", "fp32", 1e-7), ("fp64", "mesh", 1e-7), ("fp32", "fp32", 2e-3)])
def test_sent_increments_match_oracle(orc, pff, prec, krylov, tol):
    p, bc = _sent(16, 16)
    mat = dict(S.material(2 * p["h"], split="amor"), E=210e9, nu=0.3, Gc=2700.0)
    om = orc.Mesh.from_plate(p)
    ost = om.new_state()
    nincr, du = 8, 5e-7
    ro = om.qs_run(mat, ost, bc, nincr, du, tol=1e-10)
    m = pff.Mesh.from_plate(p, precision=prec)
    m.set_material(mat, 0.5)
    st = m.new_state()
    opts = pff.options(cg_tol=1e-12 if prec == "fp64" else 1e-8)
    q = pff.qs_options(newton_tol=1e-10 if prec == "fp64" else 1e-5, krylov=krylov)
    r = m.qs_run(st, bc, nincr, du, qopts=q, opts=opts)
    assert np.allclose(r["reaction"], ro["reaction"], rtol=tol), (r["reaction"], ro["reaction"])
    d = to_np(st["d"])
    assert np.abs(d - ost["d"]).max() <= 10 * tol
    assert np.all(r["iters"][:, 0] >= 1) and np.all(r["iters"][:, 1] > 0)
    # split over two calls: the same increments
    st2 = m.new_state()
    a = m.qs_run(st2, bc, 3, du, qopts=q, opts=opts)
    b = m.qs_run(st2, bc, nincr - 3, du, incr0=3, qopts=q, opts=opts)
    assert np.allclose(np.concatenate([a["reaction"], b["reaction"]]), r["reaction"], rtol=1e-12)


def test_options_are_checked(pff):
    p, bc = _sent(4, 4)
    m = pff.Mesh.from_plate(p, precision="fp64")
    m.set_material(dict(S.material(2 * p["h"], split="amor"), E=210e9, nu=0.3, Gc=2700.0), 0.5)
    st = m.new_state()
    for kw in (dict(newton_tol=0.0), dict(eta_min=0.6), dict(eta_max=1.0), dict(newton_max=0)):
        with pytest.raises(pff.PffError):
            m.qs_run(st, bc, 1, 1e-7, **kw)


def test_row_and_element_forms_agree(pff):
    """The FP32 tangent CG runs in row form (per-slot pair blocks) when the
    mesh's elements span fewer than 2^15 node ids, else in element form;
    the same SENT plate, once in its natural numbering and once renumbered
    by a random permutation, gives the same reactions and damage."""
    import torch
    p, bc = _sent(200, 200)
    rng = np.random.default_rng(3)
    N = p["xy"].shape[0]
    perm = rng.permutation(N)
    inv = np.argsort(perm)
    q = dict(p, xy=np.ascontiguousarray(p["xy"][inv]), tri=np.ascontiguousarray(perm[p["tri"]].astype(np.int32)),
             notch=np.ascontiguousarray(p["notch"][inv]),
             tedges=np.ascontiguousarray(perm[p["tedges"]].astype(np.int32)))
    t = q["tri"].astype(np.int64)
    assert int((t.max(axis=1) - t.min(axis=1)).max()) >= 2 ** 15
    mat = dict(S.material(2 * p["h"], split="amor"), E=210e9, nu=0.3, Gc=2700.0)
    out = []
    for pl, b in ((p, bc), (q, bc[inv])):
        m = pff.Mesh.from_plate(pl, precision="fp64")
        m.set_material(mat, 0.5)
        st = m.new_state()
        r = m.qs_run(st, b, 3, 2e-7, newton_tol=1e-8, opts=pff.options(cg_tol=1e-10))
        torch.cuda.synchronize()
        out.append((r["reaction"], to_np(st["d"])))
    assert np.allclose(out[1][0], out[0][0], rtol=1e-6), (out[0][0], out[1][0])
    assert np.max(np.abs(out[1][1][perm] - out[0][1])) <= 1e-6
