"""Pins of the oracle's per-element toughness field and its gradient (the
field-valued inverse of Secs. 4.2 and 7; per-element terms of Eq.
implicit_gc_l0_element_term): a uniform field is the scalar Gc, the
per-element gradient sums to dL/dGc, and matches central finite differences
of the loss, element by element and along a region."""
import numpy as np
import pytest

import pff_synth as S


def _problem(orc):
    p = S.plate(20, 8)
    mat = S.material(2 * p["h"])
    om = orc.Mesh.from_plate(p)
    dt = om.stable_dt(mat, 0.5)
    nsteps = 30
    st = om.new_state()
    om.run(dict(mat, Gc=3.0), st, nsteps, dt, tol=1e-13)
    return p, mat, om, dt, nsteps, st["d"].copy()


def test_uniform_field_is_the_scalar_toughness(orc):
    p, mat, om, dt, nsteps, dstar = _problem(orc)
    m2 = dict(mat, Gc=2.5)
    a = om.new_state()
    om.run(m2, a, nsteps, dt, tol=1e-13)
    om.set_gc_field(np.full(om.Ne, 2.5))
    b = om.new_state()
    om.run(m2, b, nsteps, dt, tol=1e-13)
    L1, g1, _, ge = om.adjoint_gc(m2, nsteps, dt, dstar, tol=1e-13, field=True)
    om.set_gc_field(None)
    L0, g0, _ = om.adjoint_gc(m2, nsteps, dt, dstar, tol=1e-13)
    for k in ("u", "v", "a", "d", "H"):
        assert np.array_equal(a[k], b[k]), k
    assert L1 == L0 and g1 == g0
    assert abs(ge.sum() - g0) <= 1e-12 * abs(g0)


def test_field_changes_the_solution(orc):
    p, mat, om, dt, nsteps, dstar = _problem(orc)
    cx = p["xy"][p["tri"]].mean(axis=1)[:, 0]
    gc = np.where(cx < 0.5 * cx.max(), 2.0, 6.0)
    om.set_gc_field(gc)
    a = om.new_state()
    om.run(mat, a, nsteps, dt, tol=1e-13)
    om.set_gc_field(None)
    b = om.new_state()
    om.run(dict(mat, Gc=2.0), b, nsteps, dt, tol=1e-13)
    # tougher right half: less damage there, the same mechanics before damage acts
    right = p["xy"][:, 0] > 0.6 * p["xy"][:, 0].max()
    assert a["d"][right].sum() < b["d"][right].sum()


def test_per_element_gradient_vs_central_fd(orc):
    p, mat, om, dt, nsteps, dstar = _problem(orc)
    gc0 = np.full(om.Ne, 2.5)
    cx = p["xy"][p["tri"]].mean(axis=1)[:, 0]
    gc0 *= 1.0 + 0.2 * np.sin(40.0 * cx)  # a non-uniform field
    om.set_gc_field(gc0)
    L, g, st, ge = om.adjoint_gc(dict(mat, Gc=2.5), nsteps, dt, dstar, tol=1e-13, field=True)
    assert st == 0
    pick = np.argsort(-np.abs(ge))[:4]

    def loss(gc):
        om.set_gc_field(gc)
        s = om.new_state()
        om.run(dict(mat, Gc=2.5), s, nsteps, dt, tol=1e-13)
        return np.mean((s["d"] - dstar) ** 2)

    for e in pick:
        h = 1e-4 * gc0[e]
        gp = gc0.copy(); gp[e] += h
        gm = gc0.copy(); gm[e] -= h
        fd = (loss(gp) - loss(gm)) / (2 * h)
        assert abs(fd - ge[e]) <= 2e-4 * abs(ge[e]), (e, fd, ge[e])
    # along a region: the directional derivative is the region's sum
    region = (cx > 0.3 * cx.max()) & (cx < 0.7 * cx.max())
    h = 1e-4
    fd = (loss(gc0 * (1 + h * region)) - loss(gc0 * (1 - h * region))) / (2 * h)
    want = float(np.sum(ge[region] * gc0[region]))
    assert abs(fd - want) <= 2e-4 * abs(want), (fd, want)
    om.set_gc_field(None)
