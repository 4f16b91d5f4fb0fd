"""Pins of the oracle's discrete adjoint (Sec. 4.2, Eqs.
implicit_forward_linear_system, implicit_adjoint_linear_system,
implicit_gc_l0_element_term) against central finite differences of the
oracle's own forward map."""
import numpy as np
import pytest

import pff_synth as S


@pytest.mark.parametrize("split", ["spectral", "amor", "iso"])
def test_elem_adjoint_is_force_jacobian_transpose(orc, split):
    p = S.plate(4, 4, Lx=1e-3, Ly=1e-3, jitter=0.1, seed=3)
    m = orc.Mesh.from_plate(p)
    mat = S.material(2e-4, split=split)
    rng = np.random.default_rng(7)
    u = rng.normal(size=(m.N, 2)) * 1e-7
    d = rng.uniform(0, 0.9, m.N)
    fbar = rng.normal(size=(m.N, 2))
    pbar = rng.normal(size=m.Ne) * 1e-9
    ub, db = m.elem_adjoint(mat, u, d, fbar, pbar)
    h = 1e-14
    for _ in range(5):
        w = rng.normal(size=(m.N, 2))
        fp, pp = m.internal_force(mat, u + h * w, d)
        fm, pm = m.internal_force(mat, u - h * w, d)
        lhs = (np.sum((fp - fm) * fbar) + np.sum((pp - pm) * pbar)) / (2 * h)
        assert abs(lhs - np.sum(w * ub)) <= 1e-5 * abs(lhs) + 1e-9
        wd = rng.normal(size=m.N)
        fp, _ = m.internal_force(mat, u, d + 1e-7 * wd)
        fm, _ = m.internal_force(mat, u, d - 1e-7 * wd)
        lhs = np.sum((fp - fm) * fbar) / 2e-7
        assert abs(lhs - np.sum(wd * db)) <= 1e-6 * abs(lhs)


def test_damage_adjoint_terms_fd(orc):
    p = S.plate(6, 4, jitter=0.1, seed=4)
    m = orc.Mesh.from_plate(p)
    mat = S.material(2e-3)
    rng = np.random.default_rng(8)
    H = rng.uniform(0, 100, m.Ne)
    lam = rng.normal(size=m.N) * (1 - p["notch"])
    xt = rng.uniform(size=m.N)
    gc, Hb = m.damage_adjoint_terms(mat, lam, xt)

    def res(Gc, H):
        mt = dict(mat, Gc=Gc)
        b, _ = m.damage_rhs(mt, H)
        return lam @ (b - m.damage_apply(mt, H, xt))

    dG = 1e-4 * mat["Gc"]
    assert abs((res(mat["Gc"] + dG, H) - res(mat["Gc"] - dG, H)) / (2 * dG) - gc) <= 1e-8 * abs(gc)
    for e in rng.choice(m.Ne, 5, replace=False):
        Hp = H.copy(); Hm = H.copy()
        Hp[e] += 1e-3; Hm[e] -= 1e-3
        fd = (res(mat["Gc"], Hp) - res(mat["Gc"], Hm)) / 2e-3
        assert abs(fd - Hb[e]) <= 1e-7 * abs(Hb).max()


@pytest.mark.slow
def test_full_adjoint_matches_central_fd(orc):
    """dL/dGc by the discrete adjoint of a 40-step run on a 20 x 8 plate
    against central FD with delta = 1e-4 Gc (CG solved to 1e-13 so that the
    forward map is smooth in Gc away from active-set switches)."""
    p = S.plate(20, 8)
    m = orc.Mesh.from_plate(p)
    mat = S.material(2 * p["h"])
    dt = m.stable_dt(mat, 0.5)
    nsteps = 40
    st = m.new_state()
    m.run(dict(mat, Gc=3.0), st, nsteps, dt, tol=1e-13)
    dstar = st["d"].copy()
    for Gc in (2.0, 3.5):
        L, g, status = m.adjoint_gc(dict(mat, Gc=Gc), nsteps, dt, dstar, tol=1e-13)
        assert status == 0 and L > 0

        def loss(G):
            s = m.new_state()
            m.run(dict(mat, Gc=G), s, nsteps, dt, tol=1e-13)
            return np.mean((s["d"] - dstar) ** 2)

        dG = 1e-4 * Gc
        fd = (loss(Gc + dG) - loss(Gc - dG)) / (2 * dG)
        assert abs(loss(Gc) - L) <= 1e-14
        assert abs(g - fd) <= 1e-4 * abs(fd), (g, fd)
