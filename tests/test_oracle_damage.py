"""Pins of the oracle's damage solve: the matrix-free operator against a
dense assembly built from the cotangent formula (Eq. assembled_fe_operator
with textbook P1 entries), the AT2/AT1 solutions against closed forms
(uniform history, the 1-D profiles of Fig. regularization_schematic and the
AT1 threshold of Sec. 2.1), and the projected CG against a bound-constrained
QP solved by scipy."""
import numpy as np
import pytest
import scipy.linalg as sla
import scipy.optimize as so

import pff_synth as S


def _dense_damage_operator(p, mat, H):
    """A = sum_e [kappa K^e + c_e M^e] with K^e from cotangents:
    K_ab = -cot(theta_c)/2 (c the third vertex), K_aa = -sum of the row;
    M^e = A_e (1 + delta_ab) / 12."""
    xy, tri = p["xy"], p["tri"]
    N = xy.shape[0]
    cross = lambda u, v: u[0] * v[1] - u[1] * v[0]
    at1 = mat["model"] == "AT1"
    kap = (0.75 if at1 else 1.0) * mat["Gc"] * mat["l0"]
    A = np.zeros((N, N))
    b = np.zeros(N)
    for e, t in enumerate(tri):
        P = xy[t]
        area = 0.5 * abs(cross(P[1] - P[0], P[2] - P[0]))
        Ke = np.zeros((3, 3))
        for a in range(3):
            bb, c = (a + 1) % 3, (a + 2) % 3
            u, v = P[bb] - P[a], P[c] - P[a]
            cot = np.dot(u, v) / abs(cross(u, v))   # angle at vertex a, opposite edge (bb, c)
            Ke[bb, c] = Ke[c, bb] = -0.5 * cot
        for a in range(3):
            Ke[a, a] = -Ke[a].sum()
        Me = area * (np.ones((3, 3)) + np.eye(3)) / 12
        ce = 2 * H[e] if at1 else mat["Gc"] / mat["l0"] + 2 * H[e]
        we = 2 * H[e] - (3 * mat["Gc"] / (8 * mat["l0"]) if at1 else 0.0)
        A[np.ix_(t, t)] += kap * Ke + ce * Me
        b[t] += we * area / 3
    return A, b


@pytest.mark.parametrize("model", ["AT2", "AT1"])
def test_matvec_and_rhs_match_dense_assembly(orc, model):
    p = S.plate(6, 4, jitter=0.1, seed=4)
    m = orc.Mesh.from_plate(p)
    mat = S.material(2e-3, model=model)
    rng = np.random.default_rng(0)
    H = rng.uniform(0, 50, m.Ne)
    A, b = _dense_damage_operator(p, mat, H)
    x = rng.normal(size=m.N)
    q = m.damage_apply(mat, H, x)
    assert np.allclose(q, A @ x, rtol=1e-12, atol=1e-12 * np.abs(A @ x).max())
    bo, dg = m.damage_rhs(mat, H)
    assert np.allclose(bo, b, rtol=1e-12, atol=1e-15)
    assert np.allclose(dg, np.diag(A), rtol=1e-12)


def test_at2_solve_matches_cholesky(orc):
    p = S.plate(10, 6, jitter=0.1, seed=6)
    m = orc.Mesh.from_plate(p)
    mat = S.material(2e-3)
    rng = np.random.default_rng(1)
    H = rng.uniform(0, 3000, m.Ne)
    A, b = _dense_damage_operator(p, mat, H)
    D = p["notch"].astype(bool)
    F = ~D
    x = np.ones(m.N)
    x[F] = sla.cho_solve(sla.cho_factor(A[np.ix_(F, F)]), b[F] - A[np.ix_(F, D)] @ np.ones(D.sum()))
    dprev = np.zeros(m.N)
    d, info, rel, st, xo = m.damage_solve(mat, H, dprev, tol=1e-14)
    assert st == 0 and rel <= 1e-14
    assert np.abs(xo - x).max() <= 1e-12
    assert np.array_equal(d, np.minimum(1, np.maximum(xo, dprev)) * F + D)
    # the natural stop count at tol 1e-8 is what an unforced run reports
    d8, info8, rel8, _, _ = m.damage_solve(mat, H, dprev, tol=1e-8)
    assert rel8 <= 1e-8 and info8[0] == info8[1]
    # forcing the count reproduces the natural run exactly
    df, infof, _, _, _ = m.damage_solve(mat, H, dprev, tol=1e-8, forced=int(info8[0]))
    assert np.array_equal(df, d8)


def test_at2_clamp(orc):
    p = S.plate(8, 4, jitter=0.1, seed=8)
    m = orc.Mesh.from_plate(p)
    mat = S.material(2e-3)
    rng = np.random.default_rng(2)
    H = rng.uniform(0, 100, m.Ne)
    dprev = rng.uniform(0, 0.5, m.N) * (1 - p["notch"]) + p["notch"]
    d, info, rel, st, x = m.damage_solve(mat, H, dprev, tol=1e-12)
    assert np.all(d >= dprev) and np.all(d <= 1)
    assert np.all(d[p["notch"] == 1] == 1)
    assert np.any(x < dprev)   # the clamp was active somewhere


@pytest.mark.parametrize("Hval", [5.0, 400.0, 3e4])
def test_at2_uniform_history(orc, Hval):
    """No notch, uniform H: (Gc/l0 + 2H) d = 2H has the constant solution."""
    p = S.plate(8, 6, jitter=0.1, seed=1, notch=False)
    m = orc.Mesh.from_plate(p)
    mat = S.material(2e-3)
    d, info, rel, st, _ = m.damage_solve(mat, np.full(m.Ne, Hval), np.zeros(m.N), tol=1e-13)
    want = 2 * Hval / (mat["Gc"] / mat["l0"] + 2 * Hval)
    assert np.abs(d - want).max() <= 1e-12


@pytest.mark.parametrize("ratio", [0.5, 0.99, 1.5, 4.0])
def test_at1_uniform_history_and_threshold(orc, ratio):
    """AT1 with uniform H: d = 0 below H_crit = 3Gc/(16 l0) (the elastic
    threshold), d = 1 - H_crit/H above it."""
    p = S.plate(8, 6, jitter=0.1, seed=1, notch=False)
    m = orc.Mesh.from_plate(p)
    mat = S.material(2e-3, model="AT1")
    Hc = 3 * mat["Gc"] / (16 * mat["l0"])
    d, info, rel, st, _ = m.damage_solve(mat, np.full(m.Ne, ratio * Hc), np.zeros(m.N), tol=1e-13)
    assert st == 0
    want = max(0.0, 1 - 1 / ratio)
    assert np.abs(d - want).max() <= 1e-11


def _strip(ny, l0=None, Lx=None, W=0.01):
    """Strip [0, Lx] x [0, 2W] with the whole mid-row held at d = 1."""
    hy = 2 * W / ny
    nx = 8
    Lx = Lx or nx * hy
    p = S.plate(nx, ny, Lx=Lx, Ly=2 * W, notch=False)
    p["notch"][(ny // 2) * (nx + 1):(ny // 2 + 1) * (nx + 1)] = 1
    return p


def test_at2_profile_1d(orc):
    """H = 0, d = 1 on the mid-line: the continuum solution on a strip of
    half-width W is cosh((W - n)/l0) / cosh(W/l0) (-> exp(-n/l0)) and the
    regularised length per unit crack length is tanh(W/l0) (-> 1).  The
    discrete error converges at O(h^2)."""
    W, l0 = 0.01, 1e-3
    errs, lens = [], []
    for ny in (40, 80, 160):
        p = _strip(ny, W=W)
        m = orc.Mesh.from_plate(p)
        mat = S.material(l0)
        d, info, rel, st, _ = m.damage_solve(mat, np.zeros(m.Ne), p["notch"].astype(float), tol=1e-13)
        assert st == 0
        nx = p["nx"]
        col = np.arange(ny + 1) * (nx + 1) + nx // 2
        n = np.abs(p["xy"][col, 1] - W)
        exact = np.cosh((W - n) / l0) / np.cosh(W / l0)
        errs.append(np.abs(d[col] - exact).max())
        Efr = m.energies(mat, np.zeros((m.N, 2)), np.zeros((m.N, 2)), d)[2]
        lens.append(Efr / (mat["Gc"] * p["Lx"]))
    assert errs[0] < 2e-2
    assert 3.3 < errs[0] / errs[1] < 4.7 and 3.3 < errs[1] / errs[2] < 4.7
    t = np.tanh(W / l0)
    le = [abs(L - t) for L in lens]
    assert le[2] < 2e-3 and le[0] / le[1] > 3.0


def test_at1_profile_1d(orc):
    """AT1, H = 0, d = 1 on the mid-line: d = <1 - n/(2 l0)>_+^2 with compact
    support and regularised length exactly 1."""
    W, l0 = 0.01, 1e-3
    errs, lens = [], []
    for ny in (40, 80, 160):
        p = _strip(ny, W=W)
        m = orc.Mesh.from_plate(p)
        mat = S.material(l0, model="AT1")
        d, info, rel, st, _ = m.damage_solve(mat, np.zeros(m.Ne), p["notch"].astype(float),
                                             tol=1e-13, max_restarts=500, max_it=100000)
        assert st == 0
        nx = p["nx"]
        col = np.arange(ny + 1) * (nx + 1) + nx // 2
        n = np.abs(p["xy"][col, 1] - W)
        exact = np.maximum(0, 1 - n / (2 * l0)) ** 2
        errs.append(np.abs(d[col] - exact).max())
        Efr = m.energies(mat, np.zeros((m.N, 2)), np.zeros((m.N, 2)), d)[2]
        lens.append(Efr / (mat["Gc"] * p["Lx"]))
        assert np.all(d[col][n > 2 * l0 + 2 * W / ny] == 0)   # compact support
    # with 2 l0 on a grid line the P1 solution of this 1-D obstacle problem is
    # nodally exact (constant d'' on the support)
    assert max(errs) < 1e-10, errs
    assert abs(lens[2] - 1) < 2e-3 and abs(lens[0] - 1) >= abs(lens[2] - 1), lens


def test_at1_matches_bound_constrained_qp(orc):
    """The projected CG solves min 1/2 x^T A x - b^T x on [d_prev, 1] with the
    notch eliminated; compare with L-BFGS-B on the same quadratic."""
    p = S.plate(8, 6, jitter=0.1, seed=12)
    m = orc.Mesh.from_plate(p)
    mat = S.material(2e-3, model="AT1")
    rng = np.random.default_rng(5)
    Hc = 3 * mat["Gc"] / (16 * mat["l0"])
    H = rng.uniform(0, 3 * Hc, m.Ne)
    dprev = (rng.uniform(0, 0.3, m.N) * (rng.uniform(size=m.N) < 0.3)) * (1 - p["notch"]) + p["notch"]
    A, b = _dense_damage_operator(p, mat, H)
    D = p["notch"].astype(bool)
    F = ~D
    AFF = A[np.ix_(F, F)]
    bF = b[F] - A[np.ix_(F, D)] @ np.ones(D.sum())
    res = so.minimize(lambda x: (0.5 * x @ AFF @ x - bF @ x, AFF @ x - bF), dprev[F], jac=True,
                      method="L-BFGS-B", bounds=list(zip(dprev[F], np.ones(F.sum()))),
                      options=dict(ftol=1e-16, gtol=1e-14, maxiter=100000))
    d, info, rel, st, _ = m.damage_solve(mat, H, dprev, tol=1e-12, max_restarts=500)
    assert st == 0
    assert np.abs(d[F] - res.x).max() < 1e-6
    # KKT: gradient g = A x - b is 0 on free nodes, >= 0 at lower, <= 0 at upper
    g = AFF @ d[F] - bF
    lo, hi = d[F] <= dprev[F], d[F] >= 1
    free = ~lo & ~hi
    sc = np.abs(bF).max()
    assert np.abs(g[free]).max() <= 1e-9 * sc
    assert np.all(g[lo] >= -1e-9 * sc) and np.all(g[hi] <= 1e-9 * sc)
