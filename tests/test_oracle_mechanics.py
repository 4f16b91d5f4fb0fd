"""Pins of the oracle's mechanics: energy splits (Eqs. spectral_split,
amor_split), degradation, internal force (Sec. 2.3) and velocity Verlet
(Eqs. vv_u, vv_a, vv_v), checked against textbook formulas, finite
differences of the strain energy, the patch test, the exact discrete
Verlet solution of a linear mode and energy conservation."""
import numpy as np
import pytest
import scipy.linalg as sla

import pff_synth as S

SPLITS = ["spectral", "amor", "iso"]


def _mat(split="spectral", **kw):
    return S.material(2e-3, split=split, **kw)


def _lame(mat):
    E, nu = mat["E"], mat["nu"]
    return E * nu / ((1 + nu) * (1 - 2 * nu)), E / (2 * (1 + nu)), E / (3 * (1 - 2 * nu))


def _tensor_energy_grad(orc, mat, e, which, h=1e-9):
    """Central FD of psi+ (which=2) / psi- (3) / psi (4) w.r.t. the tensor
    components; the shear derivative is halved because exy appears twice."""
    g = np.zeros(3)
    for c in range(3):
        ep = np.array(e, float); em = np.array(e, float)
        ep[c] += h; em[c] -= h
        g[c] = (orc.constitutive(mat, ep)[which] - orc.constitutive(mat, em)[which]) / (2 * h)
    g[2] *= 0.5
    return g


@pytest.mark.parametrize("split", SPLITS)
def test_split_sum_is_full_energy(orc, split):
    mat = _mat(split)
    lam, mu, K = _lame(mat)
    rng = np.random.default_rng(0)
    for _ in range(200):
        e = rng.normal(size=3) * 1e-4
        _, _, pp, pm, _ = orc.constitutive(mat, e)
        tr = e[0] + e[1]
        full = 0.5 * lam * tr ** 2 + mu * (e[0] ** 2 + e[1] ** 2 + 2 * e[2] ** 2)
        assert abs(pp + pm - full) <= 1e-12 * full
        assert pp >= 0 and pm >= 0


@pytest.mark.parametrize("split", SPLITS)
def test_stress_is_energy_gradient(orc, split):
    mat = _mat(split)
    rng = np.random.default_rng(1)
    for _ in range(50):
        e = rng.normal(size=3) * 1e-3
        d = rng.uniform()
        sig, sp, pp, pm, psi = orc.constitutive(mat, e, d)
        gp = _tensor_energy_grad(orc, mat, e, 2, 1e-10)
        # sigma+ = d psi+/d eps
        assert np.allclose(sp, gp, rtol=1e-5, atol=1e-5 * np.abs(sp).max())
        # sigma = g(d) sigma+ + sigma- = d psi/d eps at fixed d
        g = np.zeros(3)
        for c in range(3):
            ep = np.array(e); em = np.array(e)
            ep[c] += 1e-10; em[c] -= 1e-10
            g[c] = (orc.constitutive(mat, ep, d)[4] - orc.constitutive(mat, em, d)[4]) / 2e-10
        g[2] *= 0.5
        assert np.allclose(sig, g, rtol=1e-5, atol=1e-5 * np.abs(sig).max())


def test_spectral_special_cases(orc):
    mat = _mat("spectral")
    lam, mu, _ = _lame(mat)
    # equibiaxial tension: all energy tensile; compression: all compressive
    _, _, pp, pm, _ = orc.constitutive(mat, [1e-4, 1e-4, 0])
    assert pm == 0 and abs(pp - (0.5 * lam * 4e-8 + mu * 2e-8)) < 1e-12 * pp
    _, _, pp, pm, _ = orc.constitutive(mat, [-1e-4, -1e-4, 0])
    assert pp == 0 and pm > 0
    # uniaxial tension with principal axes rotated 45 deg: eps = [[a/2, a/2],[a/2, a/2]]
    a = 2e-4
    _, sp, pp, pm, _ = orc.constitutive(mat, [a / 2, a / 2, a / 2])
    assert pm == 0 and abs(pp - (0.5 * lam * a * a + mu * a * a)) < 1e-12 * pp
    # pure shear: eigenvalues +-s, trace 0: psi+ = mu s^2 = psi-
    s = 1e-4
    _, _, pp, pm, _ = orc.constitutive(mat, [0, 0, s])
    assert abs(pp - mu * s * s) < 1e-12 * pp and abs(pm - mu * s * s) < 1e-12 * pm


def test_amor_special_cases(orc):
    mat = _mat("amor")
    _, mu, K = _lame(mat)
    # pure shear is fully deviatoric: psi+ = 2 mu exy^2, psi- = 0
    s = 1e-4
    _, _, pp, pm, _ = orc.constitutive(mat, [0, 0, s])
    assert pm == 0 and abs(pp - 2 * mu * s * s) < 1e-12 * pp
    # equibiaxial compression: the volumetric part is psi-
    c = -1e-4
    _, _, pp, pm, _ = orc.constitutive(mat, [c, c, 0])
    assert abs(pm - 0.5 * K * (2 * c) ** 2) < 1e-12 * pm
    # 3-D deviator of diag(c, c, 0): (c/3)^2 * 2 + (2c/3)^2 = 2c^2/3
    assert abs(pp - mu * 2 * c * c / 3) < 1e-12 * pp


def test_plane_strain_lame_closed_form(orc):
    # nu = 1/4 gives lambda = mu = 2E/5 in plane strain
    mat = _mat("iso", nu=0.25)
    sig, *_ = orc.constitutive(mat, [1e-4, 0, 0])
    E = mat["E"]
    # sigma_xx = (lambda + 2 mu) e, sigma_yy = lambda e
    assert abs(sig[0] - (1 + 1e-7) * 3 * (E / 2.5) * 1e-4) < 1e-9 * abs(sig[0])
    assert abs(sig[1] - (1 + 1e-7) * (E / 2.5) * 1e-4) < 1e-9 * abs(sig[1])


def test_textbook_plane_strain_D(orc):
    """Isotropic split at d = 0: sigma = (1+eta) D eps_voigt with the textbook
    plane-strain D (engineering shear strain)."""
    mat = _mat("iso")
    E, nu = mat["E"], mat["nu"]
    D = E / ((1 + nu) * (1 - 2 * nu)) * np.array(
        [[1 - nu, nu, 0], [nu, 1 - nu, 0], [0, 0, (1 - 2 * nu) / 2]])
    rng = np.random.default_rng(2)
    for _ in range(20):
        e = rng.normal(size=3) * 1e-4
        sig = orc.constitutive(mat, e, 0.0)[0]
        want = (1 + 1e-7) * D @ np.array([e[0], e[1], 2 * e[2]])
        assert np.allclose(sig, want, rtol=1e-12, atol=1e-9)


def test_degradation(orc):
    mat = _mat("spectral")
    e = [2e-4, -1e-4, 5e-5]
    _, sp, pp, pm, _ = orc.constitutive(mat, e, 0.0)
    sig1, _, _, _, psi1 = orc.constitutive(mat, e, 1.0)
    sigm = orc.constitutive(mat, e, 0.0)[0] - (1 + 1e-7) * sp
    assert np.allclose(sig1, 1e-7 * sp + sigm, rtol=1e-12, atol=1e-6)
    assert abs(psi1 - (1e-7 * pp + pm)) < 1e-12 * (pp + pm)
    sighalf = orc.constitutive(mat, e, 0.5)[0]
    assert np.allclose(sighalf, (0.25 + 1e-7) * sp + sigm, rtol=1e-12, atol=1e-6)


@pytest.mark.parametrize("split", SPLITS)
def test_tangent_matches_fd(orc, split):
    mat = _mat(split)
    rng = np.random.default_rng(3)
    for _ in range(40):
        e = rng.normal(size=3) * 1e-3
        d = rng.uniform()
        de = rng.normal(size=3)
        ds = orc.constitutive_tangent(mat, e, d, de)
        h = 1e-7
        fd = (orc.constitutive(mat, e + h * de, d)[0] - orc.constitutive(mat, e - h * de, d)[0]) / (2 * h)
        assert np.allclose(ds, fd, rtol=1e-5, atol=1e-6 * np.abs(fd).max())
        # symmetry of the tangent (Hessian of psi): <de2, C de> = <de, C de2>
        de2 = rng.normal(size=3)
        ds2 = orc.constitutive_tangent(mat, e, d, de2)
        ip = lambda s, t: s[0] * t[0] + s[1] * t[1] + 2 * s[2] * t[2]
        assert abs(ip(de2, ds) - ip(de, ds2)) <= 1e-9 * abs(ip(de2, ds)) + 1e-3


def test_patch_test(orc):
    """Uniform strain gives zero force at every interior node."""
    p = S.plate(8, 6, jitter=0.1, seed=5)
    m = orc.Mesh.from_plate(p)
    for split in SPLITS:
        mat = _mat(split)
        x, y = p["xy"][:, 0], p["xy"][:, 1]
        u = np.stack([1e-4 * x + 3e-5 * y, -2e-5 * x + 5e-5 * y], axis=1)
        d = np.zeros(m.N)
        f, _ = m.internal_force(mat, u, d)
        interior = (x > 0) & (x < p["Lx"]) & (y > 0) & (y < p["Ly"])
        scale = np.abs(f).max()
        assert scale > 0
        assert np.abs(f[interior]).max() <= 1e-12 * scale
        # rigid motion (translation + infinitesimal rotation) gives no force at all
        ur = np.stack([1e-3 - 1e-5 * y, 2e-3 + 1e-5 * x], axis=1)
        fr, _ = m.internal_force(mat, ur, d)
        assert np.abs(fr).max() <= 1e-9 * scale  # roundoff of the 1e-3 translation


@pytest.mark.parametrize("split", SPLITS)
@pytest.mark.parametrize("n", [2, 3])
def test_force_is_energy_gradient(orc, split, n):
    """f_int = d/du sum_e A_e psi(eps_e, dbar_e) by central FD on tiny meshes."""
    p = S.plate(n, 2, Lx=1e-3, Ly=1e-3, jitter=0.1, seed=n, notch=False)
    m = orc.Mesh.from_plate(p)
    mat = _mat(split)
    rng = np.random.default_rng(n)
    u = rng.normal(size=(m.N, 2)) * 1e-7
    d = rng.uniform(0, 0.9, size=m.N)
    f, _ = m.internal_force(mat, u, d)
    z = np.zeros((m.N, 2))
    h = 1e-13
    fd = np.zeros_like(f)
    for i in range(m.N):
        for c in range(2):
            up = u.copy(); um = u.copy()
            up[i, c] += h; um[i, c] -= h
            fd[i, c] = (m.energies(mat, up, z, d)[0] - m.energies(mat, um, z, d)[0]) / (2 * h)
    assert np.allclose(f, fd, rtol=1e-5, atol=1e-6 * np.abs(f).max())


def _cst_stiffness(p, mat):
    """Textbook CST assembly K = sum_e A_e B_e^T D B_e (engineering strain)."""
    E, nu = mat["E"], mat["nu"]
    D = E / ((1 + nu) * (1 - 2 * nu)) * np.array(
        [[1 - nu, nu, 0], [nu, 1 - nu, 0], [0, 0, (1 - 2 * nu) / 2]])
    xy, tri = p["xy"], p["tri"]
    N = xy.shape[0]
    K = np.zeros((2 * N, 2 * N))
    for t in tri:
        (x1, y1), (x2, y2), (x3, y3) = xy[t]
        A2 = (x2 - x1) * (y3 - y1) - (x3 - x1) * (y2 - y1)
        b = np.array([y2 - y3, y3 - y1, y1 - y2]) / A2
        c = np.array([x3 - x2, x1 - x3, x2 - x1]) / A2
        B = np.zeros((3, 6))
        B[0, 0::2] = b; B[1, 1::2] = c; B[2, 0::2] = c; B[2, 1::2] = b
        Ke = 0.5 * A2 * B.T @ D @ B
        dofs = np.ravel([[2 * t[a], 2 * t[a] + 1] for a in range(3)])
        K[np.ix_(dofs, dofs)] += Ke
    return K


def test_cst_stiffness(orc):
    p = S.plate(4, 4, jitter=0.1, seed=7, notch=False)
    m = orc.Mesh.from_plate(p)
    mat = _mat("iso")
    K = _cst_stiffness(p, mat)
    rng = np.random.default_rng(4)
    u = rng.normal(size=(m.N, 2)) * 1e-6
    f, _ = m.internal_force(mat, u, np.zeros(m.N))
    assert np.allclose(f.ravel(), (1 + 1e-7) * K @ u.ravel(), rtol=1e-10, atol=1e-10 * np.abs(f).max())


def test_verlet_exact_mode(orc):
    """Linear system (iso split, d = 0, no load): starting from a generalised
    eigenmode phi (K phi = w^2 M phi) at rest, velocity Verlet gives exactly
    u_n = cos(n theta) phi with cos(theta) = 1 - w^2 dt^2 / 2."""
    p = S.plate(4, 2, jitter=0.1, seed=9, notch=False)
    p["tedges"] = p["tedges"][:0]; p["tvec"] = p["tvec"][:0]
    m = orc.Mesh.from_plate(p)
    mat = _mat("iso", eta=0.0)
    K = _cst_stiffness(p, mat)
    mass = np.repeat(m.lumped_mass(mat["rho"]), 2)
    w2, V = sla.eigh(K, np.diag(mass))
    k = 7
    phi = V[:, k] * 1e-6 / np.abs(V[:, k]).max()
    dt = 0.5 * m.stable_dt(mat, 1.0)
    theta = np.arccos(1 - w2[k] * dt * dt / 2)
    st = dict(u=phi.reshape(-1, 2).copy(), v=np.zeros((m.N, 2)), d=np.zeros(m.N),
              H=np.zeros(m.Ne))
    f0, _ = m.internal_force(mat, st["u"], st["d"])
    st["a"] = -f0 / mass.reshape(-1, 2)
    nsteps = 25
    m.run(mat, st, nsteps, dt, damage_on=False)
    want = np.cos(nsteps * theta) * phi.reshape(-1, 2)
    assert np.abs(st["u"] - want).max() <= 1e-9 * np.abs(phi).max()


def test_energy_conservation_second_order(orc):
    """Undamaged free vibration: the energy error of velocity Verlet is
    O(dt^2): halving dt divides the max drift by ~4."""
    p = S.plate(12, 8, jitter=0.1, seed=11, notch=False)
    p["tedges"] = p["tedges"][:0]; p["tvec"] = p["tvec"][:0]
    m = orc.Mesh.from_plate(p)
    mat = _mat("spectral")
    x, y = p["xy"][:, 0] / p["Lx"], p["xy"][:, 1] / p["Ly"]
    u0 = np.stack([np.sin(np.pi * x) * np.cos(np.pi * y), 0.5 * np.sin(2 * np.pi * y) * x],
                  axis=1) * 1e-6
    dt0 = m.stable_dt(mat, 0.5)
    T = 80 * dt0
    drifts = []
    for k in (1, 2, 4):
        dt = dt0 / k
        st = dict(u=u0.copy(), v=np.zeros((m.N, 2)), d=np.zeros(m.N), H=np.zeros(m.Ne))
        mass = m.lumped_mass(mat["rho"])
        f0, _ = m.internal_force(mat, st["u"], st["d"])
        st["a"] = -f0 / mass[:, None]
        E0 = m.energies(mat, st["u"], st["v"], st["d"])[:2].sum()
        r = m.run(mat, st, 80 * k, dt, damage_on=False, energy_every=1)
        E = r["energies"][:, 0] + r["energies"][:, 1]
        drifts.append(np.abs(E - E0).max() / E0)
    assert drifts[0] < 3e-2
    assert 3.2 < drifts[0] / drifts[1] < 4.8
    assert 3.2 < drifts[1] / drifts[2] < 4.8


def test_energy_closed_forms(orc):
    p = S.plate(6, 4, jitter=0.1, seed=2, notch=False)
    m = orc.Mesh.from_plate(p)
    A = p["Lx"] * p["Ly"]
    for model in ("AT2", "AT1"):
        mat = S.material(2e-3, model=model)
        v = np.tile([3.0, -4.0], (m.N, 1))
        x, y = p["xy"][:, 0], p["xy"][:, 1]
        e = np.array([1e-4, -3e-5, 2e-5])
        u = np.stack([e[0] * x + e[2] * y, e[2] * x + e[1] * y], axis=1)
        c = 0.3
        Eel, Ekin, Efr = m.energies(mat, u, v, np.full(m.N, c))
        psi = orc.constitutive(mat, e, c)[4]
        assert abs(Ekin - 0.5 * mat["rho"] * A * 25.0) < 1e-12 * Ekin
        assert abs(Eel - A * psi) < 1e-12 * Eel
        want = mat["Gc"] * A * (c * c / (2 * mat["l0"]) if model == "AT2" else 0.375 * c / mat["l0"])
        assert abs(Efr - want) < 1e-12 * want
