"""Pins of the oracle's plane-stress constitutive law (Sec. 2.1, "Plane
assumptions"): lambda_PS = E nu / (1 - nu^2) in the spectral and isotropic
splits; the volumetric-deviatoric split keeps the 3-D bulk modulus and adds
e_zz = -nu / (1 - nu) tr to the 3-D trace, which makes the undamaged
material exactly the textbook plane-stress solid.  Checked against the
textbook plane-stress matrix, finite differences of the energy (stress and
tangent), the plane-stress wave speed and special cases."""
import math

import numpy as np
import pytest

import pff_synth as S

SPLITS = ["spectral", "amor", "iso"]


def _mat(split="amor", **kw):
    return S.material(2e-3, split=split, plane="stress", **kw)


def _dps(mat):
    E, nu = mat["E"], mat["nu"]
    return E / (1 - nu ** 2) * np.array([[1, nu, 0], [nu, 1, 0], [0, 0, (1 - nu) / 2]])


def _g1(mat):
    """Damage with g(d) = (1 - d)^2 + eta = 1 exactly: the undamaged material."""
    return 1.0 - math.sqrt(1.0 - mat["eta"])


@pytest.mark.parametrize("split", ["amor", "iso"])
def test_undamaged_is_textbook_plane_stress(orc, split):
    """sigma+ + sigma- = D_PS eps (engineering shear) and psi+ + psi- =
    1/2 eps.D_PS.eps: the out-of-plane strain e_zz = -nu/(1-nu) tr makes
    sigma_zz vanish, so the split solid is the plane-stress solid."""
    mat = _mat(split)
    D = _dps(mat)
    d1 = _g1(mat)
    rng = np.random.default_rng(10)
    for _ in range(100):
        e = rng.normal(size=3) * 1e-4
        sig, sp, pp, pm, psi = orc.constitutive(mat, e, d1)
        v = np.array([e[0], e[1], 2 * e[2]])
        want = D @ v
        assert np.allclose(sig, want, rtol=1e-10, atol=1e-10 * np.abs(want).max())
        assert abs(pp + pm - 0.5 * v @ D @ v) <= 1e-10 * (pp + pm)
        assert pp >= 0 and pm >= 0


def test_spectral_split_sum(orc):
    mat = _mat("spectral")
    E, nu = mat["E"], mat["nu"]
    lam, mu = E * nu / (1 - nu ** 2), E / (2 * (1 + nu))
    rng = np.random.default_rng(11)
    for _ in range(100):
        e = rng.normal(size=3) * 1e-4
        _, _, pp, pm, _ = orc.constitutive(mat, e)
        tr = e[0] + e[1]
        full = 0.5 * lam * tr ** 2 + mu * (e[0] ** 2 + e[1] ** 2 + 2 * e[2] ** 2)
        assert abs(pp + pm - full) <= 1e-12 * full


def test_amor_compression_degrades_only_the_deviator(orc):
    """Equibiaxial compression e = (-a, -a, 0): tr3 < 0, so psi+ is the 3-D
    deviatoric energy mu (e:e + e_zz^2 - tr3^2 / 3) with e_zz = 2 a nu/(1-nu)."""
    mat = _mat("amor")
    nu, mu = mat["nu"], mat["E"] / (2 * (1 + mat["nu"]))
    K = mat["E"] / (3 * (1 - 2 * nu))
    a = 1e-4
    _, _, pp, pm, _ = orc.constitutive(mat, [-a, -a, 0.0])
    ez = 2 * a * nu / (1 - nu)
    tr3 = -2 * a + ez
    assert abs(pp - mu * (2 * a * a + ez * ez - tr3 * tr3 / 3)) <= 1e-12 * pp
    assert abs(pm - 0.5 * K * tr3 * tr3) <= 1e-12 * pm


@pytest.mark.parametrize("split", SPLITS)
def test_stress_and_tangent_are_energy_derivatives(orc, split):
    mat = _mat(split)
    rng = np.random.default_rng(12)
    for _ in range(40):
        e = rng.normal(size=3) * 1e-3
        d = rng.uniform()
        sig = orc.constitutive(mat, e, d)[0]
        g = np.zeros(3)
        for c in range(3):
            ep = np.array(e); em = np.array(e)
            ep[c] += 1e-10; em[c] -= 1e-10
            g[c] = (orc.constitutive(mat, ep, d)[4] - orc.constitutive(mat, em, d)[4]) / 2e-10
        g[2] *= 0.5
        assert np.allclose(sig, g, rtol=1e-5, atol=1e-5 * np.abs(sig).max())
        de = rng.normal(size=3)
        ds = orc.constitutive_tangent(mat, e, d, de)
        h = 1e-7
        fd = (orc.constitutive(mat, e + h * de, d)[0] - orc.constitutive(mat, e - h * de, d)[0]) / (2 * h)
        assert np.allclose(ds, fd, rtol=1e-5, atol=1e-6 * np.abs(fd).max())


def test_nu_zero_plane_stress_equals_plane_strain(orc):
    for split in SPLITS:
        a = S.material(2e-3, split=split, plane="stress", nu=0.0)
        b = S.material(2e-3, split=split, plane="strain", nu=0.0)
        e = [3e-4, -1e-4, 2e-4]
        ra, rb = orc.constitutive(a, e, 0.3), orc.constitutive(b, e, 0.3)
        assert np.array_equal(ra[0], rb[0]) and ra[4] == rb[4]


def test_plane_stress_wave_speed_and_subcycling_limit(orc):
    """c_p = sqrt(E / (rho (1 - nu^2))) sets the CFL step; with nu = 1/3,
    c_s^2 / c_p^2 = 1/3 as for a Poisson solid in plane strain, so the
    Rayleigh root is (c_R / c_s)^2 = 2 - 2 / sqrt(3)."""
    mat = _mat("amor", nu=1.0 / 3.0)
    p = S.plate(6, 4)
    om = orc.Mesh.from_plate(p)
    cp = math.sqrt(mat["E"] / (mat["rho"] * (1 - mat["nu"] ** 2)))
    dt = om.stable_dt(mat, 0.5)
    hmin = om.geometry()[3]
    assert abs(dt - 0.5 * hmin / cp) <= 1e-14 * dt
    ratio, nmax = orc.subcycling_limit(mat)
    exact = math.sqrt(3.0) / (0.6 * math.sqrt(2.0 - 2.0 / math.sqrt(3.0)))
    assert abs(ratio - exact) <= 1e-12 * exact and nmax == 3
