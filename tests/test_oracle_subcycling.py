"""Pins of the oracle's damage subcycling (Sec. 2.4, sec:subcycling): the
pre-simulation limit N_max = floor(c_p / (0.6 c_R)) against the closed-form
Rayleigh speed of a Poisson solid and Bergmann's approximation, and the
subcycled run against the same steps taken one at a time with the damage
solve switched on only after every n_sub-th step."""
import math

import numpy as np
import pytest

import pff_synth as S


def test_rayleigh_ratio_poisson_solid(orc):
    """nu = 1/4: c_p / c_s = sqrt(3) and (c_R / c_s)^2 = 2 - 2 / sqrt(3)."""
    mat = S.material(1e-3, nu=0.25)
    ratio, nmax = orc.subcycling_limit(mat)
    exact = math.sqrt(3.0) / (0.6 * math.sqrt(2.0 - 2.0 / math.sqrt(3.0)))
    assert abs(ratio - exact) <= 1e-12 * exact
    assert nmax == 3


@pytest.mark.parametrize("nu", [0.1, 0.2, 0.3, 0.35, 0.4, 0.45])
def test_rayleigh_ratio_vs_bergmann(orc, nu):
    """c_R / c_s ~ (0.87 + 1.12 nu) / (1 + nu) (Bergmann's approximation,
    good to a few tenths of a percent), and c_p / c_s =
    sqrt(2 (1 - nu) / (1 - 2 nu)) (plane strain)."""
    ratio, nmax = orc.subcycling_limit(S.material(1e-3, nu=nu))
    cp_cs = math.sqrt(2.0 * (1.0 - nu) / (1.0 - 2.0 * nu))
    approx = cp_cs / (0.6 * (0.87 + 1.12 * nu) / (1.0 + nu))
    assert abs(ratio - approx) <= 3e-3 * approx
    assert nmax == math.floor(ratio)


def test_limit_independent_of_stiffness_and_density(orc):
    a = orc.subcycling_limit(S.material(1e-3, nu=0.3, E=32e9, rho=2450))
    b = orc.subcycling_limit(S.material(1e-3, nu=0.3, E=3e9, rho=1180))
    assert abs(a[0] - b[0]) <= 1e-12 * a[0]


@pytest.mark.parametrize("n_sub", [1, 2, 3])
def test_subcycled_run_equals_stepwise(orc, n_sub):
    p = S.plate(24, 10)
    mat = S.material(2 * p["h"])
    om = orc.Mesh.from_plate(p)
    dt = om.stable_dt(mat, 0.5)
    nsteps = 9
    a = om.new_state()
    r = om.run(mat, a, nsteps, dt, n_sub=n_sub, tol=1e-12)
    b = om.new_state()
    Hs, ds = [], []
    for n in range(nsteps):
        om.run(mat, b, 1, dt, n0=n, damage_on=((n + 1) % n_sub == 0), tol=1e-12)
        Hs.append(b["H"].copy())
        ds.append(b["d"].copy())
    for k in ("u", "v", "a", "d", "H"):
        assert np.array_equal(a[k], b[k]), k
    # no solve (iteration count 0) after the skipped steps; d frozen there
    for n in range(nsteps):
        if (n + 1) % n_sub != 0:
            assert r["iters"][n, 0] == 0
            if n > 0:
                assert np.array_equal(ds[n], ds[n - 1])
    assert r["iters"][n_sub - 1, 0] > 0  # the first solve has work
    # the history keeps growing every step
    assert all(np.all(Hs[n + 1] >= Hs[n]) for n in range(nsteps - 1))
    assert np.any(Hs[1] > Hs[0])
