"""Pins of the oracle's quasi-static staggered loop (Sec. 3.5; the
matrix-free tangent of Sec. 2.3): a homogeneous bar on rollers pulled at its
top edge is in uniaxial stress, so its reaction, its damage after a
staggered step (the homogeneous AT2 solution) and the next reaction (the
degraded stiffness) have closed forms; Newton settles in two steps (the
first tangent, at zero strain, takes the volumetric part as compressive,
off by g(0) = 1 + eta)."""
import numpy as np
import pytest

import pff_synth as S


def _bar(orc, nx, ny, plane, Gc):
    p = S.plate(nx, ny, Lx=1e-3, Ly=2e-3, notch=False)
    mat = dict(S.material(2 * p["h"], split="amor", plane=plane), E=210e9, nu=0.3, Gc=Gc)
    N = p["xy"].shape[0]
    j = np.arange(N) // (nx + 1)
    bc = np.zeros(N, np.uint8)
    bc[j == 0] = 2            # rollers: u_y = 0 on the bottom edge
    bc[0] |= 1                # and u_x = 0 at one corner (no rigid motion)
    bc[j == ny] = 4           # loaded: u_y = U on the top edge, u_x free
    return p, mat, bc, orc.Mesh.from_plate(p)


def _eeff(mat, plane):
    E, nu = mat["E"], mat["nu"]
    return E / (1 - nu ** 2) if plane == "strain" else E


@pytest.mark.parametrize("plane", ["strain", "stress"])
def test_uniaxial_bar_reaction(orc, plane):
    p, mat, bc, om = _bar(orc, 6, 10, plane, 1e15)
    st = om.new_state()
    du = 1e-7
    r = om.qs_run(mat, st, bc, 3, du, tol=1e-12)
    eps = du * np.arange(1, 4) / 2e-3
    want = (1 + mat["eta"]) * _eeff(mat, plane) * eps * 1e-3
    assert np.allclose(r["reaction"], want, rtol=1e-9)
    assert r["newton"][0] <= 2 and np.all(r["newton"][1:] <= 1) and r["status"] == 0


def test_staggered_homogeneous_damage(orc):
    """AT2 with uniform H and natural boundaries: d = 2H / (Gc/l0 + 2H);
    the next increment's reaction carries g(d) on the whole stress."""
    p, mat, bc, om = _bar(orc, 6, 10, "strain", 2.7)
    st = om.new_state()
    du = 2e-7
    r = om.qs_run(mat, st, bc, 2, du, tol=1e-13)
    E = _eeff(mat, "strain")
    e1 = du / 2e-3
    H = 0.5 * E * e1 ** 2  # psi+ = psi in uniaxial tension (Amor)
    d1 = 2 * H / (mat["Gc"] / mat["l0"] + 2 * H)
    assert np.allclose(st["d"], st["d"].mean(), rtol=0, atol=1e-12)
    e2 = 2 * du / 2e-3
    H2 = 0.5 * E * e2 ** 2
    d2 = 2 * H2 / (mat["Gc"] / mat["l0"] + 2 * H2)
    assert abs(st["d"].mean() - d2) <= 1e-10 * d2
    g1 = (1 - d1) ** 2 + mat["eta"]
    assert abs(r["reaction"][1] - g1 * E * e2 * 1e-3) <= 1e-9 * r["reaction"][1]
    assert abs(r["reaction"][0] - (1 + mat["eta"]) * E * e1 * 1e-3) <= 1e-9 * r["reaction"][0]
