"""Pins of the oracle's mesh layer (Sec. 2.3, Eq. grad_phi; lumped mass and
CFL step of the velocity-Verlet paragraph) against closed forms, invariants
and brute force."""
import numpy as np
import pytest

import pff_synth as S


def _mesh(orc, nx=6, ny=4, jitter=0.0, seed=0):
    p = S.plate(nx, ny, jitter=jitter, seed=seed)
    return p, orc.Mesh.from_plate(p)


@pytest.mark.parametrize("jitter", [0.0, 0.1])
def test_area_sum_and_linear_reproduction(orc, jitter):
    p, m = _mesh(orc, 7, 6, jitter)
    area, grad, fext, hmin = m.geometry()
    assert np.all(area > 0)
    assert abs(area.sum() - p["Lx"] * p["Ly"]) < 1e-15
    # P1 gradients reproduce linear fields exactly: sum_a grad phi_a x_a = (1,0),
    # sum_a grad phi_a y_a = (0,1), and they sum to zero over the element.
    X = p["xy"][p["tri"]]                      # Ne x 3 x 2
    gx = np.einsum("eak,ea->ek", grad, X[:, :, 0])
    gy = np.einsum("eak,ea->ek", grad, X[:, :, 1])
    assert np.allclose(gx, [1, 0], atol=1e-9)
    assert np.allclose(gy, [0, 1], atol=1e-9)
    assert np.allclose(grad.sum(axis=1), 0, atol=1e-9)


def test_hmin_closed_form(orc):
    # right triangles with legs hx, hy: incircle diameter hx + hy - sqrt(hx^2+hy^2)
    p, m = _mesh(orc, 10, 8)
    hx, hy = p["hx"], p["hy"]
    assert abs(m.geometry()[3] - (hx + hy - np.hypot(hx, hy))) < 1e-15
    mat = S.material(2e-3)
    lam = mat["E"] * mat["nu"] / ((1 + mat["nu"]) * (1 - 2 * mat["nu"]))
    mu = mat["E"] / (2 * (1 + mat["nu"]))
    cp = np.sqrt((lam + 2 * mu) / mat["rho"])
    assert abs(m.stable_dt(mat, 0.5) - 0.5 * (hx + hy - np.hypot(hx, hy)) / cp) < 1e-20


def test_lumped_mass(orc):
    p, m = _mesh(orc, 8, 6, 0.1, seed=3)
    rho = 2450.0
    mass = m.lumped_mass(rho)
    assert abs(mass.sum() - rho * p["Lx"] * p["Ly"]) < 1e-12 * rho * p["Lx"] * p["Ly"]
    p0, m0 = _mesh(orc, 8, 6)
    m0m = m0.lumped_mass(rho)
    n = 3 * 9 + 4  # an interior node of the unjittered grid: 6 triangles
    assert abs(m0m[n] - rho * p0["hx"] * p0["hy"]) < 1e-12 * m0m[n]


def test_traction_load(orc):
    p, m = _mesh(orc, 5, 4)
    fext = m.geometry()[2]
    top = slice(4 * 6, 5 * 6)
    assert abs(fext[top, 1].sum() - 1e6 * p["Lx"]) < 1e-6
    assert abs(fext[:6, 1].sum() + 1e6 * p["Lx"]) < 1e-6
    assert abs(fext[4 * 6, 1] - 1e6 * p["hx"] / 2) < 1e-9
    assert abs(fext[4 * 6 + 2, 1] - 1e6 * p["hx"]) < 1e-9
    assert np.all(fext[:, 0] == 0)


def test_csr_brute_force(orc):
    p, m = _mesh(orc, 5, 4, 0.1)
    ptr, ent = m.csr()
    tri = p["tri"]
    for i in range(m.N):
        want = [(e << 2) | a for e in range(m.Ne) for a in range(3) if tri[e, a] == i]
        assert list(ent[ptr[i]:ptr[i + 1]]) == want


def test_colouring_valid_and_greedy(orc):
    p, m = _mesh(orc, 9, 6)
    col, ncol = m.colour()
    tri = p["tri"]
    nb = [set() for _ in range(m.Ne)]
    for e in range(m.Ne):
        for f in range(m.Ne):
            if e != f and set(tri[e]) & set(tri[f]):
                nb[e].add(f)
    # brute-force greedy in element order
    want = np.zeros(m.Ne, np.uint8)
    for e in range(m.Ne):
        used = {want[f] for f in nb[e] if f < e}
        c = 0
        while c in used:
            c += 1
        want[e] = c
    assert np.array_equal(col, want)
    assert ncol == int(col.max()) + 1
    for e in range(m.Ne):
        assert all(col[f] != col[e] for f in nb[e])


def test_inverted_element_rejected(orc):
    p = S.plate(3, 2)
    tri = p["tri"].copy()
    tri[4] = tri[4][[0, 2, 1]]
    with pytest.raises(orc.OracleError, match="element 4"):
        orc.Mesh(p["xy"], tri)


def test_ramp_closed_form(orc):
    tr = 0.05e-6
    assert orc.ramp(-1.0, tr) == 0.0 and orc.ramp(0.0, tr) == 0.0
    assert abs(orc.ramp(tr / 2, tr) - 0.5) < 1e-15
    assert abs(orc.ramp(tr / 3, tr) - 0.25) < 1e-15   # (1 - cos(pi/3)) / 2
    assert orc.ramp(tr, tr) == 1.0 and orc.ramp(5 * tr, tr) == 1.0
