"""GPU mesh build vs the oracle: incidence bit-exact, geometry, lumped mass,
traction load and the stable step (Sec. 2.3, Eq. grad_phi)."""
import numpy as np
import pytest

import pff_synth as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pff():
    import paper_2606_23458_b300 as pff
    return pff


CASES = [(100, 40, 0.0), (37, 18, 0.1), (1, 2, 0.0), (250, 130, 0.1)]


@pytest.mark.parametrize("nx,ny,jit", CASES)
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_mesh_matches_oracle(orc, pff, nx, ny, jit, prec):
    p = S.plate(nx, ny, jitter=jit, seed=7)
    om = orc.Mesh.from_plate(p)
    gm = pff.Mesh.from_plate(p, precision=prec)
    ptr, ent = gm.csr()
    optr, oent = om.csr()
    assert np.array_equal(ptr, optr) and np.array_equal(ent, oent)
    mat = S.material(2 * p["h"])
    dt = gm.set_material(mat, 0.5)
    assert abs(dt - om.stable_dt(mat, 0.5)) <= 1e-15 * dt
    area, grad, fext, minv = gm.geometry()
    oarea, ograd, ofext, ohmin = om.geometry()
    assert abs(gm.info()["hmin"] - ohmin) <= 1e-15 * ohmin
    assert np.allclose(area, oarea, rtol=1e-15, atol=0)
    tol = 1e-13 if prec == "fp64" else 1e-6
    assert np.abs(grad - ograd).max() <= tol * np.abs(ograd).max()
    assert np.abs(fext - ofext).max() <= tol * np.abs(ofext).max()
    om_mass = om.lumped_mass(mat["rho"])
    assert np.abs(minv * om_mass - 1).max() <= (1e-14 if prec == "fp64" else 1e-6)


def test_mesh_errors(pff):
    p = S.plate(4, 2)
    tri = p["tri"].copy()
    tri[3] = tri[3][[0, 2, 1]]
    with pytest.raises(pff.PffError, match="element 3"):
        pff.Mesh(p["xy"], tri)
    tri = p["tri"].copy()
    tri[5, 1] = 10 ** 6
    with pytest.raises(pff.PffError, match="element 5"):
        pff.Mesh(p["xy"], tri)
    with pytest.raises(pff.PffError):
        pff.Mesh(np.zeros((0, 2)), np.zeros((0, 3), np.int32))
    m = pff.Mesh.from_plate(p)
    with pytest.raises(pff.PffError, match="material"):
        m.set_material(dict(S.material(1e-3), nu=0.5))
