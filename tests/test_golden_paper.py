"""Values the paper prints (tests/golden/paper_benchmarks.json, each with its
citation): the materials of the synthetic workloads are those of Table
benchmark_overview, and the pre-simulation subcycling check of Sec. 2.4
gives the paper's integer limit for PMMA and c_p close to 3 x (0.6 c_R)
for the glass of the dynamic benchmarks (oracle and library alike)."""
import json
import os

import pytest

import pff_synth as S

HERE = os.path.dirname(os.path.abspath(__file__))
G = json.load(open(os.path.join(HERE, "golden", "paper_benchmarks.json")))


def _si(row):
    return dict(E=row["E_GPa"] * 1e9, nu=row["nu"], Gc=row["Gc_N_per_mm"] * 1e3)


def test_glass_plates_use_the_table_material():
    g = G["materials"]["glass"]
    m = S.material(1e-3)
    want = _si(g)
    assert m["E"] == pytest.approx(want["E"]) and m["nu"] == pytest.approx(want["nu"])
    assert m["rho"] == pytest.approx(g["rho_kg_m3"]) and m["Gc"] == pytest.approx(want["Gc"])


def test_sent_uses_the_table_material():
    q = _si(G["materials"]["steel_sent"])
    m = S.sent(20)["material"]
    assert m["E"] == pytest.approx(q["E"]) and m["nu"] == pytest.approx(q["nu"]) and m["Gc"] == pytest.approx(q["Gc"])


def test_subcycling_limits(orc):
    p = G["materials"]["pmma"]
    pmma = S.material(1e-4, split="amor", model="AT1", plane=p["plane"], E=p["E_GPa"] * 1e9, nu=p["nu"],
                      rho=p["rho_kg_m3"], Gc=p["Gc_N_per_mm"] * 1e3)
    ratio, n_max = orc.subcycling_limit(pmma)
    assert n_max == G["subcycling"]["pmma_n_max"], ratio
    glass = S.material(1e-3)
    r_glass, _ = orc.subcycling_limit(glass)
    assert abs(r_glass - G["subcycling"]["cp_over_06cR_approx"]) <= 0.05 * G["subcycling"]["cp_over_06cR_approx"]
    # the library's host-side check agrees with the oracle's
    import paper_2606_23458_b300 as pff
    assert pff.subcycling_limit(pmma)[1] == n_max
    assert pff.subcycling_limit(glass)[0] == pytest.approx(r_glass, rel=1e-10)
