"""The paper's accuracy-parameter guide (Table 3 of Sec. 4.2.1, Sec. 4.3.1, Sec. 4.4.1): the oracle against the
values Table 2 prints and against the expressions' exact integer points; the C-ABI helper against the oracle.
Host arithmetic only (no GPU)."""
import math
import os

import numpy as np
import pytest

from oracle import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "taylor_orders_table2.txt")


def _golden_rows():
    rows = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        name, tol, mac, pt, pd, pc, kt = line.split()
        rows.append((name, float(tol), float(mac), pt, pd, pc, float(kt)))
    return rows


@pytest.mark.parametrize("row", _golden_rows(), ids=lambda r: r[0])
def test_oracle_reproduces_table2(row):
    """Table 2's orders for the guide's solutes at tolerance 1e-6 (2, 6, 6), its MAC and, within the factor
    the paper's "approximately" allows, its reciprocal-space cut-off tolerance."""
    name, tol, mac, pt, pd, pc, kt = row
    g = O.parameter_guide(tol)
    assert g["mac"] == mac and g["n0"] == 500
    for key, want in (("p_tcf", pt), ("p_dcf", pd), ("p_coulomb", pc)):
        if want != "-":
            assert g[key] == int(want), (name, key)
    assert kt / 2 <= g["k_tol"] <= kt * 2, name


def test_oracle_orders_at_exact_points_and_clamp():
    """Where an expression is an integer the order is that integer; just beyond it, one more; above the
    tolerance where every expression falls below 2, the floor of 2 holds."""
    # TCF: (log10 t + 5.7) / -0.7 = 3 at log10 t = -7.8; DCF: (log10 t + 1.9) / -0.8 = 7 at -7.5;
    # Coulomb: (log10 t + 1.4) / -0.8 = 5 at -5.4
    assert O.parameter_guide(10 ** -7.8)["p_tcf"] == 3
    assert O.parameter_guide(10 ** -7.81)["p_tcf"] == 4
    assert O.parameter_guide(10 ** -7.5)["p_dcf"] == 7
    assert O.parameter_guide(10 ** -7.51)["p_dcf"] == 8
    assert O.parameter_guide(10 ** -5.4)["p_coulomb"] == 5
    assert O.parameter_guide(10 ** -5.41)["p_coulomb"] == 6
    g = O.parameter_guide(0.5)
    assert (g["p_tcf"], g["p_dcf"], g["p_coulomb"]) == (2, 2, 2)


def test_oracle_cutoff_tolerances():
    """Sec. 4.3.1: 0.04 tolerance^0.9, about a tenth of the tolerance near 1e-6; Sec. 4.4.1: one tenth."""
    for t in (1e-3, 1e-6, 1e-9):
        g = O.parameter_guide(t)
        assert g["lj_tol"] == pytest.approx(t / 10, rel=1e-15)
        assert g["k_tol"] == pytest.approx(0.04 * math.exp(0.9 * math.log(t)), rel=1e-13)
    assert 0.1 < O.parameter_guide(1e-6)["k_tol"] / 1e-6 < 0.2


def test_capi_guide_matches_oracle():
    from paper_2109_09772_gb300 import build as B
    from paper_2109_09772_gb300 import rism as R

    B.build()
    for e in np.arange(-0.5, -12.01, -0.05):
        t = float(10 ** e)
        got, ref = R.parameter_guide(t), O.parameter_guide(t)
        for k in ("p_tcf", "p_dcf", "p_coulomb", "n0"):
            assert got[k] == ref[k], (t, k)
        for k in ("mac", "k_tol", "lj_tol"):
            assert got[k] == pytest.approx(ref[k], rel=1e-14), (t, k)
    for bad in (0.0, 1.0, -1e-6, 2.0, float("nan"), float("inf")):
        with pytest.raises(R.RismError) as e:
            R.parameter_guide(bad)
        assert e.value.status == R.E_INVALID
