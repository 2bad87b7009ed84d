"""GPU parity of the all-space long-range integral (rism_lra_integral: the last integral of
eq. (excess-chemical-potential-LRA), an O(N_atom^2) sum over atom pairs) against the FP64 oracle, whose pair
overlaps are 1D wave-number quadratures.  Tolerance: rel L2 1e-6 for the per-atom sums and for T (FP32 pair
terms with float-float sums)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2109_09772_gb300 import inputs as I
from tests.helpers import max_abs_rel, rel_l2

pytestmark = pytest.mark.gpu

TOL = 1e-6


@pytest.fixture(scope="module")
def R():
    import torch

    from paper_2109_09772_gb300 import build as B
    from paper_2109_09772_gb300 import rism

    B.build()
    torch.cuda.set_device(0)
    return rism


def _check_atoms(got, ref, label):
    for k, name in ((0, "P_hc"), (1, "P_hh")):
        e = rel_l2(got[:, k], ref[:, k])
        assert e <= TOL, f"{label} {name}: rel L2 {e:.3e}"
        m = max_abs_rel(got[:, k], ref[:, k])
        assert m <= TOL, f"{label} {name}: max-abs / max {m:.3e}"


@pytest.mark.parametrize("method", ["direct", "treecode"])
def test_small_all_atoms_and_total(R, method):
    w = I.small_workload(n_atoms=150, n=(37, 21, 13), h=0.45, seed=5, ions=True, lj_rcut=4.0, net=2.0)
    r = R.from_workload(w, method=R.METHOD_DIRECT if method == "direct" else R.METHOD_TREECODE,
                        precision=R.PREC_FP32)
    T, a = r.lra_integral(atom_sums=True)
    got = a.cpu().numpy()
    # host output buffer: the same values
    hb = np.zeros((w.solute.n, 2))
    r._check(r.lib.rism_lra_integral(r.ctx, np.zeros(r.S).ctypes.data, hb.ctypes.data), "rism_lra_integral")
    np.testing.assert_array_equal(hb, got)
    r.close()
    p = O.Problem.from_workload(w)
    ref = O.lra_atom_sums(p, np.arange(w.solute.n))
    _check_atoms(got, ref, "150 atoms")
    Tref, _ = O.lra_integral(p)
    assert rel_l2(T, Tref) <= TOL, (T, Tref)


def test_globule2000_total(R):
    w = I.workload(1)
    r = R.from_workload(w, method=R.METHOD_TREECODE, precision=R.PREC_FP32)
    T = r.lra_integral()
    r.close()
    Tref, _ = O.lra_integral(O.Problem.from_workload(w))
    assert rel_l2(T, Tref) <= TOL, (T, Tref)
    np.testing.assert_allclose(T, Tref, rtol=TOL)


def test_ellipsoid13600_sampled_atoms(R):
    w = I.workload(2)
    r = R.from_workload(w, method=R.METHOD_TREECODE, precision=R.PREC_FP32)
    T, a = r.lra_integral(atom_sums=True)
    got = a.cpu().numpy()
    r.close()
    atoms = np.sort(np.random.default_rng(13).choice(w.solute.n, 64, replace=False))
    ref = O.lra_atom_sums(O.Problem.from_workload(w), atoms)
    _check_atoms(got[atoms], ref, "13,600 atoms, 64 sampled")
    assert np.all(np.isfinite(T))


def test_edge_cases(R):
    """No ionic screening: zero.  No atoms: zero.  Two atoms at one position take the R = 0 overlap."""
    w = I.small_workload(n_atoms=12, n=(8, 8, 8), h=0.5, seed=2, ions=False)
    r = R.from_workload(w, method=R.METHOD_DIRECT, precision=R.PREC_FP32)
    T, a = r.lra_integral(atom_sums=True)
    assert np.all(T == 0.0) and float(a.abs().max()) == 0.0
    r.close()
    w = I.small_workload(n_atoms=12, n=(8, 8, 8), h=0.5, seed=2, ions=True)
    w.solute.xyz[5] = w.solute.xyz[3]
    r = R.from_workload(w, method=R.METHOD_DIRECT, precision=R.PREC_FP32)
    T, a = r.lra_integral(atom_sums=True)
    p = O.Problem.from_workload(w)
    _check_atoms(a.cpu().numpy(), O.lra_atom_sums(p, np.arange(12)), "coincident atoms")
    assert rel_l2(T, O.lra_integral(p)[0]) <= TOL
    r.set_solute(np.zeros((0, 3)), [], [], [])
    assert np.all(r.lra_integral() == 0.0)
    r.close()
