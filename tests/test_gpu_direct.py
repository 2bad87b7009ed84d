"""GPU parity of the direct-sum path against the FP64 oracle (through the C ABI).

Tolerances: relative L2 per output grid <= 1e-12 for FP64 pairs, <= 1e-6 for
FP32 pairs with compensated accumulation, over all points and over the points
at least 1 A from every atom.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2109_09772_gb300 import inputs as I
from tests.helpers import check_fields, nearest_points, rel_l2

pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 1: 1e-6}  # precision -> rel L2


@pytest.fixture(scope="module")
def R():
    import torch

    from paper_2109_09772_gb300 import build as B
    from paper_2109_09772_gb300 import rism

    B.build()
    torch.cuda.set_device(0)
    return rism


def run(R, w, keys=("u", "c", "h"), **opts):
    r = R.from_workload(w, method=R.METHOD_DIRECT, **opts)
    out = r.init(u="u" in keys, c="c" in keys, h="h" in keys, lj_tail=True)
    res = {k: out[k].cpu().numpy().reshape(r.S, -1) for k in keys}
    res["lj_tail"] = out["lj_tail"]
    res["info"] = r.info()
    r.close()
    return res


@pytest.mark.parametrize("prec", [0, 1])
def test_small_ragged_all_outputs(R, prec):
    """Grid 37x21x13 (not a multiple of the 32x4x4 CTA tile), 150 atoms (3 atom tiles, ragged), 4 sites."""
    w = I.small_workload(n_atoms=150, n=(37, 21, 13), h=0.45, seed=5, ions=True, lj_rcut=4.0, net=2.0)
    p = O.Problem.from_workload(w)
    ref = O.fields(p)
    g = run(R, w, precision=prec)
    check_fields(g, ref, ("u", "c", "h"), TOL[prec], w.grid, w.solute.xyz, label=f"prec{prec}")
    np.testing.assert_allclose(g["lj_tail"], O.lj_tail(p), rtol=1e-12)
    if prec == 0:
        for k in ("u", "c", "h"):
            scale = np.abs(ref[k]).max()
            np.testing.assert_allclose(g[k], ref[k], rtol=1e-10, atol=1e-13 * scale)


@pytest.mark.parametrize("prec", [0, 1])
def test_sphere200_64cubed_full_grid(R, prec):
    """200 atoms in a 12 A sphere, 64^3 grid at 0.5 A, water sites, no LJ cut-off, no ions: u and c."""
    w = I.workload(0)
    ref = O.fields(O.Problem.from_workload(w), want=("u", "c"))
    g = run(R, w, keys=("u", "c"), precision=prec)
    check_fields(g, ref, ("u", "c"), TOL[prec], w.grid, w.solute.xyz, label=f"cfg0 prec{prec}")


@pytest.mark.parametrize("prec", [0, 1])
def test_globule2000_128cubed_sampled(R, prec):
    """2,000-atom globule, 128^3 grid, 4 sites, LJ cut-off 9 A: full GPU grids, oracle at sampled points
    (random points plus the grid point nearest to each atom, where |u| peaks)."""
    w = I.workload(1)
    idx = np.union1d(I.sample_indices(w.grid.npts, 3000, seed=2), nearest_points(w.grid, w.solute.xyz))
    ref = O.fields(O.Problem.from_workload(w), idx=idx)
    g = run(R, w, precision=prec)
    gs = {k: g[k][:, idx] for k in ("u", "c", "h")}
    check_fields(gs, ref, ("u", "c", "h"), TOL[prec], w.grid, w.solute.xyz, idx=idx, label=f"cfg1 prec{prec}")


@pytest.mark.parametrize("mode", ["none", "rcut", "tol"])
def test_lj_truncation_modes(R, mode):
    kw = {"none": dict(lj_rcut=0.0), "rcut": dict(lj_rcut=3.7), "tol": dict(lj_rcut=0.0, lj_tol=1e-3)}[mode]
    w = I.small_workload(n_atoms=70, n=(24, 18, 16), h=0.5, seed=9, ions=True, **{k: v for k, v in kw.items()
                                                                                    if k == "lj_rcut"})
    if mode == "tol":
        w.opts["lj_tol"] = 1e-3
    p = O.Problem.from_workload(w)
    ref = O.fields(p, want=("u",))
    g = run(R, w, keys=("u",), precision=0)
    if mode == "tol":
        # a per-pair cut-off found by bisection on each side may differ by an ulp; a pair exactly at it would
        # flip by |u(rc)| = tol, far below the tolerance used here
        assert rel_l2(g["u"], ref["u"]) <= 1e-12
    else:
        check_fields(g, ref, ("u",), 1e-12, w.grid, w.solute.xyz, label=mode)
    np.testing.assert_allclose(g["lj_tail"], O.lj_tail(p), rtol=1e-9)


@pytest.mark.parametrize("prec", [0, 1])
def test_grid_point_on_an_atom(R, prec):
    """An atom exactly on a grid point: u = +inf there, c and h finite and equal to the d -> 0 limits."""
    w = I.small_workload(n_atoms=20, n=(16, 12, 10), h=0.5, seed=4, ions=True, lj_rcut=5.0)
    w.solute.xyz[3] = np.array(w.grid.origin) + 0.5 * np.array([7, 5, 4])
    ref = O.fields(O.Problem.from_workload(w))
    g = run(R, w, precision=prec)
    f = (4 * 12 + 5) * 16 + 7
    assert np.all(np.isposinf(g["u"][:, f])) and np.all(np.isposinf(ref["u"][:, f]))
    keep = np.ones(g["u"].shape[1], dtype=bool)
    keep[f] = False
    assert rel_l2(g["u"][:, keep], ref["u"][:, keep]) <= TOL[prec]
    for k in ("c", "h"):
        assert np.all(np.isfinite(g[k]))
        assert rel_l2(g[k], ref[k]) <= TOL[prec]


def test_zero_atoms_gives_zero_grids(R):
    w = I.small_workload(n_atoms=5, n=(8, 8, 8), ions=True)
    r = R.from_workload(w, method=R.METHOD_DIRECT)
    r.set_solute(np.zeros((0, 3)), [], [], [])
    out = r.init(lj_tail=True)
    for k in ("u", "c", "h"):
        assert float(out[k].abs().max()) == 0.0
    assert np.all(out["lj_tail"] == 0.0)
    r.close()


def test_host_outputs_equal_device_outputs(R):
    w = I.small_workload(n_atoms=90, n=(20, 17, 9), h=0.5, seed=12, ions=True, lj_rcut=4.0)
    r = R.from_workload(w, method=R.METHOD_DIRECT, precision=R.PREC_FP32)
    dev = r.init(lj_tail=True)
    S, M = r.S, r.npts
    hu, hc, hh, tail = np.empty((S, M)), np.empty((S, M)), np.empty((S, M)), np.empty(S)
    r.init_host(hu, hc, hh, tail)
    np.testing.assert_array_equal(hu, dev["u"].cpu().numpy().reshape(S, M))
    np.testing.assert_array_equal(hc, dev["c"].cpu().numpy().reshape(S, M))
    np.testing.assert_array_equal(hh, dev["h"].cpu().numpy().reshape(S, M))
    np.testing.assert_array_equal(tail, dev["lj_tail"])
    r.close()


def test_repeatable_bitwise(R):
    w = I.small_workload(n_atoms=130, n=(21, 19, 8), h=0.5, seed=13, ions=True, lj_rcut=4.0)
    a = run(R, w, precision=1)
    b = run(R, w, precision=1)
    for k in ("u", "c", "h"):
        assert np.array_equal(a[k], b[k])


def test_status_codes(R):
    import torch

    w = I.small_workload(n_atoms=10, n=(8, 8, 8), ions=False)
    r = R.Rism(w.grid.n, w.grid.h, w.grid.origin, method=R.METHOD_DIRECT)
    with pytest.raises(R.RismError) as e:
        r.init()
    assert e.value.status == R.E_STATE
    r.set_solvent(w.solvent.q, w.solvent.sigma, w.solvent.eps, w.solvent.rho, w.solvent.is_ion)
    bad = w.solute.xyz.copy()
    bad[2, 1] = np.nan
    with pytest.raises(R.RismError) as e:
        r.set_solute(bad, w.solute.q, w.solute.sigma, w.solute.eps)
    assert e.value.status == R.E_INVALID
    neg = w.solute.sigma.copy()
    neg[0] = -1.0
    with pytest.raises(R.RismError) as e:
        r.set_solute(w.solute.xyz, w.solute.q, neg, w.solute.eps)
    assert e.value.status == R.E_INVALID
    r.set_solute(w.solute.xyz, w.solute.q, w.solute.sigma, w.solute.eps)
    with pytest.raises(R.RismError) as e:  # no ionic site: kappa = 0, h is undefined
        r.init(u=True, c=True, h=True)
    assert e.value.status == R.E_INVALID
    out = r.init(u=True, c=True, h=False)
    assert torch.isfinite(out["c"]).all()
    with pytest.raises(R.RismError) as e:
        r.set_solvent(np.zeros(9), np.ones(9), np.ones(9))
    assert e.value.status == R.E_INVALID
    r.close()


def test_bounded_wait_timeout_is_reported_and_context_survives(R):
    """The debug hook withholds the first bulk copy: the kernel's bounded wait runs out, it records the
    error and returns; the call reports RISM_E_TIMEOUT and the same context then computes normally."""
    w = I.small_workload(n_atoms=150, n=(16, 8, 8), h=0.5, seed=3, ions=True, lj_rcut=4.0)
    r = R.from_workload(w, method=R.METHOD_DIRECT, precision=R.PREC_FP32, debug_flags=1, wait_limit=2000)
    for _ in range(2):  # a second call reports the same status: no sticky CUDA error was left behind
        with pytest.raises(R.RismError) as e:
            r.init()
        assert e.value.status == R.E_TIMEOUT
    r.close()
    r = R.from_workload(w, method=R.METHOD_DIRECT, precision=R.PREC_FP32)
    out = r.init()
    ref = O.fields(O.Problem.from_workload(w))
    for k in ("u", "c", "h"):
        assert rel_l2(out[k].cpu().numpy().reshape(r.S, -1), ref[k]) <= 1e-6
    r.close()
