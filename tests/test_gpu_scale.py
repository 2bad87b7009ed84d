"""GPU parity at the full sizes of the benchmark workloads, in the launch configuration bench.py times
(treecode, FP32 pairs, degree 8, theta 0.7, autotuned launch shape), through the C ABI:

* the 2,000-atom globule on 128^3: every grid point of u, c, h against the FP64 oracle, element by element;
* the 13,600-atom ellipsoid on 224x192x160: sampled points and the point nearest each atom;
* the LJ cut-off boundary: pairs whose membership FP32 rounding of d^2 can flip, with the discrepancy bounded
  by |u_LJ(r_c)| per flipped pair (FP64 paths decide it exactly);
* rism_potential and rism_asymptotics called by name.
Tolerances: rel L2 and max-abs error / max |ref| per output grid, over all points and over points >= 1 A from
every atom: 1e-5 for the treecode, 1e-6 for FP32 direct sums, 1e-12 for FP64 direct sums.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2109_09772_gb300 import inputs as I
from tests.helpers import check_fields, lj_boundary_pairs, nearest_points, rel_l2

pytestmark = pytest.mark.gpu

TREE_TOL = 1e-5


@pytest.fixture(scope="module")
def R():
    import torch

    from paper_2109_09772_gb300 import build as B
    from paper_2109_09772_gb300 import rism

    B.build()
    torch.cuda.set_device(0)
    return rism


def _bench_context(R, w):
    """The context bench.py times: treecode, FP32 pairs, autotuned launch shape."""
    return R.from_workload(w, method=R.METHOD_TREECODE, precision=R.PREC_FP32, autotune=1)


def test_globule2000_every_point_against_oracle(R):
    w = I.workload(1)
    ref = O.fields(O.Problem.from_workload(w))
    r = _bench_context(R, w)
    r.init()  # the autotuner times its candidates on the first call
    out = r.init(lj_tail=True)
    S = r.S
    g = {k: out[k].cpu().numpy().reshape(S, -1) for k in ("u", "c", "h")}
    r.close()
    check_fields(g, ref, ("u", "c", "h"), TREE_TOL, w.grid, w.solute.xyz, label="cfg1 full grid")
    np.testing.assert_allclose(out["lj_tail"], O.lj_tail(O.Problem.from_workload(w)), rtol=1e-12)


def test_ellipsoid13600_sampled_against_oracle(R):
    w = I.workload(2)
    idx = np.union1d(I.sample_indices(w.grid.npts, 20000, seed=21), nearest_points(w.grid, w.solute.xyz))
    ref = O.fields(O.Problem.from_workload(w), idx=idx)
    r = _bench_context(R, w)
    r.init()
    out = r.init()
    import torch

    t = torch.as_tensor(idx, device="cuda")
    g = {k: out[k].reshape(r.S, -1)[:, t].cpu().numpy() for k in ("u", "c", "h")}
    r.close()
    check_fields(g, ref, ("u", "c", "h"), TREE_TOL, w.grid, w.solute.xyz, idx=idx, label="cfg2 sampled")


@pytest.mark.parametrize("method", ["direct_fp32", "treecode", "direct_fp64"])
def test_lj_cutoff_boundary_pairs(R, method):
    """Points that have an atom within FP32 rounding of the 9 A cut-off.  The FP32 paths decide membership on
    an FP32 d^2 and may flip such a pair; each flip moves u_s by |u_LJ,is(r_c)| at most.  The FP64 path decides
    it as the oracle does (d < r_c)."""
    import torch

    w = I.workload(1)
    rc = float(w.opts["lj_rcut"])
    pts, ats = lj_boundary_pairs(w.grid, w.solute.xyz, rc)
    assert pts.size > 0
    idx = np.unique(pts)
    p = O.Problem.from_workload(w)
    ref = O.fields(p, idx=idx, want=("u",))["u"]
    if method == "treecode":
        r = _bench_context(R, w)
        r.init(u=True, c=False, h=False)
    else:
        r = R.from_workload(w, method=R.METHOD_DIRECT,
                            precision=R.PREC_FP32 if method == "direct_fp32" else R.PREC_FP64)
    out = r.init(u=True, c=False, h=False)
    got = out["u"].reshape(r.S, -1)[:, torch.as_tensor(idx, device="cuda")].cpu().numpy()
    r.close()
    # |u_LJ(r_c)| per (site, boundary pair), Lorentz-Berthelot, summed per point
    bound = np.zeros((w.solvent.nsite, idx.size))
    pos = np.searchsorted(idx, pts)
    for s in range(w.solvent.nsite):
        sg = 0.5 * (w.solute.sigma[ats] + w.solvent.sigma[s])
        ep = np.sqrt(w.solute.eps[ats] * w.solvent.eps[s])
        sr6 = (sg / rc) ** 6
        np.add.at(bound[s], pos, np.abs(4.0 * ep * (sr6 * sr6 - sr6)))
    err = np.abs(got - ref)
    if method == "direct_fp64":
        assert np.all(err <= 1e-10 * np.abs(ref) + 1e-12), float(err.max())
    else:
        # rounding of the FP32 pair sums (direct), or the treecode's interpolation error (1e-5 of the grid's
        # scale), plus |u_LJ(r_c)| for every pair that may have flipped
        scale = np.sqrt(np.mean(ref ** 2, axis=1, keepdims=True))
        noise = 2e-6 * np.abs(ref) + (1e-5 if method == "treecode" else 1e-7) * scale
        assert np.all(err <= noise + 1.01 * bound), float((err - noise - bound).max())


def test_potential_and_asymptotics_by_name(R):
    """rism_potential (u + LJ tail) and rism_asymptotics (c, h) agree with rism_init's grids and with the
    oracle within the FP32 tolerance."""
    w = I.small_workload(n_atoms=150, n=(37, 21, 13), h=0.45, seed=5, ions=True, lj_rcut=4.0, net=2.0)
    ref = O.fields(O.Problem.from_workload(w))
    for method in (R.METHOD_DIRECT, R.METHOD_TREECODE):
        r = R.from_workload(w, method=method, precision=R.PREC_FP32)
        fused = r.init(lj_tail=True)
        u, tail = r.potential(lj_tail=True)
        c, h = r.asymptotics()
        S = r.S
        # the kernels are specialised on the requested outputs, so the fused call and the separate ones may
        # round differently: they agree to the FP32 tolerance
        for k, v in (("u", u), ("c", c), ("h", h)):
            a, b = v.cpu().numpy(), fused[k].cpu().numpy()
            assert rel_l2(a, b) <= 1e-6, (k, rel_l2(a, b))
        np.testing.assert_array_equal(tail, fused["lj_tail"])
        g = {"u": u.cpu().numpy().reshape(S, -1), "c": c.cpu().numpy().reshape(S, -1),
             "h": h.cpu().numpy().reshape(S, -1)}
        check_fields(g, ref, ("u", "c", "h"), 1e-6, w.grid, w.solute.xyz, label=f"by name, method {method}")
        r.close()
