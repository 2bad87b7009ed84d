"""GPU Taylor far field (RISM_APPROX_TAYLOR: the target boxes take the order-p Taylor moments of the paper's
cluster-particle treecode, Sec. 2.3, with the recurrences of Sec. 2.3.2 / Sec. 2.4 for 1/d and e^{-kappa d}/d)
against the FP64 oracle.  The Taylor expansion converges more slowly in the acceptance parameter than the
barycentric proxies, so its tests use theta 0.5 (and order 10 at theta 0.6); the tolerance is the treecode's
1e-5.  Error must fall geometrically with the order."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2109_09772_gb300 import inputs as I
from tests.helpers import check_fields, nearest_points, rel_l2

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


def run(R, w, keys=("u", "c", "h"), **opts):
    r = R.from_workload(w, method=R.METHOD_TREECODE, precision=R.PREC_FP32, approx=R.APPROX_TAYLOR, **opts)
    out = r.init(u="u" in keys, c="c" in keys, h="h" in keys)
    res = {k: out[k].cpu().numpy().reshape(r.S, -1) for k in keys}
    res["info"] = r.info()
    r.close()
    return res


@pytest.mark.parametrize("degree,theta", [(8, 0.5), (10, 0.6)])
def test_globule2000_against_oracle(R, degree, theta):
    w = I.workload(1)
    idx = np.union1d(I.sample_indices(w.grid.npts, 3000, seed=2), nearest_points(w.grid, w.solute.xyz))
    ref = O.fields(O.Problem.from_workload(w), idx=idx)
    g = run(R, w, degree=degree, theta=theta)
    assert g["info"]["cp_pairs"] > 0 and g["info"]["tree_boxes"] > 0
    check_fields({k: g[k][:, idx] for k in ("u", "c", "h")}, ref, ("u", "c", "h"), TREE_TOL, w.grid, w.solute.xyz,
                 idx=idx, label=f"taylor p{degree} theta{theta}")


def test_error_falls_geometrically_with_the_order(R):
    w = I.workload(1)
    idx = I.sample_indices(w.grid.npts, 2000, seed=3)
    ref = O.fields(O.Problem.from_workload(w), idx=idx, want=("c", "h"))
    errs = []
    for p in (2, 4, 6, 8):
        g = run(R, w, keys=("c", "h"), degree=p, theta=0.5)
        errs.append(max(rel_l2(g["c"][:, idx], ref["c"]), rel_l2(g["h"][:, idx], ref["h"])))
    assert errs[0] > errs[1] > errs[2] > errs[3], errs
    assert errs[0] / errs[3] > 100.0, errs


def test_clipped_boxes_and_repeatable(R):
    """A 150x37x70 grid whose boxes are clipped and partly too thin for an expansion; two runs agree bit for
    bit; every point against the oracle."""
    w = I.small_workload(n_atoms=500, n=(150, 37, 70), h=0.5, seed=29, ions=True, lj_rcut=5.0, net=1.0)
    w.solute.xyz[:, 0] -= 10.0
    a = run(R, w, degree=10, theta=0.5)
    b = run(R, w, degree=10, theta=0.5)
    for k in ("u", "c", "h"):
        assert np.array_equal(a[k], b[k]), k
    assert a["info"]["tree_boxes"] > 0
    ref = O.fields(O.Problem.from_workload(w))
    check_fields(a, ref, ("u", "c", "h"), TREE_TOL, w.grid, w.solute.xyz, label="taylor clipped")


def test_taylor_needs_the_target_boxes(R):
    w = I.small_workload(n_atoms=20, n=(16, 16, 16), h=0.5, seed=2, ions=True)
    for opts in (dict(method=R.METHOD_DIRECT), dict(method=R.METHOD_TREECODE, target_proxies=0)):
        with pytest.raises(R.RismError) as e:
            R.Rism(w.grid.n, w.grid.h, w.grid.origin, approx=R.APPROX_TAYLOR, **opts)
        assert e.value.status == R.E_UNSUPPORTED


def test_reverse_mode_in_taylor_context(R):
    """The reverse mode of a Taylor context (its far part runs as a direct sum) against the oracle gradient."""
    import torch

    w = I.small_workload(n_atoms=60, n=(26, 22, 18), h=0.5, seed=31, ions=True, lj_rcut=4.0, net=1.0)
    nx, ny, nz = w.grid.n
    G = {k: np.stack([I.gaussian_random_field((nz, ny, nx), w.grid.h, 5 + 10 * i + s, corr_len=1.5)
                      for s in range(w.solvent.nsite)]) for i, k in enumerate(("u", "c", "h"))}
    r = R.from_workload(w, method=R.METHOD_TREECODE, precision=R.PREC_FP32, approx=R.APPROX_TAYLOR)
    r.init()
    g = r.backward(*(torch.as_tensor(G[k], device="cuda") for k in ("u", "c", "h")))
    r.close()
    atoms = np.arange(w.solute.n)
    ref = O.grad(O.Problem.from_workload(w), atoms, G["u"], G["c"], G["h"])
    for k, v in (("xyz", ref[:, 0:3]), ("q", ref[:, 3]), ("sigma", ref[:, 4]), ("eps", ref[:, 5])):
        assert rel_l2(g[k].cpu().numpy()[atoms], v) <= 2e-5, k


def test_parameter_guide_applied(R):
    """The paper's guide at a residual tolerance of 1e-6 (Table 3: Taylor orders 2 / 6 / 6 for h / c / u, so
    one order 6 for every moment, MAC 0.3; Sec. 4.4.1: per-pair LJ cut-offs at |u_LJ(r_cut)| = 1e-7): every
    output within ten times the tolerance (TREE_TOL, 1e-5) of the FP64 oracle with the same LJ cut-offs (the
    relation between error and residual tolerance of eq. (error-tolerance))."""
    w0 = I.workload(1)
    gd = R.parameter_guide(1e-6)
    assert (gd["p_tcf"], gd["p_dcf"], gd["p_coulomb"], gd["mac"]) == (2, 6, 6, 0.3)
    w = I.Workload(w0.name, w0.solute, w0.solvent, w0.grid, dict(w0.opts, lj_rcut=0.0, lj_tol=gd["lj_tol"]))
    idx = np.union1d(I.sample_indices(w.grid.npts, 3000, seed=6), nearest_points(w.grid, w.solute.xyz))
    ref = O.fields(O.Problem.from_workload(w), idx=idx)
    g = run(R, w, degree=max(gd["p_tcf"], gd["p_dcf"], gd["p_coulomb"]), theta=gd["mac"])
    assert g["info"]["cp_pairs"] > 0
    check_fields({k: g[k][:, idx] for k in ("u", "c", "h")}, ref, ("u", "c", "h"), TREE_TOL, w.grid, w.solute.xyz,
                 idx=idx, label="guide 1e-6")
