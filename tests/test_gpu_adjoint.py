"""GPU reverse mode (rism_potential_backward) against the FP64 oracle gradient, against central differences
of the GPU's own FP64 forward, and through torch.autograd."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2109_09772_gb300 import inputs as I
from tests.helpers import rel_l2

pytestmark = pytest.mark.gpu

GRAD_TOL = 2e-5  # rel L2 per gradient kind, FP32 pair terms with float-float sums


@pytest.fixture(scope="module")
def R():
    import torch

    from paper_2109_09772_gb300 import build as B
    from paper_2109_09772_gb300 import rism

    B.build()
    torch.cuda.set_device(0)
    return rism


def _cotangents(w, seed, kinds=("u", "c", "h"), mask_near=None):
    nx, ny, nz = w.grid.n
    S = w.solvent.nsite
    G = {}
    for k, kind in enumerate(kinds):
        f = np.stack([I.gaussian_random_field((nz, ny, nx), w.grid.h, seed + 10 * k + s, corr_len=1.5)
                      for s in range(S)])
        if mask_near is not None:
            f[:, ~mask_near.reshape(nz, ny, nx)] = 0.0
        G[kind] = f
    return G


def _gpu_grad(R, w, G, **opts):
    import torch

    r = R.from_workload(w, method=R.METHOD_DIRECT, precision=R.PREC_FP32, **opts)
    dev = {k: torch.as_tensor(v, device="cuda") for k, v in G.items()}
    g = r.backward(dev.get("u"), dev.get("c"), dev.get("h"))
    torch.cuda.synchronize()
    r.close()
    return {k: v.cpu().numpy() for k, v in g.items()}


def _check(g, ref, atoms, tol=GRAD_TOL, label=""):
    parts = {"xyz": ref[:, 0:3], "q": ref[:, 3], "sigma": ref[:, 4], "eps": ref[:, 5]}
    for k, v in parts.items():
        got = g[k][atoms]
        e = rel_l2(got, v)
        assert e <= tol, f"{label} d{k}: rel L2 {e:.3e} > {tol:g}"


@pytest.mark.parametrize("lj_rcut", [0.0, 4.0])
def test_small_all_atoms_vs_oracle(R, lj_rcut):
    w = I.small_workload(n_atoms=60, n=(26, 22, 18), h=0.5, seed=31, ions=True, lj_rcut=lj_rcut, net=1.0)
    G = _cotangents(w, seed=5)
    p = O.Problem.from_workload(w)
    atoms = np.arange(w.solute.n)
    ref = O.grad(p, atoms, G["u"], G["c"], G["h"])
    g = _gpu_grad(R, w, G)
    _check(g, ref, atoms, label=f"rcut{lj_rcut}")


def test_only_c_cotangent_no_ions(R):
    """u and c only (no ionic sites, kappa = 0), as in the differentiation workload."""
    w = I.small_workload(n_atoms=40, n=(20, 20, 16), h=0.5, seed=33, ions=False, lj_rcut=5.0)
    G = _cotangents(w, seed=9, kinds=("u", "c"))
    p = O.Problem.from_workload(w)
    atoms = np.arange(w.solute.n)
    ref = O.grad(p, atoms, G["u"], G["c"], None)
    g = _gpu_grad(R, w, G)
    _check(g, ref, atoms, label="no-ions")


def test_globule2000_sampled_atoms(R):
    """2,000-atom globule on the 128^3 grid: GPU gradient of every atom, oracle for 12 sampled atoms."""
    w = I.workload(1)
    G = _cotangents(w, seed=13)
    p = O.Problem.from_workload(w)
    atoms = np.sort(np.random.default_rng(4).choice(w.solute.n, 12, replace=False))
    ref = O.grad(p, atoms, G["u"], G["c"], G["h"])
    g = _gpu_grad(R, w, G)
    _check(g, ref, atoms, tol=5e-5, label="cfg1")


def test_central_differences_of_gpu_forward(R):
    """d/dR, d/dq, d/dsigma, d/deps by central differences of the GPU FP64 direct forward, on a problem
    holding one atom at a time (L is a sum over atoms), cotangents zero within 1 A of it, LJ cut-off off."""
    import torch

    from tests.helpers import far_mask

    w = I.small_workload(n_atoms=5, n=(24, 22, 20), h=0.5, seed=41, ions=True, lj_rcut=0.0)
    for i in range(3):
        one = I.Workload(w.name, I.Solute(w.solute.xyz[i:i + 1].copy(), w.solute.q[i:i + 1].copy(),
                                          w.solute.sigma[i:i + 1].copy(), w.solute.eps[i:i + 1].copy()),
                         w.solvent, w.grid, dict(w.opts))
        G = _cotangents(one, seed=50 + i, mask_near=far_mask(one.grid, one.solute.xyz, 1.0))
        g = _gpu_grad(R, one, G)
        dev = {k: torch.as_tensor(v, device="cuda") for k, v in G.items()}

        def loss(sol):
            r = R.Rism(one.grid.n, one.grid.h, one.grid.origin, method=R.METHOD_DIRECT, precision=R.PREC_FP64,
                       lj_mode=R.LJ_NONE)
            r.set_solvent(w.solvent.q, w.solvent.sigma, w.solvent.eps, w.solvent.rho, w.solvent.is_ion)
            r.set_solute(*sol)
            out = r.init()
            val = sum(float((dev[k] * out[k]).sum()) for k in ("u", "c", "h"))
            r.close()
            return val

        base = [one.solute.xyz.copy(), one.solute.q.copy(), one.solute.sigma.copy(), one.solute.eps.copy()]
        for name, idx, comp, step in (("xyz", 0, 0, 1e-5), ("xyz", 0, 1, 1e-5), ("xyz", 0, 2, 1e-5),
                                      ("q", 1, None, 1e-5), ("sigma", 2, None, 1e-5), ("eps", 3, None, 1e-6)):
            vals = []
            for sgn in (1, -1):
                sol = [b.copy() for b in base]
                if comp is None:
                    sol[idx][0] += sgn * step
                else:
                    sol[idx][0, comp] += sgn * step
                vals.append(loss(sol))
            fd = (vals[0] - vals[1]) / (2 * step)
            got = g[name][0] if comp is None else g[name][0][comp]
            assert got == pytest.approx(fd, rel=2e-4, abs=1e-7 * max(1.0, abs(fd))), (i, name, comp, got, fd)


def test_backward_is_repeatable_bitwise(R):
    import torch

    w = I.small_workload(n_atoms=30, n=(16, 14, 12), h=0.5, seed=44, ions=True, lj_rcut=4.0)
    G = {k: torch.as_tensor(v, device="cuda") for k, v in _cotangents(w, seed=3).items()}
    r = R.from_workload(w, method=R.METHOD_DIRECT, precision=R.PREC_FP32)
    a = r.backward(G["u"], G["c"], G["h"])
    b = r.backward(G["u"], G["c"], G["h"])
    r.close()
    for k in a:
        assert torch.equal(a[k], b[k]), k


def test_autograd_wiring(R):
    """torch.autograd through rism.fields: the gradients equal rism_potential_backward's."""
    import torch

    w = I.small_workload(n_atoms=30, n=(16, 14, 12), h=0.5, seed=44, ions=True, lj_rcut=4.0)
    r = R.from_workload(w, method=R.METHOD_DIRECT, precision=R.PREC_FP32)
    xyz = torch.tensor(w.solute.xyz, dtype=torch.float64, requires_grad=True)
    q = torch.tensor(w.solute.q, dtype=torch.float64, requires_grad=True)
    sg = torch.tensor(w.solute.sigma, dtype=torch.float64, requires_grad=True)
    ep = torch.tensor(w.solute.eps, dtype=torch.float64, requires_grad=True)
    u, c, h = R.fields(xyz, q, sg, ep, r)
    G = {k: torch.randn_like(v) for k, v in (("u", u), ("c", c), ("h", h))}
    L = (G["u"] * u).sum() + (G["c"] * c).sum() + (G["h"] * h).sum()
    L.backward()
    direct = r.backward(G["u"], G["c"], G["h"])
    for name, t in (("xyz", xyz), ("q", q), ("sigma", sg), ("eps", ep)):
        a, b = t.grad.numpy(), direct[name].cpu().numpy()
        assert np.array_equal(a, b), (name, float(np.abs(a - b).max() / np.abs(b).max()))
    r.close()


def _grad(R, w, G, method, **opts):
    import torch

    r = R.from_workload(w, method=method, precision=R.PREC_FP32, **opts)
    dev = {k: torch.as_tensor(v, device="cuda") for k, v in G.items()}
    g = r.backward(dev.get("u"), dev.get("c"), dev.get("h"))
    torch.cuda.synchronize()
    r.close()
    return {k: v.cpu().numpy() for k, v in g.items()}


def test_treecode_reverse_far_field_globule2000(R):
    """Treecode context on the 2,000-atom globule: the far part runs over the grid boxes (proxies carry the
    cotangent weights aggregated through the Lagrange basis).  Against the direct reverse mode for every atom and
    against the oracle for 12 sampled atoms."""
    w = I.workload(1)
    G = _cotangents(w, seed=23)
    gt = _grad(R, w, G, R.METHOD_TREECODE)
    gd = _grad(R, w, G, R.METHOD_DIRECT)
    for k in ("xyz", "q", "sigma", "eps"):
        assert rel_l2(gt[k], gd[k]) <= 1e-5, k
    atoms = np.sort(np.random.default_rng(6).choice(w.solute.n, 12, replace=False))
    ref = O.grad(O.Problem.from_workload(w), atoms, G["u"], G["c"], G["h"])
    _check(gt, ref, atoms, tol=5e-5, label="tree reverse")


def test_treecode_reverse_ragged_and_repeatable(R):
    """Clipped boxes (a 150x37x70 grid), every atom against the oracle; two calls agree bit for bit."""
    w = I.small_workload(n_atoms=500, n=(150, 37, 70), h=0.5, seed=29, ions=True, lj_rcut=5.0, net=1.0)
    w.solute.xyz[:, 0] -= 10.0
    G = _cotangents(w, seed=31)
    a = _grad(R, w, G, R.METHOD_TREECODE)
    b = _grad(R, w, G, R.METHOD_TREECODE)
    for k in a:
        assert np.array_equal(a[k], b[k]), k
    atoms = np.arange(w.solute.n)
    ref = O.grad(O.Problem.from_workload(w), atoms, G["u"], G["c"], G["h"])
    _check(a, ref, atoms, label="tree reverse ragged")


def _fd_safe_atoms(w, count, delta, rc, seed):
    """Seeded atoms none of whose +-delta probes along x, y, z moves a grid point across the LJ cut-off (such a
    crossing makes L jump by G u_LJ(r_c), which the derivative does not contain)."""
    from tests.helpers import lj_boundary_pairs

    rel = 4.0 * delta / rc
    _, ats = lj_boundary_pairs(w.grid, w.solute.xyz, rc, rel=rel)
    bad = set(ats.tolist())
    order = np.random.default_rng(seed).permutation(w.solute.n)
    return np.sort(np.array([a for a in order if a not in bad][:count]))


def test_stack55000_backward_64_atoms_vs_oracle_and_central_differences(R):
    """The differentiation workload: 55,000 atoms (four stacked ellipsoids) on 320x320x384, forward u + c with
    FP32 pairs (treecode), backward with a smooth seeded cotangent (correlation length 3 A, amplitude 0.5) used
    for both u and c.  64 seeded atoms: the gradient against the FP64 oracle's analytic gradient, and against
    central differences (delta 1e-5 A, 1e-6 relative for q, sigma, eps) of L restricted to the atom's own terms
    (L is a sum over atoms), each term evaluated by the FP64 direct sum on a one-atom solute."""
    import torch

    w = I.workload(4)
    nx, ny, nz = w.grid.n
    S = w.solvent.nsite
    G = np.stack([I.gaussian_random_field((nz, ny, nx), w.grid.h, 700 + s, corr_len=3.0, amplitude=0.5)
                  for s in range(S)])
    Gd = torch.as_tensor(G, device="cuda")
    r = R.from_workload(w, method=R.METHOD_TREECODE, precision=R.PREC_FP32)
    r.init(u=True, c=True, h=False)
    g = {k: v.cpu().numpy() for k, v in r.backward(Gd, Gd, None).items()}
    r.close()
    rc = float(w.opts["lj_rcut"])
    delta = 1e-5
    atoms = _fd_safe_atoms(w, 64, delta, rc, seed=64)
    assert atoms.size == 64
    # the FP64 oracle's analytic gradient of the same L
    ref = O.grad(O.Problem.from_workload(w), atoms, G, G, None)
    _check(g, ref, atoms, label="55k vs oracle")

    # central differences of L_i = sum_s sum_r G_s (u_i,s + c_i,s), atom i alone, FP64 direct sums
    one = R.Rism(w.grid.n, w.grid.h, w.grid.origin, method=R.METHOD_DIRECT, precision=R.PREC_FP64,
                 lj_mode=R.LJ_RCUT, lj_rcut=rc)
    one.set_solvent(w.solvent.q, w.solvent.sigma, w.solvent.eps, w.solvent.rho, w.solvent.is_ion)
    plus = {"u": one.empty_grid(), "c": one.empty_grid()}
    minus = {"u": one.empty_grid(), "c": one.empty_grid()}

    def fields(out, x, q, s, e):
        one.set_solute(x.reshape(1, 3), [q], [s], [e])
        one.init(u=True, c=True, h=False, out=out)

    # L(+) - L(-) as one sum of pointwise differences: the r^-12 wall at the grid points next to the atom is
    # many orders above the rest of L, so differencing two totals would lose the derivative in their rounding
    def diff():
        return float((Gd * (plus["u"] - minus["u"])).sum() + (Gd * (plus["c"] - minus["c"])).sum())

    fd = np.zeros((atoms.size, 6))
    for n, a in enumerate(atoms):
        base = [w.solute.xyz[a].copy(), float(w.solute.q[a]), float(w.solute.sigma[a]), float(w.solute.eps[a])]
        for comp in range(6):
            step = delta if comp < 3 else 1e-6 * max(abs(base[comp - 2]), 1e-3)
            for sgn, out in ((1.0, plus), (-1.0, minus)):
                x, q, s, e = base[0].copy(), base[1], base[2], base[3]
                if comp == 3:
                    # the LJ terms do not depend on q, and next to the atom they are so large that the
                    # Coulomb change drowns in their rounding: probe q with the atom's LJ switched off
                    e = 0.0
                if comp < 3:
                    x[comp] += sgn * step
                elif comp == 3:
                    q += sgn * step
                elif comp == 4:
                    s += sgn * step
                else:
                    e += sgn * step
                fields(out, x, q, s, e)
            fd[n, comp] = diff() / (2.0 * step)
    one.close()
    _check(g, fd, atoms, label="55k vs central differences")
