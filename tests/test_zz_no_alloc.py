"""rism_init_noalloc: the allocation-free direct-sum entry point, for callers that cannot call cudaMalloc
(plug-ins whose host application owns the device memory, callers that must not allocate after start-up).

Its output must match the context API (rism_init, direct method) within the tolerance the parity tests use
(rel L2 1e-6 for FP32 pairs, 1e-12 for FP64 pairs) on two calls in a row: the shared scratch array keeps the
previous call's contents, so the second call checks that nothing stale leaks through.  This file is
collected last and must also pass on its own in a fresh process.
"""
import numpy as np
import pytest

from paper_2109_09772_gb300 import inputs as I
from tests.helpers import rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def R():
    import torch

    from paper_2109_09772_gb300 import build as B
    from paper_2109_09772_gb300 import rism

    B.build()
    torch.cuda.set_device(0)
    return rism


def _dev(a):
    import torch

    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")


@pytest.mark.parametrize("prec,tol", [(1, 1e-6), (0, 1e-12)])
def test_noalloc_matches_context_api_twice(R, prec, tol):
    import torch

    # two different solutes in a row, then the first again: stale scratch would show in the third call
    wa = I.small_workload(n_atoms=150, n=(37, 21, 13), h=0.45, seed=5, ions=True, lj_rcut=4.0, net=2.0)
    wb = I.small_workload(n_atoms=97, n=(37, 21, 13), h=0.45, seed=6, ions=True, lj_rcut=4.0, net=-1.0)
    refs = {}
    for name, w in (("a", wa), ("b", wb)):
        r = R.from_workload(w, method=R.METHOD_DIRECT, precision=prec)
        out = r.init(u=True, c=True, h=True)
        refs[name] = {k: out[k].cpu().numpy() for k in ("u", "c", "h")}
        r.close()
    S = wa.solvent.nsite
    nx, ny, nz = wa.grid.n
    solvent = (wa.solvent.q, wa.solvent.sigma, wa.solvent.eps, wa.solvent.rho, wa.solvent.is_ion)
    for name, w in (("a", wa), ("b", wb), ("a", wa)):
        outs = {k: torch.full((S, nz, ny, nx), float("nan"), dtype=torch.float64, device="cuda")
                for k in ("u", "c", "h")}
        R.init_noalloc(w.grid.n, w.grid.h, w.grid.origin, _dev(w.solute.xyz), _dev(w.solute.q),
                       _dev(w.solute.sigma), _dev(w.solute.eps), solvent, u=outs["u"], c=outs["c"], hh=outs["h"],
                       method=R.METHOD_DIRECT, precision=prec, lj_mode=R.LJ_RCUT, lj_rcut=4.0)
        torch.cuda.synchronize()
        for k in ("u", "c", "h"):
            got = outs[k].cpu().numpy()
            assert np.isfinite(got).all()
            assert rel_l2(got, refs[name][k]) <= tol, (name, k)


def test_noalloc_rejects_too_many_atoms(R):
    import torch

    n = R.NOALLOC_MAX_ATOMS + 1
    z = torch.zeros(n, dtype=torch.float64, device="cuda")
    xyz = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
    w = I.small_workload(n_atoms=5, n=(8, 8, 8), ions=True)
    solvent = (w.solvent.q, w.solvent.sigma, w.solvent.eps, w.solvent.rho, w.solvent.is_ion)
    u = torch.empty((w.solvent.nsite, 8, 8, 8), dtype=torch.float64, device="cuda")
    with pytest.raises(R.RismError) as e:
        R.init_noalloc(w.grid.n, w.grid.h, w.grid.origin, xyz, z, z, z, solvent, u=u, method=R.METHOD_DIRECT)
    assert e.value.status == R.E_INVALID
    assert "RISM_NOALLOC_MAX_ATOMS" in str(e.value)


def test_noalloc_refuses_host_outputs_and_bad_device_inputs(R):
    """A host output pointer is refused before any launch; NaN / negative sigma in device-resident solute
    arrays are found by the library's device-side check and refused; the next good call still works."""
    import torch

    w = I.small_workload(n_atoms=40, n=(16, 12, 10), h=0.5, seed=3, ions=True, lj_rcut=4.0)
    S = w.solvent.nsite
    nx, ny, nz = w.grid.n
    solvent = (w.solvent.q, w.solvent.sigma, w.solvent.eps, w.solvent.rho, w.solvent.is_ion)
    args = lambda xyz, sg: (w.grid.n, w.grid.h, w.grid.origin, _dev(xyz), _dev(w.solute.q), _dev(sg),
                            _dev(w.solute.eps), solvent)
    host_u = torch.zeros((S, nz, ny, nx), dtype=torch.float64)
    with pytest.raises(R.RismError) as e:
        R.init_noalloc(*args(w.solute.xyz, w.solute.sigma), u=host_u, method=R.METHOD_DIRECT)
    assert e.value.status == R.E_INVALID and "device memory" in str(e.value)
    u = torch.zeros((S, nz, ny, nx), dtype=torch.float64, device="cuda")
    bad_xyz = w.solute.xyz.copy()
    bad_xyz[7, 1] = float("nan")
    with pytest.raises(R.RismError) as e:
        R.init_noalloc(*args(bad_xyz, w.solute.sigma), u=u, method=R.METHOD_DIRECT)
    assert e.value.status == R.E_INVALID
    bad_sig = w.solute.sigma.copy()
    bad_sig[3] = -1.0
    with pytest.raises(R.RismError) as e:
        R.init_noalloc(*args(w.solute.xyz, bad_sig), u=u, method=R.METHOD_DIRECT)
    assert e.value.status == R.E_INVALID
    # the error word left in the shared scratch by the refused calls does not leak into the next call
    R.init_noalloc(*args(w.solute.xyz, w.solute.sigma), u=u, method=R.METHOD_DIRECT, lj_mode=R.LJ_RCUT,
                   lj_rcut=4.0)
    torch.cuda.synchronize()
    r = R.from_workload(w, method=R.METHOD_DIRECT, precision=R.PREC_FP32)
    ref = r.init(u=True, c=False, h=False)["u"].cpu().numpy()
    r.close()
    assert rel_l2(u.cpu().numpy(), ref) <= 1e-6
