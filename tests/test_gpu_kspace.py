"""GPU parity of the reciprocal-space asymptotics (rism_asymptotics_k: eqs. (dcf-k)/(tcf-k) on the grid's
reciprocal lattice, with and without the frequency cut-off of Sec. 2.5) against the FP64 oracle.
Tolerances (FP32 phase tables and products, float-float sums): rel L2 1e-6 per output over the compared
entries, max-abs error / max |ref| 4e-6 (the FP32 class of tests/helpers.py)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2109_09772_gb300 import inputs as I
from tests.helpers import rel_l2

pytestmark = pytest.mark.gpu

TOL, MAX_TOL = 1e-6, 4e-6


@pytest.fixture(scope="module")
def R():
    import torch

    from paper_2109_09772_gb300 import build as B
    from paper_2109_09772_gb300 import rism

    B.build()
    torch.cuda.set_device(0)
    return rism


def _check(got, ref, label):
    for s in range(ref.shape[0]):
        e = rel_l2(got[s].view(np.float64), ref[s].view(np.float64))
        assert e <= TOL, f"{label} site {s}: rel L2 {e:.3e}"
        m = float(np.abs(got[s] - ref[s]).max() / max(np.abs(ref[s]).max(), 1e-300))
        assert m <= MAX_TOL, f"{label} site {s}: max-abs / max {m:.3e}"


@pytest.mark.parametrize("grid", [(37, 21, 13), (24, 30, 18)])
def test_small_full_half_spectrum(R, grid):
    """Every entry of the half spectrum (odd and even axes, ragged CTA tiles), no cut-off."""
    w = I.small_workload(n_atoms=150, n=grid, h=0.45, seed=5, ions=True, lj_rcut=4.0, net=2.0)
    r = R.from_workload(w, method=R.METHOD_TREECODE, precision=R.PREC_FP32)
    c, h, kc = r.asymptotics_k(0.0)
    assert kc == 0.0
    S = r.S
    got = {"c": c.cpu().numpy().reshape(S, -1), "h": h.cpu().numpy().reshape(S, -1)}
    r.close()
    ref = O.kspace(O.Problem.from_workload(w))
    for k in ("c", "h"):
        _check(got[k], ref[k], f"{grid} {k}")
    assert np.all(got["c"][:, 0] == 0)


def test_two_mx_blocks_ragged_quads(R):
    """A grid whose half spectrum spans two 128-wide m_x blocks (nx = 262: 132 m_x) and whose rows end in a
    ragged quad (ny = 9): every entry against the oracle, for the whole half spectrum (4 groups of 32 m_x per
    item in the first block, 1 in the second) and two cut-offs (m_x up to about 80 and 49: items of 3, 2, 1 and
    0 groups, the second block empty)."""
    w = I.small_workload(n_atoms=60, n=(262, 9, 7), h=0.4, seed=12, ions=True, lj_rcut=4.0, net=1.0)
    p = O.Problem.from_workload(w)
    r = R.from_workload(w, method=R.METHOD_DIRECT, precision=R.PREC_FP32)
    S = r.S
    full = O.kspace(p)
    for rel in (0.0, 1e-5, 1e-3):
        tol = rel * float(np.abs(full["c"]).max())
        c, h, kc = r.asymptotics_k(tol)
        assert r.info()["launches"] == 2
        got = {"c": c.cpu().numpy().reshape(S, -1), "h": h.cpu().numpy().reshape(S, -1)}
        ref = O.kspace(p, kcut=kc) if kc > 0 else full
        if kc > 0:
            keep = np.abs(ref["h"][0]) > 0
            assert 0 < keep.sum() < keep.size
            for k in ("c", "h"):
                assert np.all(got[k][:, ~keep & (np.arange(keep.size) > 0)] == 0)
        for k in ("c", "h"):
            _check(got[k], ref[k], f"nx 262, tol {rel} {k}")
    r.close()


def test_cutoff_matches_oracle_root_and_zeroes(R):
    w = I.small_workload(n_atoms=150, n=(40, 36, 33), h=0.5, seed=8, ions=True, lj_rcut=4.0, net=-1.0)
    p = O.Problem.from_workload(w)
    full = O.kspace(p)
    tol = 1e-3 * float(np.abs(full["c"]).max())
    kc_ref = O.kspace_kcut(p, tol)
    r = R.from_workload(w, method=R.METHOD_DIRECT, precision=R.PREC_FP32)
    c, h, kc = r.asymptotics_k(tol)
    S = r.S
    got = {"c": c.cpu().numpy().reshape(S, -1), "h": h.cpu().numpy().reshape(S, -1)}
    # host output buffers: the same values
    nx, ny, nz = w.grid.n
    hc = np.zeros((S, nz, ny, nx // 2 + 1), dtype=np.complex128)
    kc2 = np.zeros(1)
    r._check(r.lib.rism_asymptotics_k(r.ctx, tol, hc.ctypes.data, None, kc2.ctypes.data), "rism_asymptotics_k")
    np.testing.assert_array_equal(hc.reshape(S, -1), got["c"])
    r.close()
    assert kc == pytest.approx(kc_ref, rel=1e-12) and kc2[0] == kc
    ref = O.kspace(p, kcut=kc)
    keep = np.abs(ref["h"][0]) > 0
    assert 0 < keep.sum() < keep.size
    for k in ("c", "h"):
        _check(got[k], ref[k], f"cut-off {k}")
        assert np.all(got[k][:, ~keep & (np.arange(keep.size) > 0)] == 0)


def test_ellipsoid13600_sampled(R):
    """The 13,600-atom solute on 224x192x160: sampled entries of the whole half spectrum and every entry of
    the lowest wave numbers, without and with a cut-off."""
    w = I.workload(2)
    nx, ny, nz = w.grid.n
    nh = nx // 2 + 1
    total = nh * ny * nz
    low = np.array([(jz * ny + jy) * nh + jx for jz in (0, 1, nz - 1) for jy in (0, 1, ny - 1) for jx in range(4)])
    idx = np.union1d(I.sample_indices(total, 1500, seed=4), low)
    p = O.Problem.from_workload(w)
    ref = O.kspace(p, idx=idx)
    r = R.from_workload(w, method=R.METHOD_TREECODE, precision=R.PREC_FP32)
    c, h, _ = r.asymptotics_k(0.0)
    import torch

    t = torch.as_tensor(idx, device="cuda")
    for k, v in (("c", c), ("h", h)):
        _check(v.reshape(r.S, -1)[:, t].cpu().numpy(), ref[k], f"13,600 atoms {k}")
    tol = 1e-4 * float(np.abs(ref["c"]).max())
    c, h, kc = r.asymptotics_k(tol)
    assert 0 < kc < 2 * np.pi / w.grid.h
    refc = O.kspace(p, kcut=kc, idx=idx)
    for k, v in (("c", c), ("h", h)):
        _check(v.reshape(r.S, -1)[:, t].cpu().numpy(), refc[k], f"13,600 atoms, cut-off {k}")
    r.close()


def test_edge_cases(R):
    w = I.small_workload(n_atoms=10, n=(12, 10, 9), h=0.5, seed=2, ions=False)
    r = R.from_workload(w, method=R.METHOD_DIRECT, precision=R.PREC_FP32)
    with pytest.raises(R.RismError) as e:  # no ionic site: kappa = 0, h(k) undefined as in real space
        r.asymptotics_k(0.0, c=True, h=True)
    assert e.value.status == R.E_INVALID
    c, _, _ = r.asymptotics_k(0.0, c=True, h=False)
    ref = O.kspace(O.Problem.from_workload(w), want=("c",))
    _check(c.cpu().numpy().reshape(r.S, -1), ref["c"], "no ions")
    r.set_solute(np.zeros((0, 3)), [], [], [])
    c, _, _ = r.asymptotics_k(0.0, c=True, h=False)
    assert float(c.abs().max()) == 0.0
    r.close()
