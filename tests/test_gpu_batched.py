"""Many solutes in one persistent, graph-captured launch (rism_potential_batched) and the autotuner."""
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2109_09772_gb300 import inputs as I
from tests.helpers import check_fields, nearest_points

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def R():
    import torch

    from paper_2109_09772_gb300 import build as B
    from paper_2109_09772_gb300 import rism

    B.build()
    torch.cuda.set_device(0)
    return rism


def _uneven(count=5, seed=0):
    """An uneven batch: 150..2,000 atoms, each with its own grid (12 A buffer, multiple of 16 points)."""
    return I.batch_workloads(count=count, seed=seed, lo=150, hi=2000)


def _single(R, w):
    r = R.from_workload(w, method=R.METHOD_TREECODE, precision=R.PREC_FP32)
    out = r.init()
    res = {k: out[k].cpu().numpy() for k in ("u", "c", "h")}
    r.close()
    return res


def test_batched_equals_per_solute_and_replays(R):
    ws = _uneven()
    rs = [R.from_workload(w, method=R.METHOD_TREECODE, precision=R.PREC_FP32) for w in ws]
    singles = [_single(R, w) for w in ws]
    out1 = R.potential_batched(rs)
    out2 = R.potential_batched(rs)  # replays the captured graph
    for k, w in enumerate(ws):
        for f in ("u", "c", "h"):
            a, b = out1[k][f].cpu().numpy(), out2[k][f].cpu().numpy()
            assert np.array_equal(a, b), (k, f)
            np.testing.assert_array_equal(a, singles[k][f])
    # new coordinates, same sizes: uploaded outside the graph, the replay must see them
    rng = np.random.default_rng(9)
    w0 = ws[0]
    moved = w0.solute.xyz + rng.normal(0.0, 0.3, size=w0.solute.xyz.shape)
    rs[0].set_solute(moved, w0.solute.q, w0.solute.sigma, w0.solute.eps)
    out3 = R.potential_batched(rs)
    w0m = I.Workload(w0.name, I.Solute(moved, w0.solute.q, w0.solute.sigma, w0.solute.eps), w0.solvent, w0.grid,
                     dict(w0.opts))
    single_moved = _single(R, w0m)
    for f in ("u", "c", "h"):
        np.testing.assert_array_equal(out3[0][f].cpu().numpy(), single_moved[f])
        np.testing.assert_array_equal(out3[1][f].cpu().numpy(), singles[1][f])
    for r in rs:
        r.close()


def test_batched_against_oracle(R):
    ws = _uneven(count=4, seed=1)
    rs = [R.from_workload(w, method=R.METHOD_TREECODE, precision=R.PREC_FP32) for w in ws]
    outs = R.potential_batched(rs)
    for w, o in zip(ws, outs):
        idx = np.union1d(I.sample_indices(w.grid.npts, 800, seed=3), nearest_points(w.grid, w.solute.xyz))
        ref = O.fields(O.Problem.from_workload(w), idx=idx)
        g = {k: o[k].cpu().numpy().reshape(w.solvent.nsite, -1)[:, idx] for k in ("u", "c", "h")}
        check_fields(g, ref, ("u", "c", "h"), 1e-5, w.grid, w.solute.xyz, idx=idx, label=w.name)
    for r in rs:
        r.close()


def test_batched_rejects_mixed_options(R):
    ws = _uneven(count=2, seed=2)
    a = R.from_workload(ws[0], method=R.METHOD_TREECODE, precision=R.PREC_FP32)
    b = R.from_workload(ws[1], method=R.METHOD_TREECODE, precision=R.PREC_FP32, degree=6)
    with pytest.raises(R.RismError) as e:
        R.potential_batched([a, b])
    assert e.value.status == R.E_INVALID
    a.close()
    b.close()


def test_autotune_picks_a_shape_and_caches_it(R, tmp_path):
    path = str(tmp_path / "tune.txt")
    os.environ["RISM_AUTOTUNE_CACHE"] = path
    w = I.workload(1)
    # a problem class no other test tunes (the in-memory cache would otherwise answer without timing)
    r = R.from_workload(w, method=R.METHOD_TREECODE, precision=R.PREC_FP32, autotune=1, degree=7, theta=0.65)
    out = r.init()
    info = r.info()
    assert info["kernel_variant"] in (0, 1, 2)
    idx = I.sample_indices(w.grid.npts, 1500, seed=8)
    ref = O.fields(O.Problem.from_workload(w), idx=idx)
    g = {k: out[k].cpu().numpy().reshape(r.S, -1)[:, idx] for k in ("u", "c", "h")}
    check_fields(g, ref, ("u", "c", "h"), 1e-5, label="autotuned")
    r.close()
    assert os.path.exists(path) and os.path.getsize(path) > 0
    line = open(path).read().strip().splitlines()[0]
    assert "S4" in line and line.split()[-2] == str(info["kernel_variant"])


def test_batched_32_solutes_500_to_8000_atoms_against_oracle(R):
    """The 32-solute batch of the benchmark plan (500..8,000 atoms, log-uniform, own grids) in one persistent
    graph-captured launch; solutes above 4,096 atoms take the radix-sort tree build inside the batched graph.
    Every solute against the FP64 oracle at sampled points and at the point nearest each atom."""
    import torch

    ws = I.batch_workloads(count=32, seed=0)
    assert sum(w.solute.n > 4096 for w in ws) >= 2
    rs = [R.from_workload(w, method=R.METHOD_TREECODE, precision=R.PREC_FP32) for w in ws]
    outs = R.potential_batched(rs)
    outs = R.potential_batched(rs, out=outs)  # the replayed graph
    torch.cuda.synchronize()
    for w, o in zip(ws, outs):
        idx = np.union1d(I.sample_indices(w.grid.npts, 600, seed=w.solute.n), nearest_points(w.grid, w.solute.xyz))
        ref = O.fields(O.Problem.from_workload(w), idx=idx)
        t = torch.as_tensor(idx, device="cuda")
        g = {k: o[k].reshape(w.solvent.nsite, -1)[:, t].cpu().numpy() for k in ("u", "c", "h")}
        check_fields(g, ref, ("u", "c", "h"), 1e-5, w.grid, w.solute.xyz, idx=idx, label=w.name)
    for r in rs:
        r.close()
