"""GPU parity of the treecode path (BL particle-cluster far field + cell-list near field) against the
FP64 oracle, through the C ABI.

The treecode is an approximation: its error at degree 8, theta 0.7 must stay within rel L2 1e-5 per output
grid; with no accepted cluster (small solutes) it reduces to the FP32 direct sum (1e-6).  Error falls
geometrically with the degree.
"""
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
    r = R.from_workload(w, method=R.METHOD_TREECODE, precision=R.PREC_FP32, **opts)
    out = r.init(u="u" in keys, c="c" in keys, h="h" in keys, lj_tail=True)
    res = {k: out[k].cpu().numpy().reshape(r.S, -1) for k in keys}
    res["info"] = r.info()
    res["lj_tail"] = out["lj_tail"]
    r.close()
    return res


def test_small_ragged_no_accepted_cluster(R):
    """150 atoms: no cluster is large enough for proxies, so every pair is direct (far list) or near
    (cells): FP32-direct accuracy on a ragged 37x21x13 grid."""
    w = I.small_workload(n_atoms=150, n=(37, 21, 13), h=0.45, seed=5, ions=True, lj_rcut=4.0, net=2.0)
    p = O.Problem.from_workload(w)
    ref = O.fields(p)
    g = run(R, w)
    assert g["info"]["proxy_pairs"] == 0
    check_fields(g, ref, ("u", "c", "h"), 1e-6, w.grid, w.solute.xyz, label="tree small")
    np.testing.assert_allclose(g["lj_tail"], O.lj_tail(p), rtol=1e-12)


def _sampled(w, count=3000, seed=2):
    return np.union1d(I.sample_indices(w.grid.npts, count, seed=seed), nearest_points(w.grid, w.solute.xyz))


def test_globule2000_degree8_theta07(R):
    """2,000-atom globule, 128^3 grid, 4 sites, LJ cut-off 9 A, degree 8, theta 0.7."""
    w = I.workload(1)
    idx = _sampled(w)
    ref = O.fields(O.Problem.from_workload(w), idx=idx)
    g = run(R, w)
    # target boxes take the far field here: proxies at the boxes, none at the octree nodes
    assert g["info"]["cp_pairs"] > 0 and g["info"]["tree_boxes"] > 0 and g["info"]["tree_proxied"] == 0
    gs = {k: g[k][:, idx] for k in ("u", "c", "h")}
    check_fields(gs, ref, ("u", "c", "h"), TREE_TOL, w.grid, w.solute.xyz, idx=idx, label="cfg1 tree")


def test_error_falls_with_degree(R):
    """Geometric convergence of the barycentric-Lagrange far field: error(degree) decreases."""
    w = I.workload(1)
    idx = I.sample_indices(w.grid.npts, 2000, seed=3)
    ref = O.fields(O.Problem.from_workload(w), idx=idx, want=("c",))
    errs = []
    for deg in (2, 4, 6, 8):
        g = run(R, w, keys=("c",), degree=deg, leaf=32)
        errs.append(rel_l2(g["c"][:, idx], ref["c"]))
    assert errs[0] > errs[1] > errs[2] > errs[3], errs
    assert errs[0] / errs[2] > 20.0, errs


def test_no_lj_cutoff_means_all_atoms_near(R):
    """Without an LJ cut-off every atom is in the near field of every batch (LJ exact), the far field still
    uses the tree."""
    w = I.small_workload(n_atoms=120, n=(20, 18, 14), h=0.5, seed=8, ions=True, lj_rcut=0.0)
    ref = O.fields(O.Problem.from_workload(w))
    g = run(R, w)
    check_fields(g, ref, ("u", "c", "h"), 1e-6, w.grid, w.solute.xyz, label="tree no-cutoff")


def test_grid_point_on_an_atom(R):
    w = I.small_workload(n_atoms=20, n=(16, 12, 10), h=0.5, seed=4, ions=True, lj_rcut=5.0)
    w.solute.xyz[3] = np.array(w.grid.origin) + 0.5 * np.array([7, 5, 4])
    ref = O.fields(O.Problem.from_workload(w))
    g = run(R, w)
    f = (4 * 12 + 5) * 16 + 7
    assert np.all(np.isposinf(g["u"][:, f]))
    keep = np.ones(g["u"].shape[1], dtype=bool)
    keep[f] = False
    assert rel_l2(g["u"][:, keep], ref["u"][:, keep]) <= 1e-6
    for k in ("c", "h"):
        assert np.all(np.isfinite(g[k]))
        assert rel_l2(g[k], ref[k]) <= 1e-6


def test_zero_atoms(R):
    w = I.small_workload(n_atoms=5, n=(9, 8, 8), ions=True)
    r = R.from_workload(w, method=R.METHOD_TREECODE)
    r.set_solute(np.zeros((0, 3)), [], [], [])
    out = r.init()
    for k in ("u", "c", "h"):
        assert float(out[k].abs().max()) == 0.0
    r.close()


def test_small_leaves_many_nodes_and_repeatable(R):
    """leaf = 8 gives a deep tree and long lists; results repeat bit for bit."""
    w = I.workload(1)
    idx = I.sample_indices(w.grid.npts, 1500, seed=4)
    ref = O.fields(O.Problem.from_workload(w), idx=idx)
    a = run(R, w, leaf=8)
    b = run(R, w, leaf=8)
    assert a["info"]["tree_nodes"] > 300
    for k in ("u", "c", "h"):
        assert np.array_equal(a[k], b[k])
    check_fields({k: a[k][:, idx] for k in ("u", "c", "h")}, ref, ("u", "c", "h"), TREE_TOL, label="leaf8")


def test_ellipsoid13600_224x192x160_sampled(R):
    """13,600-atom prolate ellipsoid (net -24) on the 224x192x160 grid, degree 8, theta 0.7."""
    w = I.workload(2)
    idx = _sampled(w, count=2500, seed=5)
    ref = O.fields(O.Problem.from_workload(w), idx=idx)
    g = run(R, w)
    gs = {k: g[k][:, idx] for k in ("u", "c", "h")}
    check_fields(gs, ref, ("u", "c", "h"), TREE_TOL, w.grid, w.solute.xyz, idx=idx, label="cfg2 tree")


def test_ellipsoid13600_degree4_theta05_long_lists(R):
    """A strict MAC (theta 0.5) and a low degree give long far lists on the 13,600-atom ellipsoid: the
    per-batch list slots grow on the first call and the result stays close to the oracle."""
    w = I.workload(2)
    idx = I.sample_indices(w.grid.npts, 1500, seed=9)
    ref = O.fields(O.Problem.from_workload(w), idx=idx, want=("c", "h"))
    g = run(R, w, keys=("c", "h"), degree=4, theta=0.5)
    for k in ("c", "h"):
        assert rel_l2(g[k][:, idx], ref[k]) <= 1e-4, k


def test_target_proxies_on_and_off_agree_with_oracle(R):
    """Cluster-particle far field (proxy targets on grid boxes of 16^3 points and up) against the particle-
    cluster form and the oracle on the 2,000-atom globule: both within the treecode tolerance, and the box
    level takes a large share of the work."""
    w = I.workload(1)
    idx = _sampled(w, count=2500, seed=11)
    ref = O.fields(O.Problem.from_workload(w), idx=idx)
    on = run(R, w, target_proxies=1)
    off = run(R, w, target_proxies=0)
    assert on["info"]["cp_pairs"] > 0 and on["info"]["tree_boxes"] > 0
    assert off["info"]["cp_pairs"] == 0
    assert on["info"]["direct_pairs"] < 0.5 * off["info"]["direct_pairs"]
    for g, lab in ((on, "boxes on"), (off, "boxes off")):
        gs = {k: g[k][:, idx] for k in ("u", "c", "h")}
        check_fields(gs, ref, ("u", "c", "h"), TREE_TOL, w.grid, w.solute.xyz, idx=idx, label=lab)


def test_target_proxies_ragged_clipped_boxes(R):
    """A grid whose sides are not multiples of 16 (boxes clipped at the edges, some too thin for proxies, so
    their points take the field of an enclosing box) with a solute off-centre: all points against the oracle."""
    w = I.small_workload(n_atoms=700, n=(150, 37, 70), h=0.5, seed=21, ions=True, lj_rcut=6.0, net=3.0)
    w.solute.xyz[:, 0] -= 12.0
    ref = O.fields(O.Problem.from_workload(w))
    g = run(R, w, target_proxies=1, leaf=16)
    assert g["info"]["cp_pairs"] > 0
    check_fields(g, ref, ("u", "c", "h"), TREE_TOL, w.grid, w.solute.xyz, label="ragged boxes")


def test_target_proxies_error_falls_with_degree(R):
    """Geometric convergence with the box-level interpolation active."""
    w = I.workload(1)
    idx = I.sample_indices(w.grid.npts, 2000, seed=13)
    ref = O.fields(O.Problem.from_workload(w), idx=idx, want=("c",))
    errs = []
    for deg in (3, 5, 7, 9):
        g = run(R, w, keys=("c",), degree=deg, target_proxies=1)
        assert g["info"]["cp_pairs"] > 0
        errs.append(rel_l2(g["c"][:, idx], ref["c"]))
    assert errs[0] > errs[1] > errs[2] > errs[3], errs


def _fresh(R, w, xyz):
    r = R.from_workload(w, method=R.METHOD_TREECODE, precision=R.PREC_FP32)
    r.set_solute(xyz, w.solute.q, w.solute.sigma, w.solute.eps)
    out = r.init(lj_tail=True)
    res = {k: out[k].cpu().numpy() for k in ("u", "c", "h")}
    res["lj_tail"] = out["lj_tail"]
    r.close()
    return res


def test_graph_replay_matches_regular_path(R):
    """From the second treecode call on, a context replays one captured graph (solute upload from pinned
    memory, tables, tree, lists, evaluation, LJ tail).  New coordinates each call: every result equals, bit
    for bit, a fresh context's first (uncaptured) call."""
    w = I.small_workload(n_atoms=600, n=(48, 40, 36), h=0.5, seed=17, ions=True, lj_rcut=6.0, net=2.0)
    r = R.from_workload(w, method=R.METHOD_TREECODE, precision=R.PREC_FP32)
    rng = np.random.default_rng(3)
    out = None
    for step in range(4):
        xyz = w.solute.xyz + rng.normal(0.0, 0.2, size=w.solute.xyz.shape)
        r.set_solute(xyz, w.solute.q, w.solute.sigma, w.solute.eps)
        out = r.init(lj_tail=True, out={k: out[k] for k in ("u", "c", "h")} if out else None)
        ref = _fresh(R, w, xyz)
        for k in ("u", "c", "h"):
            assert np.array_equal(out[k].cpu().numpy(), ref[k]), (step, k)
        np.testing.assert_array_equal(out["lj_tail"], ref["lj_tail"])
    r.close()


def test_graph_replay_larger_solute_grows_lists(R):
    """The replayed step meets a solute with longer lists than the captured one: the call grows the list
    slots, runs the regular path, and the result equals a fresh context's."""
    small = I.small_workload(n_atoms=60, n=(48, 40, 36), h=0.5, seed=19, ions=True, lj_rcut=6.0)
    big = I.small_workload(n_atoms=900, n=(48, 40, 36), h=0.5, seed=20, ions=True, lj_rcut=6.0)
    r = R.from_workload(small, method=R.METHOD_TREECODE, precision=R.PREC_FP32, leaf=8)
    r.init()
    r.init()
    r.set_solute(big.solute.xyz, big.solute.q, big.solute.sigma, big.solute.eps)
    out = r.init(lj_tail=True)
    r2 = R.from_workload(big, method=R.METHOD_TREECODE, precision=R.PREC_FP32, leaf=8)
    ref = r2.init(lj_tail=True)
    for k in ("u", "c", "h"):
        assert np.array_equal(out[k].cpu().numpy(), ref[k].cpu().numpy()), k
    r.close()
    r2.close()


def test_build_fallbacks_clustered_atoms_and_many_nodes(R):
    """The tree build's other paths against the oracle: a dense cluster of 1,100 atoms with three atoms 22 A away
    crowds the sort's buckets (the build then sorts bitonically), and leaf = 1 gives more nodes than the
    build keeps in shared memory (it builds again in global memory).  Both match the oracle and give the
    same fields as the roomy build (leaf 32 on the same solute)."""
    from dataclasses import replace

    core = I.sphere_solute(1100, 7.5, 1.0, seed=11, min_spacing=1.0)
    far = np.array([[22.0, 0.5, -1.0], [-21.5, 3.0, 2.0], [0.5, -21.0, 22.0]])  # tens of atoms share a bucket
    sol = I.Solute(np.vstack([core.xyz, far]), np.concatenate([core.q, [0.5, -0.5, 0.0]]),
                   np.concatenate([core.sigma, [3.0, 3.2, 3.4]]), np.concatenate([core.eps, [0.1, 0.15, 0.2]]))
    base = I.small_workload(n_atoms=40, n=(100, 96, 104), h=0.5, seed=3, lj_rcut=6.0)
    w = replace(base, solute=sol)
    idx = np.union1d(I.sample_indices(w.grid.npts, 2500, seed=8), nearest_points(w.grid, sol.xyz))
    ref = O.fields(O.Problem.from_workload(w), idx=idx)
    roomy = run(R, w, leaf=32)
    many = run(R, w, leaf=1)
    assert many["info"]["tree_nodes"] > 1024 >= roomy["info"]["tree_nodes"]
    for g, label in ((roomy, "leaf32"), (many, "leaf1")):
        check_fields({k: g[k][:, idx] for k in ("u", "c", "h")}, ref, ("u", "c", "h"), TREE_TOL, w.grid, sol.xyz,
                     idx=idx, label=label)
    for k in ("u", "c", "h"):
        assert rel_l2(many[k], roomy[k]) < TREE_TOL


def test_host_outputs_through_replayed_step(R):
    """Host output buffers, page-locked or pageable, take the replayed step too (from a context's second call
    on) and arrive by concurrent copies from device buffers: equal to the device outputs bit for bit, also
    after the atoms move."""
    import torch

    w = I.workload(1)
    S, M = w.solvent.nsite, w.grid.npts
    sol = w.solute
    rd = R.from_workload(w, method=R.METHOD_TREECODE, precision=R.PREC_FP32)
    rp = R.from_workload(w, method=R.METHOD_TREECODE, precision=R.PREC_FP32)
    rq = R.from_workload(w, method=R.METHOD_TREECODE, precision=R.PREC_FP32)
    pinned = [torch.empty((S, M), dtype=torch.float64).pin_memory().numpy() for _ in range(3)]
    pageable = [np.empty((S, M)) for _ in range(3)]
    tp, tq = np.zeros(S), np.zeros(S)
    for step in range(3):
        xyz = sol.xyz + (0.37 if step == 2 else 0.0)
        rd.set_solute(xyz, sol.q, sol.sigma, sol.eps)
        out = rd.init(lj_tail=True)
        rp.set_solute(xyz, sol.q, sol.sigma, sol.eps)
        rp.init_host(*pinned, tp)
        rq.set_solute(xyz, sol.q, sol.sigma, sol.eps)
        rq.init_host(*pageable, tq)
        for i, k in enumerate(("u", "c", "h")):
            ref = out[k].cpu().numpy().reshape(S, M)
            assert np.array_equal(ref, pinned[i]), (step, k, "page-locked")
            assert np.array_equal(ref, pageable[i]), (step, k, "pageable")
        np.testing.assert_array_equal(np.asarray(out["lj_tail"]), tp)
        np.testing.assert_array_equal(np.asarray(out["lj_tail"]), tq)
    for r in (rd, rp, rq):
        r.close()


@pytest.mark.parametrize("shape", [0, 1, 2])
def test_each_launch_shape(R, shape):
    """Each launch shape (8x8x8 with 4 far points per thread, 16x8x8 with two near sub-batches per batch, 8x8x8
    with 8 far points per thread), forced through the debug hook, against the oracle on the 2,000-atom globule."""
    w = I.workload(1)
    idx = I.sample_indices(w.grid.npts, 1500, seed=21)
    ref = O.fields(O.Problem.from_workload(w), idx=idx)
    g = run(R, w, debug_flags=(shape + 1) << 4)
    assert g["info"]["kernel_variant"] == shape
    check_fields({k: g[k][:, idx] for k in ("u", "c", "h")}, ref, ("u", "c", "h"), TREE_TOL, label=f"shape{shape}")


def test_build_mid_sized_solute_paths(R):
    """Between 4,096 and 16,384 atoms the build radix-sorts in shared memory and keeps the sorted codes and up to
    2,048 nodes there: 6,000 atoms with leaf 32 build there, leaf 2 overflows the node store and builds again in
    global memory; above 16,384 atoms (17,000) the sort and the nodes go through global memory, and the leaf boxes
    gather the positions in three chunks of 8,192 atoms.  Each against the oracle, and the first two agree with
    each other."""
    base = I.small_workload(n_atoms=40, n=(112, 104, 96), h=0.5, seed=3, lj_rcut=6.0)
    from dataclasses import replace

    mid = I.sphere_solute(6000, I.globule_radius(6000), 2.0, seed=21)
    w = replace(base, solute=mid)
    idx = np.union1d(I.sample_indices(w.grid.npts, 2000, seed=9), nearest_points(w.grid, mid.xyz))
    ref = O.fields(O.Problem.from_workload(w), idx=idx)
    roomy = run(R, w, leaf=32)
    many = run(R, w, leaf=2)
    assert roomy["info"]["tree_nodes"] <= 2048 < many["info"]["tree_nodes"]
    for g, label in ((roomy, "6000 leaf32"), (many, "6000 leaf2")):
        check_fields({k: g[k][:, idx] for k in ("u", "c", "h")}, ref, ("u", "c", "h"), TREE_TOL, w.grid, mid.xyz,
                     idx=idx, label=label)
    for k in ("u", "c", "h"):
        assert rel_l2(many[k], roomy[k]) < TREE_TOL
    big = I.sphere_solute(17000, I.globule_radius(17000), -3.0, seed=22)
    w = replace(I.small_workload(n_atoms=40, n=(144, 144, 144), h=0.5, seed=3, lj_rcut=6.0), solute=big)
    idx = np.union1d(I.sample_indices(w.grid.npts, 1500, seed=10), nearest_points(w.grid, big.xyz)[:500])
    ref = O.fields(O.Problem.from_workload(w), idx=idx)
    g = run(R, w)
    check_fields({k: g[k][:, idx] for k in ("u", "c", "h")}, ref, ("u", "c", "h"), TREE_TOL, w.grid, big.xyz,
                 idx=idx, label="17000")


def test_host_outputs_in_z_slabs_ragged_and_empty(R):
    """With host outputs the near field runs in four z slabs whose copies start as each slab finishes: on a grid
    of three batch layers (nz = 20: 8 + 8 + 4 planes) the last slab is empty and the last layer ragged.  The host
    grids equal the device grids bit for bit, on the regular path (first call) and the replayed one."""
    import torch

    w = I.small_workload(n_atoms=300, n=(40, 24, 20), h=0.5, seed=31, ions=True, lj_rcut=6.0, net=1.0)
    S, M = w.solvent.nsite, w.grid.npts
    sol = w.solute
    rd = R.from_workload(w, method=R.METHOD_TREECODE, precision=R.PREC_FP32)
    rh = R.from_workload(w, method=R.METHOD_TREECODE, precision=R.PREC_FP32)
    host = [torch.empty((S, M), dtype=torch.float64).pin_memory().numpy() for _ in range(3)]
    for step in range(3):
        xyz = sol.xyz + (0.21 if step == 2 else 0.0)
        rd.set_solute(xyz, sol.q, sol.sigma, sol.eps)
        out = rd.init()
        rh.set_solute(xyz, sol.q, sol.sigma, sol.eps)
        for hb in host:
            hb.fill(np.nan)
        rh.init_host(*host)
        for i, k in enumerate(("u", "c", "h")):
            assert np.array_equal(out[k].cpu().numpy().reshape(S, M), host[i]), (step, k)
    for r in (rd, rh):
        r.close()


def test_host_outputs_box_level_in_slabs_ordered(R):
    """With host outputs the target boxes run slab by slab: each z slab first takes the boxes of every level that
    it needs first, in the heaviest-first box order (1,935 boxes in five levels on the 13,600-atom ellipsoid's
    224x192x160 grid; z slabs of five batch layers, which split level-0 box layers).  The host grids equal the
    device grids bit for bit, on the regular path and the replayed one."""
    import torch

    w = I.workload(2)
    S, M = w.solvent.nsite, w.grid.npts
    sol = w.solute
    rd = R.from_workload(w, method=R.METHOD_TREECODE, precision=R.PREC_FP32)
    rh = R.from_workload(w, method=R.METHOD_TREECODE, precision=R.PREC_FP32)
    host = [torch.empty((S, M), dtype=torch.float64).pin_memory().numpy() for _ in range(3)]
    for step in range(2):
        rd.set_solute(sol.xyz, sol.q, sol.sigma, sol.eps)
        out = rd.init()
        rh.set_solute(sol.xyz, sol.q, sol.sigma, sol.eps)
        for hb in host:
            hb.fill(np.nan)
        rh.init_host(*host)
        for i, k in enumerate(("u", "c", "h")):
            assert np.array_equal(out[k].cpu().numpy().reshape(S, M), host[i]), (step, k)
    for r in (rd, rh):
        r.close()
