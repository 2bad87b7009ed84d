"""The multi-rank host logic of bench.py on CPU: two gloo ranks, each with its own seeded solute of the same
shape (independent problems, weak scaling); the step time is the slowest rank's and the job value counts every
rank's points."""
import os

import numpy as np
import pytest


def _rank(rank, world, port, q):
    import torch.distributed as dist

    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w = bench._workload(seed=rank)
        ms = 2.0 + rank  # rank 1 is the slow one
        ms_max = bench.reduce_max(dist, ms, "cpu")
        value = bench.job_value(world, w.solvent.nsite, w.grid.npts, ms_max)
        q.put((rank, ms_max, value, w.solute.n, tuple(w.grid.n), float(w.solute.xyz[0, 0]), w.solvent.nsite))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_weak_scaling():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + (os.getpid() % 1000)
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=240) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, ms0, v0, n0, g0, x0, s0), (r1, ms1, v1, n1, g1, x1, s1) = res
    assert ms0 == ms1 == 3.0  # both ranks report the slowest rank's time
    # the default workload: the 13,600-atom ellipsoid on 224 x 192 x 160 with 4 sites, one per rank
    assert n0 == n1 == 13600 and g0 == g1 == (224, 192, 160) and s0 == s1 == 4
    assert v0 == v1 == pytest.approx(2 * 4 * 224 * 192 * 160 / 3.0e-3 / 1e9)
    assert x0 != x1  # each rank has its own seeded solute


def test_single_rank_without_process_group():
    import bench

    assert bench.reduce_max(None, 1.5, "cpu") == 1.5
    assert bench.job_value(1, 4, 1000, 2.0) == pytest.approx(4 * 1000 / 2e-3 / 1e9)
    a, b = bench._workload(seed=0), bench._workload(seed=1)
    assert a.solute.n == b.solute.n and not np.allclose(a.solute.xyz, b.solute.xyz)


def test_reference_arm_json_line_on_cpu():
    """`bench.py --impl reference` (the oracle on the host cores) prints one JSON line with the bench's metric and
    unit and no transfers; a rank other than 0 prints nothing and exits 0."""
    import json
    import subprocess
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    cmd = [sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--steps", "1", "--warmup", "3",
           "--ref-points", "200"]
    r = subprocess.run(cmd, cwd=root, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    import bench

    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["value"] > 0 and d["higher_is_better"] is True and d["steps"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    r1 = subprocess.run(cmd, cwd=root, capture_output=True, text=True, timeout=300, env=dict(os.environ, RANK="1"))
    assert r1.returncode == 0 and r1.stdout.strip() == ""
