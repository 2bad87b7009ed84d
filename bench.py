"""Benchmark of the 3D-RISM initialization path on GB300.

One step = one whole initialization of one solute through the C ABI:
solute upload, per-pair tables (mixing, cut-offs), tree build, proxy charges,
interaction lists, evaluation of u, c_lr, h_lr for every grid point and
solvent site, and the LJ tail integrals.  Default workload: the
tubulin-dimer-sized solute -- 13,600 atoms in a prolate 80x65x45 A ellipsoid
(net -24) on a 224x192x160 grid at 0.5 A with water O/H + 0.1 M Na+/Cl-
sites, LJ cut-off 9 A, treecode degree 8, theta 0.7 (synthetic, seeded).
``--workload globule2000`` runs the 2,000-atom globule on 128^3 instead.

value  = grid-point x site evaluations per second (Gpts.site/s), device
         outputs, CUDA events on the library's stream, L2 flushed between
         steps (256 MB write outside the timed events).
e2e    = the same step with HOST output buffers (pinned), the device-to-host
         copy of u, c, h inside the timed region.
Under torchrun each rank runs its own seeded solute (independent problems,
no collective): weak scaling, value = all ranks' points / max rank time.

--impl reference times the FP64 CPU oracle (the reference arm of this
project) on a bounded sample of the same workload on the host cores.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "grid-pt·site evals/s & init time per solute at stated error vs FP64 direct"
UNIT = "Gpts·site/s"
# name -> (index of the seeded workload definition, name of the workload with its sizes)
WORKLOADS = {"ellipsoid13600": (2, "ellipsoid13600_224x192x160"), "globule2000": (1, "globule2000_128cubed"),
             "sphere200": (0, "sphere200_64cubed")}
DEFAULT_WORKLOAD = "ellipsoid13600"
WORKLOAD = WORKLOADS[DEFAULT_WORKLOAD][1]


def _select(name):
    global WORKLOAD
    WORKLOAD = WORKLOADS[name][1]
    return WORKLOADS[name][0]


_WIDX = [WORKLOADS[DEFAULT_WORKLOAD][0]]


def _workload(seed=0):
    from paper_2109_09772_gb300 import inputs as I

    return I.workload(_WIDX[0], seed=seed)


def reduce_max(dist, v, device):
    """The slowest rank's value (max over ranks); the rank's own value without a process group."""
    if dist is None:
        return v
    import torch

    t = torch.tensor([float(v)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(world, S, M, ms):
    """Whole-job throughput in Gpts*site/s: every rank initializes its own solute of S sites on M points
    (weak scaling, independent problems), so a step of the slowest rank delivers world * S * M values."""
    return world * S * M / (ms * 1e-3) / 1e9


def _config(w, method, precision):
    return {"workload": WORKLOAD, "atoms": w.solute.n, "grid": list(w.grid.n), "spacing_A": w.grid.h,
            "sites": w.solvent.nsite, "lj_rcut_A": w.opts.get("lj_rcut"), "degree": w.opts.get("degree"),
            "theta": w.opts.get("theta"), "method": method, "precision": precision, "autotune": True,
            "outputs": "u, c_lr, h_lr (FP64 grids) + LJ tail integrals",
            "l2": f"flushed before every timed step by a 256 MB write (outputs {3 * w.solvent.nsite * w.grid.npts * 8 / 1e6:.0f} MB, "
                  f"inputs {w.solute.n * 48 / 1e3:.0f} KB)"}


class Clocks:
    """nvidia-smi sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.idx = device_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def wait_first(self, timeout_s=3.0):
        """Block until nvidia-smi has printed its first sample, so the samples cover the timed region."""
        t0 = time.perf_counter()
        while self.proc is not None and not self.lines and time.perf_counter() - t0 < timeout_s:
            time.sleep(0.01)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


# Algorithmic work per unit, counted from the loop bodies (thread instructions of one lane).
# Far and box-level pairs (k_far32, k_cp_eval): dx 2 FADD, d^2 1 FFMA, q/d 1 FMUL, Phi1 1 FADD, d 1 FMUL,
# -kappa d 1 FMUL, Phik 1 FFMA and the MUFU rsqrt and ex2: 10 flops (FFMA = 2).  The special-function pipe
# bounds them: on this part rsqrt issues at 16 and ex2 at 32 per clock per SM (a microbenchmark of
# independent MUFU chains, see the k_far32 profile summary), so a pair costs 1/16 + 1/32 SM clocks.
# Near pairs (k_near32): a tested pair 4 (dx 2, d^2 1, compare 1); a pair inside the LJ cut-off 4 + 2 S
# (compare, rcp, r^-6 2 FMUL, per site 2 FFMA); a pair inside r_short 10 + 4 F (two compares, rsqrt, q/d,
# table coordinate 2 FMUL, index 2, fraction 2, per field c / h a cubic piece 3 FFMA + 1 accumulate).
FLOPS_FAR = 10
MUFU_CLK_PER_PAIR = 1.0 / 16.0 + 1.0 / 32.0
NEAR_TESTED, NEAR_LJ_BASE, NEAR_LJ_SITE, NEAR_SR_BASE, NEAR_SR_FIELD = 4, 4, 2, 10, 4
FLOPS_LJ_SITE = 4
FLOPS_LJ_SHARED = 2
FP32_LANES_PER_SM = 128
SMS = 152
# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum of one ncu capture of the kernel as it
# stands), per workload; None when the kernel has changed since the capture or no capture was taken.
# "box" sums the box-level launches of one step (k_cp_work and its k_order where the boxes are ordered,
# k_cp_eval, k_cp_reduce, k_l2l per level, k_tdown).
TRAFFIC_BYTES = {
    "ellipsoid13600_224x192x160": {"k_far32": 163232256, "k_near32": 719858944, "box": 125013504},
    "globule2000_128cubed": {"k_far32": 33913088, "k_near32": 181672960, "box": 17674496},
}


def _alu_peak_tflops(sm_mhz):
    return SMS * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12


def run_gpu(args):
    import numpy as np
    import torch

    from paper_2109_09772_gb300 import build as B
    from paper_2109_09772_gb300 import rism as R

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    B.build()
    w = _workload(seed=rank)
    method = R.METHOD_TREECODE if args.method == "treecode" else R.METHOD_DIRECT
    prec = R.PREC_FP32 if args.precision == "fp32" else R.PREC_FP64
    # the autotuner picks the target-batch shape and leaf size during the (untimed) warm-up
    r = R.from_workload(w, method=method, precision=prec, debug_flags=2, autotune=0 if args.no_autotune else 1)
    S, M = w.solvent.nsite, w.grid.npts
    xyz, q, sg, ep = w.solute.xyz, w.solute.q, w.solute.sigma, w.solute.eps
    fields = ("u", "c", "h") if r.info()["kappa"] > 0 else ("u", "c")  # h needs ionic screening
    out = {k: r.empty_grid() for k in fields}
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    st = torch.cuda.current_stream()

    def step():
        r.set_solute(xyz, q, sg, ep)
        return r.init(u=True, c=True, h="h" in fields, lj_tail=True, out=out)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = Clocks(torch.cuda.current_device())
    clocks.start()
    clocks.wait_first()
    times, evals, launches, far_ms, near_ms, box_ms = [], [], 0, [], [], []
    torch.cuda.synchronize()
    t_wall0 = time.perf_counter()
    for _ in range(args.steps):
        flush.fill_(1.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        step()
        e1.record(st)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
        inf = r.info()
        evals.append(inf["eval_ms"])
        if inf["far_ms"] > 0:
            far_ms.append(inf["far_ms"])
            near_ms.append(inf["near_ms"])
            box_ms.append(inf["box_ms"])
        launches += inf["launches"]
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall0
    ck = clocks.stop()
    ms = reduce_max(dist, sum(times) / len(times), "cuda")
    value = job_value(world, S, M, ms)

    e2e = None
    if not args.no_e2e:
        # end to end: host (pinned) output buffers, device-to-host copies inside the timed region
        hu = torch.empty((S, M), dtype=torch.float64).pin_memory()
        hc = torch.empty((S, M), dtype=torch.float64).pin_memory()
        hh = torch.empty((S, M), dtype=torch.float64).pin_memory() if "h" in fields else None
        tail = np.zeros(S)
        P = lambda t: t.numpy()

        def step_host():
            r.set_solute(xyz, q, sg, ep)
            r.init_host(P(hu), P(hc), None if hh is None else P(hh), tail)

        for _ in range(2):
            step_host()
        et = []
        for _ in range(max(3, min(args.steps, 10))):
            flush.fill_(1.0)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            step_host()
            et.append(time.perf_counter() - t0)
        e2e_ms = reduce_max(dist, 1e3 * sum(et) / len(et), "cuda")
        e2e = {"value": job_value(world, S, M, e2e_ms), "unit": UNIT, "ms_per_step": e2e_ms,
               "h2d_bytes_per_step": int(xyz.nbytes + q.nbytes + sg.nbytes + ep.nbytes),
               "d2h_bytes_per_step": int(len(fields) * S * M * 8 + S * 8)}

    # accuracy of this step against the FP64 oracle at sampled points (rank 0 only; not timed)
    acc = None
    if rank == 0 and not args.no_check:
        from oracle import oracle as O
        from paper_2109_09772_gb300 import inputs as I

        # random points plus the grid point nearest each atom (where |u| peaks)
        nx, ny, nz = w.grid.n
        ijk = np.rint((w.solute.xyz - np.asarray(w.grid.origin)) / w.grid.h).astype(np.int64)
        ijk = np.clip(ijk, 0, np.array([nx - 1, ny - 1, nz - 1]))
        idx = np.union1d(I.sample_indices(M, args.check_points, seed=7), (ijk[:, 2] * ny + ijk[:, 1]) * nx + ijk[:, 0])
        ref = O.fields(O.Problem.from_workload(w), idx=idx)
        acc = {"points": int(idx.size)}
        for k in fields:
            g = out[k].reshape(S, -1)[:, torch.as_tensor(idx, device="cuda")].cpu().numpy()
            acc[k] = float(np.linalg.norm(g - ref[k]) / np.linalg.norm(ref[k]))
            acc[k + "_max_abs_over_max"] = float(np.abs(g - ref[k]).max() / np.abs(ref[k]).max())

    # rooflines of the evaluation kernels (CUDA events on the library stream); "roofline" is the dominant one
    inf = r.info()
    peaks, src = _peaks()
    pairs_far = inf["direct_pairs"] + inf["proxy_pairs"]
    sm_mhz = peaks.get("sm_max_mhz", 2070.0)
    clk = sm_mhz * 1e6
    mean = lambda v: (sum(v) / len(v)) if v else 0.0
    kern = {}
    if method == R.METHOD_TREECODE and far_ms:
        xu_peak = SMS * clk / MUFU_CLK_PER_PAIR / 1e9  # Gpairs/s
        issue_peak = SMS * 4 * 32 * clk / 1e12  # T thread-instructions/s
        nf = 2  # the step requests c and h
        near_inst = (inf["near_tested"] * NEAR_TESTED + inf["lj_pairs"] * (NEAR_LJ_BASE + NEAR_LJ_SITE * S) +
                     inf["sr_pairs"] * (NEAR_SR_BASE + NEAR_SR_FIELD * nf))
        for name, t_ms, work, peak, unit, bound, traffic, desc in (
                ("k_far32", mean(far_ms), pairs_far, xu_peak, "Gpairs/s", "alu", TRAFFIC_BYTES[WORKLOAD]["k_far32"],
                 "far field of the target batches: direct and source-proxy pairs; MUFU-bound"),
                ("box level (k_cp_eval + interpolation)", mean(box_ms), inf["cp_pairs"], xu_peak, "Gpairs/s", "alu",
                 TRAFFIC_BYTES[WORKLOAD]["box"], "proxy-target pairs, timed with the downward pass and interpolation"),
                ("k_near32", mean(near_ms), near_inst, issue_peak, "Tinst/s", "alu", TRAFFIC_BYTES[WORKLOAD]["k_near32"],
                 "near field + epilogue: algorithmic instructions of the tested / LJ / short-range pairs against "
                 "the issue rate (4 schedulers x 32 lanes x clock per SM)")):
            if t_ms <= 0:
                continue
            scale = 1e9 if unit == "Gpairs/s" else 1e12
            ach = work / (t_ms * 1e-3) / scale
            kern[name] = {"bound": bound, "achieved": ach, "peak": peak, "unit": unit, "frac": ach / peak,
                          "traffic": traffic, "kernel_ms": t_ms, "work_per_launch": work, "what": desc,
                          "peak_source": f"{SMS} SMs at {sm_mhz:.0f} MHz ({src} sm_max_mhz)"}
        kname = max(kern, key=lambda k: kern[k]["kernel_ms"])
        roof = dict(kern[kname], kernel=kname)
    else:
        kern_ms = mean(evals)
        flops = pairs_far * (FLOPS_FAR + FLOPS_LJ_SHARED + FLOPS_LJ_SITE * S)
        peak = _alu_peak_tflops(sm_mhz)
        achieved = flops / (kern_ms * 1e-3) / 1e12 if kern_ms > 0 else None
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": (achieved / peak) if achieved else None, "traffic": None,
                "kernel": "k_direct32 / k_direct64 (whole direct sum)", "kernel_ms": kern_ms,
                "peak_source": f"FP32 FMA pipe: {SMS} SMs x {FP32_LANES_PER_SM} lanes x 2 x {sm_mhz:.0f} MHz ({src})"}
    timing = {"step_ms": ms, "far_ms": (sum(far_ms) / len(far_ms)) if far_ms else None,
              "near_ms": (sum(near_ms) / len(near_ms)) if near_ms else None,
              "box_ms": (sum(box_ms) / len(box_ms)) if box_ms else None,
              "eval_ms": sum(evals) / len(evals) if evals else None}
    res = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": ("f32 (FP32 pair terms, float-float sums, each output rounded to FP32 and stored as FP64)"
                     if prec == R.PREC_FP32 else "f64"),
           "data": "synthetic (seeded globule, protein density)",
           "config": _config(w, args.method, args.precision), "e2e": e2e, "gpu_launches": launches,
           "clocks": ck, "roofline": roof, "roofline_kernels": kern, "timing": timing,
           "error_vs_fp64_oracle_rel_l2": acc,
           "counts": {k: inf[k] for k in ("direct_pairs", "proxy_pairs", "cp_pairs", "near_pairs", "near_tested",
                                            "lj_pairs", "sr_pairs", "tree_nodes", "tree_proxied", "tree_leaves",
                                            "tree_boxes", "kernel_variant")},
           "wall_s": t_wall}
    if rank == 0 and not args.no_fp64:
        # the plain FP64 direct sum on the same GPU, one timed step (the comparison of the headline)
        r64 = R.from_workload(w, method=R.METHOD_DIRECT, precision=R.PREC_FP64)
        r64.init(out=out)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        r64.set_solute(xyz, q, sg, ep)
        r64.init(out=out, lj_tail=True)
        e1.record(st)
        torch.cuda.synchronize()
        t64 = e0.elapsed_time(e1)
        res["fp64_direct_ms"] = t64
        res["speedup_vs_fp64_direct"] = t64 / ms
        r64.close()
    if rank == 0 and world == 1 and not args.no_cpu:
        res["cpu_baseline"] = cpu_baseline(args.cpu_seconds)
    r.close()
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(res))


def cpu_baseline(seconds=15.0, seed=0):
    """The FP64 oracle as it stands on the host cores, on a bounded sample of grid points of the same
    workload; value in the bench's unit."""
    import numpy as np

    from oracle import oracle as O
    from paper_2109_09772_gb300 import inputs as I

    w = _workload(seed)
    p = O.Problem.from_workload(w)
    cores = os.cpu_count() or 1
    # calibrate: grow the sample until one run takes a second (start-up costs no longer dominate), then
    # size the measured sample for about `seconds` of work
    n = 2000
    while True:
        idx = I.sample_indices(w.grid.npts, n, seed=11)
        t0 = time.perf_counter()
        O.fields(p, idx=idx, nthreads=cores)
        t = time.perf_counter() - t0
        if t >= 1.0 or n >= w.grid.npts:
            break
        n = min(w.grid.npts, n * 4)
    n = int(min(w.grid.npts, max(2000, n * seconds / max(t, 1e-3))))
    idx = I.sample_indices(w.grid.npts, n, seed=12)
    t0 = time.perf_counter()
    O.fields(p, idx=idx, nthreads=cores)
    t = time.perf_counter() - t0
    S = w.solvent.nsite
    return {"value": S * n / t / 1e9, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{n} random grid points of {WORKLOAD} (all {w.solute.n} atoms, {S} sites, u+c+h), "
                      f"{t:.1f} s"}


def run_reference(args):
    """Reference arm: the FP64 CPU oracle, bounded sample per step, on the host cores."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import numpy as np

    from oracle import oracle as O
    from paper_2109_09772_gb300 import inputs as I

    O.build()
    w = _workload(0)
    p = O.Problem.from_workload(w)
    cores = os.cpu_count() or 1
    S = w.solvent.nsite
    npts = max(100, int(args.ref_points))
    for k in range(args.warmup):
        O.fields(p, idx=I.sample_indices(w.grid.npts, min(npts, 200), seed=100 + k), nthreads=cores)
    ts = []
    for k in range(args.steps):
        idx = I.sample_indices(w.grid.npts, npts, seed=200 + k)
        t0 = time.perf_counter()
        O.fields(p, idx=idx, nthreads=cores)
        ts.append(time.perf_counter() - t0)
    ms = 1e3 * sum(ts) / len(ts)
    value = S * npts / (ms * 1e-3) / 1e9
    sample = f"{npts} random grid points per step of {WORKLOAD} (all {w.solute.n} atoms, {S} sites, u+c+h)"
    print(json.dumps({"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1,
                      "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
                      "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                      "config": _config(w, "oracle (direct FP64, CPU)", "fp64"),
                      "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                                       "sample": sample},
                      "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))


# ------------------------------------------------------------------ suites
# Measurements of the other workloads of the benchmark plan (not the default line).

def _events_ms(fn, reps=3):
    import torch

    st = torch.cuda.current_stream()
    ts = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(st)
        fn()
        e1.record(st)
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    return min(ts)


def _rel(a, b):
    import numpy as np

    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def suite_pareto(args):
    """13,600-atom prolate ellipsoid, 224x192x160 grid: FP64 direct vs FP32 direct vs FP32 treecode at
    degrees 4, 6, 8 and theta 0.5..0.8 (time per initialization, error vs the FP64 oracle at sampled points)."""
    import numpy as np
    import torch

    from oracle import oracle as O
    from paper_2109_09772_gb300 import build as B
    from paper_2109_09772_gb300 import inputs as I
    from paper_2109_09772_gb300 import rism as R

    B.build()
    torch.cuda.set_device(0)
    w = I.workload(2)
    S, M = w.solvent.nsite, w.grid.npts
    rng = np.random.default_rng(5)
    idx = np.union1d(I.sample_indices(M, 3000, seed=6), rng.choice(M, 0, replace=False))
    ref = O.fields(O.Problem.from_workload(w), idx=idx)
    tidx = torch.as_tensor(idx, device="cuda")

    def run(**opts):
        r = R.from_workload(w, **opts)
        out = r.init()
        torch.cuda.synchronize()
        xyz, q, sg, ep = w.solute.xyz, w.solute.q, w.solute.sigma, w.solute.eps

        def step():
            r.set_solute(xyz, q, sg, ep)
            r.init(out=out)

        ms = _events_ms(step, reps=args.reps)
        err = {k: _rel(out[k].reshape(S, -1)[:, tidx].cpu().numpy(), ref[k]) for k in ("u", "c", "h")}
        info = r.info()
        r.close()
        return ms, err, info

    ms64, e64, _ = run(method=R.METHOD_DIRECT, precision=R.PREC_FP64)
    print(json.dumps({"suite": "pareto", "workload": "ellipsoid13600_224x192x160", "method": "direct",
                      "precision": "fp64", "ms": ms64, "gpts_site_s": S * M / (ms64 * 1e-3) / 1e9, "err": e64}),
          flush=True)
    ms32, e32, _ = run(method=R.METHOD_DIRECT, precision=R.PREC_FP32)
    print(json.dumps({"suite": "pareto", "method": "direct", "precision": "fp32", "ms": ms32,
                      "speedup_vs_fp64_direct": ms64 / ms32, "err": e32}), flush=True)
    cases = [(deg, th, 1) for deg in (4, 6, 8) for th in (0.5, 0.6, 0.7, 0.8)] + [(8, 0.7, 0)]
    for deg, th, tp in cases:
        ms, e, info = run(method=R.METHOD_TREECODE, precision=R.PREC_FP32, degree=deg, theta=th, autotune=1,
                          target_proxies=tp, debug_flags=2)
        print(json.dumps({"suite": "pareto", "method": "treecode", "precision": "fp32", "degree": deg,
                          "theta": th, "target_proxies": tp, "ms": ms, "speedup_vs_fp64_direct": ms64 / ms,
                          "gpts_site_s": S * M / (ms * 1e-3) / 1e9, "err": e,
                          "direct_pairs": info["direct_pairs"], "proxy_pairs": info["proxy_pairs"],
                          "cp_pairs": info["cp_pairs"], "near_pairs": info["near_pairs"],
                          "box_ms": info["box_ms"], "far_ms": info["far_ms"], "near_ms": info["near_ms"],
                          "tree_boxes": info["tree_boxes"], "variant": info["kernel_variant"],
                          "batch": info["batch"]}), flush=True)


def suite_batched(args):
    """32 solutes, 500..8,000 atoms (log-uniform), own grids: one graph-captured persistent launch against 32
    sequential treecode initializations."""
    import numpy as np
    import torch

    from oracle import oracle as O
    from paper_2109_09772_gb300 import build as B
    from paper_2109_09772_gb300 import inputs as I
    from paper_2109_09772_gb300 import rism as R

    B.build()
    torch.cuda.set_device(0)
    ws = I.batch_workloads(count=32, seed=0)
    rs = [R.from_workload(w, method=R.METHOD_TREECODE, precision=R.PREC_FP32) for w in ws]
    outs = [r.init() for r in rs]
    torch.cuda.synchronize()

    def seq():
        for r, o in zip(rs, outs):
            r.set_solute(*(getattr(r, "_sol")))
            r.init(out=o)

    for r, w in zip(rs, ws):
        r._sol = (w.solute.xyz, w.solute.q, w.solute.sigma, w.solute.eps)
    ms_seq = _events_ms(seq, reps=args.reps)
    bouts = [R.potential_batched(rs)]  # capture
    torch.cuda.synchronize()

    def bat():
        for r in rs:
            r.set_solute(*r._sol)
        bouts[0] = R.potential_batched(rs, out=bouts[0])

    ms_bat = _events_ms(bat, reps=args.reps)
    pts = sum(w.solvent.nsite * w.grid.npts for w in ws)
    # parity of the batched outputs on three solutes (sampled points)
    errs = []
    for k in (0, 15, 31):
        w = ws[k]
        idx = I.sample_indices(w.grid.npts, 1000, seed=k)
        ref = O.fields(O.Problem.from_workload(w), idx=idx)
        o = bouts[0][k]
        errs.append({f: _rel(o[f].reshape(w.solvent.nsite, -1)[:, torch.as_tensor(idx, device="cuda")].cpu().numpy(),
                             ref[f]) for f in ("u", "c", "h")})
    print(json.dumps({"suite": "batched", "solutes": len(ws), "atoms": [w.solute.n for w in ws],
                      "grids": [w.grid.n[0] for w in ws], "ms_sequential": ms_seq, "ms_batched_graph": ms_bat,
                      "speedup": ms_seq / ms_bat, "gpts_site_s_batched": pts / (ms_bat * 1e-3) / 1e9,
                      "err_sampled": errs}), flush=True)
    for r in rs:
        r.close()


def suite_adjoint(args):
    """55,000 atoms (four stacked ellipsoids), 320x320x384 grid: forward u + c with FP32 pairs and the
    backward pass for a smooth seeded cotangent (correlation length 3 A, amplitude 0.5) used for both u and c;
    gradients of sampled atoms against the FP64 oracle."""
    import numpy as np
    import torch

    from oracle import oracle as O
    from paper_2109_09772_gb300 import build as B
    from paper_2109_09772_gb300 import inputs as I
    from paper_2109_09772_gb300 import rism as R

    B.build()
    torch.cuda.set_device(0)
    w = I.workload(4)
    nx, ny, nz = w.grid.n
    S = w.solvent.nsite
    G = np.stack([I.gaussian_random_field((nz, ny, nx), w.grid.h, 700 + s, corr_len=3.0, amplitude=0.5)
                  for s in range(S)])
    Gd = torch.as_tensor(G, device="cuda")
    r = R.from_workload(w, method=R.METHOD_TREECODE, precision=R.PREC_FP32)
    out = {"u": r.empty_grid(), "c": r.empty_grid()}
    r.init(u=True, c=True, h=False, out=out)
    sol = (w.solute.xyz, w.solute.q, w.solute.sigma, w.solute.eps)

    def fwd():
        r.set_solute(*sol)
        r.init(u=True, c=True, h=False, out=out)

    ms_fwd = _events_ms(fwd, reps=args.reps)
    g = r.backward(Gd, Gd, None)
    torch.cuda.synchronize()
    ms_bwd = _events_ms(lambda: r.backward(Gd, Gd, None), reps=max(1, args.reps - 1))
    atoms = np.sort(np.random.default_rng(64).choice(w.solute.n, args.adj_atoms, replace=False))
    t0 = time.perf_counter()
    ref = O.grad(O.Problem.from_workload(w), atoms, G, G, None)
    t_or = time.perf_counter() - t0
    gg = {k: v.cpu().numpy() for k, v in g.items()}
    err = {"xyz": _rel(gg["xyz"][atoms], ref[:, 0:3]), "q": _rel(gg["q"][atoms], ref[:, 3]),
           "sigma": _rel(gg["sigma"][atoms], ref[:, 4]), "eps": _rel(gg["eps"][atoms], ref[:, 5])}
    pairs = w.solute.n * w.grid.npts
    print(json.dumps({"suite": "adjoint", "workload": "stack55000_320x320x384", "ms_forward_u_c": ms_fwd,
                      "ms_backward": ms_bwd, "backward_pairs_per_s": pairs / (ms_bwd * 1e-3),
                      "atoms_checked": int(atoms.size), "grad_rel_l2_vs_oracle": err,
                      "oracle_seconds": t_or}), flush=True)
    r.close()


def suite_precision(args):
    """Split of the treecode's error against the FP64 oracle (configs 1 and 2, sampled points and the point
    nearest each atom): interpolation (treecode vs the FP32 direct sum of the same pairs) and FP32 rounding
    (FP32 direct sum vs oracle), next to the FP64 direct sum vs oracle."""
    import numpy as np
    import torch

    from oracle import oracle as O
    from paper_2109_09772_gb300 import build as B
    from paper_2109_09772_gb300 import inputs as I
    from paper_2109_09772_gb300 import rism as R

    B.build()
    torch.cuda.set_device(0)
    for wi in (1, 2):
        w = I.workload(wi)
        S, M = w.solvent.nsite, w.grid.npts
        nx, ny, nz = w.grid.n
        ijk = np.clip(np.rint((w.solute.xyz - np.asarray(w.grid.origin)) / w.grid.h).astype(np.int64), 0,
                      np.array([nx - 1, ny - 1, nz - 1]))
        idx = np.union1d(I.sample_indices(M, 20000, seed=31), (ijk[:, 2] * ny + ijk[:, 1]) * nx + ijk[:, 0])
        t = torch.as_tensor(idx, device="cuda")
        ref = O.fields(O.Problem.from_workload(w), idx=idx)
        got = {}
        for name, kw in (("direct_fp64", dict(method=R.METHOD_DIRECT, precision=R.PREC_FP64)),
                         ("direct_fp32", dict(method=R.METHOD_DIRECT, precision=R.PREC_FP32)),
                         ("treecode_fp32", dict(method=R.METHOD_TREECODE, precision=R.PREC_FP32))):
            r = R.from_workload(w, **kw)
            out = r.init()
            got[name] = {k: out[k].reshape(S, -1)[:, t].cpu().numpy() for k in ("u", "c", "h")}
            r.close()
        rel = lambda a, b: float(np.linalg.norm(a - b) / np.linalg.norm(b))
        res = {"suite": "precision", "workload": w.name, "points": int(idx.size)}
        for k in ("u", "c", "h"):
            res[k] = {"direct_fp64_vs_oracle": rel(got["direct_fp64"][k], ref[k]),
                      "direct_fp32_vs_oracle": rel(got["direct_fp32"][k], ref[k]),
                      "treecode_vs_direct_fp32": rel(got["treecode_fp32"][k], got["direct_fp32"][k]),
                      "treecode_vs_oracle": rel(got["treecode_fp32"][k], ref[k])}
        print(json.dumps(res), flush=True)


def suite_taylor(args):
    """The two far-field approximation families on the same target boxes, acceptance test and near field:
    barycentric-Lagrange Chebyshev proxies and the paper's Taylor moments (Sec. 2.3), degrees / orders 4..10 at
    theta 0.5 and 0.7, on the 2,000-atom globule and the 13,600-atom ellipsoid: time per initialization (and
    the box-level part) against the error at sampled points."""
    import numpy as np
    import torch

    from oracle import oracle as O
    from paper_2109_09772_gb300 import build as B
    from paper_2109_09772_gb300 import inputs as I
    from paper_2109_09772_gb300 import rism as R

    B.build()
    torch.cuda.set_device(0)
    for wi in (1, 2):
        w = I.workload(wi)
        S = w.solvent.nsite
        idx = I.sample_indices(w.grid.npts, 3000, seed=2)
        ref = O.fields(O.Problem.from_workload(w), idx=idx)
        t = torch.as_tensor(idx, device="cuda")
        for approx in (R.APPROX_BARYCENTRIC, R.APPROX_TAYLOR):
            for th in (0.5, 0.7):
                for p in (4, 6, 8, 10):
                    r = R.from_workload(w, method=R.METHOD_TREECODE, precision=R.PREC_FP32, degree=p, theta=th,
                                        approx=approx, debug_flags=2)
                    out = r.init()
                    torch.cuda.synchronize()
                    sol = (w.solute.xyz, w.solute.q, w.solute.sigma, w.solute.eps)

                    def step():
                        r.set_solute(*sol)
                        r.init(out=out)

                    ms = _events_ms(step, reps=args.reps)
                    inf = r.info()
                    err = {k: _rel(out[k].reshape(S, -1)[:, t].cpu().numpy(), ref[k]) for k in ("c", "h")}
                    print(json.dumps({"suite": "taylor", "workload": w.name,
                                      "approx": "taylor" if approx == R.APPROX_TAYLOR else "barycentric",
                                      "theta": th, "order": p, "ms": ms, "box_ms": inf["box_ms"],
                                      "err_rel_l2": err}), flush=True)
                    r.close()


def suite_kspace(args):
    """Reciprocal-space asymptotics (eqs. (dcf-k)/(tcf-k)) of the 13,600-atom ellipsoid on the half spectrum of
    its 224x192x160 grid: the whole half spectrum, and with the frequency cut-off of Sec. 2.5 at tolerances
    1e-4 and 1e-2 of the largest |c(k)|; CUDA events around the call's kernels; FMA-pipe roofline of the
    structure-factor sum (4 FP32 FMAs per kept (k, atom) pair); sampled errors against the FP64 oracle."""
    import numpy as np
    import torch

    from oracle import oracle as O
    from paper_2109_09772_gb300 import build as B
    from paper_2109_09772_gb300 import inputs as I
    from paper_2109_09772_gb300 import rism as R

    B.build()
    torch.cuda.set_device(0)
    w = I.workload(2)
    nx, ny, nz = w.grid.n
    nh = nx // 2 + 1
    r = R.from_workload(w, method=R.METHOD_TREECODE, precision=R.PREC_FP32, debug_flags=2)
    p = O.Problem.from_workload(w)
    idx = I.sample_indices(nh * ny * nz, 1500, seed=4)
    t = torch.as_tensor(idx, device="cuda")
    peaks, src = _peaks()
    clk = peaks.get("sm_max_mhz", 2070.0) * 1e6
    fma_peak = SMS * FP32_LANES_PER_SM * clk  # FMA/s
    c0, _, _ = r.asymptotics_k(0.0)
    cmax = float(c0.abs().max())
    kx = 2 * np.pi * np.arange(nh) / (nx * w.grid.h)
    ky = 2 * np.pi * np.fft.fftfreq(ny, d=w.grid.h)
    kz = 2 * np.pi * np.fft.fftfreq(nz, d=w.grid.h)
    k2 = (kz[:, None, None] ** 2 + ky[None, :, None] ** 2 + kx[None, None, :] ** 2).ravel()
    for rel in (0.0, 1e-4, 1e-2):
        tol = rel * cmax
        ms = []
        for _ in range(max(3, args.reps)):
            c, h, kc = r.asymptotics_k(tol)
            torch.cuda.synchronize()
            ms.append(r.info()["eval_ms"])
        ms = min(ms)
        kept = int(np.count_nonzero(k2 <= kc * kc)) if kc > 0 else k2.size
        fma = 4.0 * kept * w.solute.n
        ref = O.kspace(p, kcut=kc, idx=idx)
        err = {k: float(np.linalg.norm(v.reshape(r.S, -1)[:, t].cpu().numpy() - ref[k]) / np.linalg.norm(ref[k]))
               for k, v in (("c", c), ("h", h))}
        print(json.dumps({"suite": "kspace", "workload": "ellipsoid13600_224x192x160", "k_tol_rel": rel,
                          "k_cut": kc, "kept_k": kept, "half_spectrum": int(k2.size), "ms": ms,
                          "roofline": {"bound": "alu", "unit": "FMA/s", "achieved": fma / (ms * 1e-3),
                                       "peak": fma_peak, "frac": fma / (ms * 1e-3) / fma_peak,
                                       "peak_source": f"FP32 FMA pipe, {SMS} SMs x 128 lanes at "
                                                      f"{clk / 1e6:.0f} MHz ({src})"},
                          "err_sampled_rel_l2": err}), flush=True)
    r.close()


def suite_lra(args):
    """The all-space long-range integral (last integral of eq. (excess-chemical-potential-LRA)), O(N_atom^2)
    atom pairs, for the 13,600-atom ellipsoid and the 55,000-atom stack; MUFU-bound pair roofline."""
    import torch

    from paper_2109_09772_gb300 import build as B
    from paper_2109_09772_gb300 import inputs as I
    from paper_2109_09772_gb300 import rism as R

    B.build()
    torch.cuda.set_device(0)
    peaks, src = _peaks()
    clk = peaks.get("sm_max_mhz", 2070.0) * 1e6
    xu_peak = SMS * clk / MUFU_CLK_PER_PAIR
    for idx in (2, 4):
        w = I.workload(idx)
        r = R.from_workload(w, method=R.METHOD_DIRECT, precision=R.PREC_FP32)
        T = r.lra_integral()
        ms = _events_ms(lambda: r.lra_integral(), reps=max(3, args.reps))
        pairs = float(w.solute.n) ** 2
        print(json.dumps({"suite": "lra", "workload": w.name, "atoms": w.solute.n, "T_A3": list(T), "ms": ms,
                          "pairs_per_s": pairs / (ms * 1e-3),
                          "roofline": {"bound": "alu", "unit": "pairs/s", "achieved": pairs / (ms * 1e-3),
                                       "peak": xu_peak, "frac": pairs / (ms * 1e-3) / xu_peak,
                                       "peak_source": "rsqrt + ex2 per pair on the special-function pipe"}}),
              flush=True)
        r.close()


def suite_mufu(args):
    """Issue rates of rsqrt / ex2 / rcp / FFMA / DFMA (thread ops per clock per SM): compiles and runs the
    microbenchmark in microbench/ (the denominators of the pair kernels' rooflines)."""
    import tempfile

    src = os.path.join(ROOT, "microbench", "mufu_rates.cu")
    with tempfile.TemporaryDirectory() as d:
        exe = os.path.join(d, "mufu_rates")
        subprocess.run(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-o", exe, src], check=True)
        r = subprocess.run([exe], capture_output=True, text=True, check=True)
    print(r.stdout.strip(), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--method", default="treecode", choices=["treecode", "direct"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--ref-points", type=int, default=30000)
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS))
    ap.add_argument("--check-points", type=int, default=20000)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-check", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="default launch shape (profiling runs)")
    ap.add_argument("--suite", default=None, choices=["pareto", "batched", "adjoint", "mufu", "kspace", "lra", "precision",
                                                      "taylor"])
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--adj-atoms", type=int, default=16)
    args = ap.parse_args()
    _WIDX[0] = _select(args.workload)
    if args.suite:
        {"pareto": suite_pareto, "batched": suite_batched, "adjoint": suite_adjoint, "mufu": suite_mufu,
         "kspace": suite_kspace, "lra": suite_lra, "precision": suite_precision,
         "taylor": suite_taylor}[args.suite](args)
        return
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
