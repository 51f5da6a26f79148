#!/usr/bin/env python
"""Benchmark of the treecode BEM hot path on one GB300 (or N replicas).

Workload (the two-sphere configuration the metric is quoted on): a spherical
molecule of radius 4 A (icosphere, 20480 panels) with a central +1e charge,
eps_in 4, next to a sphere of radius 4 A (20480 panels) with imposed charge
0.05 C/m^2, centres 12 A apart, eps_out 80, kappa 0.125 1/A; K=7, 19-point
near rule, 9 points per edge, treecode theta 0.5, P 6; GMRES tol 1e-6 with
FP32 inner solves and FP64 residual refinement.

One step = the whole hot path: Morton sort + octree + geometry + lists +
near-field precompute (pgb_tree_reset + pgb_tree_build, nothing cached), the FP32+refinement GMRES solve (pgb_solve) and
the energies (pgb_energy), inputs resident on the device.  value = treecode
matvecs per second inside those steps (all operator applications of the solve,
FP32 and FP64, divided by the step time).  L2 is flushed (512 MB write)
before each timed step; the flush is outside the timed intervals.

--impl reference times the CPU FP64 oracle (direct-sum rows of the same
operator) on a bounded sample of the same workload.
"""
import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "treecode matvecs/sec and GMRES solve ms at 1e-5 energy err, FP32+refine vs FP64"
UNIT = "matvecs/s"
WORKLOAD = "two spheres r=4 A, 2 x 20480 panels, sigma=0.05 C/m^2, R=12 A"
PARAMS = dict(K=7, K_near=19, n_edge=9, P=6, theta=0.5, leaf_size=32, group_size=32, p2p_item=64, m2p_item=64,
              precond=0, graphs=2, lanes=4, overlap=0, batch=1, residual=1)
TOL = 1e-6
RESTART = 100
MAX_ITER = 2000


def device_peaks(dev):
    """FP32 ALU peak of the device from its SM count (cudaDevAttrMultiProcessorCount
    through torch) and the maximum SM clock (sm_max_mhz of MEASURED_PEAKS.json,
    else 2070 MHz): SMs x 128 FP32 lanes x 2 flop (FMA) x clock."""
    import torch
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    mhz = float(load_peaks().get("sm_max_mhz", 2070.0))
    tf = n_sm * 128 * 2 * mhz * 1e6 / 1e12
    note = (f"{n_sm} SMs (device attribute) x 128 FP32 lanes x 2 flop x {mhz:.0f} MHz (sm_max_mhz of "
            f"MEASURED_PEAKS.json): derived, the file holds no FP32 figure")
    return {"fp32_tflops": tf, "sm_count": n_sm, "sm_max_mhz": mhz, "note": note}


def workload_bodies(level=5):
    import synth
    v, f = synth.icosphere(level, 4.0)
    mol = dict(kind="dielectric", verts=v, tris=f, eps_in=4.0, qxyz=np.zeros((1, 3)), q=np.array([1.0]), bc=0.0)
    srf = dict(kind="sigma", verts=v + np.array([12.0, 0.0, 0.0]), tris=f, eps_in=1.0, qxyz=np.zeros((0, 3)),
               q=np.zeros(0), bc=0.05)
    return [mol, srf]


# ------------------------------------------------------------------ flops
def p2p_flops(laplace):
    """FP32 operations per target x source-point pair of the P2P tile loop
    (rsqrt and exp counted as one each): difference 3, r^2 5, rsqrt 1, n.d 5,
    1/r^2 and t 2, Yukawa 10, Laplace 3."""
    return 26 + (3 if laplace else 0)


def m2p_flops(P, laplace):
    """Operations per (target, far node) of the far-field evaluation as the
    kernel runs it (far_eval: monomials of S = R/r^2 in nested order, one
    product each, summed per degree against the node's coefficients), counted
    term by term: setup 22 (R 3, r^2 5, rsqrt 1, 1/r^2 1, S 3, r 1, x 1, x^2 1,
    g_1 1, exp 1, prefactor 2, final product 2), T - 1 monomial products,
    2 per Yukawa multiply-add, the radial factors g_p (3 each for p >= 2) and
    their multiply-adds (2 each for p >= 1); Laplace adds 2 per term and 1."""
    T = (P + 1) * (P + 2) * (P + 3) // 6
    yuk = 22 + (T - 1) + 2 * T + 2 * min(P, 1) + 5 * max(P - 1, 0)
    return yuk + ((2 * T + 1) if laplace else 0)


def p2p_kernel_flops(info):
    yp = info["p2p_pairs"] - info["p2p_laplace_pairs"]
    return yp * p2p_flops(False) + info["p2p_laplace_pairs"] * p2p_flops(True)


def m2p_kernel_flops(info, P):
    ym = info["m2p_pairs"] - info["m2p_laplace_pairs"]
    return ym * m2p_flops(P, False) + info["m2p_laplace_pairs"] * m2p_flops(P, True)


# ------------------------------------------------------------------ clocks
class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(index), "--query-gpu=" + self.FIELDS,
                                       "--format=csv,noheader,nounits", "-lms", "50"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        rows = [r.split(",") for r in open(self.f.name).read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], None, set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
            except (ValueError, IndexError):
                continue
            for nm, val in zip(names, r[5:9]):
                if "Active" in val and "Not" not in val:
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ profile
def kernel_source_hash():
    """First 16 hex digits of the SHA-256 of the treecode kernels' sources
    (treecode.cuh, then ds.cuh): the key under which a committed ncu summary
    records the source it was taken on."""
    h = hashlib.sha256()
    for f in ("treecode.cuh", "ds.cuh"):
        h.update(open(os.path.join(ROOT, "paper_1506_03745_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def recorded_traffic(kernel):
    """dram bytes per launch of `kernel` from the committed ncu summary
    (profiles/<kernel>_two_sphere.txt), if it was taken on the current kernel
    source."""
    name = kernel.split("<")[0]
    path = os.path.join(ROOT, "profiles", f"{name}_fp32_two_sphere.txt")
    if not os.path.exists(path):
        return None
    h = kernel_source_hash()
    kv = {}
    for line in open(path):
        if "=" in line and not line.startswith("#"):
            k, v = line.split("=", 1)
            kv[k.strip()] = v.strip()
    if kv.get("kernel_sources_sha256_16") != h or "dram_bytes_per_launch_full" not in kv:
        return None
    return float(kv["dram_bytes_per_launch_full"])


def recorded_counters(fname):
    """key = value lines of a committed ncu summary (profiles/fname) when its
    recorded source hash matches the current kernels (else empty)."""
    path = os.path.join(ROOT, "profiles", fname)
    if not os.path.exists(path):
        return {}
    h = kernel_source_hash()
    kv = {}
    for line in open(path):
        if "=" in line and not line.startswith("#"):
            k, v = line.split("=", 1)
            kv[k.strip()] = v.strip()
    if kv.get("kernel_sources_sha256_16") != h:
        return {}
    out = {}
    for k, v in kv.items():
        try:
            out[k] = float(v)
        except ValueError:
            pass
    return out


def load_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


# ------------------------------------------------------------------ reference (oracle)
def cpu_info():
    """Host cores the oracle runs on (os.cpu_count) and the CPU model."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if model is None:
        try:
            for line in open("/proc/cpuinfo"):
                if line.lower().startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
        except OSError:
            pass
    return os.cpu_count() or 1, model or "unknown"


def _oracle_rows_task(task):
    """Worker: direct-sum FP64 oracle rows of the two-sphere workload for the
    molecule targets [t0, t1) (both rows of each); returns seconds."""
    t0, t1, seed = task
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from problems import oracle_system
    so = oracle_system(workload_bodies(), theta=0.0)
    x = np.random.default_rng(seed).normal(size=so.n)
    c0 = time.perf_counter()
    so.apply_rows(x, 0, np.arange(t0, t1))
    return time.perf_counter() - c0


def _dense_rows_task(task):
    """Worker: rows of the dense oracle system (oracle.bem.System.assemble_rows)
    for a chunk of target panels of one body of a small workload."""
    name, body, rows = task
    so = _dense_system(name)
    per = [np.zeros(0, dtype=np.int64) for _ in so.bodies]
    per[body] = np.asarray(rows)
    return so.assemble_rows(per)


def _dense_system(name):
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from problems import oracle_system, spheres
    if name == "kirkwood":   # config 1: one sphere, 1280 panels, central charge
        return oracle_system(spheres(level_mol=3, surface=False), theta=0.0)
    return oracle_system(spheres(level_mol=3, level_srf=3, kind="sigma"), theta=0.0)   # 2 x 1280 panels


def _pool(n):
    """Spawned worker processes (the parent holds a CUDA context), one BLAS
    thread each."""
    import multiprocessing as mp
    old = {v: os.environ.get(v) for v in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS")}
    for v in old:
        os.environ[v] = "1"
    try:
        return mp.get_context("spawn").Pool(n)
    finally:
        for v, val in old.items():
            if val is None:
                os.environ.pop(v, None)
            else:
                os.environ[v] = val


def oracle_matvec_rate(pool, cores, rows_per_task=6, rounds=1, seed=0):
    """Direct-sum oracle rows sampled over all host cores: tasks of
    rows_per_task molecule targets, `cores` tasks per round.  Returns
    (matvecs per second of wall time, targets sampled, wall seconds)."""
    tasks = [(k * rows_per_task, (k + 1) * rows_per_task, seed) for k in range(cores * rounds)]
    c0 = time.perf_counter()
    pool.map(_oracle_rows_task, tasks, chunksize=1)
    wall = time.perf_counter() - c0
    n_t = rows_per_task * len(tasks)
    return (n_t / 40960) / wall, n_t, wall


def oracle_dense_solves(pool, cores):
    """Dense FP64 assembly (rows split over the host cores) and LAPACK LU
    solve (threaded BLAS of the parent) of two small workloads: ms each."""
    import scipy.linalg
    out = []
    for name, label in (("kirkwood", "Kirkwood sphere, 1280 panels (2560 unknowns)"),
                        ("two_spheres_l3", "two spheres r=4 A, 2 x 1280 panels (3840 unknowns)")):
        so = _dense_system(name)
        tasks = []
        for b, pn in enumerate(so.panels):
            for ch in np.array_split(np.arange(pn.N), max(1, cores)):
                if len(ch):
                    tasks.append((name, b, ch))
        c0 = time.perf_counter()
        parts = pool.map(_dense_rows_task, tasks, chunksize=1)
        A = np.zeros((so.n, so.n))
        rhs = np.zeros(so.n)
        for idx, Ar, br in parts:
            A[idx] = Ar
            rhs[idx] = br
        c1 = time.perf_counter()
        lu = scipy.linalg.lu_factor(A)
        scipy.linalg.lu_solve(lu, rhs)
        c2 = time.perf_counter()
        out.append({"workload": label, "unknowns": int(so.n), "assembly_ms": 1e3 * (c1 - c0),
                    "lu_solve_ms": 1e3 * (c2 - c1), "solve_ms": 1e3 * (c2 - c0)})
    return out


def cpu_baseline_record(target_s=10.0):
    """The oracle on the host cores: the direct-sum matvec rate of the
    two-sphere workload (sampled rows, about target_s of wall time on all
    cores) and the dense assembly + LU solve times of two small workloads."""
    cores, model = cpu_info()
    pool = _pool(cores)
    try:
        oracle_matvec_rate(pool, cores, rows_per_task=1)       # start the workers
        n_t, wall, seed = 0, 0.0, 1
        while wall < target_s:
            _, n, w = oracle_matvec_rate(pool, cores, rows_per_task=16, seed=seed)
            n_t += n
            wall += w
            seed += 1
        rate = (n_t / 40960) / wall
        dense = oracle_dense_solves(pool, cores)
    finally:
        pool.close()
        pool.join()
    return {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle", "cpu_model": model,
            "sample": f"{n_t} of 40960 target panels (both rows each) in {wall:.1f} s on {cores} worker processes, "
                      f"direct-sum FP64 oracle rows (dense O(N^2) operator, not a treecode), extrapolated to whole "
                      f"matvecs",
            "dense_lu": dense}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    cores, model = cpu_info()
    pool = _pool(cores)
    try:
        for _ in range(args.warmup):
            oracle_matvec_rate(pool, cores, rows_per_task=1)
        tot, n_tot = 0.0, 0
        for _ in range(args.steps):
            _, n_t, wall = oracle_matvec_rate(pool, cores, rows_per_task=2)
            tot += wall
            n_tot += n_t
    finally:
        pool.close()
        pool.join()
    value = (n_tot / 40960) / tot
    sample = (f"{n_tot // args.steps} of 40960 target panels per step (both rows of each) on {cores} worker "
              f"processes, direct-sum FP64 oracle over all 286720 source points, extrapolated to whole matvecs")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
                             "cpu_model": model},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def reduce_across_ranks(dist, total_ms, matvecs, device):
    """Whole-job numbers of N replicas: the slowest rank's time and the sum of
    the operator applications of all ranks."""
    import torch
    t = torch.tensor([total_ms], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    m = torch.tensor([float(matvecs)], device=device, dtype=torch.float64)
    dist.all_reduce(m)
    return float(t.item()), int(round(m.item()))


# ------------------------------------------------------------------ GPU arm
def rank_chunks(n_poses, batch, rank, world):
    """Contiguous pose range [lo, hi) of `rank`: whole chunks of `batch` poses
    (the unions the sweep solves), as even as the chunk count allows."""
    chunks = (n_poses + batch - 1) // batch
    c0 = chunks * rank // world
    c1 = chunks * (rank + 1) // world
    return min(n_poses, c0 * batch), min(n_poses, c1 * batch)


def gather_rows(dist, F, lo, hi, n, width, device):
    """Rows [lo, hi) of the (n, k) array F from every rank (at most `width`
    rows each), assembled in order (rank 0 receives; others return None).
    Result collection after the timed region: no exchange inside a solve."""
    import torch
    world = dist.get_world_size()
    k = F.shape[1]
    width = max(width, 1)
    buf = torch.zeros((width, k), dtype=torch.float64, device=device)
    buf[:hi - lo] = torch.as_tensor(F[lo:hi], dtype=torch.float64, device=device)
    meta = torch.tensor([lo, hi], dtype=torch.int64, device=device)
    bufs = [torch.zeros_like(buf) for _ in range(world)]
    metas = [torch.zeros_like(meta) for _ in range(world)]
    dist.all_gather(bufs, buf)
    dist.all_gather(metas, meta)
    if dist.get_rank() != 0:
        return None
    out = np.zeros((n, k))
    for b, m in zip(bufs, metas):
        a, c = int(m[0]), int(m[1])
        out[a:c] = b[:c - a].cpu().numpy()
    return out


def run_gpu(args):
    import torch
    import paper_1506_03745_gb300 as pgb
    from paper_1506_03745_gb300.context import context as gpu_context

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    bodies = workload_bodies()
    ctx = gpu_context(bodies, **PARAMS)
    n = pgb.pgb_num_unknowns(ctx)
    x = torch.empty(n, dtype=torch.float64, device=dev)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)

    def step(mode):
        pgb.pgb_tree_reset(ctx)   # the whole geometry pipeline runs in every step
        pgb.pgb_tree_build(ctx)
        code, st = pgb.pgb_solve(ctx, mode, TOL, MAX_ITER, RESTART, x)
        if code != 0:
            raise RuntimeError(f"solve did not converge: {st}")
        e = pgb.pgb_energy(ctx, x)
        return st, e

    for _ in range(args.warmup):
        step(pgb.PGB_FP32_REFINE)
    torch.cuda.synchronize()
    # ---- timed region
    pgb.pgb_timing(ctx, True, read=True)      # reset counters, timing on
    clocks = Clocks(local)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    total_ms, matvecs, stats = 0.0, 0, []
    for _ in range(args.steps):
        flush.zero_()
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        st, e32 = step(pgb.PGB_FP32_REFINE)
        s1.record(stream)
        s1.synchronize()
        total_ms += s0.elapsed_time(s1)
        matvecs += st["matvecs"]
        stats.append(st)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    timing = pgb.pgb_timing(ctx, False, read=True)
    t_max, mv_all = reduce_across_ranks(dist, total_ms, matvecs, dev) if dist else (total_ms, matvecs)
    value = mv_all / (t_max / 1e3)

    # ---- FP64 reference solve on the same GPU (reported beside the value)
    flush.zero_()
    torch.cuda.synchronize()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    st64, e64 = step(pgb.PGB_FP64)
    f1.record(stream)
    f1.synchronize()
    fp64_ms = f0.elapsed_time(f1)
    x64 = x.clone()
    step(pgb.PGB_FP32_REFINE)
    e_err = {k: abs(e32[k] - e64[k]) / max(abs(e64[k]), 1e-300) for k in ("solvation", "surface", "total")}
    pc = precond_solve(pgb, bodies, dev, stream, flush, e64) if not PARAMS.get("precond") else None
    ov = variant_solve(pgb, bodies, dev, stream, flush, e64, overlap=1) if not PARAMS.get("overlap") else None
    native = variant_solve(pgb, bodies, dev, stream, flush, e64, residual=0) if PARAMS.get("residual") else None

    info = pgb.pgb_tree_stats(ctx)
    peaks = device_peaks(dev)
    peak_tflops = peaks["fp32_tflops"]
    kern = {}
    for name, stage, fl in (("k_p2p<float> (P2P, near leaves)", "p2p", p2p_kernel_flops(info)),
                            ("k_m2p<float,6> (M2P, far nodes)", "m2p", m2p_kernel_flops(info, PARAMS["P"]))):
        ms, calls = timing[stage]
        kern[stage] = dict(kernel=name, total_ms=ms, calls=calls, flops=fl,
                           avg_ms=ms / calls if calls else None,
                           achieved=fl / (ms / calls / 1e3) / 1e12 if calls else None)
    dom = max(kern.values(), key=lambda k: k["total_ms"])
    traffic = recorded_traffic(dom["kernel"].split(" ")[0])
    # the FP64-class product of the refinement residual: same algorithmic
    # counts.  residual = 1: double-single kernels on the FP32 pipe, set
    # against the FP32 peak with the FP32 operations they issue per FP64-class
    # operation (ncu, profiles/ds_residual_two_sphere.txt); residual = 0:
    # native FP64 kernels against the FP64 pipe (2 FMA lanes per SM per clock)
    fp64_peak = peaks["sm_count"] * 2 * 2 * peaks["sm_max_mhz"] * 1e6 / 1e12
    tag = "ds" if PARAMS["residual"] else "double"
    ds_prof = recorded_counters("ds_residual_two_sphere.txt")
    for name, stage, fl in ((f"k_p2p<{tag}> (P2P, FP64-class residual)", "p2p_fp64", p2p_kernel_flops(info)),
                            (f"k_m2p<{tag},6> (M2P, FP64-class residual)", "m2p_fp64",
                             m2p_kernel_flops(info, PARAMS["P"]))):
        ms, calls = timing[stage]
        ach = fl / (ms / calls / 1e3) / 1e12 if calls else None
        rec = dict(kernel=name, total_ms=ms, calls=calls, flops=fl, avg_ms=ms / calls if calls else None,
                   achieved_fp64_class=ach, unit="TFLOP/s")
        if PARAMS["residual"]:
            key = stage.split("_")[0]
            rec.update(bound="alu (FP32 pipe, double-single)", fp32_peak=peak_tflops,
                       fp32_ops_per_fp64_class_op=ds_prof.get(f"{key}_fp32_ops_per_op"),
                       ncu_fma_pipe=ds_prof.get(f"{key}_fma_pipe"), ncu_issue_active=ds_prof.get(f"{key}_issue"),
                       note="FP64-class operations counted as the FP32 kernels' flops; ncu figures from the "
                            "committed capture when it was taken on the current source, else null")
            if ach and rec["fp32_ops_per_fp64_class_op"]:
                rec["fp32_pipe_frac"] = ach * rec["fp32_ops_per_fp64_class_op"] / peak_tflops
        else:
            rec.update(bound="alu (FP64 pipe)", peak=fp64_peak, frac=(ach / fp64_peak) if ach else None)
        kern[stage] = rec

    # the assembly of the FP32 product (item partial sums, near-field
    # correction SpMV, rows): the memory-bound kernel, against the measured
    # copy bandwidth.  Algorithmic bytes per launch: per correction entry its
    # index and FP32 values (4 + 16 B); per panel its FP32 densities (12 B),
    # CSR offset and group data (8 + 4 + 4 + 16 B) and permutation/body
    # (8 B); per unknown x read and y written (16 B); per work item its 64
    # FP64 partial sums (512 B).  The whole working set stays in L2.
    hbm = load_peaks().get("hbm_gbs")
    ms, calls = timing["assemble"]
    asm_bytes = (20 * info["n_corrections"] + 60 * info["n_panels"] + 16 * info["n_unknowns"] +
                 512 * (info["n_p2p_items"] + info["n_m2p_items"]))
    if calls and hbm:
        ach = asm_bytes / (ms / calls / 1e3) / 1e9
        kern["assemble"] = dict(kernel="k_assemble<float> (near-field SpMV + rows)", total_ms=ms, calls=calls,
                                bytes=asm_bytes, avg_ms=ms / calls, achieved=ach, unit="GB/s", bound="hbm",
                                peak=hbm, frac=ach / hbm, peak_source="MEASURED_PEAKS.json hbm_gbs (of measured)",
                                note="L2-resident working set (about 25 MB per launch): the fraction is of HBM")

    # ---- end to end through the public API with host inputs
    e2e_ms = []
    h2d = sum(b["verts"].nbytes + b["tris"].astype(np.int32).nbytes + b["qxyz"].nbytes + b["q"].nbytes
              for b in bodies)
    d2h = 32 + 24  # energies + solve stats
    e2e_mv = 0
    for i in range(args.warmup + args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        c2 = gpu_context(bodies, **PARAMS)
        xx = torch.empty(n, dtype=torch.float64, device=dev)
        code, st = pgb.pgb_solve(c2, pgb.PGB_FP32_REFINE, TOL, MAX_ITER, RESTART, xx)
        ee = pgb.pgb_energy(c2, xx)
        pgb.pgb_destroy(c2)
        torch.cuda.synchronize()
        if i >= args.warmup:
            e2e_ms.append(1e3 * (time.perf_counter() - t0))
            e2e_mv += st["matvecs"]
    e2e_value = e2e_mv / (sum(e2e_ms) / 1e3) * (mv_all / max(matvecs, 1))

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline_record()

    st0 = stats[0]
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n_unknowns": n, "theta": PARAMS["theta"], "P": PARAMS["P"],
                   "leaf_size": PARAMS["leaf_size"], "p2p_item": PARAMS["p2p_item"], "m2p_item": PARAMS["m2p_item"],
                   "precond": PARAMS["precond"], "overlap": PARAMS["overlap"], "K": PARAMS["K"], "tol": TOL, "restart": RESTART,
                   "residual": "double-single FP64-class product (PGB_FP64_DS)" if PARAMS["residual"]
                               else "native FP64 product",
                   "step": "full tree build (sort, octree, lists, near field; nothing cached) + "
                           "FP32/FP64-refined GMRES solve + energies",
                   "l2": "flushed (512 MB write) before every timed step",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "solve": {"fp32_refine_ms": t_max / args.steps, "fp64_ms": fp64_ms,
                  "speedup_vs_fp64": fp64_ms / (t_max / args.steps),
                  "iterations": st0["iterations"], "outer_steps": st0["outer_steps"],
                  "matvecs": st0["matvecs"], "matvecs_fp64": st0["matvecs_fp64"],
                  "fp64_iterations": st64["iterations"], "rel_residual": st0["rel_residual"],
                  "energy_rel_err_vs_fp64": e_err, "energies_kcal_mol": e32,
                  "block_diagonal_precond": pc,
                  "overlapped_fp64_residual": ov,
                  "native_fp64_residual": native},
        "stage_ms_per_step": {k: v[0] / args.steps for k, v in timing.items() if k not in ("kernel_launches", "host_launches")},
        "gpu_launches": timing["kernel_launches"],
        "host_launch_calls": timing["host_launches"],
        "roofline": {"kernel": dom["kernel"], "bound": "alu", "achieved": dom["achieved"],
                     "peak": peak_tflops, "unit": "TFLOP/s",
                     "frac": (dom["achieved"] / peak_tflops) if dom["achieved"] else None,
                     "traffic": traffic, "flops_per_launch": dom["flops"], "launches": dom["calls"],
                     "avg_launch_ms": dom["avg_ms"],
                     "peak_source": peaks["note"], "sm_count": peaks["sm_count"],
                     "sm_max_mhz": peaks["sm_max_mhz"],
                     "note": "dominant kernel of the FP32 treecode product (the inner products of a step); "
                             "the FP64-class residual kernels are in other_kernels, against the FP32 pipe",
                     "other_kernels": {k: {kk: vv for kk, vv in v.items() if kk != "kernel"} | {"kernel": v["kernel"]}
                                       for k, v in kern.items() if v is not dom}},
        "tree": info,
        "clocks": clk,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": d2h,
                "ms_per_step": statistics.mean(e2e_ms)},
        "cpu_baseline": cpu,
        # the paper's only stated timing, as context (another workload and machine)
        "paper_context": {"timing": "less than one minute per run",
                          "hardware": "Intel Xeon X5650 CPUs + 1 NVIDIA Tesla C2075 (Fermi)",
                          "workload": "protein G B1 D4' (4 elem/A^2) near a charged block (2 elem/A^2), "
                                      "N_crit 300, P 4, theta 0.5, GMRES tol 1e-5 (structure and meshes not "
                                      "available here)"},
        # the FP32 + refinement solve against the plain FP64 solve on the same
        # GPU, last so that a tail of the line keeps it
        "solve_vs_fp64": {"fp32_refine_ms": t_max / args.steps, "fp64_ms": fp64_ms,
                          "speedup_vs_fp64": fp64_ms / (t_max / args.steps),
                          "energy_rel_err_vs_fp64": e_err},
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    pgb.pgb_destroy(ctx)
    if dist:
        dist.destroy_process_group()


# ------------------------------------------------------------------ other workloads
def star_bodies(density, seed=3, nq=900):
    """Star-shaped molecule r = 15 A (1 + sum_{l<=6} a_lm Y_lm), `density`
    panels per A^2, nq charges inside (>= 1.5 A from the mesh), eps_in 4."""
    import synth
    nu = synth.nu_for_density(seed, density)
    v, f = synth.star_surface(seed, nu)
    coeffs = synth.star_coefficients(seed)
    xyz, q = synth.interior_charges(seed, nq, v, f, radius_fn=lambda d: synth.star_radius(d, coeffs, 15.0))
    return dict(kind="dielectric", verts=v, tris=f, eps_in=4.0, qxyz=xyz, q=q, bc=0.0)


def sphere_body(radius=40.0, nu=39, sigma=-0.05):
    import synth
    u, f = synth.geodesic_sphere(nu)
    return dict(kind="sigma", verts=u * radius, tris=f, eps_in=1.0, qxyz=np.zeros((0, 3)), q=np.zeros(0), bc=sigma)


def place_for_gap(verts, R, radius, gap):
    """x offset D of the rotated molecule so that its closest vertex is `gap`
    from a sphere of `radius` at the origin (bisection)."""
    v = np.asarray(verts) @ np.asarray(R).T
    lo, hi = radius + gap - v[:, 0].min() - 50.0, radius + gap - v[:, 0].min() + 50.0
    for _ in range(80):
        mid = 0.5 * (lo + hi)
        d = np.sqrt(((v + np.array([mid, 0, 0])) ** 2).sum(1)).min() - radius
        lo, hi = (mid, hi) if d < gap else (lo, mid)
    return 0.5 * (lo + hi)


def _timed(fn):
    import torch
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    out = fn()
    e1.record()
    e1.synchronize()
    return out, e0.elapsed_time(e1)


def run_star(args):
    """Config: star molecule at 2, 4, 8 panels/A^2 with 900 charges, FP32 +
    refinement (tol 1e-6) against the plain FP64 solve on the same GPU."""
    import torch
    import paper_1506_03745_gb300 as pgb
    from paper_1506_03745_gb300.context import context as gpu_context
    rows = []
    for dens in (2, 4, 8):
        body = star_bodies(dens)
        ctx = gpu_context([body], **PARAMS)
        n = pgb.pgb_num_unknowns(ctx)
        x = torch.empty(n, dtype=torch.float64, device="cuda")
        for _ in range(args.warmup):
            pgb.pgb_solve(ctx, pgb.PGB_FP32_REFINE, TOL, MAX_ITER, RESTART, x)
        ms = []
        for _ in range(args.steps):
            (code, st), t = _timed(lambda: (pgb.pgb_tree_build(ctx),
                                            pgb.pgb_solve(ctx, pgb.PGB_FP32_REFINE, TOL, MAX_ITER, RESTART, x))[1])
            (e32), te = _timed(lambda: pgb.pgb_energy(ctx, x))
            ms.append(t + te)
        (c64, st64), t64 = _timed(lambda: pgb.pgb_solve(ctx, pgb.PGB_FP64, TOL, MAX_ITER, RESTART, x))
        e64 = pgb.pgb_energy(ctx, x)
        info = pgb.pgb_tree_stats(ctx)
        rows.append({"density": dens, "panels": info["n_panels"], "ms_per_step": statistics.median(ms),
                     "fp64_solve_ms": t64, "iterations": st["iterations"], "matvecs": st["matvecs"],
                     "matvecs_per_s": st["matvecs"] / (statistics.median(ms) / 1e3),
                     "solvation_kcal_mol": e32["solvation"], "solvation_rel_err_vs_fp64":
                         abs(e32["solvation"] - e64["solvation"]) / abs(e64["solvation"]),
                     "coulomb_kcal_mol": e32["coulomb"]})
        pgb.pgb_destroy(ctx)
    print(json.dumps({"workload": "star molecule r=15 A, 900 charges, 2/4/8 panels/A^2, single body",
                      "step": "tree build + FP32/FP64-refined solve (tol 1e-6) + energies", "params": PARAMS,
                      "results": rows}), flush=True)


def run_stern(args):
    """Nested interfaces: the star molecule (2 panels/A^2, 900 charges) inside
    a Stern layer -- the same star surface at r0 = 17 A (about 2 A further
    out, ion-free, eps 80) -- 10 A from a sphere r = 40 A (30420 panels,
    sigma -0.05 C/m^2): FP32 + refinement (tol 1e-6) with one treecode pass
    per region, against FP64 and against the same system without the layer."""
    import torch
    import synth
    import paper_1506_03745_gb300 as pgb
    from paper_1506_03745_gb300.context import context as gpu_context
    mol = star_bodies(2)
    nu = synth.nu_for_density(3, 2)
    vs, fs = synth.star_surface(3, nu, 17.0)
    stern = dict(kind="dielectric", verts=vs, tris=fs, eps_in=80.0, qxyz=np.zeros((0, 3)), q=np.zeros(0), bc=0.0)
    srf = sphere_body()
    D = place_for_gap(vs, np.eye(3), 40.0, 10.0)
    for b in (mol, stern):
        b["R"], b["t"] = np.eye(3), np.array([D, 0.0, 0.0])
    out = {}
    for name, bodies in (("stern", [dict(mol, parent=1), stern, srf]), ("plain", [mol, srf])):
        ctx = gpu_context(bodies, **PARAMS)
        n = pgb.pgb_num_unknowns(ctx)
        x = torch.empty(n, dtype=torch.float64, device="cuda")
        for _ in range(args.warmup):
            pgb.pgb_solve(ctx, pgb.PGB_FP32_REFINE, TOL, MAX_ITER, RESTART, x)
        ms = []
        for _ in range(args.steps):
            (code, st), t = _timed(lambda: (pgb.pgb_tree_build(ctx),
                                            pgb.pgb_solve(ctx, pgb.PGB_FP32_REFINE, TOL, MAX_ITER, RESTART, x))[1])
            e32, te = _timed(lambda: pgb.pgb_energy(ctx, x))
            ms.append(t + te)
        (c64, st64), t64 = _timed(lambda: pgb.pgb_solve(ctx, pgb.PGB_FP64, TOL, MAX_ITER, RESTART, x))
        e64 = pgb.pgb_energy(ctx, x)
        out[name] = {"panels": pgb.pgb_tree_stats(ctx)["n_panels"], "unknowns": n,
                     "ms_per_step": statistics.median(ms), "fp64_solve_ms": t64, "iterations": st["iterations"],
                     "status": code, "energies_kcal_mol": e32,
                     "energy_rel_err_vs_fp64": {k: abs(e32[k] - e64[k]) / max(abs(e64[k]), 1e-300)
                                                for k in ("solvation", "surface", "total")}}
        pgb.pgb_destroy(ctx)
    print(json.dumps({"workload": "star molecule (2 panels/A^2, 900 charges) in a 2 A Stern layer, 10 A from a "
                                  "sphere r=40 A (30420 panels, sigma -0.05 C/m^2)",
                      "step": "tree build + FP32/FP64-refined solve (tol 1e-6) + energies", "results": out}),
          flush=True)


def run_gradient(args):
    """Config: star molecule (2 panels/A^2, 900 charges) 10 A from a sphere
    r = 40 A (30420 panels, sigma -0.05 C/m^2): adjoint gradient time."""
    import torch
    import paper_1506_03745_gb300 as pgb
    from paper_1506_03745_gb300.context import context as gpu_context
    mol = star_bodies(2)
    srf = sphere_body()
    D = place_for_gap(mol["verts"], np.eye(3), 40.0, 10.0)
    mol["R"], mol["t"] = np.eye(3), np.array([D, 0.0, 0.0])
    prm = dict(PARAMS)
    ctx = gpu_context([mol, srf], **prm)
    n = pgb.pgb_num_unknowns(ctx)
    x = torch.empty(n, dtype=torch.float64, device="cuda")
    nq = len(mol["q"])
    for _ in range(args.warmup):
        pgb.pgb_solve(ctx, pgb.PGB_FP32_REFINE, TOL, MAX_ITER, RESTART, x)
        pgb.pgb_grad(ctx, x, nq, 2, pgb.PGB_FP32, 1e-6, MAX_ITER, RESTART)
    ts, tg = [], []
    for _ in range(args.steps):
        (code, st), t1 = _timed(lambda: pgb.pgb_solve(ctx, pgb.PGB_FP32_REFINE, TOL, MAX_ITER, RESTART, x))
        res, t2 = _timed(lambda: pgb.pgb_grad(ctx, x, nq, 2, pgb.PGB_FP32, 1e-6, MAX_ITER, RESTART))
        ts.append(t1)
        tg.append(t2)
    _, dq, dbc, dt, ast = res
    e = pgb.pgb_energy(ctx, x, 2)
    print(json.dumps({"workload": "star molecule (2 panels/A^2, 900 charges) 10 A from a sphere r=40 A "
                                  "(30420 panels, sigma -0.05 C/m^2)",
                      "panels": pgb.pgb_tree_stats(ctx)["n_panels"], "solve_ms": statistics.median(ts),
                      "grad_ms": statistics.median(tg), "solve_iterations": st["iterations"],
                      "adjoint_iterations": ast["iterations"], "adjoint_rel_residual": ast["rel_residual"],
                      "F_total_kcal_mol": e["total"], "dF_dt_molecule": dt[0].tolist(),
                      "dF_dsigma": float(dbc[1]), "sum_q_dFdq_plus_sigma_dFdsigma_over_2F":
                          float((mol["q"] @ dq + srf["bc"] * dbc[1]) / (2 * e["total"]))}), flush=True)
    pgb.pgb_destroy(ctx)


def orientation_landscape(F, n_orient, n_gap, T=300.0):
    """Boltzmann weights of the orientations at each gap (poses ordered
    orientation-major, gap-minor), computed by the library
    (pgb_orientation_landscape)."""
    import paper_1506_03745_gb300 as pgb
    return pgb.pgb_orientation_landscape(F, n_orient, n_gap, T)


def run_poses(args):
    """Config subset: one synthetic molecule (~5000 panels, 900 charges) in
    `--poses` orientations x 4 gaps (6, 8, 10, 14 A) near a sphere r = 40 A
    (30420 panels, sigma -0.05 C/m^2), batched with pgb_solve_batch in pure
    FP32 (tol 1e-5); the energy error against FP64 is measured on 2 poses."""
    import torch
    import synth
    import paper_1506_03745_gb300 as pgb
    from paper_1506_03745_gb300.context import context as gpu_context
    nu = int(round(math.sqrt(5000 / 20)))
    v, f = synth.star_surface(100, nu)
    coeffs = synth.star_coefficients(100)
    xyz, q = synth.interior_charges(100, 900, v, f, radius_fn=lambda d: synth.star_radius(d, coeffs, 15.0))
    mol = dict(kind="dielectric", verts=v, tris=f, eps_in=4.0, qxyz=xyz, q=q, bc=0.0)
    srf = sphere_body()
    Rs = synth.random_rotations(7, args.poses)
    poses_R, poses_t = [], []
    for R in Rs:
        for gap in (6.0, 8.0, 10.0, 14.0):
            poses_R.append(R)
            poses_t.append([place_for_gap(v, R, 40.0, gap), 0.0, 0.0])
    poses_R, poses_t = np.array(poses_R), np.array(poses_t)
    mol["R"], mol["t"] = poses_R[0], poses_t[0]
    ctx = gpu_context([mol, srf], **PARAMS)
    B = len(poses_R)
    pgb.pgb_solve_batch(ctx, 0, poses_R[:2], poses_t[:2], pgb.PGB_FP32, 1e-5, MAX_ITER, RESTART)  # warm-up
    pgb.pgb_timing(ctx, True, read=True)
    (code, F, st), ms = _timed(lambda: pgb.pgb_solve_batch(ctx, 0, poses_R, poses_t, pgb.PGB_FP32, 1e-5,
                                                           MAX_ITER, RESTART))
    tim = pgb.pgb_timing(ctx, False, read=True)
    code64, F64, _ = pgb.pgb_solve_batch(ctx, 0, poses_R[:2], poses_t[:2], pgb.PGB_FP64, 1e-9, MAX_ITER, RESTART)
    err = [abs(F[i, 3] - F64[i, 3]) / abs(F64[i, 3]) for i in range(2)]
    print(json.dumps({"workload": f"1 molecule ({pgb.pgb_tree_stats(ctx)['n_panels'] - 30420} panels, 900 "
                                  f"charges) x {args.poses} orientations x 4 gaps near a sphere r=40 A "
                                  f"(30420 panels)", "poses": B, "lanes": PARAMS["lanes"],
                      "batch": PARAMS["batch"], "ms": ms, "poses_per_s": B / (ms / 1e3),
                      "mean_iterations": float(np.mean([s["iterations"] for s in st])),
                      "energy_rel_err_vs_fp64_first_2_poses": err, "status": code,
                      "stage_ms_per_pose": {k: v[0] / B for k, v in tim.items() if k not in ("kernel_launches", "host_launches") and v[0]},
                      "kernel_launches_per_pose": tim["kernel_launches"] / B,
                      "host_launch_calls_per_pose": tim["host_launches"] / B,
                      "F_total_range_kcal_mol": [float(F[:, 3].min()), float(F[:, 3].max())],
                      "orientation_landscape": orientation_landscape(F[:, 3], args.poses, 4)}), flush=True)
    pgb.pgb_destroy(ctx)


def run_poses_uneven(args):
    """Pose sweep over 8 distinct synthetic molecules of uneven size (star
    surfaces r0 = 15 A from the molecule generator, about 5000 ... 40000
    panels in geometric steps, 900 charges each) near a sphere r = 40 A
    (30420 panels, sigma -0.05 C/m^2): `--poses` orientations x 4 gaps (6, 8,
    10, 14 A) per molecule, FP32 + refinement with the double-single
    residual and the block-diagonal preconditioner (tol 1e-6: every pose's
    energy within 1e-5 of FP64; `--precond 0` gives the plain GMRES at tol
    1e-5).  Batched: pgb_solve_poses
    with chunks of `batch` poses (default 8, one pose of every molecule per
    chunk: one launch per stage over eight molecules of different sizes);
    beside it the same poses molecule by molecule through pgb_solve_batch
    with 4 lanes.  The batched FP64 solve (tol 1e-9) is timed beside the
    batched FP32 + refinement solve on the leading 8 chunks: speedup and
    per-pose energy error.  Under torchrun the poses are split across the
    ranks in contiguous runs of whole chunks (independent problems: no
    exchange inside a solve); rank 0 tunes the parameters for all, the time
    is the slowest rank's, and the energies are gathered after the timed
    region."""
    import torch
    import synth
    import paper_1506_03745_gb300 as pgb
    from paper_1506_03745_gb300.context import context as gpu_context
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    batch = PARAMS["batch"] if PARAMS["batch"] > 1 else 8
    sizes = np.geomspace(5000, 40000, 8)
    srf = sphere_body()
    verts, npan, mols = [], [], []
    for k, N in enumerate(sizes):
        nu = int(round(math.sqrt(N / 20)))
        seed = 300 + k
        v, f = synth.star_surface(seed, nu)
        coeffs = synth.star_coefficients(seed)
        xyz, q = synth.interior_charges(seed, 900, v, f,
                                        radius_fn=lambda d, c=coeffs: synth.star_radius(d, c, 15.0))
        mols.append(dict(kind="dielectric", verts=v, tris=f, eps_in=4.0, qxyz=xyz, q=q, bc=0.0))
        verts.append(v)
        npan.append(len(f))
    # treecode parameters and work-item sizes by the autotuner, on the first
    # molecule 8 A from the sphere: the fastest FP32 solve whose total energy
    # is within 1e-5 of the most accurate candidate's (theta 0.5, P 7)
    # the block-diagonal preconditioner halves the iterations (55 -> 27 per
    # pose); with it the relative-residual tolerance that keeps every pose's
    # energy within 1e-5 of the FP64 solve is tighter (on the leading 64 poses
    # 1e-5 left 2.6e-5, 3e-6 left 6.5e-6, 2e-6 left 8.9e-6 on another pose
    # set, 1e-6 left 4.9e-6): 1e-6 by default
    prm = dict(PARAMS)
    if args.precond is None:
        prm["precond"] = 1
    tol = args.pose_tol if args.pose_tol is not None else (1e-6 if prm["precond"] else 1e-5)
    tune = None
    if not args.no_autotune and rank == 0:
        m0 = dict(mols[0], R=np.eye(3), t=np.array([place_for_gap(verts[0], np.eye(3), 40.0, 8.0), 0.0, 0.0]))
        ct = gpu_context([m0, srf], **prm)
        thetas, Ps, leaves = [0.5, 0.6, 0.7], [5, 6, 7], [32, 64]
        (chosen, rep), t_ms = _timed(lambda: pgb.pgb_autotune(ct, thetas, Ps, leaves, reps=3, tol=tol,
                                                              target_rel_err=1e-5))
        pgb.pgb_destroy(ct)
        for k in ("theta", "P", "leaf_size", "p2p_item", "m2p_item"):
            prm[k] = chosen[k]
        tune = {"chosen": {k: prm[k] for k in ("theta", "P", "leaf_size", "p2p_item", "m2p_item")},
                "candidates": [{"theta": t_, "P": p_, "leaf": l_, "matvec_ms": rep[i, 0], "solve_ms": rep[i, 1],
                                "energy_rel_diff": rep[i, 2]}
                               for i, (t_, p_, l_) in enumerate((t_, p_, l_) for t_ in thetas for p_ in Ps
                                                                 for l_ in leaves)],
                "ms": t_ms}
    if dist is not None:  # every rank solves with rank 0's parameters
        box = [prm]
        dist.broadcast_object_list(box, src=0)
        prm = box[0]
    ctxs = [gpu_context([mols[k], srf], **dict(prm, batch=batch if k == 0 else 1)) for k in range(8)]
    Rs = synth.random_rotations(17, args.poses)
    R, t, pc = [], [], []
    for Ro in Rs:
        for gap in (6.0, 8.0, 10.0, 14.0):
            for k in range(8):
                R.append(Ro)
                t.append([place_for_gap(verts[k], Ro, 40.0, gap), 0.0, 0.0])
                pc.append(k)
    R, t, pc = np.array(R), np.array(t), np.array(pc, dtype=np.int32)
    B = len(R)
    mode = pgb.PGB_FP32_REFINE
    lo, hi = rank_chunks(B, batch, rank, world)
    pgb.pgb_solve_poses(ctxs, pc[:batch], 0, R[:batch], t[:batch], mode, tol, MAX_ITER, RESTART)  # warm-up
    pgb.pgb_timing(ctxs[0], True, read=True)
    if dist is not None:
        torch.cuda.synchronize(dev)
        dist.barrier()
    code, F, st, ms = 0, np.zeros((0, 4)), [], 0.0
    if hi > lo:
        (code, F, st), ms = _timed(lambda: pgb.pgb_solve_poses(ctxs, pc[lo:hi], 0, R[lo:hi], t[lo:hi], mode, tol,
                                                               MAX_ITER, RESTART))
    tim = pgb.pgb_timing(ctxs[0], False, read=True)
    n_local = hi - lo
    if dist is not None:
        torch.cuda.synchronize(dev)
        dist.barrier()
        tm = torch.tensor([ms], dtype=torch.float64, device=dev)
        dist.all_reduce(tm, op=dist.ReduceOp.MAX)
        ms = float(tm.item())
        chunks = (B + batch - 1) // batch
        width = ((chunks + world - 1) // world) * batch
        Fl = np.zeros((B, 4))
        Fl[lo:hi] = F
        its_l = np.zeros((B, 2))
        its_l[lo:hi, 0] = [s_["iterations"] for s_ in st]
        its_l[lo:hi, 1] = [s_["rel_residual"] for s_ in st]
        cd = torch.tensor([abs(code)], dtype=torch.float64, device=dev)
        dist.all_reduce(cd, op=dist.ReduceOp.MAX)
        Fg = gather_rows(dist, Fl, lo, hi, B, width, dev)
        Ig = gather_rows(dist, its_l, lo, hi, B, width, dev)
        if rank != 0:
            for c in ctxs:
                pgb.pgb_destroy(c)
            dist.destroy_process_group()
            return
        F = Fg
        st = [{"iterations": int(v[0]), "rel_residual": float(v[1])} for v in Ig]
        code = -int(cd.item()) if cd.item() else 0
    # the same poses molecule by molecule with concurrent lanes (molecule 0
    # needs a context of its own without the batch parameter)
    lanes = None
    if not args.no_lanes and world == 1:
        c0 = gpu_context([mols[0], srf], **dict(prm, batch=1))
        F_l = np.zeros_like(F)
        ms_l = 0.0
        for k in range(8):
            sel = np.nonzero(pc == k)[0]
            ck = c0 if k == 0 else ctxs[k]
            pgb.pgb_solve_batch(ck, 0, R[sel[:2]], t[sel[:2]], mode, tol, MAX_ITER, RESTART)  # warm-up
            (_, Fk, _), msk = _timed(lambda: pgb.pgb_solve_batch(ck, 0, R[sel], t[sel], mode, tol, MAX_ITER,
                                                                 RESTART))
            F_l[sel] = Fk
            ms_l += msk
        pgb.pgb_destroy(c0)
        lanes = {"ms": ms_l, "poses_per_s": B / (ms_l / 1e3),
                 "max_rel_diff_total_energy": float(np.max(np.abs(F_l[:, 3] - F[:, 3]) / np.abs(F[:, 3])))}
    # the batched FP64 solve (tol 1e-9) beside the batched FP32 + refinement
    # solve on the same leading poses (up to 8 chunks): time and per-pose
    # energy error
    n64 = min(B, 8 * batch)
    (_, F32s, _), ms32 = _timed(lambda: pgb.pgb_solve_poses(ctxs, pc[:n64], 0, R[:n64], t[:n64], mode, tol,
                                                            MAX_ITER, RESTART))
    (code64, F64, st64), ms64 = _timed(lambda: pgb.pgb_solve_poses(ctxs, pc[:n64], 0, R[:n64], t[:n64],
                                                                   pgb.PGB_FP64, 1e-9, MAX_ITER, RESTART))
    err = np.abs(F[:n64, 3] - F64[:, 3]) / np.abs(F64[:, 3])
    vs64 = {"poses": n64, "fp32_refine_ms": ms32, "fp64_ms": ms64, "speedup": ms64 / ms32, "fp64_status": code64,
            "fp64_mean_iterations": float(np.mean([s_["iterations"] for s_ in st64])),
            "energy_rel_err_max": float(err.max()), "energy_rel_err_median": float(np.median(err))}
    its = np.array([s["iterations"] for s in st])
    print(json.dumps({"workload": f"8 molecules ({min(npan)}-{max(npan)} panels, 900 charges each) x {args.poses} "
                                  f"orientations x 4 gaps near a sphere r=40 A (30420 panels)",
                      "poses": B, "batch": batch, "n_gpus": world, "tol": tol, "precond": prm.get("precond", 0),
                      "split": "contiguous whole chunks per rank, slowest rank's time" if world > 1 else None,
                      "ms": ms, "poses_per_s": B / (ms / 1e3),
                      "lanes_4_per_molecule": lanes, "mode": "FP32 + refinement (double-single residual)",
                      "max_rel_residual": float(max(s_["rel_residual"] for s_ in st)),
                      "molecule_panels": npan, "mean_iterations": float(its.mean()), "autotune": tune,
                      "iterations_range": [int(its.min()), int(its.max())], "status": code,
                      "batched_vs_fp64": vs64,
                      # rank 0's own poses
                      "stage_ms_per_pose": {k: v[0] / max(n_local, 1) for k, v in tim.items() if k not in ("kernel_launches", "host_launches") and v[0]},
                      "kernel_launches_per_pose": tim["kernel_launches"] / max(n_local, 1),
                      "host_launch_calls_per_pose": tim["host_launches"] / max(n_local, 1),
                      # per molecule, per gap: Boltzmann weights over the orientations (poses are
                      # ordered orientation, gap, molecule)
                      "orientation_landscape": {f"molecule_{k}": orientation_landscape(F[k::8, 3], args.poses, 4)
                                                for k in range(8)}}), flush=True)
    for c in ctxs:
        pgb.pgb_destroy(c)
    if dist is not None:
        dist.destroy_process_group()


def _two_sphere_analytical(case):
    """(F_int, solvation, surface, isolated molecule, isolated surface) of the
    analytical two-sphere solution for `case`, and the volts of one internal
    potential unit, from tests/golden/two_sphere_analytical.txt (written from
    the series solution of Section 4 by make_two_sphere_analytical.py)."""
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tests", "golden", "two_sphere_analytical.txt")
    volt, row = None, None
    for line in open(path):
        if line.startswith("# one internal potential unit"):
            volt = float(line.split("=")[1].split()[0])
        elif line.split()[:2] == [case, "60"]:
            row = [float(v) for v in line.split()[2:]]
    return row, volt


def run_replica(args):
    """The paper's grid-convergence case (Section 5.1, Table 1): a dielectric
    sphere r = 5 A (eps 4, unit charge at its centre) and a sphere r = 4 A held
    at phi0 = 1 internal potential unit, 12 A apart, kappa 0.125, eps 80, at
    icosphere levels 3..6 (1280 ... 81920 panels per sphere), with the
    paper's parameters (far rule 3 points, close-by rule `--near` points,
    9 Gauss points per edge in-element, N_crit 300, P 15, theta 0.5, GMRES tol
    1e-9; FP32 + refinement with the double-single residual).  Per level the
    interaction energy F_int = F(pair) - F(molecule alone) - F(surface alone)
    (Eq. 17) against the analytical value, and the observed order of
    convergence of the three finest meshes."""
    import math
    import torch
    import synth
    import paper_1506_03745_gb300 as pgb
    from paper_1506_03745_gb300.context import context as gpu_context
    ana, volt = _two_sphere_analytical("paper_5_4_phi1")
    prm = dict(PARAMS, K=3, K_near=args.near, n_edge=9, leaf_size=300, P=15, theta=0.5)
    tol = 1e-9
    levels = [int(v) for v in args.levels.split(",")]
    rows = []
    for level in levels:
        vm, fm = synth.icosphere(level, 5.0)
        vs, fs = synth.icosphere(level, 4.0)
        mol = dict(kind="dielectric", verts=vm, tris=fm, eps_in=4.0, qxyz=np.zeros((1, 3)), q=np.array([1.0]), bc=0.0)
        srf = dict(kind="phi", verts=vs + np.array([12.0, 0.0, 0.0]), tris=fs, eps_in=1.0, qxyz=np.zeros((0, 3)),
                   q=np.zeros(0), bc=volt)
        out = {"level": level, "panels_per_sphere": len(fm)}
        F = {}
        t_all = 0.0
        for name, bodies in (("pair", [mol, srf]), ("molecule", [mol]), ("surface", [srf])):
            ctx = gpu_context(bodies, **prm)
            n = pgb.pgb_num_unknowns(ctx)
            x = torch.empty(n, dtype=torch.float64, device="cuda")
            (code, st), ms = _timed(lambda: pgb.pgb_solve(ctx, pgb.PGB_FP32_REFINE, tol, MAX_ITER, RESTART, x))
            e = pgb.pgb_energy(ctx, x)
            pgb.pgb_destroy(ctx)
            F[name] = e
            t_all += ms
            out[name] = {"status": code, "iterations": st["iterations"], "rel_residual": st["rel_residual"],
                         "solve_ms": ms, "solvation": e["solvation"], "surface": e["surface"]}
        f_int = (F["pair"]["solvation"] + F["pair"]["surface"]) - F["molecule"]["solvation"] - F["surface"]["surface"]
        out["F_int_kcal_mol"] = f_int
        out["rel_error_vs_analytical"] = abs(f_int - ana[0]) / abs(ana[0])
        out["solve_ms_total"] = t_all
        rows.append(out)
        print(json.dumps(out), file=sys.stderr, flush=True)
    orders = {}
    for k in range(len(rows) - 1):
        e0, e1 = rows[k]["rel_error_vs_analytical"], rows[k + 1]["rel_error_vs_analytical"]
        orders[f"levels_{rows[k]['level']}_{rows[k + 1]['level']}"] = math.log(e0 / e1) / math.log(4.0)
    richardson = None
    if len(rows) >= 3:
        f1, f2, f3 = (r["F_int_kcal_mol"] for r in rows[-3:])
        if (f1 - f2) * (f2 - f3) > 0:
            richardson = math.log((f1 - f2) / (f2 - f3)) / math.log(4.0)
    print(json.dumps({"workload": "paper grid-convergence case: spheres r=5 A (eps 4, central charge 1 e) and r=4 A "
                                  "(phi0 = 1 internal unit), 12 A apart, kappa 0.125, eps 80",
                      "params": {k: prm[k] for k in ("K", "K_near", "n_edge", "leaf_size", "P", "theta")},
                      "tol": tol, "mode": "FP32 + refinement (double-single residual)",
                      "F_int_analytical_kcal_mol": ana[0], "levels": rows,
                      "observed_order_vs_analytical": orders,
                      "observed_order_richardson_three_finest": richardson,
                      "paper_observed_order": 1.007}), flush=True)


def run_scaling(args):
    """The two-sphere configuration at icosphere levels 4..7 (2 x 5120 ... 2 x
    327680 panels): the step (tree + FP32/FP64-refined solve + energies) and
    the FP32 product alone, to show the growth with N."""
    import torch
    import paper_1506_03745_gb300 as pgb
    from paper_1506_03745_gb300.context import context as gpu_context
    out = []
    for level in (4, 5, 6, 7):
        bodies = workload_bodies(level)
        ctx = gpu_context(bodies, **PARAMS)
        n = pgb.pgb_num_unknowns(ctx)
        x = torch.empty(n, dtype=torch.float64, device="cuda")

        def step():
            pgb.pgb_tree_reset(ctx)
            pgb.pgb_tree_build(ctx)
            code, st = pgb.pgb_solve(ctx, pgb.PGB_FP32_REFINE, TOL, MAX_ITER, RESTART, x)
            return code, st, pgb.pgb_energy(ctx, x)

        step()
        ms, res = [], None
        for _ in range(max(1, args.steps)):
            res, t = _timed(step)
            ms.append(t)
        x32 = torch.randn(n, dtype=torch.float32, device="cuda")
        y32 = torch.empty_like(x32)
        pgb.pgb_matvec(ctx, x32, y32, pgb.PGB_FP32)
        _, tmv = _timed(lambda: [pgb.pgb_matvec(ctx, x32, y32, pgb.PGB_FP32) for _ in range(10)])
        code, st, e = res
        info = pgb.pgb_tree_stats(ctx)
        out.append({"panels": info["n_panels"], "unknowns": n, "ms_per_step": statistics.median(ms),
                    "iterations": st["iterations"], "status": code, "fp32_matvec_ms": tmv / 10,
                    "near_pairs": info["p2p_pairs"], "far_evaluations": info["m2p_pairs"],
                    "solvation_kcal_mol": e["solvation"]})
        pgb.pgb_destroy(ctx)
        del x, x32, y32
        torch.cuda.empty_cache()
    print(json.dumps({"workload": "two spheres r=4 A, sigma 0.05 C/m^2, R=12 A, icosphere levels 4-7",
                      "results": out}), flush=True)


def run_brick(args):
    """Flat-faced charged body at zero ionic strength: the star molecule
    (2 panels/A^2, 900 charges) 10 A above a 100 x 100 x 10 A box with
    sigma -0.05 C/m^2 (squares of 1.4 A, two triangles each), kappa = 0.
    Step = tree build + FP32/FP64-refined solve + energies; the FP64 solve of
    the same step beside it."""
    import torch
    import synth
    import paper_1506_03745_gb300 as pgb
    from paper_1506_03745_gb300.context import context as gpu_context
    mol = star_bodies(2)
    zmin = float(mol["verts"][:, 2].min())
    v, f = synth.brick(100.0, 100.0, 10.0, 1.4, center=(0.0, 0.0, zmin - 10.0 - 5.0))
    srf = dict(kind="sigma", verts=v, tris=f, eps_in=1.0, qxyz=np.zeros((0, 3)), q=np.zeros(0), bc=-0.05)
    ctx = gpu_context([mol, srf], kappa=0.0, **PARAMS)
    n = pgb.pgb_num_unknowns(ctx)
    x = torch.empty(n, dtype=torch.float64, device="cuda")

    def step(mode):
        pgb.pgb_tree_reset(ctx)
        pgb.pgb_tree_build(ctx)
        code, st = pgb.pgb_solve(ctx, mode, TOL, MAX_ITER, RESTART, x)
        return code, st, pgb.pgb_energy(ctx, x)

    for _ in range(args.warmup):
        step(pgb.PGB_FP32_REFINE)
    ms, res = [], None
    for _ in range(args.steps):
        res, t = _timed(lambda: step(pgb.PGB_FP32_REFINE))
        ms.append(t)
    (c64, st64, e64), t64 = _timed(lambda: step(pgb.PGB_FP64))
    code, st, e = res
    print(json.dumps({"workload": "star molecule (2 panels/A^2, 900 charges) 10 A above a 100 x 100 x 10 A box "
                                  "(sigma -0.05 C/m^2), kappa = 0",
                      "panels": pgb.pgb_tree_stats(ctx)["n_panels"], "brick_panels": int(len(f)),
                      "ms_per_step": statistics.median(ms), "fp64_ms": t64, "iterations": st["iterations"],
                      "fp64_iterations": st64["iterations"], "status": [code, c64],
                      "energies_kcal_mol": e,
                      "energy_rel_err_vs_fp64": {k: abs(e[k] - e64[k]) / max(abs(e64[k]), 1e-300)
                                                 for k in ("solvation", "surface", "total")}}), flush=True)
    pgb.pgb_destroy(ctx)


def precond_solve(pgb, bodies, dev, stream, flush, e64, steps=3):
    """The same step with the block-diagonal right preconditioner (precond=1)."""
    return variant_solve(pgb, bodies, dev, stream, flush, e64, steps, precond=1)


def variant_solve(pgb, bodies, dev, stream, flush, e64, steps=3, **override):
    """The same step with some parameters changed (e.g. precond=1, or
    overlap=1: the FP64 product of the refinement residual started early on a
    side stream): median device ms over `steps` steps after one warm-up, its
    iterations, products, products per second, and the energy difference to
    the FP64 solve."""
    import torch
    from paper_1506_03745_gb300.context import context as gpu_context
    ctx = gpu_context(bodies, **dict(PARAMS, **override))
    n = pgb.pgb_num_unknowns(ctx)
    x = torch.empty(n, dtype=torch.float64, device=dev)
    ms, st, e = [], None, None
    for i in range(steps + 1):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        pgb.pgb_tree_reset(ctx)
        pgb.pgb_tree_build(ctx)
        code, st = pgb.pgb_solve(ctx, pgb.PGB_FP32_REFINE, TOL, MAX_ITER, RESTART, x)
        e = pgb.pgb_energy(ctx, x)
        b.record(stream)
        b.synchronize()
        if code != 0:
            raise RuntimeError(f"solve with {override} did not converge: {st}")
        if i:
            ms.append(a.elapsed_time(b))
    pgb.pgb_destroy(ctx)
    return {"params": override, "ms_per_step": statistics.median(ms), "iterations": st["iterations"],
            "matvecs": st["matvecs"], "matvecs_per_s": st["matvecs"] / (statistics.median(ms) / 1e3),
            "rel_residual": st["rel_residual"],
            "energy_rel_err_vs_fp64": {k: abs(e[k] - e64[k]) / max(abs(e64[k]), 1e-300)
                                       for k in ("solvation", "surface", "total")}}


def run_matvec(args):
    """Operator applications only: W + K FP32 treecode matvecs of the
    workload (tree built once, untimed); prints matvecs/s and per-stage times."""
    import torch
    import paper_1506_03745_gb300 as pgb
    from paper_1506_03745_gb300.context import context as gpu_context
    dev = torch.device("cuda", 0)
    ctx = gpu_context(workload_bodies(), **PARAMS)
    n = pgb.pgb_num_unknowns(ctx)
    prec = {"fp32": pgb.PGB_FP32, "fp64": pgb.PGB_FP64, "fp64_ds": pgb.PGB_FP64_DS}[args.precision]
    dt = torch.float32 if prec == pgb.PGB_FP32 else torch.float64
    x = torch.randn(n, dtype=dt, device=dev)
    y = torch.empty_like(x)
    for _ in range(args.warmup):
        pgb.pgb_matvec(ctx, x, y, prec)
    torch.cuda.synchronize()
    pgb.pgb_timing(ctx, True, read=True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        pgb.pgb_matvec(ctx, x, y, prec)
    e1.record()
    torch.cuda.synchronize()
    t = pgb.pgb_timing(ctx, False, read=True)
    ms = e0.elapsed_time(e1) / args.steps
    print(json.dumps({"mode": "matvec", "precision": args.precision, "ms_per_matvec": ms,
                      "matvecs_per_s": 1e3 / ms,
                      "stage_ms_per_matvec": {k: v[0] / args.steps for k, v in t.items() if k not in ("kernel_launches", "host_launches")},
                      "tree": pgb.pgb_tree_stats(ctx)}), flush=True)
    pgb.pgb_destroy(ctx)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--mode", default="solve", choices=["solve", "matvec"])
    ap.add_argument("--workload", default="two_sphere", choices=["two_sphere", "star", "gradient", "poses", "poses_uneven", "brick",
                                                            "scaling", "stern", "replica"])
    ap.add_argument("--levels", default="3,4,5,6", help="icosphere levels of --workload replica")
    ap.add_argument("--near", type=int, default=37, help="close-by rule points of --workload replica (19 or 37)")
    ap.add_argument("--poses", type=int, default=8, help="orientations for --workload poses")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64", "fp64_ds"])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--leaf", type=int, default=None, help="override leaf_size (parameter sweeps)")
    ap.add_argument("--P", type=int, default=None, help="override the Taylor order (parameter sweeps)")
    ap.add_argument("--theta", type=float, default=None, help="override theta (parameter sweeps)")
    ap.add_argument("--p2p-item", type=int, default=None, help="override P2P tiles per work item (sweeps)")
    ap.add_argument("--m2p-item", type=int, default=None, help="override far nodes per M2P work item (sweeps)")
    ap.add_argument("--precond", type=int, default=None, help="1: block-diagonal GMRES preconditioner")
    ap.add_argument("--graphs", type=int, default=None, help="0: plain launches instead of the upward-pass graph")
    ap.add_argument("--lanes", type=int, default=None, help="concurrent pose lanes of pgb_solve_batch")
    ap.add_argument("--overlap", type=int, default=None, help="0: FP64 residual after the inner solve")
    ap.add_argument("--batch", type=int, default=None, help="poses per block-diagonal union solve (pose workloads)")
    ap.add_argument("--residual", type=int, default=None, help="0: native FP64 outer residual, 1: double-single")
    ap.add_argument("--no-autotune", action="store_true", help="pose sweep over 8 molecules: library parameters")
    ap.add_argument("--no-lanes", action="store_true", help="pose sweep over 8 molecules: skip the lanes comparison")
    ap.add_argument("--pose-tol", type=float, default=None,
                    help="GMRES relative-residual tolerance of the 8-molecule pose sweep (default 1e-6 with its "
                         "preconditioner, 1e-5 without)")
    args = ap.parse_args()
    for k, v in (("leaf_size", args.leaf), ("P", args.P), ("theta", args.theta), ("p2p_item", args.p2p_item),
                 ("m2p_item", args.m2p_item), ("precond", args.precond),
                 ("graphs", args.graphs), ("lanes", args.lanes), ("overlap", args.overlap), ("batch", args.batch),
                 ("residual", args.residual)):
        if v is not None:
            PARAMS[k] = v
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "star":
        run_star(args)
    elif args.workload == "gradient":
        run_gradient(args)
    elif args.workload == "brick":
        run_brick(args)
    elif args.workload == "scaling":
        run_scaling(args)
    elif args.workload == "stern":
        run_stern(args)
    elif args.workload == "replica":
        run_replica(args)
    elif args.workload == "poses":
        run_poses(args)
    elif args.workload == "poses_uneven":
        run_poses_uneven(args)
    elif args.mode == "matvec":
        run_matvec(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
