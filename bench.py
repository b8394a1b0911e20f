"""Benchmark of the quasi-static tet-FEM indentation solve on B300.

Default workload (--workload fingertip): one step = one complete indentation
solve (all 20 load steps: FP64 residual, FP32 tangent, block-Jacobi PCG in
Chronopoulos-Gear form, line search) of the single-fingertip sphere workload:
a two-layer half-capsule fingertip (R = 7 mm, L = 40 mm, 38,880 tets / 8,740
nodes) pressed 2 mm by a sphere of radius 4 mm in 20 load steps, to a
relative residual of 1e-6. The mesh is resident on the device when the timed
region starts; outputs go to device buffers. The end-to-end figure goes
through the same public C ABI from host arrays (mesh upload, indenter, solve,
host outputs, release) every step.

Batched workloads print their own line:
  --workload batch   one step = 256 random indentations of that fingertip
                     (sphere / cylinder / box edge, tilt <= 30 deg, depth
                     0.5-3 mm) in one replayed CUDA graph of the persistent
                     batched kernel (fem_batch_run).
  --workload uneven  one step = 64 fingertips of uneven size (R 5-10 mm,
                     5k-200k tets log-uniform), one random indentation each,
                     in one launch; the slot shape comes from fem_batch_tune.
  --workload dynamic the fingertip solve as 20 backward-Euler time steps of
                     1e-4 s (the paper's implicit time step) from rest, with
                     the lumped mass of a 1100 kg/m^3 body; same line format.
  --workload calibrated  the same solve on the paper's calibrated model: one
                     co-rotational shell, E=1.55 MPa, nu=0.316.
  --workload friction    the fingertip solve with Coulomb friction mu=0.783.
  --workload serve   Poisson streams of requests over a resident pool of 16
                     fingertip meshes (5k-200k tets) through the request
                     server (continuous batching), one session per offered
                     rate; latency p50/p99 and throughput beside the plain
                     one-solve-per-launch path on the same arrival trace.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl cuda|reference]
                    [--workload fingertip|dynamic|calibrated|friction|batch|uneven|serve]

Multi-GPU runs (torchrun) are independent replicas: every rank solves its own
indentation, no collectives on the data path (weak scaling).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "indentation solves/s at residual 1e-6; kernel HBM GB/s vs peak; p50/p99 latency"
UNIT = "solves/s"
TOL = 1e-6
WORKLOAD = ("fingertip_sphere: two-layer half-capsule fingertip R=7 mm L=40 mm (1 mm skin "
            "E=1.5 MPa nu=0.45 over 2 mm inner E=0.2 MPa nu=0.48, core fixed), 38880 tets / "
            "8740 nodes; sphere r=4 mm pressed 2 mm normal to a seeded skin point in 20 load steps")
DYN_DT, DYN_DENSITY = 1e-4, 1.1e-9     # s; t/mm^3 (1100 kg/m^3)
FRICTION_MU = 0.783                    # the paper's calibrated Coulomb coefficient
# single-solve variants of the fingertip workload: description, oracle
# arguments, stored oracle solution (its Newton count extrapolates the CPU leg)
VARIANTS = {
    "fingertip": (WORKLOAD, {}, "fingertip_sphere_oracle.npz"),
    "dynamic": (WORKLOAD + f"; dynamic: each load step one backward-Euler time step of {DYN_DT:g} s from "
                f"rest, lumped mass of density {DYN_DENSITY:g} t/mm^3",
                {"dt": DYN_DT, "density": DYN_DENSITY}, "fingertip_sphere_dynamic_oracle.npz"),
    "calibrated": ("fingertip_calibrated: the same geometry and load as one co-rotational linear-elastic shell "
                   "(E=1.55 MPa, nu=0.316, the paper's calibrated parameters) over the fixed core",
                   {}, "fingertip_calibrated_oracle.npz"),
    "friction": (WORKLOAD + f"; lagged smoothed Coulomb friction mu={FRICTION_MU} (slip smoothing 0.01 h_bar)",
                 {"mu_f": FRICTION_MU}, "fingertip_sphere_friction_oracle.npz"),
}


def variant_case(name, seed=None):
    """(mesh, indenter) of a single-solve variant."""
    import workloads as W
    kw = {} if seed is None else {"seed": seed}
    return W.fingertip_calibrated(**kw) if name == "calibrated" else W.fingertip_sphere(**kw)


def variant_options(F, name):
    opt = F.fem_default_options()
    if name == "dynamic":
        opt.dt, opt.density = DYN_DT, DYN_DENSITY
    elif name == "friction":
        opt.mu_f = FRICTION_MU
    return opt


def replica_seed(rank: int) -> int:
    """Skin-point seed of the indentation a replica solves (1001 = the
    single-fingertip workload; rank r solves its own seeded draw)."""
    return 1001 + rank


def max_over_ranks(value: float, world: int, device=None) -> float:
    """MAX of a host scalar over all ranks (timing only, not on the data path)."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"fem_bench_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows)}


def algorithmic_bytes(n_tets, n_nodes, products, newton_iters, evals):
    """Per-launch algorithmic bytes of the solve kernel.

    Stored-tangent accounting of the indentation problem (FP32 = 4 B): per
    element-tangent product (each PCG iteration and each Chebyshev step of the
    preconditioner) 264 B/tet + 160 B/node (tangent 45 floats + Dm^-1 9 floats,
    tet ids, CSR, p read / y write, fused vector updates); per Newton iteration
    464 B/tet + 48 B/node extra (u read, tangent write, FP64 forces, CSR); per
    line-search energy pass 60 B/tet."""
    return (products * (264 * n_tets + 160 * n_nodes) + newton_iters * (464 * n_tets + 48 * n_nodes)
            + evals * 60 * n_tets)


def compact_bytes(n_tets, n_nodes, products, newton_iters, evals):
    """The same, for this library's compressed tangent (30 floats + ushort4 local
    ids per tet, node vectors in shared memory): per tangent product 128 B/tet
    read + 32 B/node published/loaded; per Newton iteration the FP64 pass (Dm^-1
    72 B, V 8 B, ids 8 B, info 4 B) + tangent write 128 B; per energy pass
    92 B/tet."""
    return (products * (128 * n_tets + 32 * n_nodes) + newton_iters * (220 * n_tets + 48 * n_nodes)
            + evals * 92 * n_tets)


# device-side sources of the profiled kernels and of the shared-memory layout
# they run with (host code that only prepares the same inputs is left out)
KERNEL_SOURCES = ("fem_internal.h", "fem_math.cuh", "fem_solve.cu")


def source_digest():
    """SHA-256 over the kernel sources (the kernels as built)."""
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2103_16747_b300", "csrc")
    for f in KERNEL_SOURCES:
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(f.encode() + fh.read())
    return h.hexdigest()[:16]


def profiled_traffic(summary="solve_kernel_fingertip_sphere.md", key="traffic_bytes_per_launch"):
    """DRAM bytes (per launch, or per solve) from a committed ncu summary, or
    None if the kernel sources changed since that capture."""
    path = os.path.join(ROOT, "profiles", summary)
    if not os.path.exists(path):
        return None
    vals = {}
    for line in open(path):
        if ":" in line and line.strip().startswith(("- source_digest", "- " + key)):
            k, v = line.strip()[2:].split(":", 1)
            vals[k.strip()] = v.strip().strip("`")
    if vals.get("source_digest") != source_digest():
        return None
    try:
        return float(vals[key])
    except (KeyError, ValueError):
        return None


def _oracle_steps(job):
    """One worker of cpu_oracle_batch_rate: the oracle's first load steps of
    one solve, timed (run in a spawned process)."""
    mesh, ind, n_load_steps = job
    from oracle import Problem
    t0 = time.perf_counter()
    r = Problem(mesh, ind).solve(tol=1e-10, load_steps=n_load_steps)
    return time.perf_counter() - t0, int(np.sum(r.newton_iters[:n_load_steps]))


def cpu_oracle_batch_rate(meshes, draws, n_jobs=16, n_load_steps=2):
    """The oracle as it stands on independent solves, one process per solve
    across the host cores (spawned, so no process inherits a CUDA context):
    the first n_load_steps of n_jobs seeded solves, extrapolated to the full
    load schedule by load steps."""
    import multiprocessing as mp
    cores = os.cpu_count() or 1
    jobs = [(meshes[i], draws[i], n_load_steps) for i in range(min(n_jobs, len(draws)))]
    t0 = time.perf_counter()
    with mp.get_context("spawn").Pool(processes=min(cores, len(jobs))) as pool:
        res = pool.map(_oracle_steps, jobs)
    wall = time.perf_counter() - t0
    full = [t * d.n_steps / n_load_steps for (t, _), d in zip(res, draws)]
    # throughput of a pool of min(cores, jobs) workers running such solves back to back
    workers = min(cores, len(jobs))
    value = workers / (sum(full) / len(full))
    return {"value": value, "unit": UNIT, "cores": workers, "kind": "oracle",
            "sample": (f"{len(jobs)} of the step's solves, load steps 1-{n_load_steps} each ({sum(n for _, n in res)} "
                       f"Newton iterations, {wall:.1f} s wall on {workers} processes), extrapolated to their full "
                       f"schedules by load steps; one spawned process per solve, nproc {cores}")}


def cpu_oracle_rate(mesh, ind, n_load_steps, variant="fingertip"):
    """Time the oracle (as it stands) on the first n_load_steps of the same
    solve and extrapolate to a full solve by Newton iterations, using the
    oracle's Newton count for the full solve stored in tests/golden."""
    try:
        from threadpoolctl import threadpool_info
    except ImportError:                     # not installed on every host
        def threadpool_info():
            return [{"num_threads": int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))}]
    from oracle import Problem
    _, kwargs, golden = VARIANTS[variant]
    p = Problem(mesh, ind, **kwargs)
    t0 = time.perf_counter()
    r = p.solve(tol=1e-10, load_steps=n_load_steps)
    dt = time.perf_counter() - t0
    its = int(np.sum(r.newton_iters[:n_load_steps]))
    full_its = None
    g = os.path.join(ROOT, "tests", "golden", golden)
    if os.path.exists(g):
        full_its = int(np.sum(np.load(g)["newton_iters"]))
    per_it = dt / max(its, 1)
    est = per_it * (full_its if full_its else its * ind.n_steps / n_load_steps)
    threads = max([t.get("num_threads", 1) for t in threadpool_info()] or [1])
    return {"value": 1.0 / est, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": (f"load steps 1-{n_load_steps} of 20 of the same solve ({its} Newton iterations, "
                       f"{dt:.1f} s), extrapolated by the oracle's {full_its} Newton iterations for the "
                       f"full solve; scipy SuperLU is single-threaded, BLAS pool {threads} threads, "
                       f"nproc {os.cpu_count()}"),
            "seconds": dt}


def run_reference(args, rank, world):
    """The oracle as it stands on the host cores (rank 0 only)."""
    if rank != 0:
        return
    variant = args.workload if args.workload in VARIANTS else "fingertip"
    mesh, ind = variant_case(variant)
    for _ in range(args.warmup):
        cpu_oracle_rate(mesh, ind, 1, variant)
    times, rates = [], []
    cores = 1
    for _ in range(args.steps):
        r = cpu_oracle_rate(mesh, ind, 1, variant)
        times.append(r["seconds"])
        rates.append(r["value"])
        cores = r["cores"]
    value = float(args.steps / sum(1.0 / v for v in rates))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 / value,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": VARIANTS[variant][0], "tol": TOL},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "each step: load step 1 of 20 of the solve, extrapolated by "
                                       "Newton iterations to a full solve"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_cuda(args, rank, world, local):
    import torch
    import workloads as W
    import paper_2103_16747_b300 as F

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    variant = args.workload
    mesh, ind = variant_case(variant, seed=replica_seed(rank))
    stream = torch.cuda.Stream(device=dev)
    solver = F.IndentationSolver(mesh, cuda_stream=stream)
    solver.set_indenter(ind)
    info = solver.info()
    opt = variant_options(F, variant)
    n = mesh.n_nodes
    d_u = torch.zeros((n, 3), dtype=torch.float64, device=dev)
    d_f = torch.zeros((ind.n_steps, 3), dtype=torch.float64, device=dev)
    d_fc = torch.zeros((n, 3), dtype=torch.float64, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # > 126 MB L2

    def solve_once():
        return F.fem_solve(solver.handle, ind.n_steps, TOL, opt, d_u, d_f, d_fc)[1]

    for _ in range(max(args.warmup, 0)):
        st = solve_once()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    kernel_ms, stats = [], []
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        for k in range(args.steps):
            with torch.cuda.stream(stream):
                flush.fill_(float(k))                 # evict L2 between timed steps
            ev[k][0].record(stream)
            st = solve_once()
            ev[k][1].record(stream)
            kernel_ms.append(st.kernel_ms)
            stats.append(st)
        torch.cuda.synchronize()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total = max_over_ranks(sum(step_ms) / 1000.0, world, dev)
    value = world * args.steps / total

    # end to end through the public API from host arrays, every step
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()   # noqa: E731
    h_nodes, h_tets = pin(mesh.nodes), pin(mesh.tets.astype(np.int32))
    h_mat, h_fixed = pin(mesh.tet_material.astype(np.int32)), pin(mesh.fixed_nodes.astype(np.int32))
    h_u = torch.zeros((n, 3), dtype=torch.float64).pin_memory()
    h_f = torch.zeros((ind.n_steps, 3), dtype=torch.float64).pin_memory()
    h_fc = torch.zeros((n, 3), dtype=torch.float64).pin_memory()
    h2d = (h_nodes.numel() * 8 + h_tets.numel() * 4 + h_mat.numel() * 4 + h_fixed.numel() * 4
           + mesh.materials.size * 8 + (12 + 3 + 3 + ind.n_steps) * 8)
    d2h = (h_u.numel() + h_f.numel() + h_fc.numel()) * 8
    e2e_times = []
    for k in range(args.warmup + args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        hd = F.fem_create_mesh(h_nodes, h_tets, h_mat, mesh.materials, h_fixed, None, stream)
        F.fem_set_indenter(hd, ind.shape, ind.pose, np.asarray(ind.params), ind.direction, ind.depth_schedule)
        F.fem_solve(hd, ind.n_steps, TOL, opt, h_u, h_f, h_fc)
        F.fem_destroy_mesh(hd)
        t1 = time.perf_counter()
        if k >= args.warmup:
            e2e_times.append(t1 - t0)
    e2e_total = max_over_ranks(sum(e2e_times), world, dev)

    # roofline of the dominant kernel (the persistent solve kernel)
    s0 = stats[-1]
    evals = s0.newton_iters + s0.backtracks + ind.n_steps
    kms = statistics.mean(kernel_ms)
    alg = algorithmic_bytes(mesh.n_tets, n, s0.tangent_products, s0.newton_iters, evals)
    cmp_b = compact_bytes(mesh.n_tets, n, s0.tangent_products, s0.newton_iters, evals)
    peak, peak_kind = peaks()
    achieved = alg / (kms / 1000.0) / 1e9
    # the committed capture is of the default variant
    traffic = profiled_traffic() if variant == "fingertip" else None
    lat = sorted(step_ms)
    p = lambda q: lat[min(len(lat) - 1, int(math.ceil(q * len(lat))) - 1)]   # noqa: E731
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total * 1000.0 / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32 (tangent, PCG vectors) + f64 (residual, "
            "energy, reductions, displacement)", "data": "synthetic",
            "config": {"workload": VARIANTS[variant][0], "tol": TOL, "n_parts": info.n_parts,
                       "l2": "flushed between timed steps (256 MiB write, L2 is 126 MB)",
                       "replicas": world, "newton_iters": s0.newton_iters, "cg_iters": s0.cg_iters,
                       "tangent_products": s0.tangent_products, "backtracks": s0.backtracks,
                       "preconditioner": f"Chebyshev degree {opt.precond_degree} on block-Jacobi, "
                                         f"interval [4/{opt.precond_ratio:g}, 4]"},
            "latency_ms": {"p50": p(0.5), "p99": p(0.99)},
            "e2e": {"value": world * args.steps / e2e_total, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(d2h)},
            "gpu_launches": 3 * args.steps,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic, "kernel": "solve_kernel",
                         "kernel_ms": kms, "algorithmic_bytes": alg, "peak_kind": peak_kind,
                         "compact_accounting_GBs": cmp_b / (kms / 1000.0) / 1e9},
            "clocks": clk.summary()}
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = {k: v for k, v in cpu_oracle_rate(mesh, ind, 2, variant).items() if k != "seconds"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    solver.close()
    if world > 1:
        torch.distributed.destroy_process_group()


FP32_PEAK_TFLOPS = 148 * 128 * 2 * 2.032e9 / 1e12   # SMs x FP32 lanes x FMA x max SM clock


def flops_per_solve(n_tets, n_nodes, products, newton_iters):
    """FP32 work of the hot path: ~300 flop/tet + ~40 flop/node per tangent
    product, ~600 flop/tet per Newton iteration (tangent build)."""
    return products * (300 * n_tets + 40 * n_nodes) + newton_iters * 600 * n_tets


def run_batch(args, rank, world, local):
    """Batched workloads: many independent solves per step in one launch."""
    import torch
    import workloads as W
    import paper_2103_16747_b300 as F

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    opt = F.fem_default_options()
    opt.max_newton = 200            # deep random draws need more Newton steps in their last load steps
    if args.workload == "batch":
        mesh, _ = W.fingertip_sphere()
        draws = W.draw_indentations(mesh, args.n_solves, seed=1002 + 1000 * rank)
        meshes = [mesh] * len(draws)
        workload = (f"batch: {len(draws)} random indentations (sphere r 2-6 / cylinder r 1-4 / 20 mm box edge, "
                    f"tilt <= 30 deg, depth 0.5-3 mm, 20 load steps) of the fingertip of the single-solve "
                    f"workload ({mesh.n_tets} tets / {mesh.n_nodes} nodes), one replayed CUDA graph per step")
    else:
        jobs = W.uneven_fingertips(args.n_solves, seed=1003 + 1000 * rank)
        meshes = [m for m, _ in jobs]
        draws = [d for _, d in jobs]
        workload = (f"uneven: {len(draws)} fingertips R 5-10 mm, {min(m.n_tets for m in meshes)}-"
                    f"{max(m.n_tets for m in meshes)} tets (log-uniform 5k-200k, {sum(m.n_tets for m in meshes)} "
                    f"total), one random indentation each, one launch per step")
    uniq = {id(m): m for m in meshes}
    handles = {k: F.fem_create_mesh(m.nodes, m.tets, m.tet_material, m.materials, m.fixed_nodes)
               for k, m in uniq.items()}
    hs = [handles[id(m)] for m in meshes]
    # both batched workloads take their slot shape from the autotuner, unless
    # a fixed group size is asked for (profiling: then the plan's launches are
    # the only ones)
    t0 = time.perf_counter()
    if args.batch_parts:
        opt.batch_engine, opt.batch_parts = F.FEM_BATCH_GROUPS, args.batch_parts
        tune = {"skipped": f"uniform groups of {args.batch_parts} CTAs (--batch-parts)"}
    else:
        opt, rep = F.fem_batch_tune(hs, draws, TOL, opt, proxy_steps=4)
        tune = {"seconds": time.perf_counter() - t0,
                "chosen": {"engine": opt.batch_engine, "parts": opt.batch_parts,
                           "tets_per_cta": opt.batch_tets_per_cta},
                "candidates": [{"engine": rep.engine[k], "parts": rep.parts[k],
                                "tets_per_cta": rep.tets_per_cta[k], "proxy_solves_per_s": rep.rate[k]}
                               for k in range(rep.n_candidates)]}
    plan = F.FemBatch(hs, [d.n_steps for d in draws], opt)
    info = plan.info()
    outs = [torch.zeros((m.n_nodes, 3), dtype=torch.float64, device=dev) for m in meshes]
    frcs = [torch.zeros((d.n_steps, 3), dtype=torch.float64, device=dev) for d in draws]
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    for _ in range(max(args.warmup, 0)):
        plan.run(draws, TOL, outs, frcs, check=False)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    step_s, stats = [], None
    with ClockSampler(local) as clk:
        for k in range(args.steps):
            flush.fill_(float(k))
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            rc, stats = plan.run(draws, TOL, outs, frcs, check=False)
            torch.cuda.synchronize()
            step_s.append(time.perf_counter() - t0)
    kernel_ms = stats[0].kernel_ms
    total = max_over_ranks(sum(step_s), world, dev)
    n = len(draws)
    value = world * n * args.steps / total
    ok = sum(1 for s_ in stats if s_.status == 0)
    alg = sum(algorithmic_bytes(m.n_tets, m.n_nodes, s_.tangent_products, s_.newton_iters,
                                s_.newton_iters + s_.backtracks + d.n_steps)
              for m, s_, d in zip(meshes, stats, draws))
    flops = sum(flops_per_solve(m.n_tets, m.n_nodes, s_.tangent_products, s_.newton_iters)
                for m, s_ in zip(meshes, stats))
    peak, peak_kind = peaks()
    achieved = alg / (kernel_ms / 1000.0) / 1e9
    # the plain one-solve-per-launch path (fem_solve, one cooperative launch
    # per solve) on every draw of the step, kernel time
    single_s = 0.0
    for i in range(n):
        s1 = F.IndentationSolver(meshes[i])
        s1.set_indenter(draws[i])
        r = s1.solve(TOL, opt, check=False)
        single_s += r["stats"].kernel_ms / 1000.0
        s1.close()
    # end to end: public one-shot call from host arrays (meshes uploaded every step)
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()   # noqa: E731
    h_out = [torch.zeros((m.n_nodes, 3), dtype=torch.float64).pin_memory() for m in meshes]
    h_frc = [torch.zeros((d.n_steps, 3), dtype=torch.float64).pin_memory() for d in draws]
    h2d = sum(m.nodes.size * 8 + m.tets.size * 4 + m.tet_material.size * 4 + m.fixed_nodes.size * 4
              for m in uniq.values()) + sum((12 + 3 + 3 + d.n_steps) * 8 for d in draws)
    d2h = sum(o.numel() * 8 for o in h_out) + sum(f.numel() * 8 for f in h_frc)
    h_in = {k: (pin(m.nodes), pin(m.tets.astype(np.int32)), pin(m.tet_material.astype(np.int32)),
                pin(m.fixed_nodes.astype(np.int32))) for k, m in uniq.items()}
    e2e_s = 0.0
    for _ in range(args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        eh = {k: F.fem_create_mesh(h_in[k][0], h_in[k][1], h_in[k][2], m.materials, h_in[k][3])
              for k, m in uniq.items()}
        F.fem_solve_batch([eh[id(m)] for m in meshes], draws, TOL, opt, h_out, h_frc, check=False)
        for h_ in eh.values():
            F.fem_destroy_mesh(h_)
        e2e_s += time.perf_counter() - t0
    e2e_s = max_over_ranks(e2e_s, world, dev)
    # DRAM traffic from the committed capture of the same slot shape (uniform
    # 37-CTA groups on this fingertip, 8 solves), scaled by the solves of the
    # launch; None for other shapes or changed sources
    traffic = None
    if args.workload == "batch" and info.engine == 1 and info.parts == 37:
        per_solve = profiled_traffic("group_kernel_fingertip_batch.md", "traffic_bytes_per_solve")
        traffic = per_solve * n if per_solve is not None else None
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total * 1000.0 / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 (tangent, PCG vectors) + f64 (residual, energy, reductions, displacement)",
            "data": "synthetic",
            "config": {"workload": workload, "tol": TOL, "solves_per_step": n, "converged": ok,
                       "engine": {1: "cta_groups", 2: "clusters"}[info.engine], "ctas_per_solve": info.parts,
                       "slots": info.slots, "graph": bool(info.graph), "resident_tangent": bool(info.resident_tangent),
                       "cg_iters_total": sum(s_.cg_iters for s_ in stats),
                       "newton_iters_total": sum(s_.newton_iters for s_ in stats),
                       "l2": "flushed between timed steps (256 MiB write, L2 is 126 MB)", "autotune": tune},
            "single_path_same_draws": {"value": n / single_s, "unit": UNIT, "solves": n,
                                       "note": "fem_solve (one cooperative launch per solve) on every draw "
                                               "of the step, sum of kernel times"},
            "e2e": {"value": world * n * args.steps / e2e_s, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(d2h)},
            "gpu_launches": (1 + n) * args.steps,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "kernel": "group_kernel" if info.engine == 1 else "cluster_kernel",
                         "kernel_ms": kernel_ms, "algorithmic_bytes": alg, "peak_kind": peak_kind,
                         "fp32_tflops": flops / (kernel_ms / 1000.0) / 1e12, "fp32_peak_tflops": FP32_PEAK_TFLOPS},
            "clocks": clk.summary()}
    if rank == 0 and not args.no_cpu_baseline:
        # the oracle's direct solve is for meshes up to the fingertip's size
        small = [k for k, m in enumerate(meshes) if m.n_tets <= 40000]
        line["cpu_baseline"] = cpu_oracle_batch_rate([meshes[k] for k in small], [draws[k] for k in small])
    if rank == 0:
        print(json.dumps(line), flush=True)
    plan.close()
    for h_ in handles.values():
        F.fem_destroy_mesh(h_)
    if world > 1:
        torch.distributed.destroy_process_group()


def percentile(xs, q):
    xs = sorted(xs)
    if not xs:
        return None
    return xs[min(len(xs) - 1, max(0, int(math.ceil(q * len(xs))) - 1))]


def run_serve(args, rank, world, local):
    """Request server under Poisson arrivals (one session per offered rate)."""
    import torch
    import workloads as W
    import paper_2103_16747_b300 as F

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    jobs = W.uneven_fingertips(16, seed=1004 + 1000 * rank)
    pool = [m for m, _ in jobs]
    kinds = [(k, d) for k, m in enumerate(pool) for d in W.draw_indentations(m, 4, seed=2000 + k)]
    handles = [F.fem_create_mesh(m.nodes, m.tets, m.tet_material, m.materials, m.fixed_nodes) for m in pool]
    opt = F.fem_default_options()
    opt.max_newton = 200
    sopt = F.fem_default_options()
    sopt.max_newton = 200
    sopt.batch_parts = args.serve_class_cap
    if args.serve_tets_per_cta:
        sopt.batch_tets_per_cta = args.serve_tets_per_cta
    # the plain path: one fem_solve (cooperative launch) per request kind, kernel time
    t_plain = []
    for k, d in kinds:
        s1 = F.IndentationSolver(pool[k])
        s1.set_indenter(d)
        t_plain.append(s1.solve(TOL, opt, check=False)["stats"].kernel_ms / 1000.0)
        s1.close()
    srv = F.FemServer(handles, 20, sopt, result_bytes=1 << 30)
    info = srv.info()
    rng = np.random.Generator(np.random.PCG64(1004 + 1000 * rank))
    sessions = []
    with ClockSampler(local) as clk:
        for rate in args.rates:
            n_req = int(rng.poisson(rate * args.serve_seconds))
            arrivals = np.cumsum(rng.exponential(1.0 / rate, size=n_req))
            arrivals = arrivals[arrivals < args.serve_seconds]
            picks = rng.integers(0, len(kinds), size=len(arrivals))
            srv.start(args.serve_seconds + args.drain_seconds)
            t0 = time.perf_counter()
            ids, rejected = [], 0
            for a, p_ in zip(arrivals, picks):
                dt = t0 + a - time.perf_counter()
                if dt > 0:
                    time.sleep(dt)
                k, d = kinds[p_]
                rc, rid = srv.submit(k, d, TOL)
                if rc == 0:
                    ids.append((rid, p_))
                else:
                    rejected += 1
            lat, ok, t_first, t_last = [], 0, None, None
            for rid, p_ in ids:
                k, d = kinds[p_]
                left = max(1, int(1000 * (t0 + args.serve_seconds + args.drain_seconds - time.perf_counter())))
                rc, _, _, st, tm = srv.result(rid, pool[k].n_nodes, d.n_steps, wait_ms=left)
                if rc == F.FEM_PENDING:
                    continue
                lat.append(1000.0 * (tm[2] - tm[0]))
                ok += rc == 0
                t_first = tm[0] if t_first is None else min(t_first, tm[0])
                t_last = tm[2] if t_last is None else max(t_last, tm[2])
            srv.stop()
            done = len(lat)
            # the plain path on the same trace: one GPU worker, FIFO, each
            # request taking its kind's measured fem_solve time
            fin, plain_lat = 0.0, []
            for a, p_ in zip(arrivals, picks):
                fin = max(fin, a) + t_plain[p_]
                plain_lat.append(1000.0 * (fin - a))
            sessions.append({
                "offered_per_s": rate, "requests": int(len(arrivals)), "rejected": rejected, "completed": done,
                "converged": int(ok), "throughput": done / (t_last - t_first) if done > 1 else None,
                "p50_ms": percentile(lat, 0.5), "p99_ms": percentile(lat, 0.99),
                "plain_path": {"throughput": len(arrivals) / fin if fin > 0 else None,
                               "p50_ms": percentile(plain_lat, 0.5), "p99_ms": percentile(plain_lat, 0.99)}})
            print(json.dumps({"session": sessions[-1]}), file=sys.stderr, flush=True)
    best = max((x["throughput"] or 0.0) for x in sessions)
    line = {"metric": METRIC, "value": best, "unit": UNIT, "n_gpus": world, "steps": len(sessions), "warmup": 0,
            "ms_per_step": 1000.0 * args.serve_seconds, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None,
            "dtype": "f32 (tangent, PCG vectors) + f64 (residual, energy, reductions, displacement)",
            "data": "synthetic",
            "config": {"workload": (f"serve: Poisson requests over a resident pool of 16 fingertips "
                                    f"({min(m.n_tets for m in pool)}-{max(m.n_tets for m in pool)} tets), "
                                    f"4 random indentations per mesh, {args.serve_seconds:.0f} s per offered rate"),
                       "tol": TOL, "tets_per_cta_target": sopt.batch_tets_per_cta,
                       "size_classes": list(info.class_parts[:info.n_classes]),
                       "groups": list(info.class_groups[:info.n_classes]), "result_slots": info.result_slots,
                       "plain_path": "fem_solve per request in arrival order, measured kernel time per request kind "
                                     "(queueing simulated on the same trace)"},
            "sessions": sessions,
            "latency_ms": {"p50": sessions[0]["p50_ms"], "p99": sessions[0]["p99_ms"],
                           "at_offered_per_s": sessions[0]["offered_per_s"]},
            "gpu_launches": len(sessions), "clocks": clk.summary()}
    if rank == 0:
        print(json.dumps(line), flush=True)
    srv.close()
    for h_ in handles:
        F.fem_destroy_mesh(h_)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["cuda", "reference"], default="cuda")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", choices=["fingertip", "dynamic", "calibrated", "friction", "batch", "uneven",
                                           "serve"], default="fingertip")
    ap.add_argument("--rates", type=float, nargs="+", default=[1.0, 2.0, 4.0, 8.0, 16.0],
                    help="offered request rates (req/s) of the serve workload")
    ap.add_argument("--serve-seconds", type=float, default=20.0)
    ap.add_argument("--drain-seconds", type=float, default=90.0)
    ap.add_argument("--serve-class-cap", type=int, default=64,
                    help="largest CTA group of the request server (power of two)")
    ap.add_argument("--serve-tets-per-cta", type=int, default=650,
                    help="size-class target of the request server (0: the library default, 1300); "
                         "650 gives larger groups per request than batches use")
    ap.add_argument("--batch-parts", type=int, default=0,
                    help="batched workloads: uniform CTA groups of this size instead of the autotuner")
    ap.add_argument("--n-solves", type=int, default=None,
                    help="solves per step of the batched workloads (default 256 / 64)")
    args = ap.parse_args()
    if args.n_solves is None:
        args.n_solves = 256 if args.workload == "batch" else 64
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
    elif args.workload in VARIANTS:
        run_cuda(args, rank, world, local)
    elif args.workload == "serve":
        run_serve(args, rank, world, local)
    else:
        run_batch(args, rank, world, local)


if __name__ == "__main__":
    main()
