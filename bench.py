"""Benchmark of the quasi-static tet-FEM indentation solve on B300.

Default workload (--workload batch): one step = 256 random indentations of the
single-fingertip mesh (two-layer half-capsule, R = 7 mm, L = 40 mm, 38,880 tets
/ 8,740 nodes; sphere r 2-6 / cylinder r 1-4 / 20 mm box edge, tilt <= 30 deg,
depth 0.5-3 mm, 20 load steps each) to a relative residual of 1e-6, in one
replayed CUDA graph of the persistent batched kernel (fem_batch_run), slot
shape from the autotuner, FP32 stored tangent. Meshes and workspace are
resident when the timed region starts; outputs go to device buffers. Beside it
the line carries the plain path (one fem_solve launch per indentation) on the
same draws, the end-to-end figure through the public one-shot call from pinned
host arrays, the roofline of the batched kernel and the oracle on the host
cores.

Other workloads print the same kind of line:
  --workload fingertip   one step = the single sphere indentation of that
                         fingertip (2 mm, r = 4 mm, 20 load steps), fem_solve.
  --workload dynamic     the same as 20 backward-Euler time steps of 1e-4 s from
                         rest (lumped mass, 1100 kg/m^3).
  --workload calibrated  the same on the paper's calibrated model: one
                         co-rotational shell, E = 1.55 MPa, nu = 0.316.
  --workload friction    the same with Coulomb friction mu = 0.783.
  --workload uneven      one step = 64 fingertips of uneven size (R 5-10 mm,
                         5k-200k tets log-uniform), one random indentation each.
  --workload serve       Poisson streams of requests over a resident pool of 16
                         fingertip meshes through the request server (continuous
                         batching), one session per offered rate, and the plain
                         one-solve-per-request path run on the same arrival trace.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl cuda|reference]
                    [--workload batch|fingertip|dynamic|calibrated|friction|uneven|serve]

Multi-GPU runs (torchrun) are independent replicas: every rank solves its own
draws, no collectives on the data path (weak scaling).
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
DTYPE = "f32 (tangent, PCG vectors) + f64 (residual, energy, line search, displacement)"
WORKLOAD = ("fingertip_sphere: two-layer half-capsule fingertip R=7 mm L=40 mm (1 mm skin "
            "E=1.5 MPa nu=0.45 over 2 mm inner E=0.2 MPa nu=0.48, core fixed), 38880 tets / "
            "8740 nodes; sphere r=4 mm pressed 2 mm normal to a seeded skin point in 20 load steps")
DYN_DT, DYN_DENSITY = 1e-4, 1.1e-9     # s; t/mm^3 (1100 kg/m^3)
FRICTION_MU = 0.783                    # the paper's calibrated Coulomb coefficient
VARIANTS = {
    "fingertip": (WORKLOAD, {}),
    "dynamic": (WORKLOAD + f"; dynamic: each load step one backward-Euler time step of {DYN_DT:g} s from "
                f"rest, lumped mass of density {DYN_DENSITY:g} t/mm^3", {"dt": DYN_DT, "density": DYN_DENSITY}),
    "calibrated": ("fingertip_calibrated: the same geometry and load as one co-rotational linear-elastic shell "
                   "(E=1.55 MPa, nu=0.316, the paper's calibrated parameters) over the fixed core", {}),
    "friction": (WORKLOAD + f"; lagged smoothed Coulomb friction mu={FRICTION_MU} (slip smoothing 0.01 h_bar)",
                 {"mu_f": FRICTION_MU}),
}
BATCH_MAX_NEWTON = 400   # the deepest random draws need up to ~370 Newton steps at their hardest load step
L2_NOTE = "flushed between timed steps (256 MiB write, L2 is 126 MB)"


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


def batch_jobs(workload, n, rank):
    """(meshes, draws, description) of a batched workload; rank r draws its own."""
    import workloads as W
    if workload == "batch":
        mesh, _ = W.fingertip_sphere()
        draws = W.draw_indentations(mesh, n, seed=1002 + 1000 * rank)
        return [mesh] * len(draws), draws, (
            f"batch: {len(draws)} random indentations (sphere r 2-6 / cylinder r 1-4 / 20 mm box edge, "
            f"tilt <= 30 deg, depth 0.5-3 mm, 20 load steps) of the fingertip of the single-solve "
            f"workload ({mesh.n_tets} tets / {mesh.n_nodes} nodes), one replayed CUDA graph per step")
    jobs = W.uneven_fingertips(n, seed=1003 + 1000 * rank)
    meshes = [m for m, _ in jobs]
    return meshes, [d for _, d in jobs], (
        f"uneven: {len(jobs)} fingertips R 5-10 mm, {min(m.n_tets for m in meshes)}-"
        f"{max(m.n_tets for m in meshes)} tets (log-uniform 5k-200k, {sum(m.n_tets for m in meshes)} "
        f"total), one random indentation each, one launch per step")


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


# ------------------------------------------------------------ roofline accounting
#
# Two accountings of the bytes a solve moves, both from the iteration counts the
# library reports (fem_stats): products = tangent products (PCG iterations and
# preconditioner steps), newton = Newton iterations (each builds the tangent),
# evals = FP64 evaluation passes (one per Newton iteration, one per line-search
# halving, one per load step).

def stored_tangent_bytes(n_tets, n_nodes, products, newton, evals):
    """The indentation problem's reference accounting with a stored 45-float
    FP32 tangent: per product 264 B/tet + 160 B/node (tangent 45 floats + Dm^-1
    9 floats, tet ids, node->tet lists, p read / y write, fused vector updates);
    per Newton iteration 464 B/tet + 48 B/node (u read, tangent write, FP64
    forces, lists); per energy pass 60 B/tet."""
    return (products * (264 * n_tets + 160 * n_nodes) + newton * (464 * n_tets + 48 * n_nodes)
            + evals * 60 * n_tets)


def own_bytes(n_tets, n_nodes, products, newton, evals, tan_bytes):
    """This library's own bytes. Per tangent product: the stored tangent
    (tan_bytes per tet: 30 floats in 8 float4 = 128 B, or 64 B in FP16), local
    node ids 8 B and four node->tet entries 16 B per tet; per node the published
    vector (12 B), its halo read (12 B) and the accumulator (8 B). Per Newton
    iteration (tangent build): Dm^-1 72 B, volume 8 B, ids 8 B, material 4 B
    per tet read, the tangent written, 48 B per node. Per evaluation pass: the
    same 92 B per tet read, 96 B of FP64 corner forces written by the tet's
    owner and 96 B read back, 48 B per node (u read, residual and contact
    written)."""
    return (products * ((tan_bytes + 24) * n_tets + 32 * n_nodes)
            + newton * ((92 + tan_bytes) * n_tets + 48 * n_nodes)
            + evals * (284 * n_tets + 48 * n_nodes))


def product_bytes(n_tets, n_nodes, tan_bytes):
    return (tan_bytes + 24) * n_tets + 32 * n_nodes


FP32_PEAK_TFLOPS = 148 * 128 * 2 * 2.032e9 / 1e12   # SMs x FP32 lanes x FMA x max SM clock


def flops_per_solve(n_tets, n_nodes, products, newton):
    """FP32 work of the hot path: ~300 flop/tet + ~40 flop/node per tangent
    product, ~600 flop/tet per Newton iteration (tangent build)."""
    return products * (300 * n_tets + 40 * n_nodes) + newton * 600 * n_tets


def evals_of(st, n_steps):
    return st.newton_iters + st.backtracks + n_steps


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


def profiled_value(summary, key):
    """A figure from a committed ncu summary, or None if the kernel sources
    changed since that capture."""
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


def phase_fractions(rows, peak, time_ms):
    """Per-phase bandwidth: rows = [(bytes, share of the kernel time)]; the
    phase time is share x time_ms."""
    out = {}
    for name, (b, share) in rows.items():
        t = share * time_ms / 1000.0
        gbs = b / t / 1e9 if t > 0 else None
        out[name] = {"bytes": b, "time_ms": share * time_ms, "achieved_GBs": gbs,
                     "frac": (gbs / peak) if gbs else None}
    return out


# ------------------------------------------------------------ CPU oracle legs

def _oracle_sample(job):
    """One worker of the oracle legs: the oracle as it stands on the first
    load steps of one solve (Problem set-up included), timed."""
    mesh, ind, n_load_steps, kwargs = job
    from oracle import Problem
    t0 = time.perf_counter()
    r = Problem(mesh, ind, **kwargs).solve(tol=1e-10, load_steps=n_load_steps)
    return time.perf_counter() - t0, int(np.sum(r.newton_iters[:n_load_steps]))


def _one_thread_per_worker():
    """Pool initializer: one BLAS thread per worker process (one process per
    core; SuperLU itself is single-threaded)."""
    try:
        from threadpoolctl import threadpool_limits
        threadpool_limits(1)
    except Exception:
        pass


class OraclePool:
    """Spawned worker processes for the oracle (spawned, so no worker inherits
    a CUDA context); one solve sample per worker at a time."""

    def __init__(self, n):
        import multiprocessing as mp
        self.n = max(1, int(n))
        init = _one_thread_per_worker if self.n > 1 else None
        self.pool = mp.get_context("spawn").Pool(processes=self.n, initializer=init)

    def run(self, jobs):
        t0 = time.perf_counter()
        res = self.pool.map(_oracle_sample, jobs, chunksize=1)
        return time.perf_counter() - t0, res

    def close(self):
        self.pool.close()
        self.pool.join()


def blas_threads():
    try:
        from threadpoolctl import threadpool_info
        return max([t.get("num_threads", 1) for t in threadpool_info()] or [1])
    except Exception:
        return int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))


def oracle_sample_rate(pool, meshes, draws, picks, n_load_steps, kwargs=None):
    """Solves/s of the oracle on a bounded sample: load steps 1..n_load_steps
    of each picked solve, all picks at once on the pool. The sample's share of
    a full solve is n_load_steps / K (K load steps per solve), so the rate is
    (picks x n_load_steps / K) / wall. Later load steps take more Newton
    iterations than the first ones, so this overstates the oracle's rate."""
    jobs = [(meshes[k], draws[k], n_load_steps, kwargs or {}) for k in picks]
    wall, res = pool.run(jobs)
    solves = sum(n_load_steps / draws[k].n_steps for k in picks)
    return solves / wall, wall, sum(n for _, n in res)


def cpu_baseline_line(value, cores, sample):
    return {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample}


# ------------------------------------------------------------ reference arm

def run_reference(args, rank, world):
    """The oracle as it stands on the host cores (rank 0 only); every step is a
    bounded sample of the same workload, timed as it runs."""
    if rank != 0:
        return
    cores = os.cpu_count() or 1
    if args.workload in VARIANTS:
        mesh, ind = variant_case(args.workload)
        meshes, draws, desc, kwargs = [mesh], [ind], VARIANTS[args.workload][0], VARIANTS[args.workload][1]
        width = 1
    elif args.workload in ("batch", "uneven"):
        meshes, draws, desc = batch_jobs(args.workload, args.n_solves, 0)
        # the oracle's direct solve is for meshes up to the fingertip's size
        keep = [k for k, m in enumerate(meshes) if m.n_tets <= 40000]
        meshes, draws = [meshes[k] for k in keep], [draws[k] for k in keep]
        kwargs = {}
        width = min(cores, 16, len(draws))
    else:
        print(json.dumps({"impl": "reference", "unavailable": "the serving workload has no CPU reference: "
                          "its comparison is the plain one-solve-per-request GPU path"}), flush=True)
        return
    pool = OraclePool(width)
    walls, solves_done, newton = [], 0.0, 0
    for step in range(args.warmup + args.steps):
        picks = [(step * width + j) % len(draws) for j in range(width)]
        rate, wall, its = oracle_sample_rate(pool, meshes, draws, picks, 1, kwargs)
        if step >= args.warmup:
            walls.append(wall)
            solves_done += rate * wall
            newton += its
    pool.close()
    value = solves_done / sum(walls)
    sample = (f"each step: load step 1 of {draws[0].n_steps} of {width} solve(s) of the workload at once "
              f"({width} spawned process(es), set-up included; steps rotate through the draws), scaled to "
              f"full solves by load steps ({newton} Newton iterations in the timed steps); scipy SuperLU is "
              f"single-threaded, BLAS {'1 thread per process' if width > 1 else f'pool {blas_threads()} threads'}, "
              f"nproc {cores}")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * statistics.mean(walls),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": desc, "tol": TOL},
            "cpu_baseline": cpu_baseline_line(value, width, sample),
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------ single solve (C1 and variants)

def run_single(args, rank, world, local):
    import torch
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
        solve_once()
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

    # roofline of the dominant kernel (the persistent solve kernel), own bytes
    s0 = stats[-1]
    ev_n = evals_of(s0, ind.n_steps)
    kms = statistics.mean(kernel_ms)
    peak, peak_kind = peaks()
    own = own_bytes(mesh.n_tets, n, s0.tangent_products, s0.newton_iters, ev_n, 128)
    stored = stored_tangent_bytes(mesh.n_tets, n, s0.tangent_products, s0.newton_iters, ev_n)
    achieved = own / (kms / 1000.0) / 1e9
    ph = {name: s0.phase_ms[k] / max(s0.phase_ms[7], 1e-30) for k, name in enumerate(F.PHASES)}
    phases = phase_fractions({
        "tangent_product": (s0.tangent_products * product_bytes(mesh.n_tets, n, 128),
                            ph["product_element"] + ph["product_gather"]),
        "element_eval": (ev_n * (284 * mesh.n_tets + 48 * n), ph["eval"]),
        "tangent_build": (s0.newton_iters * ((92 + 128) * mesh.n_tets + 48 * n), ph["tangent"])}, peak, kms)
    traffic = (profiled_value("solve_kernel_fingertip_sphere.md", "traffic_bytes_per_launch")
               if variant == "fingertip" else None)
    lat = sorted(step_ms)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total * 1000.0 / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": DTYPE, "data": "synthetic",
            "config": {"workload": VARIANTS[variant][0], "tol": TOL, "n_parts": info.n_parts, "l2": L2_NOTE,
                       "replicas": world, "newton_iters": s0.newton_iters, "cg_iters": s0.cg_iters,
                       "tangent_products": s0.tangent_products, "backtracks": s0.backtracks,
                       "preconditioner": f"Chebyshev degree {opt.precond_degree} on block-Jacobi, "
                                         f"interval [4/{opt.precond_ratio:g}, 4]"},
            "latency_ms": {"p50": percentile(lat, 0.5), "p99": percentile(lat, 0.99)},
            "e2e": {"value": world * args.steps / e2e_total, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(d2h)},
            "gpu_launches": 3 * args.steps,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic, "kernel": "solve_kernel",
                         "kernel_ms": kms, "algorithmic_bytes": own, "accounting": "own (FP32 30-float tangent)",
                         "peak_kind": peak_kind, "phases": phases,
                         "stored_tangent_accounting": {"bytes": stored,
                                                       "achieved": stored / (kms / 1000.0) / 1e9,
                                                       "frac": stored / (kms / 1000.0) / 1e9 / peak}},
            "clocks": clk.summary()}
    if rank == 0 and not args.no_cpu_baseline:
        pool = OraclePool(1)
        rate, wall, its = oracle_sample_rate(pool, [mesh], [ind], [0], 2, VARIANTS[variant][1])
        pool.close()
        line["cpu_baseline"] = cpu_baseline_line(
            rate, 1, f"load steps 1-2 of {ind.n_steps} of the same solve (set-up included, {its} Newton "
                     f"iterations, {wall:.1f} s), scaled to a full solve by load steps (later steps take more "
                     f"Newton iterations: this overstates the oracle's rate); scipy SuperLU single-threaded, "
                     f"nproc {os.cpu_count()}")
    if rank == 0:
        print(json.dumps(line), flush=True)
    solver.close()
    if world > 1:
        torch.distributed.destroy_process_group()


# ------------------------------------------------------------ batched solves (C2, C3)

def run_batch(args, rank, world, local):
    import torch
    import paper_2103_16747_b300 as F

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    opt = F.fem_default_options()
    opt.max_newton = BATCH_MAX_NEWTON
    opt.tangent_fp16 = 1 if args.fp16_tangent else 0
    tan_bytes = 64 if args.fp16_tangent else 128
    meshes, draws, workload = batch_jobs(args.workload, args.n_solves, rank)
    uniq = {id(m): m for m in meshes}
    handles = {k: F.fem_create_mesh(m.nodes, m.tets, m.tet_material, m.materials, m.fixed_nodes)
               for k, m in uniq.items()}
    hs = [handles[id(m)] for m in meshes]
    # slot shape from the autotuner, unless a fixed group size is asked for
    # (profiling: then the plan's launches are the only ones)
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
    step_dev_ms, step_wall, stats = [], [], None
    with ClockSampler(local) as clk:
        for k in range(args.steps):
            flush.fill_(float(k))                     # evict L2 between timed steps
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            rc, stats = plan.run(draws, TOL, outs, frcs, check=False)
            torch.cuda.synchronize()
            step_wall.append(time.perf_counter() - t0)
            # device time of the replayed graph (CUDA events on the plan's stream
            # around the launch: workspace reset, uploads, persistent kernel, reorder)
            step_dev_ms.append(stats[0].kernel_ms)
    total = max_over_ranks(sum(step_dev_ms) / 1000.0, world, dev)
    n = len(draws)
    value = world * n * args.steps / total
    ok = sum(1 for s_ in stats if s_.status == 0)
    kms = statistics.mean(step_dev_ms)
    peak, peak_kind = peaks()
    per = [(m, s_, d, evals_of(s_, d.n_steps)) for m, s_, d in zip(meshes, stats, draws)]
    own = sum(own_bytes(m.n_tets, m.n_nodes, s_.tangent_products, s_.newton_iters, e, tan_bytes)
              for m, s_, d, e in per)
    stored = sum(stored_tangent_bytes(m.n_tets, m.n_nodes, s_.tangent_products, s_.newton_iters, e)
                 for m, s_, d, e in per)
    flops = sum(flops_per_solve(m.n_tets, m.n_nodes, s_.tangent_products, s_.newton_iters) for m, s_, d, e in per)
    achieved = own / (kms / 1000.0) / 1e9
    # per-phase bandwidth: each solve reports the shares of its own time spent
    # in each phase (clock of its part 0); groups run side by side for the whole
    # launch, so a phase's share of the launch is the product-weighted mean share
    wsum = sum(s_.tangent_products for _, s_, _, _ in per) or 1

    def share(*names):
        idx = [F.PHASES.index(x) for x in names]
        return sum(s_.tangent_products * sum(s_.phase_ms[i] for i in idx) for _, s_, _, _ in per) / wsum

    phases = phase_fractions({
        "tangent_product": (sum(s_.tangent_products * product_bytes(m.n_tets, m.n_nodes, tan_bytes)
                                for m, s_, _, _ in per), share("product_element", "product_gather")),
        "element_eval": (sum(e * (284 * m.n_tets + 48 * m.n_nodes) for m, s_, _, e in per), share("eval")),
        "tangent_build": (sum(s_.newton_iters * ((92 + tan_bytes) * m.n_tets + 48 * m.n_nodes)
                              for m, s_, _, _ in per), share("tangent"))}, peak, kms)
    # the plain one-solve-per-launch path (fem_solve: one cooperative launch
    # per solve, all SMs) on every draw of the step, kernel time
    single_s, single_ok = 0.0, 0
    for i in range(n):
        s1 = F.IndentationSolver(meshes[i])
        s1.set_indenter(draws[i])
        r = s1.solve(TOL, opt, check=False)
        single_s += r["stats"].kernel_ms / 1000.0
        single_ok += int(r["rc"] == 0)
        s1.close()
    # end to end: the public one-shot call from pinned host arrays, meshes
    # uploaded, the plan built and released inside every step
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()   # noqa: E731
    h_out = [torch.zeros((m.n_nodes, 3), dtype=torch.float64).pin_memory() for m in meshes]
    h_frc = [torch.zeros((d.n_steps, 3), dtype=torch.float64).pin_memory() for d in draws]
    h2d = sum(m.nodes.size * 8 + m.tets.size * 4 + m.tet_material.size * 4 + m.fixed_nodes.size * 4
              for m in uniq.values()) + sum((12 + 3 + 3 + d.n_steps) * 8 for d in draws)
    d2h = sum(o.numel() * 8 for o in h_out) + sum(f.numel() * 8 for f in h_frc)
    h_in = {k: (pin(m.nodes), pin(m.tets.astype(np.int32)), pin(m.tet_material.astype(np.int32)),
                pin(m.fixed_nodes.astype(np.int32))) for k, m in uniq.items()}
    e2e_steps = max(1, min(args.steps, args.e2e_steps))
    e2e_s = 0.0
    for _ in range(e2e_steps):
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
    # 37-CTA groups on this fingertip, 8 solves, FP32 tangent), scaled by the
    # solves of the launch; None for other shapes or changed sources
    traffic = None
    if args.workload == "batch" and info.engine == 1 and info.parts == 37 and not args.fp16_tangent:
        per_solve = profiled_value("group_kernel_fingertip_batch.md", "traffic_bytes_per_solve")
        traffic = per_solve * n if per_solve is not None else None
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total * 1000.0 / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": DTYPE, "data": "synthetic",
            "config": {"workload": workload, "tol": TOL, "solves_per_step": n, "converged": ok,
                       "tangent_storage": "fp16 (per-tet scale)" if args.fp16_tangent else "fp32",
                       "max_newton_per_step": BATCH_MAX_NEWTON,
                       "engine": {1: "cta_groups", 2: "clusters"}[info.engine], "ctas_per_solve": info.parts,
                       "slots": info.slots, "graph": bool(info.graph), "resident_tangent": bool(info.resident_tangent),
                       "cg_iters_total": sum(s_.cg_iters for s_ in stats),
                       "newton_iters_total": sum(s_.newton_iters for s_ in stats),
                       "tangent_products_total": sum(s_.tangent_products for s_ in stats),
                       "wall_ms_per_step": 1000.0 * statistics.mean(step_wall),
                       "l2": L2_NOTE, "autotune": tune},
            "plain_path_same_draws": {"value": n / single_s, "unit": UNIT, "solves": n, "converged": single_ok,
                                      "note": "fem_solve (one cooperative launch on all SMs per solve) on every "
                                              "draw of the step, same options and tolerance, sum of kernel times"},
            "e2e": {"value": world * n * e2e_steps / e2e_s, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(d2h), "steps": e2e_steps,
                    "note": "fem_create_mesh from pinned host arrays, fem_solve_batch (plan, graph, run, release) "
                            "with pinned host outputs, fem_destroy_mesh, every step"},
            # per step: the persistent kernel (once per phase of the plan; one
            # phase here) and one reorder kernel per solve
            "gpu_launches": (1 + n) * args.steps,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "kernel": "group_kernel" if info.engine == 1 else "cluster_kernel",
                         "kernel_ms": kms, "algorithmic_bytes": own,
                         "accounting": f"own ({'FP16' if args.fp16_tangent else 'FP32'} tangent, {tan_bytes} B/tet)",
                         "peak_kind": peak_kind, "phases": phases,
                         "stored_tangent_accounting": {"bytes": stored,
                                                       "achieved": stored / (kms / 1000.0) / 1e9,
                                                       "frac": stored / (kms / 1000.0) / 1e9 / peak},
                         "fp32_tflops": flops / (kms / 1000.0) / 1e12, "fp32_peak_tflops": FP32_PEAK_TFLOPS},
            "clocks": clk.summary()}
    if rank == 0 and not args.no_cpu_baseline:
        small = [k for k, m in enumerate(meshes) if m.n_tets <= 40000]
        width = min(os.cpu_count() or 1, 16, len(small))
        pool = OraclePool(width)
        picks = small[:width]
        rate, wall, its = oracle_sample_rate(pool, meshes, draws, picks, 2)
        pool.close()
        line["cpu_baseline"] = cpu_baseline_line(
            rate, width, f"load steps 1-2 of {width} of the step's solves (meshes up to 40k tets) at once, one "
                         f"spawned process each, set-up included ({its} Newton iterations, {wall:.1f} s wall), "
                         f"scaled to full solves by load steps (later steps take more Newton iterations: this "
                         f"overstates the oracle's rate); SuperLU single-threaded, nproc {os.cpu_count()}")
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


# ------------------------------------------------------------ serving (C4)

def run_serve(args, rank, world, local):
    """Request server under Poisson arrivals (one session per offered rate),
    then the plain path on the same arrival trace: one fem_solve per request,
    in arrival order, each started once it has arrived and the GPU is free."""
    import torch
    import workloads as W
    import paper_2103_16747_b300 as F

    torch.cuda.set_device(local)
    jobs = W.uneven_fingertips(16, seed=1004 + 1000 * rank)
    pool = [m for m, _ in jobs]
    kinds = [(k, d) for k, m in enumerate(pool) for d in W.draw_indentations(m, 4, seed=2000 + k)]
    handles = [F.fem_create_mesh(m.nodes, m.tets, m.tet_material, m.materials, m.fixed_nodes) for m in pool]
    opt = F.fem_default_options()
    opt.max_newton = BATCH_MAX_NEWTON
    sopt = F.fem_default_options()
    sopt.max_newton = BATCH_MAX_NEWTON
    sopt.batch_parts = args.serve_class_cap
    if args.serve_tets_per_cta:
        sopt.batch_tets_per_cta = args.serve_tets_per_cta
    srv = F.FemServer(handles, 20, sopt, result_bytes=1 << 30)
    info = srv.info()
    # each mesh's class as the server forms it (CTAs per solve; beyond 64 x
    # the tets-per-CTA target, the large- or huge-mesh group), to break
    # latencies down
    T = sopt.batch_tets_per_cta if sopt.batch_tets_per_cta > 0 else 1300
    p_large = info.class_parts[info.large_class] if info.large_class >= 0 else 0
    p_huge = info.class_parts[info.huge_class] if info.huge_class >= 0 else 0
    label = {}
    for k, m in enumerate(pool):
        p = 1
        while p < min(args.serve_class_cap, 64) and p * T < m.n_tets and 2 * p <= m.n_nodes:
            p *= 2
        if m.n_tets <= 64 * T:
            label[k] = f"{p:02d}_ctas"
        elif p_large and m.n_tets <= p_large * T:
            label[k] = f"large_{p_large}_ctas"
        else:
            label[k] = f"huge_{p_huge}_ctas"
    rng = np.random.Generator(np.random.PCG64(1004 + 1000 * rank))
    sessions = []
    prev_launches, prev_suspended = info.launches, info.suspended
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
            lat, ok, t_first, t_last, by = [], 0, None, None, {}
            for rid, p_ in ids:
                k, d = kinds[p_]
                left = max(1, int(1000 * (t0 + args.serve_seconds + args.drain_seconds - time.perf_counter())))
                rc, _, _, st, tm = srv.result(rid, pool[k].n_nodes, d.n_steps, wait_ms=left)
                if rc == F.FEM_PENDING:
                    continue
                lat.append(1000.0 * (tm[2] - tm[0]))
                by.setdefault(label[k], []).append(lat[-1])
                ok += rc == 0
                t_first = tm[0] if t_first is None else min(t_first, tm[0])
                t_last = tm[2] if t_last is None else max(t_last, tm[2])
            srv.stop()
            after = srv.info()
            launches, suspended = after.launches - prev_launches, after.suspended - prev_suspended
            prev_launches, prev_suspended = after.launches, after.suspended
            # the plain path on the same trace, run for real: one GPU worker,
            # requests in arrival order, each fem_solve on the pool's resident mesh
            plain, plain_lat = plain_path_on_trace(F, handles, pool, kinds, arrivals, picks, opt,
                                                   args.serve_seconds + args.drain_seconds)
            plain_by = {}
            for p_, x in zip(picks, plain_lat):
                plain_by.setdefault(label[kinds[p_][0]], []).append(x)
            plain["by_class"] = class_latencies(plain_by)
            sessions.append({
                "offered_per_s": rate, "requests": int(len(arrivals)), "rejected": rejected,
                "completed": len(lat), "converged": int(ok),
                "throughput": len(lat) / (t_last - t_first) if len(lat) > 1 else None,
                "p50_ms": percentile(lat, 0.5), "p99_ms": percentile(lat, 0.99),
                "by_class": class_latencies(by), "launches": launches, "suspended_solves": suspended,
                "plain_path": plain})
            print(json.dumps({"session": sessions[-1]}), file=sys.stderr, flush=True)
    best = max((x["throughput"] or 0.0) for x in sessions)
    line = {"metric": METRIC, "value": best, "unit": UNIT, "n_gpus": world, "steps": len(sessions), "warmup": 0,
            "ms_per_step": 1000.0 * args.serve_seconds, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": DTYPE, "data": "synthetic",
            "config": {"workload": (f"serve: Poisson requests over a resident pool of 16 fingertips "
                                    f"({min(m.n_tets for m in pool)}-{max(m.n_tets for m in pool)} tets), "
                                    f"4 random indentations per mesh, {args.serve_seconds:.0f} s per offered rate"),
                       "tol": TOL, "tets_per_cta_target": sopt.batch_tets_per_cta,
                       "size_classes": list(info.class_parts[:info.n_classes]),
                       "groups": list(info.class_groups[:info.n_classes]),
                       "launch_shapes": [{"ctas": info.shape_ctas[k],
                                          "groups": list(info.shape_groups[k][:info.n_classes])}
                                         for k in range(info.n_shapes)],
                       "result_slots": info.result_slots,
                       "plain_path": "fem_solve per request in arrival order on the same trace, run on the GPU "
                                     "(latency = completion - arrival)"},
            "sessions": sessions,
            "latency_ms": {"p50": sessions[0]["p50_ms"], "p99": sessions[0]["p99_ms"],
                           "at_offered_per_s": sessions[0]["offered_per_s"]},
            # one persistent launch per session and one per change of launch
            # shape (the plain-path comparison is not counted)
            "gpu_launches": sum(x["launches"] for x in sessions), "clocks": clk.summary()}
    if rank == 0:
        print(json.dumps(line), flush=True)
    srv.close()
    for h_ in handles:
        F.fem_destroy_mesh(h_)


def plain_path_on_trace(F, handles, pool, kinds, arrivals, picks, opt, limit_s):
    """One fem_solve per request on the trace, in arrival order, in real time."""
    lat, done, t_end = [], 0, None
    t0 = time.perf_counter()
    outs = {k: np.zeros((m.n_nodes, 3)) for k, m in enumerate(pool)}
    frc = np.zeros((20, 3))
    for a, p_ in zip(arrivals, picks):
        now = time.perf_counter() - t0
        if now > limit_s:
            break
        if now < a:
            time.sleep(a - now)
        k, d = kinds[p_]
        F.fem_set_indenter(handles[k], d.shape, d.pose, np.asarray(d.params), d.direction, d.depth_schedule)
        F.fem_solve(handles[k], d.n_steps, TOL, opt, outs[k], frc[:d.n_steps], None, check=False)
        t_end = time.perf_counter() - t0
        lat.append(1000.0 * (t_end - a))
        done += 1
    first = float(arrivals[0]) if len(arrivals) else 0.0
    return ({"completed": done, "throughput": done / (t_end - first) if done > 1 and t_end > first else None,
             "p50_ms": percentile(lat, 0.5), "p99_ms": percentile(lat, 0.99)}, lat)


def class_latencies(by):
    """Latency percentiles per size class (label -> latencies in ms)."""
    return {k: {"n": len(v), "p50_ms": percentile(v, 0.5), "p99_ms": percentile(v, 0.99), "max_ms": max(v)}
            for k, v in sorted(by.items())}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["cuda", "reference"], default="cuda")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", choices=["batch", "fingertip", "dynamic", "calibrated", "friction", "uneven",
                                           "serve"], default="batch")
    ap.add_argument("--fp16-tangent", action="store_true",
                    help="batched workloads: store the tangent in FP16 with a per-tet scale")
    ap.add_argument("--e2e-steps", type=int, default=3,
                    help="batched workloads: end-to-end steps timed (at most --steps)")
    ap.add_argument("--rates", type=float, nargs="+", default=[2.0, 8.0, 16.0, 32.0],
                    help="offered request rates (req/s) of the serve workload")
    ap.add_argument("--serve-seconds", type=float, default=60.0)
    ap.add_argument("--drain-seconds", type=float, default=90.0)
    ap.add_argument("--serve-class-cap", type=int, default=64,
                    help="largest CTA group of the request server (power of two)")
    ap.add_argument("--serve-tets-per-cta", type=int, default=0,
                    help="size-class target of the request server (0: the library default, 1300 tets per CTA; "
                         "smaller targets give each request a larger group but send more meshes to the "
                         "large- and huge-mesh launch shapes)")
    ap.add_argument("--batch-parts", type=int, default=0,
                    help="batched workloads: uniform CTA groups of this size instead of the autotuner")
    ap.add_argument("--n-solves", type=int, default=None,
                    help="solves per step of the batched workloads (default 256 / 64)")
    args = ap.parse_args()
    if args.n_solves is None:
        args.n_solves = 64 if args.workload == "uneven" else 256
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
    elif args.workload in VARIANTS:
        run_single(args, rank, world, local)
    elif args.workload == "serve":
        run_serve(args, rank, world, local)
    else:
        run_batch(args, rank, world, local)


if __name__ == "__main__":
    main()
