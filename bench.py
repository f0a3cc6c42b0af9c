"""Benchmark: time-to-solution of asynchronous vs synchronous RAS on one GB300.

Workload (one step = one full solve to relative residual 1e-8, inputs resident
in HBM): 2D Poisson 5-point on a 1024 x 1024 grid (1,048,576 unknowns), b
uniform in [-1, 1] from SplitMix64 seed 1, regular2d 16 x 16 = 256 subdomains,
overlap 4, local CG with 20 steps per update. The headline `value` is the
asynchronous mixed-precision solver (FP32 local CG, FP64 residual / update /
convergence tests); the plain synchronous FP64 solver and the other variants
are reported beside it.

--impl reference runs the CPU oracle (sequential FP64 synchronous RAS with the
same local solver) on the host cores: set up once (untimed, reported), then
each step is a bounded sample of iterations, whose per-iteration time is
extrapolated to the oracle's iteration count for this workload
(tests/golden/config2_sync_fp64_cg20_iterations.txt, written by the oracle).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import problems  # noqa: E402

METRIC = ("time-to-solution at rel. residual 1e-8 & HBM GB/s: async vs sync RAS; "
          "serving p50/p99")
N_GRID, PX, GAMMA, M_INNER, TOL, SEED = 1024, 16, 4, 20, 1e-8, 1
WORKLOAD = ("2D Poisson 5-point 1024x1024 (1,048,576 unknowns), uniform RHS seed 1, "
            "regular2d 16x16 = 256 subdomains, overlap 4, local CG 20 steps")
GOLDEN_ITERS = os.path.join(ROOT, "tests", "golden", "config2_sync_fp64_cg20_iterations.txt")
KERNEL_SRC = os.path.join(ROOT, "paper_2003_05361_gb300", "csrc", "ras_kernels.cu")


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), \
        int(os.environ.get("LOCAL_RANK", 0))


def max_over_ranks(v: float, device=None) -> float:
    """Max of v over the ranks of the default process group (v itself when
    there is no group or one rank): the time a step took on the slowest GPU."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return v
    t = torch.tensor([float(v)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def problem():
    A = problems.poisson2d(N_GRID)
    b = problems.rhs_uniform(A.n, SEED)
    return A, b


def oracle_iterations():
    with open(GOLDEN_ITERS) as f:
        return int([ln for ln in f if ln.strip() and not ln.startswith("#")][0])


# ---------------------------------------------------------------- CPU oracle

def oracle_setup(A, part):
    """The oracle's set-up half of Algorithm 1 for the benchmark workload
    (overlap maps, local matrices; sync FP64 RAS with local CG-20), timed
    apart from the iterations as Sec. 3.1 times its solves."""
    import oracle

    return oracle.RasSetup(A, part, PX * PX, GAMMA, oracle.CG, oracle.FP64, M_INNER)


def oracle_sample(h, b, x, budget_s: float, nthreads: int):
    """Times the oracle's synchronous RAS iterations on the already set-up
    handle h, continuing from x (updated in place): one iteration, then as
    many as fit in the rest of budget_s in one call. Returns (seconds per
    iteration, iterations run). The per-iteration cost does not depend on the
    sample length: set-up is excluded and every iteration does the same work."""
    t0 = time.perf_counter()
    h.iterate(b, x, max_iter=1, nthreads=nthreads)
    t1 = time.perf_counter() - t0
    k2 = max(1, int((budget_s - t1) / max(t1, 1e-4)))
    t0 = time.perf_counter()
    h.iterate(b, x, max_iter=k2, nthreads=nthreads)
    t2 = time.perf_counter() - t0
    return (t1 + t2) / (1 + k2), 1 + k2


def oracle_baseline(A, b, part, budget_s: float):
    """cpu_baseline: the oracle timed on the host cores, single-threaded and
    OpenMP-parallel over the subdomains of an iteration on every core,
    extrapolated from a bounded sample of iterations to the oracle's own
    iteration count for this workload; set-up timed once, separately."""
    cores = os.cpu_count() or 1
    iters = oracle_iterations()
    h = oracle_setup(A, part)
    x = np.zeros(A.n)
    out = {}
    for label, nt in (("all_cores", cores), ("single_thread", 1)):
        spi, k = oracle_sample(h, b, x, budget_s / 2, nt)
        out[label] = {"value": spi * iters * 1e3, "unit": "ms", "cores": nt,
                      "ms_per_iteration": spi * 1e3, "iterations_sampled": k}
    h.close()
    line = dict(out["all_cores"])
    line.update({
        "kind": "oracle",
        "sample": f"{out['all_cores']['iterations_sampled']} (all cores) and "
                  f"{out['single_thread']['iterations_sampled']} (one thread) sync FP64 RAS "
                  f"iterations (local CG-20) of the same workload after one untimed set-up, "
                  f"per-iteration time x the oracle's {iters} iterations to 1e-8",
        "setup_ms": h.setup_s * 1e3,
        "single_thread": out["single_thread"],
    })
    return line


def run_reference(args):
    rank, world, _ = dist_env()
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("gloo")
        if rank != 0:
            dist.barrier()
            return
    import oracle

    A, b = problem()
    part = oracle.partition_regular2d(N_GRID, N_GRID, PX, PX)
    iters = oracle_iterations()
    cores = os.cpu_count() or 1
    budget = float(os.environ.get("RAS_REF_STEP_S", "1.5"))
    h = oracle_setup(A, part)  # untimed, as in Sec. 3.1
    x = np.zeros(A.n)
    for _ in range(args.warmup):
        oracle_sample(h, b, x, budget / 4, cores)
    vals, samples, spis = [], [], []
    for _ in range(args.steps):
        spi, k = oracle_sample(h, b, x, budget, cores)
        vals.append(spi * iters * 1e3)
        samples.append(k)
        spis.append(spi * 1e3)
    h.close()
    v = statistics.median(vals)
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "ms", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": v, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "mode": "sync", "local_solver": "CG-20",
                   "local_precision": "fp64", "parallelism": "host cores (OpenMP)"},
        "cpu_baseline": {"value": v, "unit": "ms", "cores": cores, "kind": "oracle",
                         "sample": f"{statistics.median(samples)} sync RAS iterations per step "
                                   f"after one untimed set-up ({h.setup_s * 1e3:.0f} ms), "
                                   f"per-iteration time x the oracle's {iters} iterations",
                         "setup_ms": h.setup_s * 1e3,
                         "ms_per_iteration": statistics.median(spis)},
        "e2e": {"value": v, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


# ---------------------------------------------------------------- clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.out = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.out.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.out:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------- roofline model

def subdomain_bytes(A, ras, ctx, kind, prec_bytes, m, staged, col_bytes=2, grid=False):
    """Algorithmic bytes of one local update of each subdomain:
    residual = nnz(rows of Omega_p) (8 + 4) + 4 (n_p + 1) + 8 (n_p + |E_p|) + 8 n_p
    (grid layout, where every column is computed: nnz 8 + 8 (n_p + |E_p|) + 8 n_p),
    local CG = nnz(A_p) (s_v + c), once when A_p is staged in shared memory,
    m times when it is re-read every step (c = 2 bytes of int16 column per
    entry, 0 in the diagonal-offset form); ILU(0)-PCG = 2 nnz(A_p) (s + 2) m
    (A_p and the factors every step); band = 2 n_p (w_p + 1) s_f (the L
    and L^T, or L and U, bands);
    update = 8 |O_p| written."""
    rp, ci = A.row_ptr, A.col
    rownnz = np.diff(rp)
    out = []
    for p in range(ctx.num_parts):
        om, ow, ifc = ras.ras_get_maps(ctx, p)
        n_p, e_p, o_p = om.size, ifc.size, int(ow.sum())
        nnz_rows = int(rownnz[om].sum())
        inside = np.zeros(A.n, bool)
        inside[om] = True
        # nnz(A_p): entries of Omega_p's rows whose column lies in Omega_p
        starts, ends = rp[om], rp[om + 1]
        idx = np.concatenate([np.arange(s, e) for s, e in zip(starts, ends)])
        nnz_p = int(inside[ci[idx]].sum())
        if grid:
            res = nnz_rows * 8 + 8 * (n_p + e_p) + 8 * n_p
        else:
            res = nnz_rows * 12 + 4 * (n_p + 1) + 8 * (n_p + e_p) + 8 * n_p
        if kind == ras.RAS_LOCAL_CG:
            loc = nnz_p * (prec_bytes + col_bytes) * (1 if staged else m)
        elif kind == ras.RAS_LOCAL_ILU0_CG:
            # A_p and the ILU(0) factors (same pattern) read every PCG step
            loc = 2 * nnz_p * (prec_bytes + 2) * m
        elif kind in (ras.RAS_LOCAL_BANDCHOL, ras.RAS_LOCAL_BANDLU):
            # local half-bandwidth of A_p in ascending global order
            loc_col = np.searchsorted(om, ci[idx])
            loc_row = np.repeat(np.arange(n_p), ends - starts)
            w_p = int(np.max(np.where(inside[ci[idx]], loc_row - loc_col, 0)))
            loc = 2 * n_p * (w_p + 1) * prec_bytes
        else:
            loc = 0
        out.append(res + loc + 8 * o_p)
    return np.array(out, dtype=np.float64)


def profile_traffic(variant: str):
    """DRAM bytes per local update of the persistent kernel from a committed
    ncu summary (profiles/*.txt) taken on the current kernel source and the
    same variant; None when there is none."""
    import glob

    src_hash = hashlib.sha256(open(KERNEL_SRC, "rb").read()).hexdigest()[:16]
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", "*.txt"))):
        kv = {}
        for ln in open(path):
            if ":" in ln and not ln.startswith((" ", "#")):
                k, v = ln.split(":", 1)
                kv[k.strip()] = v.strip()
        if kv.get("kernel_src_sha256_16") == src_hash and kv.get("variant") == variant:
            try:
                return float(kv["dram_bytes_per_update"])
            except (KeyError, ValueError):
                return None
    return None


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


# ---------------------------------------------------------------- GPU arm

def run_ours(args):
    import torch

    import paper_2003_05361_gb300 as ras

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)

    A, b = problem()
    part = ras.ras_partition_regular2d(N_GRID, N_GRID, PX, PX)
    bd = torch.tensor(b, device=dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MB > L2

    variants = {
        "async_fp32": (ras.RAS_ASYNC, ras.RAS_FP32),
        "sync_fp64": (ras.RAS_SYNC, ras.RAS_FP64),
        "async_fp64": (ras.RAS_ASYNC, ras.RAS_FP64),
        "sync_fp32": (ras.RAS_SYNC, ras.RAS_FP32),
    }
    ctxs = {p: ras.ras_setup(A, part, PX * PX, GAMMA, ras.RAS_LOCAL_CG, p, M_INNER, stream=stream)
            for p in (ras.RAS_FP32, ras.RAS_FP64)}

    def barrier():
        if world > 1:
            import torch.distributed as dist

            dist.barrier()

    def solve(mode, prec):
        x = torch.zeros(A.n, dtype=torch.float64, device=dev)
        flush.fill_(1.0)  # L2 flush outside the timed region
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        try:
            info = ras.ras_solve(ctxs[prec], bd, x, TOL, mode)
        except ras.RasError as err:
            if err.info is None:
                raise
            info = err.info  # a solve that stopped without converging
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1), info, x

    head_mode, head_prec = variants["async_fp32"]
    for _ in range(args.warmup):
        solve(head_mode, head_prec)
    barrier()
    torch.cuda.synchronize()
    times, infos, failed = [], [], []
    with ClockSampler(local) as clocks:
        for _ in range(args.steps):
            t, info, x = solve(head_mode, head_prec)
            if info.status == 0:
                times.append(t)
                infos.append(info)
            else:
                failed.append({"ms": t, "status": info.status, "relres": info.relres,
                               "updates_median": info.updates_median})
    barrier()
    # every rank joins the reduction; a rank with no converged solve reports
    # +inf, so all ranks see the failure together
    med = max_over_ranks(statistics.median(times) if times else float("inf"), dev)
    if not times or med == float("inf"):
        raise RuntimeError(f"no timed solve converged on some rank: {failed}")

    # relative residual of the last result (FP64 on the device)
    relres = ras.ras_relres(ctxs[head_prec], bd, x)

    # other variants, one solve each
    var_out, var_x = {}, {"async_fp32": x.cpu().numpy()}
    if not args.quick:
        for name, (mode, prec) in variants.items():
            if name == "async_fp32":
                continue
            t, info, xv = solve(mode, prec)
            var_x[name] = xv.cpu().numpy()
            var_out[name] = {"ms": t, "status": info.status, "iterations": info.iterations,
                             "updates_median": info.updates_median, "relres": info.relres,
                             "kernel_ms": info.kernel_ms}

    # end to end through the host-buffer entry point (pinned host memory)
    e2e = None
    if not args.quick:
        bh = torch.tensor(b).pin_memory()
        e2e_t, e2e_failed = [], 0
        for _ in range(min(args.steps, 5)):
            xh = torch.zeros(A.n, dtype=torch.float64).pin_memory()
            flush.fill_(1.0)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            info_h = ras.ras_solve_host(ctxs[head_prec], bh, xh, TOL, head_mode)
            dt = (time.perf_counter() - t0) * 1e3
            if info_h.status == 0:
                e2e_t.append(dt)
            else:
                e2e_failed += 1
        e2e_v = max_over_ranks(statistics.median(e2e_t) if e2e_t else float("inf"), dev)
        e2e = {"value": e2e_v if e2e_v != float("inf") else None, "unit": "ms",
               "h2d_bytes_per_step": 2 * 8 * A.n, "d2h_bytes_per_step": 8 * A.n,
               "failed_steps": e2e_failed, "steps": len(e2e_t) + e2e_failed}

    # roofline of the persistent kernel
    info = infos[len(infos) // 2]
    counts = ras.ras_get_update_counts(ctxs[head_prec])
    launch = ras.ras_get_launch(ctxs[head_prec])
    staged = launch["kernel_variant"] in (3, 5)
    dia = launch["kernel_variant"] == 5  # diagonal-offset form: no column bytes
    # diagonal-offset form: grid layout, no column or index bytes
    per_upd = subdomain_bytes(A, ras, ctxs[head_prec], ras.RAS_LOCAL_CG, 4, M_INNER, staged,
                              col_bytes=0 if dia else 2, grid=dia)
    alg_bytes = float(np.dot(counts, per_upd))
    kernel_s = info.kernel_ms / 1e3
    achieved = alg_bytes / kernel_s / 1e9
    peak, peak_src = measured_peaks()
    tpu = profile_traffic("async_fp32")
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "traffic": (tpu * float(counts.sum())) if tpu else None,
            "kernel": ("ras_main_kernel<CG staged in shared memory%s, float, %d>"
                       % (" (diagonal-offset form)" if dia else "", launch["cta_threads"])
                       if staged else "ras_main_kernel<CG, float, %d>" % launch["cta_threads"]),
            "kernel_ms": info.kernel_ms,
            "algorithmic_bytes": alg_bytes, "peak_source": peak_src}

    sections = {}
    if not args.quick and world == 1:
        # every section is reported, never fatal to the headline line
        for name, fn in (("band_config4", lambda: band_config4(dev, stream, args.band_iters)),
                         ("config3", lambda: config3_section(dev, stream)),
                         ("config4", lambda: config4_section(dev, stream, args.config4_full)),
                         ("serving", lambda: serving_section(args)),
                         ("nonsymmetric", lambda: nonsymmetric(dev, stream)),
                         ("oras", lambda: oras_section(dev, stream))):
            if name not in args.sections:
                continue
            try:
                sections[name] = fn()
            except Exception as e:
                sections[name] = {"error": f"{type(e).__name__}: {e}"}

    launches_per_solve = 5  # init, sysnorm, main, residual, sysnorm (async)
    line = {
        "metric": METRIC, "value": med, "unit": "ms", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": med, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64+f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "mode": "async", "local_solver": "CG-20",
                   "local_precision": "fp32", "outer_precision": "fp64", "tol": TOL,
                   "l2": "flushed before every step (256 MB write); working set 0.2 GB > L2",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "iterations_median_updates": info.updates_median,
        "updates": {"min": info.updates_min, "median": info.updates_median,
                    "max": info.updates_max, "stale": info.stale_updates},
        "restarts": info.restarts, "relres": relres,
        "step_ms_all": times, "failed_steps": failed, "variants": var_out, "e2e": e2e,
        "gpu_launches": launches_per_solve * args.steps,
        "roofline": roof, "clocks": clocks.summary(),
    }
    line.update(sections)
    if "serving" in sections and "async_fp32" in sections["serving"]:
        sv = sections["serving"]
        line["serving_p50_p99"] = {"valid": sv.get("valid"), **{
            k: {"p50_ms": sv[k].get("p50_ms"), "p99_ms": sv[k].get("p99_ms"),
                "solves_per_s": sv[k].get("solves_per_s"), "rejected": sv[k].get("rejected"),
                "failed": sv[k].get("failed")}
            for k in ("async_fp32", "sync_fp64") if k in sv}}
    if rank == 0 and world == 1 and not args.no_cpu:
        import oracle

        line["cpu_baseline"] = oracle_baseline(
            A, b, oracle.partition_regular2d(N_GRID, N_GRID, PX, PX),
            float(os.environ.get("RAS_CPU_SAMPLE_S", "12")))
        line["error_vs_oracle"] = oracle_errors(var_x, lambda: oracle.poisson2d_direct(N_GRID, b))
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist

        dist.barrier()
        dist.destroy_process_group()


def oracle_errors(xs: dict, direct) -> dict:
    """Error of every reported result against the oracle's FP64 direct
    solution x* = A^{-1} b (the RAS fixed point), computed on the host after
    the timed region: relative 2-norm ||x - x*|| / ||x*|| and element-wise
    max |x - x*| / max |x*|."""
    xs_ = direct()
    nrm, mx = float(np.linalg.norm(xs_)), float(np.abs(xs_).max())
    out = {"reference": "oracle FP64 direct solve of the global system"}
    for k, xv in xs.items():
        out[k] = {"rel_2norm": float(np.linalg.norm(xv - xs_)) / nrm,
                  "rel_max": float(np.abs(xv - xs_).max()) / mx}
    return out


def _timed_solve(ras, ctx, bd, n, dev, tol, mode, flush, max_updates=0):
    """One solve from x = 0 after an L2 flush; a solve that stops with an
    error returns its info (status, error site) instead of raising."""
    import torch

    x = torch.zeros(n, dtype=torch.float64, device=dev)
    flush.fill_(1.0)  # L2 flush outside the timed region
    torch.cuda.synchronize()
    try:
        info = ras.ras_solve(ctx, bd, x, tol, mode, max_updates)
    except ras.RasError as err:
        if err.info is None:
            raise
        info = err.info
    return info, x


def _info_row(info):
    return {"ms": info.solve_ms, "kernel_ms": info.kernel_ms, "status": info.status,
            "error_site": info.error_site, "grid": info.grid,
            "iterations": info.iterations,
            "updates": [info.updates_min, info.updates_median, info.updates_max],
            "restarts": info.restarts, "relres": info.relres}


def config3_section(dev, stream):
    """Config 3: 3D Poisson 7-point 128^3 (2,097,152 unknowns), b uniform seed
    3, seeded BFS-growth partition into 512 uneven parts (seed 3), overlap 1,
    local ILU(0)-PCG in FP32 with FP64 outer residual / update; the launch
    shape and inner step count picked by ras_autotune, then time to 1e-8
    synchronous and asynchronous (one solve each, L2 flushed). Roofline: the
    local solve's model of 2 nnz(A_p) (s + 2) bytes per PCG step (A_p and
    the ILU(0) factors: 84 m bytes per row at 7 nnz per row and s = 4) plus the
    residual rows and owned writes. Errors against the oracle's closed-form
    FP64 solve."""
    import torch

    import paper_2003_05361_gb300 as ras

    N, P = 128, 512
    A = problems.poisson3d(N)
    b = problems.rhs_uniform(A.n, 3)
    t0 = time.perf_counter()
    part = ras.ras_partition_bfs(A, P, 3)
    ctx = ras.ras_setup(A, part, P, 1, ras.RAS_LOCAL_ILU0_CG, ras.RAS_FP32, 10, stream=stream)
    setup_ms = (time.perf_counter() - t0) * 1e3
    bd = torch.tensor(b, device=dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    xs = torch.zeros(A.n, dtype=torch.float64, device=dev)
    t0 = time.perf_counter()
    tune = ras.ras_autotune(ctx, xs, ras.RAS_ASYNC, 20, True)
    tune_ms = (time.perf_counter() - t0) * 1e3
    launch = ras.ras_get_launch(ctx)
    out = {"workload": "3D Poisson 7-point 128^3 (2,097,152 unknowns), uniform RHS seed 3, "
                       "BFS-growth 512 parts (seed 3), overlap 1, ILU(0)-PCG FP32 local solves, "
                       "FP64 outer, tol 1e-8, autotuned launch",
           "setup_ms": setup_ms, "autotune_ms": tune_ms,
           "autotune": {"cta_threads": tune.cta_threads, "inner_iters": tune.inner_iters,
                        "candidates": tune.candidates, "schedule": tune.schedule,
                        "grid": tune.grid, "per_cta": tune.per_cta}, "launch": launch}
    peak, peak_src = measured_peaks()
    xsol = {}
    for mname, mode in (("sync", ras.RAS_SYNC), ("async", ras.RAS_ASYNC)):
        info, x = _timed_solve(ras, ctx, bd, A.n, dev, TOL, mode, flush)
        out[mname] = _info_row(info)
        xsol[mname] = x.cpu().numpy()
        counts = ras.ras_get_update_counts(ctx)
        per_upd = subdomain_bytes(A, ras, ctx, ras.RAS_LOCAL_ILU0_CG, 4, launch["inner_iters"],
                                  False)
        alg = float(np.dot(counts, per_upd))
        ach = alg / (info.kernel_ms / 1e3) / 1e9
        out[mname]["roofline"] = {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s",
                                  "frac": ach / peak, "peak_source": peak_src,
                                  "algorithmic_bytes": alg, "traffic": None}
    ras.ras_destroy(ctx)
    import oracle

    out["error_vs_oracle"] = oracle_errors(xsol, lambda: oracle.poisson3d_direct(N, b))
    return out


def config4_section(dev, stream, full: bool = False, cap: int = 200):
    """Config 4: 2D diffusion 2048^2 (4,194,304 unknowns), k = exp(GRF sigma 1,
    ell 1/32, seed 4), b uniform seed 4, regular 32x32 = 1024 subdomains,
    overlap 4, banded Cholesky factorised in FP64 and stored in FP32, BF16 or
    FP64. Time to 1e-8 (one solve each, L2 flushed) for FP32 factors,
    synchronous and asynchronous; BF16 and FP64 factors, which take the same
    number of synchronous iterations (the outer iteration is FP64), are timed
    over `cap` synchronous iterations and their time to 1e-8 estimated as
    time per iteration x the FP32 count (full=True solves them to 1e-8 too).
    A direct solve of the full system is out of the oracle's reach (a 69 GB
    band), so the full-size results are compared with each other and their
    FP64 residuals reported; the error against the oracle's FP64 direct solve
    is taken on the same recipe at 256^2 with the same 64 x 64 subdomains and
    overlap (4 x 4 parts), where the oracle's banded Cholesky of the whole
    system is feasible, for every storage precision."""
    import torch

    import paper_2003_05361_gb300 as ras

    out = {"workload": "2D diffusion 2048x2048 (4,194,304 unknowns), k = exp(GRF sigma 1, ell 1/32, "
                       "seed 4), uniform RHS seed 4, regular2d 32x32 = 1024 subdomains, overlap 4, "
                       "banded Cholesky (factors FP64 / FP32 / BF16), tol 1e-8"}
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    peak, peak_src = measured_peaks()
    precs = (("fp32", ras.RAS_FP32, 4), ("bf16", ras.RAS_BF16_STORE, 2), ("fp64", ras.RAS_FP64, 8))
    for n, px in ((2048, 32), (256, 4)):
        A = problems.diffusion2d(n, problems.grf_coefficient(n, 4))
        b = problems.rhs_uniform(A.n, 4)
        part = ras.ras_partition_regular2d(n, n, px, px)
        bd = torch.tensor(b, device=dev)
        xsol, rows = {}, {}
        for name, prec, sb in precs:
            ctx = ras.ras_setup(A, part, px * px, 4, ras.RAS_LOCAL_BANDCHOL, prec, stream=stream)
            modes = (("sync", ras.RAS_SYNC), ("async", ras.RAS_ASYNC)) if name == "fp32" else \
                (("sync", ras.RAS_SYNC),)
            for mname, mode in modes:
                capped = n == 2048 and name != "fp32" and not full
                info, x = _timed_solve(ras, ctx, bd, A.n, dev, TOL, mode, flush,
                                       cap if capped else 0)
                row = _info_row(info)
                if n == 2048:
                    counts = ras.ras_get_update_counts(ctx)
                    per_upd = subdomain_bytes(A, ras, ctx, ras.RAS_LOCAL_BANDCHOL, sb, 1, True)
                    alg = float(np.dot(counts, per_upd))
                    ach = alg / (info.kernel_ms / 1e3) / 1e9
                    row["roofline"] = {"bound": "hbm", "achieved": ach, "peak": peak,
                                       "unit": "GB/s", "frac": ach / peak,
                                       "peak_source": peak_src, "algorithmic_bytes": alg,
                                       "kernel": f"ras_main_kernel<band, {name}, "
                                                 f"{ras.ras_get_launch(ctx)['cta_threads']}>"}
                    row["ms_per_iteration"] = info.kernel_ms / max(info.updates_median, 1)
                    if capped:
                        row["capped_at"] = cap
                        it32 = rows["sync_fp32"]["iterations"]
                        row["estimated_ms_to_tol"] = row["ms_per_iteration"] * it32
                if not (n == 2048 and capped):
                    xsol[f"{mname}_{name}"] = x.cpu().numpy()
                rows[f"{mname}_{name}"] = row
            ras.ras_destroy(ctx)
        if n == 2048:
            out.update(rows)
            ref = xsol.get("sync_fp64", xsol["sync_fp32"])
            nr = float(np.linalg.norm(ref))
            out["difference_between_results"] = {
                "reference": "sync_fp64" if "sync_fp64" in xsol else "sync_fp32",
                **{k: float(np.linalg.norm(v - ref)) / nr for k, v in xsol.items()}}
        else:
            import oracle

            out["error_vs_oracle_256"] = oracle_errors(
                xsol, lambda: oracle.band_direct_solve(A, b))
            out["error_vs_oracle_256"]["iterations"] = {k: r["iterations"] for k, r in rows.items()}
    return out


def serving_section(args):
    """Config 5 in a bounded form: the seeded Poisson-arrival stream of 2D
    Poisson solves (side uniform in 64..512, 64 x 64 subdomains, overlap 2,
    banded Cholesky), served by continuous batching. First the saturation
    throughput of plain sync FP64 (every request present at t = 0); then
    async mixed precision (FP32 factors) and sync FP64 each on an open-loop
    stream at 0.8 x that throughput (the 0.8 point of the rates 0.5 / 0.8 /
    0.95 x saturation). p50 / p99 latency = completion - arrival."""
    import paper_2003_05361_gb300 as ras
    from paper_2003_05361_gb300.serve import Server, request_stream

    nsat, nreq = args.serve_sat_requests, args.serve_requests_bench
    sat_srv = Server(mode=ras.RAS_SYNC, prec=ras.RAS_FP64, step_limit=args.serve_step,
                     workers=args.serve_workers)
    sat = sat_srv.run(request_stream(nsat, rate=1e6, seed=7))
    rate = 0.8 * sat["solves_per_s"]
    out = {"workload": f"{nreq} seeded Poisson-arrival 2D Poisson solves per arm, side U{{64..512}}, "
                       f"64x64 subdomains, overlap 2, banded Cholesky, tol 1e-8, rate 0.8 x the "
                       f"sync-FP64 saturation throughput",
           "saturation_sync_fp64": {"requests": nsat, "solves_per_s": sat["solves_per_s"],
                                    "rejected": sat.get("rejected"), "failed": sat.get("failed")},
           "rate_per_s": rate}
    for name, mode, prec in (("async_fp32", ras.RAS_ASYNC, ras.RAS_FP32),
                             ("sync_fp64", ras.RAS_SYNC, ras.RAS_FP64)):
        srv = Server(mode=mode, prec=prec, step_limit=args.serve_step, workers=args.serve_workers)
        out[name] = srv.run(request_stream(nreq, rate=rate, seed=5))
    # rejected requests are not in the latencies; the stock stream has none
    out["valid"] = all(out[k].get("rejected", 0) == 0 for k in ("async_fp32", "sync_fp64"))
    return out


def band_config4(dev, stream, iters: int):
    """Kernel-level roofline of the banded-Cholesky path on the config-4
    workload: 2D variable-coefficient diffusion 2048^2 (k = exp(GRF), sigma 1,
    correlation length 1/32, seed 4), b uniform seed 4, regular 32x32 = 1024
    subdomains, overlap 4; `iters` synchronous iterations (capped solve) with
    factors stored in FP32 and in BF16, each timed with CUDA events inside the
    library. Algorithmic bytes per update: residual rows + band model
    2 n_p (w_p + 1) s_f + owned-row writes."""
    import torch

    import paper_2003_05361_gb300 as ras

    n = 2048
    A = problems.diffusion2d(n, problems.grf_coefficient(n, 4))
    b = problems.rhs_uniform(A.n, 4)
    part = ras.ras_partition_regular2d(n, n, 32, 32)
    bd = torch.tensor(b, device=dev)
    peak, peak_src = measured_peaks()
    out = {"workload": "2D diffusion 2048x2048 (4,194,304 unknowns), k = exp(GRF sigma 1, "
                       "ell 1/32, seed 4), regular2d 32x32 = 1024 subdomains, overlap 4, "
                       f"banded Cholesky, sync, {iters} iterations per timed launch"}
    for name, prec, sb in (("fp32", ras.RAS_FP32, 4), ("bf16", ras.RAS_BF16_STORE, 2)):
        ctx = ras.ras_setup(A, part, 1024, 4, ras.RAS_LOCAL_BANDCHOL, prec, stream=stream)
        per_upd = subdomain_bytes(A, ras, ctx, ras.RAS_LOCAL_BANDCHOL, sb, 1, True)
        ms = []
        for _ in range(3):
            x = torch.zeros(A.n, dtype=torch.float64, device=dev)
            info = ras.ras_solve(ctx, bd, x, 1e-8, ras.RAS_SYNC, iters)
            ms.append(info.kernel_ms)
        counts = ras.ras_get_update_counts(ctx)
        alg = float(np.dot(counts, per_upd))
        k_ms = statistics.median(ms)
        achieved = alg / (k_ms / 1e3) / 1e9
        launch = ras.ras_get_launch(ctx)
        tpu = profile_traffic(f"sync_band_{name}_cfg4")
        out[name] = {"ms_per_iteration": k_ms / iters, "kernel_ms": k_ms,
                     "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                                  "frac": achieved / peak, "peak_source": peak_src,
                                  "traffic": (tpu * float(counts.sum())) if tpu else None,
                                  "algorithmic_bytes": alg,
                                  "kernel": f"ras_main_kernel<band, {name}, {launch['cta_threads']}>",
                                  "grid": launch["grid"]}}
        ras.ras_destroy(ctx)
    return out


def nonsymmetric(dev, stream, reps: int = 3):
    """Generic (nonsymmetric) systems, Sec. 4.1's LU / GMRES local solvers:
    upwind convection-diffusion 1024^2 (bx = 0.5, by = 0.25: velocity
    (512.5, 256.25) on the unit square, cell Peclet numbers 0.5 / 0.25), b
    uniform seed 2, regular 16x16 = 256 subdomains, overlap 4, tol 1e-8. Time
    to solution, sync vs async, with banded-LU local solves (factors in FP32,
    BF16, FP64) and with 20 GMRES steps in FP32: the median of `reps` solves
    after one untimed solve, L2 flushed (256 MB write) before each. Roofline of
    the banded-LU FP32 synchronous kernel: algorithmic bytes (residual rows +
    band model 2 n_p (w_p + 1) s_f + owned-row writes) per kernel time."""
    import torch

    import paper_2003_05361_gb300 as ras

    n = 1024
    A = problems.convdiff2d(n, 0.5, 0.25)
    b = problems.rhs_uniform(A.n, 2)
    part = ras.ras_partition_regular2d(n, n, 16, 16)
    bd = torch.tensor(b, device=dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    peak, peak_src = measured_peaks()
    out = {"workload": "2D upwind convection-diffusion 1024x1024 (1,048,576 unknowns, "
                       "nonsymmetric M-matrix), bx 0.5, by 0.25, uniform RHS seed 2, regular2d "
                       "16x16 = 256 subdomains, overlap 4, tol 1e-8, median of %d solves, L2 "
                       "flushed before each" % reps}
    cases = (("bandlu_fp32", ras.RAS_LOCAL_BANDLU, ras.RAS_FP32, 1, 4),
             ("bandlu_bf16", ras.RAS_LOCAL_BANDLU, ras.RAS_BF16_STORE, 1, 2),
             ("bandlu_fp64", ras.RAS_LOCAL_BANDLU, ras.RAS_FP64, 1, 8),
             ("gmres20_fp32", ras.RAS_LOCAL_GMRES, ras.RAS_FP32, 20, 4))
    for name, kind, prec, m, sb in cases:
        ctx = ras.ras_setup(A, part, 256, 4, kind, prec, m, stream=stream)
        row = {}
        for mname, mode in (("sync", ras.RAS_SYNC), ("async", ras.RAS_ASYNC)):
            runs = []
            for rep in range(reps + 1):
                x = torch.zeros(A.n, dtype=torch.float64, device=dev)
                flush.fill_(1.0)
                torch.cuda.synchronize()
                info = ras.ras_solve(ctx, bd, x, TOL, mode)
                if rep > 0:
                    runs.append(info)
            runs.sort(key=lambda i: i.solve_ms)
            med = runs[len(runs) // 2]
            row[mname] = {"ms": med.solve_ms, "kernel_ms": med.kernel_ms,
                          "ms_all": [r.solve_ms for r in runs], "status": med.status,
                          "failed": sum(1 for r in runs if r.status != 0),
                          "iterations": med.iterations, "relres": med.relres,
                          "updates": [med.updates_min, med.updates_median, med.updates_max]}
            if name == "bandlu_fp32" and mode == ras.RAS_SYNC:
                counts = ras.ras_get_update_counts(ctx)
                per_upd = subdomain_bytes(A, ras, ctx, ras.RAS_LOCAL_BANDLU, sb, 1, True)
                alg = float(np.dot(counts, per_upd))
                achieved = alg / (med.kernel_ms / 1e3) / 1e9
                launch = ras.ras_get_launch(ctx)
                row["roofline"] = {"bound": "hbm", "achieved": achieved, "peak": peak,
                                   "unit": "GB/s", "frac": achieved / peak,
                                   "peak_source": peak_src, "traffic": None,
                                   "algorithmic_bytes": alg,
                                   "kernel": f"ras_main_kernel<band (LU records), float, "
                                             f"{launch['cta_threads']}>",
                                   "grid": launch["grid"]}
        out[name] = row
        ras.ras_destroy(ctx)
    return out


def oras_section(dev, stream, max_updates: int = 12000):
    """Optimized RAS (the paper's future work, Sec. 6) on the benchmark problem
    (2D Poisson 1024^2, b seed 1, regular 16x16 = 256 subdomains, overlap 4)
    with banded-Cholesky local solves in FP32: time to 1e-8 for interface
    parameters alpha = 0 (RAS), 0.5, 0.8, 0.9, sync and async, one timed solve
    after an untimed one, L2 flushed before each; every solve capped at
    `max_updates` updates per subdomain (a diverging alpha ends RAS_ENOCONV)."""
    import torch

    import paper_2003_05361_gb300 as ras

    A, b = problem()
    part = ras.ras_partition_regular2d(N_GRID, N_GRID, PX, PX)
    bd = torch.tensor(b, device=dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    out = {"workload": "2D Poisson 5-point 1024x1024 (1,048,576 unknowns), uniform RHS seed 1, "
                       "regular2d 16x16 = 256 subdomains, overlap 4, banded Cholesky FP32 local "
                       "solves on optimized local matrices A_p + alpha diag(exterior couplings), "
                       "tol 1e-8, one timed solve per point, L2 flushed before each",
           "points": []}
    for alpha in (0.0, 0.5, 0.8, 0.9):
        ctx = ras.ras_setup(A, part, PX * PX, GAMMA, ras.RAS_LOCAL_BANDCHOL, ras.RAS_FP32,
                            stream=stream, oras_alpha=alpha)
        for mname, mode in (("sync", ras.RAS_SYNC), ("async", ras.RAS_ASYNC)):
            for rep in range(2):
                x = torch.zeros(A.n, dtype=torch.float64, device=dev)
                flush.fill_(1.0)
                torch.cuda.synchronize()
                info = ras.ras_solve(ctx, bd, x, TOL, mode, max_updates)
            out["points"].append({"alpha": alpha, "mode": mname, "ms": info.solve_ms,
                                  "status": info.status, "iterations": info.iterations,
                                  "relres": info.relres})
        ras.ras_destroy(ctx)
    return out


def run_sweep(args):
    """One-GPU analogues of the paper's partitioning and overlap experiments
    (Sec. 4.2, regular1d vs regular2d vs a graph partitioner; Sec. 4.3,
    overlap) on the benchmark's 2D Poisson problem (1024^2, b seed 1) in 256
    subdomains: regular2d 16x16, regular1d (256 strips of 4 rows) and seeded
    BFS growth (seed 1). Local solvers: banded Cholesky in FP32 (the paper's
    direct local solver) at overlap 1 / 2 / 4 / 8 / 16 and CG-20 in FP32 at
    overlap 1 / 2 / 4 / 8; synchronous vs asynchronous, and for overlap 4 with
    the banded solver also the decentralized detection scheme (Sec. 3.3.2).
    A combination outside a local solver's limits (local half-bandwidth > 160
    for the banded solver; a local problem that does not fit in shared
    memory for CG) is reported as an error row. One solve per synchronous
    point; asynchronous points are the median (by time) of --sweep-reps
    solves (10, as Sec. 4.1 averages its runs) with the minimum and maximum."""
    import torch

    import paper_2003_05361_gb300 as ras

    torch.cuda.set_device(0)
    A, b = problem()
    bd = torch.tensor(b, device="cuda")
    parts = {"regular2d": ras.ras_partition_regular2d(N_GRID, N_GRID, PX, PX),
             "regular1d": ras.ras_partition_regular2d(N_GRID, N_GRID, 1, PX * PX),
             "bfs": ras.ras_partition_bfs(A, PX * PX, 1)}
    solvers = {"band_fp32": (ras.RAS_LOCAL_BANDCHOL, 1, (1, 2, 4, 8, 16)),
               "cg20_fp32": (ras.RAS_LOCAL_CG, M_INNER, (1, 2, 4, 8))}
    # --sweep-only partition:local (e.g. regular2d:cg20_fp32) runs a subset
    if args.sweep_only:
        keep = [tuple(t.split(":")) for t in args.sweep_only.split(",")]
        parts = {k: v for k, v in parts.items() if any(k == pk for pk, _ in keep)}
        solvers = {k: v for k, v in solvers.items() if any(k == sk for _, sk in keep)}
    rows = []

    def run(ctx, mode, reps):
        out = []
        for _ in range(reps):
            x = torch.zeros(A.n, dtype=torch.float64, device="cuda")
            try:
                out.append(ras.ras_solve(ctx, bd, x, TOL, mode))
            except ras.RasError as err:
                if err.info is None:
                    raise
                out.append(err.info)
        out.sort(key=lambda i: i.kernel_ms)
        return out[len(out) // 2], [i.kernel_ms for i in out], sum(i.status != 0 for i in out)

    for pname, part in parts.items():
        for sname, (kind, m, gammas) in solvers.items():
            for gamma in gammas:
                try:
                    ctx = ras.ras_setup(A, part, PX * PX, gamma, kind, ras.RAS_FP32, m)
                except ras.RasError as err:
                    row = {"partition": pname, "local": sname, "overlap": gamma, "error": str(err)}
                    rows.append(row)
                    print(json.dumps(row), flush=True)
                    continue
                modes = [("sync", ras.RAS_SYNC, 1), ("async", ras.RAS_ASYNC, args.sweep_reps)]
                if gamma == 4 and kind == ras.RAS_LOCAL_BANDCHOL:
                    modes.append(("async_decentral", ras.RAS_ASYNC_DECENTRAL, args.sweep_reps))
                for mname, mode, reps in modes:
                    info, all_ms, nfail = run(ctx, mode, reps)
                    ph = ras.ras_get_phase_times(ctx).astype(np.float64)
                    upd = np.maximum(ras.ras_get_update_counts(ctx), 1).astype(np.float64)
                    per = (ph / upd[:, None]).mean(0) / 1e3
                    row = {"partition": pname, "local": sname, "overlap": gamma, "mode": mname,
                           "status": info.status, "ms": info.kernel_ms,
                           "ms_min": min(all_ms), "ms_max": max(all_ms), "runs": reps,
                           "failed_runs": nfail,
                           "iterations": info.iterations, "updates_min": info.updates_min,
                           "updates_max": info.updates_max, "restarts": info.restarts,
                           "relres": info.relres, "grid": info.grid,
                           "us_per_update": {"gather": per[0], "solve": per[1], "update": per[2]},
                           "max_local_bandwidth": int(ras.ras_get_info(ctx)["max_bandwidth"])}
                    if mode != ras.RAS_SYNC:
                        # spread of the per-subdomain update counts (Figs. 6c / 7c)
                        cnt = ras.ras_get_update_counts(ctx)
                        hist, edges = np.histogram(cnt, bins=8)
                        row["update_histogram"] = {"counts": hist.tolist(),
                                                   "edges": [float(e) for e in edges]}
                        row["stale_updates"] = info.stale_updates
                    rows.append(row)
                    print(json.dumps(row), flush=True)
                ras.ras_destroy(ctx)
    print(json.dumps({"sweep": "partition x local solver x overlap x mode (2D Poisson 1024^2, "
                               "256 subdomains, FP32 local solves)", "rows": rows}), flush=True)


def run_profile_case(args):
    """Small cases for ncu, each launch capped at `--profile-updates` local
    updates per subdomain (a few ms):
      cg_cfg2   the benchmark workload, async, FP32 local CG-20 (default);
      band_cfg1 2D Poisson 128^2, 2x2, overlap 2, banded Cholesky FP32, sync;
      band_cfg4s the config-4 subdomain shape on a quarter of the grid: 2D
                diffusion 1024^2 (k = exp(GRF), seed 4), 16x16 = 256 subdomains
                of 64x64, overlap 4, banded Cholesky FP32, sync (1.1 GB of
                factor records, well over L2); its DRAM bytes per update stand
                for the full config-4 launch;
      gmres_nonsym 2D upwind convection-diffusion 1024^2 (bx 0.5, by 0.25),
                16x16 = 256 subdomains, overlap 4, 20 GMRES steps in FP32, sync."""
    import torch

    import paper_2003_05361_gb300 as ras

    if args.case == "band_cfg4s":
        A = problems.diffusion2d(1024, problems.grf_coefficient(1024, 4))
        b = problems.rhs_uniform(A.n, 4)
        part = ras.ras_partition_regular2d(1024, 1024, 16, 16)
        ctx = ras.ras_setup(A, part, 256, 4, ras.RAS_LOCAL_BANDCHOL, ras.RAS_FP32)
        mode, variant = ras.RAS_SYNC, "sync_band_fp32_cfg4"
    elif args.case == "gmres_nonsym":
        A = problems.convdiff2d(1024, 0.5, 0.25)
        b = problems.rhs_uniform(A.n, 2)
        part = ras.ras_partition_regular2d(1024, 1024, 16, 16)
        ctx = ras.ras_setup(A, part, 256, 4, ras.RAS_LOCAL_GMRES, ras.RAS_FP32, 20)
        mode, variant = ras.RAS_SYNC, "sync_gmres20_fp32_nonsym"
    elif args.case == "band_cfg1":
        A = problems.poisson2d(128)
        b, _, _ = problems.rhs_eigen2d(128)
        part = ras.ras_partition_regular2d(128, 128, 2, 2)
        ctx = ras.ras_setup(A, part, 4, 2, ras.RAS_LOCAL_BANDCHOL, ras.RAS_FP32)
        mode, variant = ras.RAS_SYNC, "sync_band_fp32_cfg1"
    else:
        A, b = problem()
        part = ras.ras_partition_regular2d(N_GRID, N_GRID, PX, PX)
        ctx = ras.ras_setup(A, part, PX * PX, GAMMA, ras.RAS_LOCAL_CG, ras.RAS_FP32, M_INNER)
        mode, variant = ras.RAS_ASYNC, "async_fp32"
    bd = torch.tensor(b, device="cuda")
    tot = 0
    for _ in range(2):
        x = torch.zeros(A.n, dtype=torch.float64, device="cuda")
        info = ras.ras_solve(ctx, bd, x, TOL, mode, args.profile_updates)
        tot = int(ras.ras_get_update_counts(ctx).sum())
    torch.cuda.synchronize()
    print(json.dumps({"profile_case": variant, "updates_per_launch": tot,
                      "kernel_ms": info.kernel_ms, "status": info.status}))


def run_serving(args):
    """Serving workload: a seeded Poisson stream of 2D Poisson solves with sides
    uniform in 64..512 (64 x 64 subdomains, overlap 2, banded Cholesky),
    served by continuous batching; async mixed precision (FP32 factors) vs
    sync FP64. Reports p50 / p99 latency (completion - arrival) and solves/s.
    The stream length and rate are bounded so the run takes about a minute."""
    import torch

    import paper_2003_05361_gb300 as ras
    from paper_2003_05361_gb300.serve import Server, request_stream

    torch.cuda.set_device(0)
    out = {}
    for name, mode, prec in (("async_fp32", ras.RAS_ASYNC, ras.RAS_FP32),
                             ("sync_fp64", ras.RAS_SYNC, ras.RAS_FP64)):
        reqs = request_stream(args.serve_requests, rate=args.serve_rate, seed=5)
        srv = Server(mode=mode, prec=prec, step_limit=args.serve_step, workers=args.serve_workers)
        stats = srv.run(reqs)
        out[name] = stats
        print(json.dumps({"serving": name, **stats}), flush=True)
    # a request rejected on arrival is not served, so it is left out of the
    # latencies: report the count beside p99 and flag the line when the
    # stock stream (sides 64..512 always fit the slots) had any
    rejected = {k: v.get("rejected", 0) for k, v in out.items()}
    line = {"metric": "serving p50/p99 latency and solves/s (continuous batching)",
            "unit": "ms", "value": out["async_fp32"].get("p99_ms"), "higher_is_better": False,
            "rejected": rejected, "valid": all(r == 0 for r in rejected.values()),
            "config": {"workload": f"{args.serve_requests} seeded Poisson-arrival 2D Poisson solves, "
                                   f"side U{{64..512}}, rate {args.serve_rate}/s, 64x64 subdomains, "
                                   "overlap 2, banded Cholesky, tol 1e-8",
                       "setup_workers": args.serve_workers},
            "variants": out}
    print(json.dumps(line), flush=True)


def run_serve_sweep(args):
    """Serving at several loads: the sync-FP64 saturation throughput is
    measured first (every request of a burst present at t = 0), then async
    mixed precision (FP32 factors) and sync FP64 each serve an open-loop
    Poisson stream at 0.5, 0.8 and 0.95 x that throughput (the rates of the
    serving reading), --serve-requests requests per point."""
    import torch

    import paper_2003_05361_gb300 as ras
    from paper_2003_05361_gb300.serve import Server, request_stream

    torch.cuda.set_device(0)
    sat = Server(mode=ras.RAS_SYNC, prec=ras.RAS_FP64, step_limit=args.serve_step,
                 workers=args.serve_workers).run(request_stream(args.serve_sat_requests, rate=1e6,
                                                                seed=7))
    mu = sat["solves_per_s"]
    print(json.dumps({"saturation_sync_fp64": sat}), flush=True)
    rows = []
    for frac in (0.5, 0.8, 0.95):
        for name, mode, prec in (("async_fp32", ras.RAS_ASYNC, ras.RAS_FP32),
                                 ("sync_fp64", ras.RAS_SYNC, ras.RAS_FP64)):
            srv = Server(mode=mode, prec=prec, step_limit=args.serve_step,
                         workers=args.serve_workers)
            st = srv.run(request_stream(args.serve_requests, rate=frac * mu, seed=5))
            row = {"load": frac, "rate_per_s": frac * mu, "arm": name, **st}
            rows.append(row)
            print(json.dumps(row), flush=True)
    print(json.dumps({"serve_sweep": f"{args.serve_requests} requests per point, side U{{64..512}}, "
                                     f"sync-FP64 saturation {mu:.3f} solves/s", "rows": rows}),
          flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--quick", action="store_true", help="headline only (no variants, no e2e)")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU baseline sample")
    ap.add_argument("--profile", action="store_true", help="run the small ncu case only")
    ap.add_argument("--profile-updates", type=int, default=20)
    ap.add_argument("--case", default="cg_cfg2", choices=["cg_cfg2", "band_cfg1", "band_cfg4s", "gmres_nonsym"])
    ap.add_argument("--band-iters", type=int, default=200,
                    help="sync iterations of the config-4 band roofline launch")
    ap.add_argument("--sweep", action="store_true",
                    help="overlap / partition / detection sweep on the benchmark problem")
    ap.add_argument("--sweep-only", default="",
                    help="with --sweep: comma-separated partition:local pairs to run "
                         "(e.g. regular2d:cg20_fp32)")
    ap.add_argument("--sweep-reps", type=int, default=10,
                    help="asynchronous solves per sweep point (median, min, max)")
    ap.add_argument("--serve", action="store_true", help="run the serving workload only")
    ap.add_argument("--serve-sweep", action="store_true",
                    help="serving at 0.5 / 0.8 / 0.95 x the sync-FP64 saturation throughput")
    ap.add_argument("--serve-requests", type=int, default=300)
    ap.add_argument("--serve-rate", type=float, default=20.0)
    ap.add_argument("--serve-step", type=int, default=20)
    ap.add_argument("--serve-workers", type=int, default=2, help="host threads doing request setup")
    ap.add_argument("--serve-sat-requests", type=int, default=40,
                    help="requests of the saturation run in the default benchmark")
    ap.add_argument("--serve-requests-bench", type=int, default=60,
                    help="requests per serving arm in the default benchmark")
    ap.add_argument("--config4-full", action="store_true",
                    help="solve config 4 to 1e-8 with every storage precision")
    ap.add_argument("--sections", default="config3,config4,serving,nonsymmetric,oras",
                    help="comma-separated extra sections of the default run")
    args = ap.parse_args()
    args.sections = [x for x in args.sections.split(",") if x]
    if args.sweep:
        run_sweep(args)
    elif args.serve_sweep:
        run_serve_sweep(args)
    elif args.serve:
        run_serving(args)
    elif args.profile:
        run_profile_case(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
