#!/usr/bin/env python
"""Benchmark of the D-NGD step on one GB300 (one JSON line on stdout).

Workload: 5-D Poisson -Laplace(u) = f on [0,1]^5, u = sum_i sin(pi x_i), tanh MLP
5-256-256-256-1 (n = 133,377), 3,000 interior + 1,000 boundary points
(m = 4,000), Glorot init (seed 0), lambda = 1e-5 (the paper's rule
lambda_k = min(loss, 1e-5) at this loss).  One timed step = one D-NGD
iteration: dngd_step (FP64 jets + J, the exact Gram K + lambda I from 8-bit
slices on the tcgen05 tensor cores, FP64 factor with sliced trailing updates,
refined solve for v, f_vv, refined solve for a, GA test) followed by the
31-point grid line search and the parameter update (dngd_line_search).

Reported: steps/s of the mixed path (value, device-resident inputs), the same
through host buffers (e2e), the FP64 GPU path's steps/s and step errors
against a full FP64 CPU oracle step at the same theta, Gram TFLOP/s against
the measured tensor peak, p50/p99 step latency and clocks under load.

--impl reference: the FP64 CPU oracle on the host cores (the slow baseline).
"""
import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "D-NGD steps/s mixed vs FP64 at equal step error; Gram TFLOP/s; p99 step latency"
UNIT = "steps/s"
DTYPES = {"oz": "f32 jets and Jacobian / bf16 tensor (exact integer slices, 4 per entry, 13 products) / f64 "
                "factor, f32 preconditioner / f64 Gram operator",
          "oz64": "f64 jets and Jacobian / bf16 tensor (exact integer slices, 4 per entry, 15 products) / f64 "
                  "factor, f32 preconditioner / f64 Gram operator",
          "bf16": "bf16/f32 (double-float accumulation in the refinement)",
          "tf32": "tf32/f32 (double-float accumulation in the refinement)"}
L2_NOTE = {"oz": "working set larger than L2 (J: 2.13 GB FP32, slices 4.27 GB BF16, Gram 128 MB FP64 per step)",
           "oz64": "working set larger than L2 (J: 4.27 GB FP64, slices 4.27 GB BF16, Gram 128 MB FP64 per step)",
           "bf16": "working set larger than L2 (J: 2.13 GB FP32 + 1.07 GB BF16 per step)",
           "tf32": "working set larger than L2 (J: 2.13 GB FP32 per step)"}
def _prec(dngd, name):
    """The precision mode of a --precision name."""
    return {"oz": dngd.MIXED_OZ, "oz64": dngd.MIXED_OZ64, "bf16": dngd.MIXED_BF16, "tf32": dngd.MIXED_TF32}[name]


WORKLOAD = "poisson5d_dense: -Lap u = f on [0,1]^5, MLP 5-256-256-256-1 (n=133377), 3000+1000 pts (m=4000)"


# DRAM bytes (read + write) of one exact-Gram product launch on the 5-D
# workload, from an ncu capture of k_gram_oz (profiles/k_gram_oz_poisson5d_oz64.md);
# keyed by --precision, valid for the kernel as committed with that summary.
GRAM_TRAFFIC = {"oz64": 39.47e9}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), float(p["bf16_tflops"]), float(p["bf16_tflops_sustained"]), "measured"
    except Exception:
        return 6800.0, 1900.0, 1700.0, "fallback"


def _grid():
    return np.array([2.0 ** (-j) for j in range(31)])


class ClockSampler:
    """nvidia-smi sampling of SM clocks / throttle reasons during a region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None
        self.gpu = gpu_index

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "50"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is not None:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except Exception:
                self.p.kill()
        self.f.flush()
        self.f.seek(0)
        rows = [ln.strip().split(", ") for ln in self.f.read().splitlines() if ln.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
                for nm, val in zip(names, r[5:9]):
                    if val.strip().lower() == "active":
                        reasons.add(nm)
            except Exception:
                continue
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


def max_over_ranks(ms, dist, device):
    """The job's time is the slowest rank's (replicas run independently)."""
    if dist is None:
        return float(ms)
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(world, ms_per_step):
    """Whole-job steps/s: every rank advances its own replica one step per ms_per_step."""
    return world * 1000.0 / ms_per_step


def oracle_full_step(wl, lam, with_kappa=False):
    """One full FP64 oracle step (stage timings in seconds)."""
    from oracle import residual as ores, step as ostep
    prob = ores.problem_from_spec(wl)
    t = {}
    t0 = time.perf_counter()
    r, J = ores.residual_and_jacobian(wl["theta"], prob, wl["X"], wl["target"])
    t["jacobian"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    K = ostep.gram(J, lam)
    t["gram"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    L = ostep.cholesky(K)
    del K
    t["cholesky"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    alpha = ostep.chol_solve(L, r)
    v = -(J.T @ alpha)
    t["solve_v"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    fvv = ores.second_directional(wl["theta"], prob, wl["X"], wl["target"], v)
    t["fvv"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    beta = ostep.chol_solve(L, fvv)
    a = -(J.T @ beta)
    delta, ratio, acc = ostep.ga_accept(v, a)
    t["solve_a"] = time.perf_counter() - t0
    out = dict(delta=delta, v=v, a=a, alpha=alpha, accepted=acc, ratio=ratio)
    if with_kappa:
        # not part of the step (untimed): an upper bound of cond(K + lambda I)
        out["kappa_upper"], out["norm_K"] = _kappa_upper(J, lam)
    return out, t


def _threads():
    """Threads of the BLAS numpy calls: threadpoolctl where installed, else
    the OpenBLAS library numpy loaded, asked through its own query."""
    try:
        from threadpoolctl import threadpool_info
        return max((i.get("num_threads", 0) for i in threadpool_info()), default=None)
    except Exception:
        pass
    import ctypes
    try:
        with open("/proc/self/maps") as f:
            libs = sorted({ln.split()[-1] for ln in f if "openblas" in ln.lower() and ln.split()[-1].startswith("/")})
    except OSError:
        libs = []
    for path in libs:
        try:
            lib = ctypes.CDLL(path)
        except OSError:
            continue
        for name in ("scipy_openblas_get_num_threads64_", "scipy_openblas_get_num_threads",
                     "openblas_get_num_threads64_", "openblas_get_num_threads"):
            fn = getattr(lib, name, None)
            if fn is not None:
                fn.restype = ctypes.c_int
                return int(fn())
    v = os.environ.get("OPENBLAS_NUM_THREADS") or os.environ.get("OMP_NUM_THREADS")
    return int(v) if v else None


def _sub_workload(wl, per_class):
    """The first `per_class` points of every residual class of a workload (same
    network, parameters and class constants): a bounded sample of it."""
    import copy
    sub = copy.deepcopy(wl)
    rows, start = [], 0
    for c in sub["classes"]:
        take = min(per_class, int(c["count"]))
        rows.extend(range(start, start + take))
        start += int(c["count"])
        c["count"] = take
    sub["X"] = np.ascontiguousarray(wl["X"][rows])
    sub["target"] = np.ascontiguousarray(wl["target"][rows])
    return sub


def run_reference(args, wl):
    """--impl reference: the FP64 CPU oracle (the paper's method written plainly)."""
    # untimed warm-up on a bounded sample (32 points per class: imports, BLAS
    # thread pool), then at most 2 timed full steps (~50 s of CPU work each)
    warm = max(3, args.warmup)
    small = _sub_workload(wl, 32)
    from oracle import residual as ores
    for _ in range(warm):
        oracle_full_step(small, args.lam)
    steps = min(args.steps, 2)
    times = []
    for _ in range(steps):
        t0 = time.perf_counter()
        r0 = ores.residual(wl["theta"], ores.problem_from_spec(wl), wl["X"], wl["target"])
        oracle_full_step(wl, _lam_for(args, 0.5 * float(r0 @ r0)))
        times.append(time.perf_counter() - t0)
    ms = 1000.0 * float(np.mean(times))
    cores = len(os.sched_getaffinity(0))
    value = 1000.0 / ms
    sample = (f"{steps} full FP64 oracle step(s) of the workload from theta_0 (--steps capped at 2: one step is "
              f"~{ms / 1000:.0f} s of CPU work), after {warm} untimed warm-up steps on the first 32 points of each "
              f"residual class; line search not included")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": steps, "warmup": warm, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "lam": _lam_config(args), "step": "dngd_step + 31-point line search + update",
                   "parallelism": "single GPU"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
                         "blas_threads": _threads()},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def run_batch(args, rank, world, local_rank):
    """64 independent 2-D Poisson instances (k ~ U{1..8}, width ~ U{32,64,128},
    m ~ U[256,2048]) stepped by one CUDA-graph launch per batch step."""
    import torch
    from oracle import residual as ores, step as ostep
    from paper_2505_21404_gb300 import dngd, workloads
    torch.cuda.set_device(local_rank)
    dev = torch.device(f"cuda:{local_rank}")
    lam = args.lam
    wls = workloads.poisson2d_batch(64, seed=0, lam=lam)
    bprec = _prec(dngd, args.precision)
    descs = [dngd.make_desc(wl, precision=bprec, refine_tol=args.refine_tol, refine_max_it=60) for wl in wls]
    ths = [torch.tensor(wl["theta"], device=dev) for wl in wls]
    Xs = [torch.tensor(wl["X"], device=dev) for wl in wls]
    tgs = [torch.tensor(wl["target"], device=dev) for wl in wls]
    ds = [torch.zeros(len(wl["theta"]), dtype=torch.float64, device=dev) for wl in wls]
    # CPU oracle on a sample of 4 instances (timing + error reference)
    cpu, refs = None, {}
    if rank == 0 and world == 1 and not args.no_oracle:
        t0 = time.perf_counter()
        for i in (0, 1, 2, 3):
            wl = wls[i]
            refs[i] = ostep.dense_step(wl["theta"], ores.problem_from_spec(wl), wl["X"], wl["target"], lam)["delta"]
        t_or = (time.perf_counter() - t0) / 4
        cpu = {"value": 1.0 / t_or, "unit": "instance-steps/s", "cores": len(os.sched_getaffinity(0)),
               "kind": "oracle", "sample": "FP64 oracle steps of instances 0-3 (mean time per instance step)"}
    batch = dngd.Batch(descs)
    for _ in range(args.warmup):
        batch.step(ths, Xs, tgs, ds)
    torch.cuda.synchronize(dev)
    clocks = ClockSampler(local_rank)
    clocks.start()
    time.sleep(0.3)
    l0 = dngd.dngd_launch_count()
    t0 = time.perf_counter()
    lat = []
    infos = None
    for _ in range(args.steps):
        ts = time.perf_counter()
        infos = batch.step(ths, Xs, tgs, ds)
        lat.append(1000.0 * (time.perf_counter() - ts))
    torch.cuda.synchronize(dev)
    t_batch = (time.perf_counter() - t0) / args.steps
    launches = dngd.dngd_launch_count() - l0
    clk = clocks.stop()
    # the same 64 instances stepped alone, one after another, through the same
    # captured-graph API (the first call of a context is its synchronous step);
    # exact-Gram instances with the factor form the batch uses
    if bprec in (dngd.MIXED_OZ, dngd.MIXED_OZ64):
        for d in descs:
            d.factor_update = dngd.FACTOR_DF
    alone = [dngd.Context(d) for d in descs]
    da = [torch.zeros_like(d) for d in ds]
    for i, c in enumerate(alone):
        c.step_async(ths[i], Xs[i], tgs[i], da[i])
        c.step_wait()
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for i, c in enumerate(alone):
        c.step_async(ths[i], Xs[i], tgs[i], da[i])
        c.step_wait()
    torch.cuda.synchronize(dev)
    t_alone = time.perf_counter() - t0
    same = sum(int(torch.equal(a, b)) for a, b in zip(da, ds))
    errs = {i: float(np.linalg.norm(ds[i].cpu().numpy() - r) / np.linalg.norm(r)) for i, r in refs.items()}
    gram_flops = sum(float(wl["X"].shape[0]) * (wl["X"].shape[0] + 1) * len(wl["theta"]) for wl in wls)
    hbm, bf16_burst, bf16_sust, src = _peaks()
    value = world * 64.0 / t_batch
    line = {
        "metric": METRIC, "value": value, "unit": "instance-steps/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1000.0 * t_batch, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": DTYPES[args.precision], "data": "synthetic",
        "config": {"workload": "poisson2d_batch: 64 x (-Lap u = f on [0,1]^2, u = sin(k pi x) sin(k pi y), "
                               "MLP 2-w-w-1, w ~ U{32,64,128}, m ~ U[256,2048])", "lam": lam,
                   "step": "one batch step = one CUDA-graph launch with 64 parallel instance steps (no line "
                           "search); exact-Gram instances factored together, one launch per kernel and "
                           "64-column step"},
        "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
        "alone_sequential_instance_steps_per_s": 64.0 / t_alone, "speedup_vs_alone": t_alone / t_batch,
        "instances_bitwise_equal_alone": same, "step_error_vs_oracle": errs,
        "refine_iters_mean": float(np.mean([sum(i["solve_iters"]) for i in infos])),
        "roofline": {"bound": "tensor", "kernel": "all instance steps (aggregate Gram flops / batch step time)",
                     "achieved": gram_flops / t_batch / 1e12, "peak": bf16_sust, "unit": "TFLOP/s",
                     "frac": gram_flops / t_batch / 1e12 / bf16_sust, "peak_source": f"{src} bf16 sustained",
                     "traffic": None},
        "cpu_baseline": cpu,
        "gpu_launches": int(launches), "clocks": clk,
    }
    if rank == 0:
        print(json.dumps(line))


def run_heat(args, rank, world, local_rank):
    """Matrix-free Nystrom-PCG step of the 1+1-D heat workload (n = 12.6M):
    timed with the 3xTF32 tensor-core operator; the compensated FP32 SIMT
    operator's step at the same theta as the accuracy reference (untimed);
    PCG iterations and step time for ell in {128, 256, 512, 1024}."""
    import torch
    from paper_2505_21404_gb300 import dngd, workloads
    torch.cuda.set_device(local_rank)
    dev = torch.device(f"cuda:{local_rank}")
    # the heat problem's damping rule is min(loss, 1e-3) (App. A.3)
    cap = 1e-3 if args.lam_rule == "paper" else 0.0
    lam = 1e-3 if args.lam_rule == "paper" else args.lam
    wl = workloads.heat_pcg(lam=lam)
    m = wl["X"].shape[0]
    th = torch.tensor(wl["theta"], device=dev)
    X = torch.tensor(wl["X"], device=dev)
    tg = torch.tensor(wl["target"], device=dev)
    n = len(wl["theta"])

    def make(ell, op):
        c = dngd.Context(dngd.make_desc(wl, precision=dngd.MIXED_BF16, solver=dngd.PCG, pcg_rank=ell, pcg_tol=1e-6,
                                        pcg_max_it=500, lambda_cap=cap, pcg_operator=op))
        c.set_landmarks(workloads.landmarks(m, ell, seed=3))
        return c

    ctx = make(args.ell, dngd.PCG_OP_TC3)
    ctx.set_timing(True)
    d = torch.zeros(n, dtype=torch.float64, device=dev)
    # ~1.2 s per step: at least 3 warm-up steps, at most 5 timed ones
    warm = max(3, args.warmup)
    for _ in range(warm):
        ctx.step(th, X, tg, d)
    torch.cuda.synchronize(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    steps = max(1, min(args.steps, 5))
    clocks = ClockSampler(local_rank)
    clocks.start()
    l0 = dngd.dngd_launch_count()
    e0.record()
    infos = [ctx.step(th, X, tg, d) for _ in range(steps)]
    e1.record()
    torch.cuda.synchronize(dev)
    launches = dngd.dngd_launch_count() - l0
    clk = clocks.stop()
    ms = e0.elapsed_time(e1) / steps

    def kv_time(c):
        v = torch.randn(m, dtype=torch.float64, device=dev, generator=torch.Generator(device=dev).manual_seed(5))
        w = torch.zeros_like(v)
        c.kvp(v, w)
        torch.cuda.synchronize(dev)
        e0.record()
        for _ in range(3):
            c.kvp(v, w)
        e1.record()
        torch.cuda.synchronize(dev)
        return e0.elapsed_time(e1) / 3, w

    kv_ms, w_tc = kv_time(ctx)
    lam_used = infos[-1]["lambda_used"]
    ctx.close()
    # the compensated operator at the same theta (accuracy reference, untimed)
    ref = make(args.ell, dngd.PCG_OP_COMPENSATED)
    d_ref = torch.zeros_like(d)
    info_ref = ref.step(th, X, tg, d_ref)
    kv_ms_ref, w_ref = kv_time(ref)
    ref.close()
    step_dev = float(((d - d_ref).norm() / d_ref.norm()).item())
    kv_dev = float(((w_tc - w_ref).norm() / w_ref.norm()).item())
    sweep = []
    for ell in (128, 256, 512, 1024):
        c = make(ell, dngd.PCG_OP_TC3)
        dd = torch.zeros_like(d)
        c.step(th, X, tg, dd)
        torch.cuda.synchronize(dev)
        e0.record()
        inf = c.step(th, X, tg, dd)
        e1.record()
        torch.cuda.synchronize(dev)
        sweep.append({"ell": ell, "ms_per_step": e0.elapsed_time(e1), "pcg_iters": inf["solve_iters"],
                      "nystrom_shift": inf["shift_used"]})
        c.close()
    # K v: J^T v and J u, three 2048 x 2048 hidden-layer GEMMs each over
    # R = 26,624 point-stream rows (2 R w^2 flop apiece); 3xTF32 executes
    # three TF32 products per flop
    kv_flops = 2.0 * 3 * 2 * 26624 * 2048 * 2048
    hbm, bf16_burst, bf16_sust, src = _peaks()
    tf32_peak = bf16_sust / 2.0
    line = {
        "metric": METRIC, "value": 1000.0 / ms, "unit": "steps/s", "n_gpus": 1, "steps": steps, "warmup": warm,
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 jets / 3xTF32 tensor-core operator (FP32 accumulation) / f64 CG vectors", "data": "synthetic",
        "config": {"workload": "heat_pcg: u_t = 0.1 u_xx, MLP 2-2048x4-1 (n=12597249), 6144+1024+1024 pts",
                   "lam": ("min(loss, 1e-3) per step (the heat problem's rule, App. A.3)" if cap else lam),
                   "lam_used": lam_used, "ell": args.ell, "pcg_tol": 1e-6},
        "kv_ms": kv_ms, "pcg_iters": infos[-1]["solve_iters"], "pcg_relres": infos[-1]["solve_relres"],
        "phase_ms": infos[-1]["phase_ms"], "nystrom_shift": infos[-1]["shift_used"],
        "vs_compensated_operator": {
            "step_deviation": step_dev, "kv_deviation": kv_dev, "kv_ms": kv_ms_ref,
            "pcg_iters": info_ref["solve_iters"],
            "note": "same theta, same landmarks; the compensated FP32 SIMT operator (Kahan sums, FP64 row "
                    "reductions) as the reference: the full-size FP64 Jacobian (8,192 x 12.6M) does not fit"},
        "ell_sweep": sweep,
        "roofline": {"bound": "tensor", "kernel": "k_tc3 (3xTF32 factor-form K v: J^T v and J u, TMEM chunks of 128 K-elements)",
                     "achieved": kv_flops / (kv_ms * 1e-3) / 1e12, "peak": tf32_peak, "unit": "TFLOP/s",
                     "frac": kv_flops / (kv_ms * 1e-3) / 1e12 / tf32_peak,
                     "executed_tflops": 3 * kv_flops / (kv_ms * 1e-3) / 1e12,
                     "executed_frac": 3 * kv_flops / (kv_ms * 1e-3) / 1e12 / tf32_peak,
                     "peak_source": f"{src} bf16 sustained / 2 (TF32)", "traffic": None},
        "cpu_baseline": None, "gpu_launches": launches, "clocks": clk,
    }
    print(json.dumps(line))


def run_c1(args, rank, world, local_rank):
    """2-D Poisson, FP64, lambda = 1e-8, GA on (m = 500, n = 1,185): step
    latency p50/p99 over graph-replayed steps at fixed theta, and the 20-step
    trajectory (step + line search) with its loss and L2 error."""
    import torch
    from paper_2505_21404_gb300 import dngd, workloads
    torch.cuda.set_device(local_rank)
    dev = torch.device(f"cuda:{local_rank}")
    stream = torch.cuda.current_stream(dev)
    wl = workloads.poisson2d_fp64()
    m, n = wl["X"].shape[0], len(wl["theta"])
    desc = dngd.make_desc(wl, precision=dngd.FP64)
    th0 = torch.tensor(wl["theta"], device=dev)
    X = torch.tensor(wl["X"], device=dev)
    tg = torch.tensor(wl["target"], device=dev)
    delta = torch.zeros(n, dtype=torch.float64, device=dev)
    ctx = dngd.Context(desc, stream=stream.cuda_stream)
    # the first asynchronous step of a context runs synchronously; then W warm-up replays
    for _ in range(1 + args.warmup):
        ctx.step_async(th0, X, tg, delta)
        ctx.step_wait()
    reps = max(1000, args.steps)
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(reps + 1)]
    clocks = ClockSampler(local_rank)
    clocks.start()
    time.sleep(0.3)
    l0 = dngd.dngd_launch_count()
    torch.cuda.synchronize(dev)
    evs[0].record(stream)
    for k in range(reps):
        ctx.step_async(th0, X, tg, delta)
        evs[k + 1].record(stream)
    torch.cuda.synchronize(dev)
    launches = dngd.dngd_launch_count() - l0
    clk = clocks.stop()
    lat = np.array([evs[k].elapsed_time(evs[k + 1]) for k in range(reps)])
    total_ms = evs[0].elapsed_time(evs[reps])
    info = ctx.step_wait()
    # end to end through the public call with host buffers (inputs copied in,
    # the step copied out, status read back) for the same number of steps
    th_h, X_h, tg_h, d_h = wl["theta"].copy(), np.ascontiguousarray(wl["X"]), np.ascontiguousarray(wl["target"]), \
        np.zeros(n)
    ctx.step(th_h, X_h, tg_h, d_h)
    t0 = time.perf_counter()
    for _ in range(reps):
        ctx.step(th_h, X_h, tg_h, d_h, want_info=False)
    e2e_ms = 1000.0 * (time.perf_counter() - t0) / reps
    # 20 D-NGD iterations (step + 31-point line search) from theta_0
    etas = _grid()
    theta, theta_next = th0.clone(), torch.zeros_like(th0)
    traj = []
    ev_a, ev_b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for k in range(20):
        ev_a.record(stream)
        inf = ctx.step(theta, X, tg, delta)
        eta = ctx.line_search(theta, X, tg, delta, etas, theta_next)
        ev_b.record(stream)
        torch.cuda.synchronize(dev)
        traj.append({"loss": inf["loss"], "eta": eta, "ga_accepted": inf["ga_accepted"],
                     "ms": ev_a.elapsed_time(ev_b)})
        theta, theta_next = theta_next, theta
    l2 = None
    cpu = None
    if not args.no_oracle:
        from oracle import evaluate, residual as ores, step as ostep
        g = evaluate.midpoint_grid(2, 64)
        l2 = {"theta0": evaluate.rel_l2_error(wl["theta"], wl["widths"], g, evaluate.sine_product(g)),
              "after_20": evaluate.rel_l2_error(theta.cpu().numpy(), wl["widths"], g, evaluate.sine_product(g)),
              "grid": "64 x 64 midpoints of [0,1]^2"}
        prob = ores.problem_from_spec(wl)
        t0 = time.perf_counter()
        k_or = 0
        while time.perf_counter() - t0 < 10.0 or k_or < 3:
            ostep.dense_step(wl["theta"], prob, wl["X"], wl["target"], wl["lam"], use_ga=True)
            k_or += 1
        t_or = (time.perf_counter() - t0) / k_or
        cpu = {"value": 1.0 / t_or, "unit": "steps/s", "cores": len(os.sched_getaffinity(0)), "kind": "oracle",
               "sample": f"{k_or} FP64 oracle steps at theta_0 (mean)", "blas_threads": _threads()}
    ctx.close()
    syrk = float(m) * (m + 1) * n
    ms = total_ms / reps
    fp64_peak = 1250.0
    line = {
        "metric": METRIC, "value": 1000.0 / ms, "unit": "steps/s", "n_gpus": 1, "steps": reps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": "poisson2d_fp64: -Lap u = f on [0,1]^2, u = sin(pi x) sin(pi y), MLP 2-32-32-1 "
                               "(n=1185), 400+100 pts (m=500)", "lam": 1e-8, "precision": "fp64",
                   "step": "dngd_step_async (graph replay) at fixed theta_0; GA on",
                   "l2": "working set (J 4.7 MB) fits in L2: latency-bound, no flush"},
        "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
        "ga_accepted_at_theta0": info["ga_accepted"],
        "trajectory": traj, "l2_error": l2,
        "roofline": {"bound": "alu", "kernel": "whole step (FP64 syrk m(m+1)n + Cholesky + jets, launch-latency bound)",
                     "achieved": syrk / (ms * 1e-3) / 1e9, "peak": fp64_peak, "unit": "GFLOP/s",
                     "frac": syrk / (ms * 1e-3) / 1e9 / fp64_peak,
                     "peak_source": "nominal GB300 FP64 rate (1.25 TFLOP/s)", "traffic": None},
        "cpu_baseline": cpu,
        "e2e": {"value": 1000.0 / e2e_ms, "unit": "steps/s", "h2d_bytes_per_step": 8 * (n + 2 * m + m),
                "d2h_bytes_per_step": 8 * n},
        "gpu_launches": int(launches), "clocks": clk,
    }
    print(json.dumps(line))


def _regime_grid(cells=""):
    """Cells (m, w) of the regime map: m in {300, 1800, 3300, 6300} points by
    hidden width w in {15, 51, 71} (n = w^2 + 5w + 1 = 301, 2,857, 5,397), or
    the subset 'm:w,m:w' given on the command line."""
    if cells:
        out = []
        for c in cells.split(","):
            m, w = (int(x) for x in c.split(":"))
            if m < 5 or w < 1:
                raise ValueError(f"regime_map cell {c!r}: need m >= 5 points and width w >= 1")
            out.append((m, w))
        return out
    return [(m, w) for m in (300, 1800, 3300, 6300) for w in (15, 51, 71)]


def _regime_cpu_baseline(m=1800, w=15, seconds=10.0):
    """The FP64 oracle on the host cores for one regime-map cell: its dense
    step (jets, J, dual solve and GA) and, on the same J, r and f_vv, the
    primal solves, each repeated for about `seconds`."""
    from oracle import residual as ores, step as ostep
    from paper_2505_21404_gb300 import workloads
    ni = (4 * m) // 5
    wl = workloads.poisson_sine(2, [2, w, w, 1], ni, m - ni, k=2, seed=m + w, lam=1e-5)
    prob = ores.problem_from_spec(wl)
    t0, k_d = time.perf_counter(), 0
    while k_d < 1 or time.perf_counter() - t0 < seconds / 2:
        ref = ostep.dense_step(wl["theta"], prob, wl["X"], wl["target"], wl["lam"], use_ga=True)
        k_d += 1
    t_dual = (time.perf_counter() - t0) / k_d
    t0, k_p = time.perf_counter(), 0
    while k_p < 1 or time.perf_counter() - t0 < seconds / 2:
        ostep.primal_step(ref["J"], ref["r"], wl["lam"])
        ostep.primal_step(ref["J"], ref["fvv"], wl["lam"])
        k_p += 1
    t_primal_solves = (time.perf_counter() - t0) / k_p
    return {"value": 1.0 / t_dual, "unit": "steps/s", "cores": len(os.sched_getaffinity(0)), "kind": "oracle",
            "sample": f"m = {m}, n = {len(wl['theta'])}: {k_d} FP64 oracle dense steps (dual, GA) "
                      f"{1e3 * t_dual:.1f} ms each; the two primal solves on the same J "
                      f"{1e3 * t_primal_solves:.1f} ms ({k_p} repeats)",
            "blas_threads": _threads()}


def run_regime(args, rank, world, local_rank):
    """Primal vs dual regime map (Sec. 3, primal vs dual perspectives; the
    appendix's Navier-Stokes (m x n) sweep): the FP64 dense step solved in parameter space
    ((J^T J + lambda I), n x n) and in residual space ((J J^T + lambda I),
    m x m) on a grid of (m, n), each timed with CUDA events over --steps
    steps after the warm-up.  Synthetic 2-D Poisson residuals on MLPs
    2-w-w-1 (n = w^2 + 5w + 1) stand in for the paper's Navier-Stokes sweep."""
    import torch
    from paper_2505_21404_gb300 import dngd, workloads
    torch.cuda.set_device(local_rank)
    dev = torch.device(f"cuda:{local_rank}")
    stream = torch.cuda.current_stream(dev)
    grid = _regime_grid(args.cells)
    steps = max(1, min(args.steps, 3))
    cells = []
    clocks = ClockSampler(local_rank)
    clocks.start()
    l0 = dngd.dngd_launch_count()
    for m, w in grid:
        ni = (4 * m) // 5
        wl = workloads.poisson_sine(2, [2, w, w, 1], ni, m - ni, k=2, seed=m + w, lam=1e-5)
        n = len(wl["theta"])
        th, X, tg = (torch.tensor(np.ascontiguousarray(wl[k]), device=dev) for k in ("theta", "X", "target"))
        cell = {"m": m, "n": n}
        outs = {}
        for name, space in (("primal", dngd.SPACE_PRIMAL), ("dual", dngd.SPACE_DUAL)):
            ctx = dngd.Context(dngd.make_desc(wl, precision=dngd.FP64, solve_space=space),
                               stream=stream.cuda_stream)
            delta = torch.zeros(n, dtype=torch.float64, device=dev)
            for _ in range(args.warmup):
                ctx.step(th, X, tg, delta, want_info=False)
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize(dev)
            ev0.record(stream)
            for _ in range(steps):
                ctx.step(th, X, tg, delta, want_info=False)
            ev1.record(stream)
            torch.cuda.synchronize(dev)
            cell[name + "_ms"] = ev0.elapsed_time(ev1) / steps
            # one more step with the phase events: the Gram GEMM (J^T J or J J^T, lower
            # triangle) alone
            ctx.set_timing(True)
            inf = ctx.step(th, X, tg, delta)
            cell[name + "_gram_ms"] = inf["phase_ms"][1]
            outs[name] = delta.cpu().numpy()
            ctx.close()
        cell["winner"] = "primal" if cell["primal_ms"] < cell["dual_ms"] else "dual"
        cell["auto"] = "primal" if n < m else "dual"
        cell["step_diff"] = float(np.linalg.norm(outs["primal"] - outs["dual"]) / np.linalg.norm(outs["dual"]))
        cells.append(cell)
    launches = dngd.dngd_launch_count() - l0
    clk = clocks.stop()
    cpu = None if args.no_oracle else _regime_cpu_baseline()
    agree = sum(c["winner"] == c["auto"] for c in cells)
    # FP64 rate of the Gram GEMMs: n(n+1)m flop (primal) or m(m+1)n flop (dual), the lower triangle
    fp64_peak = 1250.0
    for c in cells:
        c["primal_gram_gflops"] = c["n"] * (c["n"] + 1) * c["m"] / (c["primal_gram_ms"] * 1e6)
        c["dual_gram_gflops"] = c["m"] * (c["m"] + 1) * c["n"] / (c["dual_gram_ms"] * 1e6)
    top = max(cells, key=lambda c: c["n"] * c["n"] * c["m"])
    line = {
        "metric": "automatic space choice = faster space (cells)", "value": agree / len(cells), "unit": "fraction",
        "n_gpus": 1, "steps": steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "regime_map: 2-D Poisson, MLP 2-w-w-1, lambda = 1e-5, GA on, FP64 dense step in "
                               "both spaces, cells (m, w) = " + ", ".join(f"({m}, {w})" for m, w in grid),
                   "l2": "each cell's timed steps repeat the step; no flush (the spaces are compared, not the "
                         "roofline)"},
        "cells": cells,
        "roofline": {"bound": "alu", "kernel": f"k_gemm<double> (A^T B, lower): J^T J of the primal step at "
                                               f"m = {top['m']}, n = {top['n']}",
                     "achieved": top["primal_gram_gflops"], "peak": fp64_peak, "unit": "GFLOP/s",
                     "frac": top["primal_gram_gflops"] / fp64_peak,
                     "peak_source": "GB300 FP64 rate: 152 SMs x 2 FP64 FMA/clock x 2,070 MHz (1.26 TFLOP/s)",
                     "traffic": None},
        "cpu_baseline": cpu,
        "gpu_launches": int(launches), "clocks": clk,
    }
    print(json.dumps(line))


def run_serving(args, rank, world, local_rank):
    """Serving loop: an arrival stream of PINN solve jobs (exponential
    inter-arrival times; 2-D / 5-D Poisson 50/50, k ~ U{1..8},
    m ~ U[512, 8192], width ~ U{64,128,256,512}, depth ~ U{2,3}; 50 D-NGD
    iterations each) offered to one dngd_server for a fixed window per
    arrival rate.  Reports completed iterations/s, device step latency
    p50/p99, job queueing delay and the admitted/queued/rejected counts."""
    import torch
    from paper_2505_21404_gb300 import dngd, workloads
    torch.cuda.set_device(local_rank)
    rates = [float(r) for r in args.rates.split(",")]
    hbm, bf16_burst, bf16_sust, src = _peaks()
    clocks = ClockSampler(local_rank)
    clocks.start()
    results = []
    l0 = dngd.dngd_launch_count()
    for rate in rates:
        n_jobs = int(min(args.max_jobs, max(4, rate * args.window * 1.2 + 2)))
        jobs = workloads.serving_jobs(n_jobs, rate_per_s=rate, seed=7, lam=args.lam)
        sprec = _prec(dngd, args.precision)
        descs = [dngd.make_desc(wl, precision=sprec, refine_tol=args.refine_tol, refine_max_it=60)
                 for _, wl, _ in jobs]
        srv = dngd.Server(hbm_budget_bytes=0, max_slots=args.slots)
        ids = []
        t0 = time.perf_counter()
        for (t_arr, wl, n_steps), desc in zip(jobs, descs):
            if t_arr >= args.window:
                break
            dt = t0 + t_arr - time.perf_counter()
            if dt > 0:
                time.sleep(dt)
            ids.append((srv.submit(desc, wl["theta"], wl["X"], wl["target"], n_steps), wl))
        rest = t0 + args.window - time.perf_counter()
        if rest > 0:
            time.sleep(rest)
        elapsed = time.perf_counter() - t0
        st = srv.stats()
        polls = [(srv.poll(j), wl) for j, wl in ids]
        flops = sum(p["steps_done"] * wl["X"].shape[0] * (wl["X"].shape[0] + 1) * len(wl["theta"])
                    for p, wl in polls)
        qd = [p["queue_s"] for p, _ in polls if p["state"] != "queued"]
        # completed jobs: time from submission to the last iteration
        lat = [p["queue_s"] + p["run_s"] for p, _ in polls if p["state"] == "done"]
        srv.close()
        results.append({
            "rate_jobs_per_s": rate, "window_s": elapsed, "submitted": len(ids),
            "steps_per_s": st["steps_total"] / elapsed, "steps_total": st["steps_total"],
            "p50_step_ms": st["p50_ms"], "p99_step_ms": st["p99_ms"],
            "queue_delay_p50_s": float(np.percentile(qd, 50)) if qd else None,
            "job_latency_p50_s": float(np.percentile(lat, 50)) if lat else None,
            "job_latency_p99_s": float(np.percentile(lat, 99)) if lat else None,
            "admitted": st["admitted"], "queued": st["queued"], "rejected": st["rejected"],
            "done": st["done"], "failed": st["failed"], "running_at_end": st["running"],
            "gram_tflops": flops / elapsed / 1e12,
        })
    launches = dngd.dngd_launch_count() - l0
    clk = clocks.stop()
    head = max(results, key=lambda r: r["steps_per_s"])
    line = {
        "metric": METRIC, "value": head["steps_per_s"], "unit": "job-steps/s", "n_gpus": 1,
        "steps": int(sum(r["steps_total"] for r in results)), "warmup": 0,
        "ms_per_step": 1000.0 / head["steps_per_s"] if head["steps_per_s"] else None, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": DTYPES[args.precision],
        "data": "synthetic",
        "config": {"workload": "serving: Poisson 2-D/5-D jobs, m ~ U[512,8192], MLP width ~ U{64..512}, depth 2-3, "
                               "50 iterations (step + 31-point line search) each", "lam": args.lam,
                   "slots": args.slots, "window_s": args.window, "hbm_budget": "80% of free"},
        "sweep": results,
        "roofline": {"bound": "tensor", "kernel": "all jobs' Gram flops m(m+1)n per completed iteration / window",
                     "achieved": head["gram_tflops"], "peak": bf16_sust, "unit": "TFLOP/s",
                     "frac": head["gram_tflops"] / bf16_sust, "peak_source": f"{src} bf16 sustained",
                     "traffic": None},
        "cpu_baseline": None, "gpu_launches": int(launches), "clocks": clk,
    }
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--lam", type=float, default=1e-5,
                    help="the cap of the damping rule (--lam-rule paper) or the fixed damping (--lam-rule fixed)")
    ap.add_argument("--lam-rule", default="paper", choices=["paper", "fixed"],
                    help="paper (default): lambda_k = min(loss, --lam) every step (App. A.3); fixed: lambda = --lam")
    ap.add_argument("--save-theta", default=None, help="write the parameters after the timed steps (.npy)")
    ap.add_argument("--gram-traffic", type=float, default=None,
                    help="DRAM bytes of one exact-Gram launch on the 5-D workload (from an ncu capture)")
    ap.add_argument("--precision", default="oz64", choices=["oz", "oz64", "bf16", "tf32"],
                    help="oz64 (default): FP64 jets and J, exact Gram from four 8-bit slices on the BF16 tensor "
                         "cores (15 products), FP64 factor, PCG on the exact Gram; oz: the same with FP32 jets and "
                         "J (13 products); bf16 / tf32: low-precision Gram, FP32-J operator")
    ap.add_argument("--fp64-steps", type=int, default=2)
    ap.add_argument("--no-oracle", action="store_true", help="skip the CPU oracle leg (no step error)")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--refine-max-it", type=int, default=400)
    ap.add_argument("--refine-tol", type=float, default=1e-5)
    ap.add_argument("--workload", default="poisson5d",
                    choices=["poisson5d", "poisson5d_w128", "poisson2d_fp64", "poisson2d_batch", "heat_pcg",
                             "serving", "regime_map"],
                    help="poisson5d (default, the headline): dense 5-D step; poisson5d_w128: same points, hidden "
                         "width 128 (profiling case); poisson2d_batch: 64 independent 2-D instances stepped as one "
                         "graph; heat_pcg: matrix-free Nystrom-PCG step of the 1+1-D heat problem (n = 12.6M); regime_map: "
                         "the FP64 step in parameter space vs residual space over a grid of (m, n)")
    ap.add_argument("--points", type=int, default=0,
                    help="poisson5d: total collocation points instead of 4,000 (3:1 interior:boundary; a smaller "
                         "case for profiler captures, not a bench line)")
    ap.add_argument("--ell", type=int, default=512, help="Nystrom landmarks for heat_pcg")
    ap.add_argument("--cells", default="", help="regime_map: only these cells, 'm:w,m:w' (MLP 2-w-w-1)")
    ap.add_argument("--rates", default="0.1,0.3,1,5,200", help="serving: offered job arrival rates (jobs/s)")
    ap.add_argument("--window", type=float, default=20.0, help="serving: seconds per arrival rate")
    ap.add_argument("--slots", type=int, default=16, help="serving: concurrent jobs")
    ap.add_argument("--max-jobs", type=int, default=400, help="serving: cap on jobs generated per rate")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))

    from paper_2505_21404_gb300 import workloads
    if args.workload == "poisson5d" and args.points > 0:
        ni = (3 * args.points) // 4
        wl = workloads.poisson_sine(5, [5, 256, 256, 256, 1], ni, args.points - ni, k=1, seed=0, lam=args.lam)
    elif args.workload == "poisson5d":
        wl = workloads.poisson5d_dense(seed=0, lam=args.lam)
    else:
        wl = workloads.poisson_sine(5, [5, 128, 128, 128, 1], 3000, 1000, k=1, seed=0, lam=args.lam)

    if args.workload == "poisson2d_fp64":
        return run_c1(args, rank, world, local_rank)
    if args.workload == "poisson2d_batch":
        return run_batch(args, rank, world, local_rank)
    if args.workload == "heat_pcg":
        return run_heat(args, rank, world, local_rank)
    if args.workload == "serving":
        return run_serving(args, rank, world, local_rank)
    if args.workload == "regime_map":
        return run_regime(args, rank, world, local_rank)
    if args.impl == "reference":
        if rank == 0:
            run_reference(args, wl)
        return

    return run_dense(args, wl, rank, world, local_rank)


def _lam_config(args):
    return (f"min(loss, {args.lam:g}) per step (the paper's rule, App. A.3)" if args.lam_rule == "paper"
            else args.lam)


def _lam_for(args, loss):
    """The damping of a step at a parameter vector with loss L: the paper's
    rule min(L, cap) (App. A.3 tables), or the fixed lambda."""
    if args.lam_rule == "paper":
        return loss if (0.0 < loss < args.lam) else args.lam
    return args.lam


def _kappa_upper(J, lam, iters=12, seed=0):
    """(||J J^T|| + lam) / lam with ||J J^T|| from power iteration on J J^T:
    an upper bound of cond(K + lam I) (its smallest eigenvalue is >= lam)."""
    x = np.random.default_rng(seed).normal(size=J.shape[0])
    nrm = 0.0
    for _ in range(iters):
        y = J @ (J.T @ x)
        nrm = float(np.linalg.norm(y) / np.linalg.norm(x))
        x = y / np.linalg.norm(y)
    return (nrm + lam) / lam, nrm


def run_dense(args, wl, rank, world, local_rank):
    """The dense D-NGD iteration of the 5-D workload (the headline line)."""
    import torch
    from paper_2505_21404_gb300 import dngd
    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device(f"cuda:{local_rank}"))
    dev = torch.device(f"cuda:{local_rank}")
    stream = torch.cuda.current_stream(dev)
    cap = args.lam if args.lam_rule == "paper" else 0.0
    do_oracle = rank == 0 and world == 1 and not args.no_oracle

    # CPU oracle at theta_0 first (rank 0, N = 1 only): timing + error reference
    ref0, cpu, lam0 = None, None, args.lam
    if do_oracle:
        from oracle import residual as ores
        r0 = ores.residual(wl["theta"], ores.problem_from_spec(wl), wl["X"], wl["target"])
        lam0 = _lam_for(args, 0.5 * float(r0 @ r0))
        ref0, stages = oracle_full_step(wl, lam0, with_kappa=True)
        t_or = float(sum(stages.values()))   # the step's stages (the kappa estimate is not timed)
        cpu = {"value": 1.0 / t_or, "unit": UNIT, "cores": len(os.sched_getaffinity(0)), "kind": "oracle",
               "sample": f"1 full FP64 oracle step of the workload at theta_0 ({t_or:.1f} s; stages " +
                         ", ".join(f"{k} {v:.1f}s" for k, v in stages.items()) +
                         "); line search not included",
               "blas_threads": _threads()}

    prec = _prec(dngd, args.precision)
    m, n = int(wl["X"].shape[0]), dngd.dngd_num_params(dngd.make_desc(wl))
    th0 = torch.tensor(wl["theta"], device=dev)
    X = torch.tensor(wl["X"], device=dev)
    tg = torch.tensor(wl["target"], device=dev)
    etas = _grid()

    def make_ctx(p):
        c = dngd.Context(dngd.make_desc(wl, precision=p, refine_tol=args.refine_tol,
                                        refine_max_it=args.refine_max_it, lambda_cap=cap),
                         stream=stream.cuda_stream)
        c.set_timing(True)
        return c

    # two contexts with the same history: A is timed on device-resident
    # inputs (value), B runs the same iterations from host buffers (e2e)
    ctx = make_ctx(prec)
    delta = torch.zeros(n, dtype=torch.float64, device=dev)
    theta = th0.clone()
    theta_next = torch.zeros_like(theta)

    # the mixed step at theta_0 (its error against the oracle)
    info0 = ctx.step(th0, X, tg, delta)
    torch.cuda.synchronize(dev)
    d_mixed0 = delta.cpu().numpy().copy()

    def one_step(c, th, out_th, dl):
        info = c.step(th, X, tg, dl)
        c.line_search(th, X, tg, dl, etas, out_th)
        return info

    for _ in range(args.warmup):
        one_step(ctx, theta, theta_next, delta)
        theta, theta_next = theta_next, theta
    torch.cuda.synchronize(dev)
    theta_start = theta.cpu().numpy().copy()
    if dist is not None:
        dist.barrier()
    clocks = ClockSampler(local_rank)
    clocks.start()
    time.sleep(0.3)
    launches0 = dngd.dngd_launch_count()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    step_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.steps)]
    infos = []
    torch.cuda.synchronize(dev)
    ev0.record(stream)
    for k in range(args.steps):
        step_ev[k][0].record(stream)
        infos.append(one_step(ctx, theta, theta_next, delta))
        step_ev[k][1].record(stream)
        theta, theta_next = theta_next, theta
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    launches = dngd.dngd_launch_count() - launches0
    clk = clocks.stop()
    total_ms = max_over_ranks(ev0.elapsed_time(ev1), dist, dev)
    ms_per_step = total_ms / args.steps
    lat = np.array([a.elapsed_time(b) for a, b in step_ev])
    value = job_value(world, ms_per_step)
    gram_ms = float(np.mean([i["phase_ms"][1] for i in infos]))
    gram_kernel_ms = float(np.mean([i["gram_kernel_ms"] for i in infos]))
    phase = np.mean(np.array([i["phase_ms"] for i in infos]), axis=0).tolist()
    iters = np.mean(np.array([i["solve_iters"] for i in infos]), axis=0).tolist()
    theta_late = theta.cpu().numpy().copy()

    # the mixed step at the late theta (the parameters after the timed steps)
    info_late = ctx.step(theta, X, tg, delta)
    torch.cuda.synchronize(dev)
    d_mixed_late = delta.cpu().numpy().copy()
    ctx.close()
    if args.save_theta:
        np.save(args.save_theta, theta_late)

    # end to end through host buffers: a second context with the same
    # history runs the same warm-up, then the same timed iterations with the
    # inputs copied in and delta / theta copied out every step
    e2e_ms = float("nan")
    h2d = 8 * (n + m * 5 + m) + 8 * (2 * n + m * 5 + m)   # step inputs + line-search inputs
    d2h = 8 * n + 8 * n                                       # delta + updated theta
    e2e_same = None
    if not args.no_e2e:
        ctxB = make_ctx(prec)
        X_h = np.ascontiguousarray(wl["X"])
        tg_h = np.ascontiguousarray(wl["target"])
        th_h = wl["theta"].copy()
        th_next_h = np.zeros(n)
        d_h = np.zeros(n)
        ctxB.step(th_h, X_h, tg_h, d_h, want_info=False)
        for _ in range(args.warmup):
            ctxB.step(th_h, X_h, tg_h, d_h, want_info=False)
            ctxB.line_search(th_h, X_h, tg_h, d_h, etas, th_next_h)
            th_h, th_next_h = th_next_h, th_h
        same_start = bool(np.array_equal(th_h, theta_start))
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            ctxB.step(th_h, X_h, tg_h, d_h, want_info=False)
            ctxB.line_search(th_h, X_h, tg_h, d_h, etas, th_next_h)
            th_h, th_next_h = th_next_h, th_h
        torch.cuda.synchronize(dev)
        e2e_ms = 1000.0 * (time.perf_counter() - t0) / args.steps
        e2e_same = {"same_start_theta": same_start, "same_end_theta": bool(np.array_equal(th_h, theta_late))}
        ctxB.close()

    # FP64 GPU path at theta_0 and at the late theta
    fp64 = None
    d64 = {}
    if not args.no_fp64:
        ctx64 = dngd.Context(dngd.make_desc(wl, precision=dngd.FP64, lambda_cap=cap), stream=stream.cuda_stream)
        ctx64.set_timing(True)
        dd = torch.zeros(n, dtype=torch.float64, device=dev)
        t64 = []
        i64 = None
        for name, th in (("theta0", th0), ("late", torch.tensor(theta_late, device=dev))):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            for k in range(args.fp64_steps):
                e0.record(stream)
                i64 = ctx64.step(th, X, tg, dd)
                ctx64.line_search(th, X, tg, dd, etas, theta_next)
                e1.record(stream)
                torch.cuda.synchronize(dev)
                t64.append(e0.elapsed_time(e1))
            d64[name] = (dd.cpu().numpy().copy(), i64)
        fp64 = {"steps_per_s": 1000.0 / float(np.mean(t64)), "ms_per_step": float(np.mean(t64)),
                "gram_ms": i64["phase_ms"][1], "phase_ms": i64["phase_ms"],
                "timed": f"{args.fp64_steps} step + line search at theta_0 and at the late theta each"}
        ctx64.close()

    # the oracle at the late theta, with the lambda the rule gives there
    ref_late, lam_late = None, None
    if do_oracle:
        from oracle import residual as ores
        wl_late = dict(wl)
        wl_late["theta"] = theta_late
        r_late = ores.residual(theta_late, ores.problem_from_spec(wl), wl["X"], wl["target"])
        lam_late = _lam_for(args, 0.5 * float(r_late @ r_late))
        ref_late, _ = oracle_full_step(wl_late, lam_late, with_kappa=True)

    def errs(ref, dmix, name, lam, info):
        out = {"lam": lam, "lam_gpu_mixed": info.get("lambda_used"), "ga_accepted_oracle": bool(ref["accepted"]),
               "refine_iters": info["solve_iters"], "shift": info["shift_used"]}
        nr = np.linalg.norm(ref["delta"])
        out["mixed_vs_oracle"] = float(np.linalg.norm(dmix - ref["delta"]) / nr)
        out["mixed_vs_oracle_entrywise"] = float(np.max(np.abs(dmix - ref["delta"]) /
                                                        (np.abs(ref["delta"]) + np.sqrt(np.mean(ref["delta"] ** 2)))))
        if name in d64:
            dd, ii = d64[name]
            out["fp64_vs_oracle"] = float(np.linalg.norm(dd - ref["delta"]) / nr)
            out["mixed_vs_fp64_gpu"] = float(np.linalg.norm(dmix - dd) / np.linalg.norm(dd))
        out["kappa_upper"], out["norm_K"] = ref.get("kappa_upper"), ref.get("norm_K")
        return out

    err = {}
    if ref0 is not None:
        err["theta0"] = errs(ref0, d_mixed0, "theta0", lam0, info0)
    if ref_late is not None:
        err["late"] = errs(ref_late, d_mixed_late, "late", lam_late, info_late)

    hbm, bf16_burst, bf16_sust, src = _peaks()
    alg_flops = float(m) * (m + 1) * n
    exec_flops = alg_flops * {dngd.MIXED_OZ: 13, dngd.MIXED_OZ64: 15}.get(prec, 1)
    # the product kernel alone (CUDA events around its launch)
    kern_ms = gram_kernel_ms if gram_kernel_ms > 0 else gram_ms
    achieved = alg_flops / (kern_ms * 1e-3) / 1e12
    executed = exec_flops / (kern_ms * 1e-3) / 1e12
    peak = bf16_sust / 2.0 if prec == dngd.MIXED_TF32 else bf16_sust
    # the refinement's J^T p / J u GEMVs over the FP32 J (BF16 / TF32 paths)
    jt_ms = float(np.mean([i["jt_ms"] for i in infos]))
    j_ms = float(np.mean([i["j_ms"] for i in infos]))
    gemv_bytes = 4.0 * m * n + 8.0 * (m + n)
    gemv_gbs = 2 * gemv_bytes / ((jt_ms + j_ms) * 1e-3) / 1e9 if jt_ms + j_ms > 0 else 0.0
    iters_total = float(np.mean([sum(i["solve_iters"]) for i in infos]))

    roof_gemv = {"bound": "hbm", "kernel": "k_gemv_t_f32 + k_gemv_n_f32 on the FP32 J (refinement operator / "
                                           "map-back J^T alpha)",
                 "achieved": gemv_gbs, "peak": hbm, "unit": "GB/s", "frac": gemv_gbs / hbm,
                 "bytes_per_launch": gemv_bytes, "launch_ms": [jt_ms, j_ms],
                 "launches_per_step": 2 * iters_total + 2,
                 "peak_source": f"{src} HBM copy bandwidth", "traffic": None}
    if prec in (dngd.MIXED_OZ, dngd.MIXED_OZ64):
        # the two refinement solves (persistent PCG: per iteration the double-float
        # Gram, 8 m^2 B, and both triangles of the FP32 inverse factor, 2 x 2 m^2 B)
        # plus each solve's map-back J^T x over the FP32 J (4 m n B), against the
        # solve phases' CUDA-event time
        solve_ms = float(np.mean([i["phase_ms"][3] + i["phase_ms"][5] for i in infos]))
        solve_bytes = iters_total * 12.0 * m * m + 2 * gemv_bytes * (2 if prec == dngd.MIXED_OZ64 else 1)
        solve_gbs = solve_bytes / (solve_ms * 1e-3) / 1e9 if solve_ms > 0 else 0.0
        mapback = "k_gemv_t (map-back J^T x over the FP64 J)" if prec == dngd.MIXED_OZ64 else \
            "k_gemv_t_f32 (map-back J^T x over the FP32 J)"
        roof_gemv = {"bound": "hbm", "kernel": f"k_pcg_persist (both solves) + {mapback}",
                     "achieved": solve_gbs, "peak": hbm, "unit": "GB/s", "frac": solve_gbs / hbm,
                     "bytes_per_step": solve_bytes, "solve_ms": solve_ms,
                     "algorithmic": "per PCG iteration 8 m^2 + 4 m^2 B (exact Gram operator, L^-1 and L^-T "
                                    "triangles); per solve 8 m n B (FP64 J) or 4 m n B (FP32 J) for J^T x",
                     "peak_source": f"{src} HBM copy bandwidth", "traffic": None}
        traffic = args.gram_traffic
        if traffic is None and args.workload == "poisson5d" and args.points <= 0:
            traffic = GRAM_TRAFFIC.get(args.precision)
        roof_gram = {"bound": "tensor",
                     "kernel": "k_gram_oz (exact Gram: tcgen05 BF16 products of 8-bit slices)",
                     "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                     "algorithmic": "m(m+1)n flop per Gram (the syrk of the 5-D workload, 2.135e12)",
                     "flops_per_launch": alg_flops, "launch_ms": kern_ms,
                     "phase_ms": gram_ms, "phase": "k_oz_slice + k_gram_oz (slicing and products)",
                     "executed_tflops": executed, "executed_frac": executed / peak,
                     "executed": ("15 m(m+1)n BF16 tensor flop (the 15 slice products of levels <= 5 of four "
                                  "slices)" if prec == dngd.MIXED_OZ64 else
                                  "13 m(m+1)n BF16 tensor flop (the 13 products of four slices)"),
                     "peak_source": f"{src} bf16 sustained",
                     "traffic": traffic,
                     "traffic_source": ("profiles/k_gram_oz_poisson5d_oz64.md (ncu dram__bytes_read.sum + "
                                        "dram__bytes_write.sum, one launch of the 5-D workload)")
                     if traffic is not None else None}
    else:
        roof_gram = {"bound": "tensor", "kernel": "k_gram_tc (tcgen05 syrk, lower 128x256 tiles)",
                     "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                     "flops_per_launch": alg_flops, "launch_ms": kern_ms, "phase_ms": gram_ms,
                     "peak_source": f"{src} bf16 sustained" + (" / 2 for tf32" if prec == dngd.MIXED_TF32 else ""),
                     "traffic": None}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": DTYPES[args.precision],
        "data": "synthetic",
        "config": {"workload": (WORKLOAD if args.points <= 0 else f"poisson5d with {args.points} points")
                               if args.workload == "poisson5d" else args.workload,
                   "lam": _lam_config(args),
                   "precision": f"mixed-{args.precision}",
                   "step": "dngd_step + 31-point line search + update",
                   "l2": L2_NOTE[args.precision],
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
        "gram_tflops": achieved, "fp64": fp64, "step_error": err,
        "speedup_vs_fp64": (value / world) / fp64["steps_per_s"] if fp64 else None,
        "refine_iters": iters, "phase_ms": phase,
        "per_step": [{"iters": i["solve_iters"], "shift": i["shift_used"], "factor_attempts": i["factor_attempts"],
                      "loss": i["loss"], "lam": i["lambda_used"], "ms": float(l)} for i, l in zip(infos, lat)],
        "ga_accepted_at_theta0": info0["ga_accepted"],
        "roofline": roof_gram if prec in (dngd.MIXED_OZ, dngd.MIXED_OZ64) else roof_gemv,
        "roofline_other": roof_gemv if prec in (dngd.MIXED_OZ, dngd.MIXED_OZ64) else roof_gram,
        "cpu_baseline": cpu,
        "e2e": {"value": 1000.0 / e2e_ms * world, "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h,
                "same_iterations_as_value": e2e_same},
        "gpu_launches": int(launches),
        "clocks": clk,
    }
    if rank == 0:
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
