#!/usr/bin/env python
"""Benchmark of the compressed H-matrix-vector product y += A~ x on GB300.

Workload (stand-in for the paper's Laplace single layer potential on the sphere, Section 5.1):
n = 262144 Fibonacci points on the unit sphere, kernel 1/(4 pi |x-y|) off the diagonal and the
mean off-diagonal row sum on it, bounding-box cluster tree with leaf size 64, standard
admissibility with eta = 2, ACA + SVD recompression at eps = 1e-6, dense leaves in AFL and
lowrank leaves in AFL-APLR; x ~ N(0,1) (seed 1). One step = one product (x permutation,
phase 1, phase 2). The compressed matrix (~1.6 GB) is far larger than L2 (129 MB), so every
step streams it from HBM.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
For N > 1 launch with torch.distributed.run: every rank runs an independent replica (the
product does not shard on one node here), value = bytes of all ranks / max time over ranks.
Prints one JSON line on rank 0.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "compressed H-matvec GB/s & % HBM peak vs plain FP64 H-matvec; p99 solve ms"
UNIT = "GB/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=262144)
    ap.add_argument("--eps", type=float, default=1e-6)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--quick", action="store_true", help="skip the FP64/plain/multi-RHS/format/serve legs")
    ap.add_argument("--no-serve", action="store_true", help="skip the short serving leg")
    ap.add_argument("--tune", action="store_true",
                    help="time the autotuner's candidate layouts and launch shapes on the matrix and run the "
                         "headline with the fastest (reported under 'autotuned')")
    ap.add_argument("--acc", default="fp32", choices=["fp32", "fp64"],
                    help="accumulation of the headline product: fp32 in-block / fp64 across blocks (default), "
                         "or fp64 throughout (the paper's arithmetic)")
    ap.add_argument("--workload", default="laplace", choices=["laplace", "batch48", "serve", "small", "scale", "multi"],
                    help="laplace: one n=262144 sphere matrix (default); batch48: 48 Matern matrices of "
                         "uneven size with 1/8/32 right-hand sides in one batched launch sequence; serve: "
                         "Poisson requests (70%% products, 30%% CG solves) against resident Matern matrices; "
                         "small: n=4096 2D exponential kernel, latency with L2 flushed; scale: n=2^21 sphere, "
                         "1 and 32 right-hand sides")
    ap.add_argument("--serve-mats", type=int, default=16)
    ap.add_argument("--serve-min-n", type=int, default=16384)
    ap.add_argument("--serve-max-n", type=int, default=262144)
    ap.add_argument("--serve-requests", type=int, default=64, help="requests per arrival rate")
    ap.add_argument("--serve-rates", default="20,100,500", help="arrival rates (requests/s) to sweep")
    ap.add_argument("--serve-budget-gb", type=float, default=150.0)
    ap.add_argument("--serve-solve-frac", type=float, default=0.3, help="share of CG solves among the requests")
    return ap.parse_args()


def workload_config(args, world: int) -> dict:
    accs = "FP32 in-block / FP64 cross-block" if getattr(args, "acc", "fp32") == "fp32" else "FP64 throughout"
    return {"workload": f"laplace-sphere n={args.n} eps={args.eps:g} AFL-APLR, {accs}",
            "n": args.n, "eps": args.eps, "kernel": "1/(4 pi r), diag = mean row sum", "points": "fibonacci sphere",
            "leaf_size": 64, "eta": 2.0, "lowrank": "ACA + SVD recompression", "rhs": 1,
            "l2": "inputs larger than L2 (compressed matrix ~1.6 GB >> 129 MB)",
            "parallelism": f"replicas x{world}" if world > 1 else "single GPU"}


# ------------------------------------------------------------------------------------------
# distributed helpers (also exercised by a 2-rank gloo test on CPU)
# ------------------------------------------------------------------------------------------
def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def aggregate(elapsed_s: float, units: float, world: int):
    """(max elapsed over ranks, sum of units over ranks); a no-op for one process."""
    if world <= 1:
        return elapsed_s, units
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([elapsed_s], dtype=torch.float64, device=dev)
    u = torch.tensor([units], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# ------------------------------------------------------------------------------------------
# clocks during the timed region
# ------------------------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join("/tmp", f"hlr_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for ln in f:
                parts = [p.strip() for p in ln.split(",")]
                if len(parts) < 8:
                    continue
                try:
                    sm.append(float(parts[0]))
                    smax.append(float(parts[1]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[4:8]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)), "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks() -> dict:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return {"hbm_gbs": float(d["hbm_gbs"]), "source": "measured"}
    return {"hbm_gbs": 6800.0, "source": "fallback"}


def recorded_traffic(kernel: str, alg_bytes: float, eps: float) -> float | None:
    """DRAM bytes per launch of `kernel` from the committed ncu capture: its traffic / algorithmic
    ratio times this launch's algorithmic bytes (traffic grows with the units a launch processes),
    if the capture was taken on the current kernel source (matched by the source hash recorded
    beside it) and at the same eps (the code widths set the padding). None otherwise."""
    import hashlib
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    src = os.path.join(ROOT, "paper_2308_10960_gb300", "csrc", "hlr_kernels.cu")
    h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    e = d.get(kernel)
    if not e or e.get("source_sha256_16") != h or abs(e.get("captured_eps", -1.0) - eps) > 1e-12 * eps:
        return None
    return float(e["traffic_over_algorithmic"]) * alg_bytes


def multi_rhs_bytes(info: dict, n: int, r: int) -> float:
    """Algorithmic bytes of Y += A~ X with r columns: the compressed streams, headers and Sigma
    once, the permutation once, and 8n (x) + 16n (y read and write) per column."""
    return float(info["algorithmic_bytes"]) - 32.0 * n + 8.0 * n + r * 24.0 * n


# ------------------------------------------------------------------------------------------
# CPU baseline and the reference arm: the C oracle (oracle/cmatvec.c) on the host cores
# ------------------------------------------------------------------------------------------
def c_oracle_matrix(Hh, eps):
    """The benchmark matrix compressed by the C oracle's own encoder (from the FP64 blocks the
    host builder made; the oracle shares no code with the GPU library)."""
    from oracle import cbaseline as cb
    t0 = time.perf_counter()
    M = cb.CMatrix(Hh.n, Hh.perm, Hh.block_views(), eps)
    return M, time.perf_counter() - t0


def c_oracle_rate(M, x, plain: bool, threads: int, reps: int, budget_s: float):
    """Median GB/s of y += A~ x by the C oracle over up to `reps` products (fewer if one
    product takes long, at least one), with the product's algorithmic bytes."""
    y = np.zeros(M.n)
    times = []
    t_start = time.perf_counter()
    for _ in range(reps):
        y[:] = 0.0
        t0 = time.perf_counter()
        M.matvec(x, y, plain=plain, threads=threads)
        times.append(time.perf_counter() - t0)
        if time.perf_counter() - t_start > budget_s:
            break
    med = float(np.median(times))
    return M.algorithmic_bytes(plain) / med / 1e9, med, len(times), y


def cpu_baseline(args, Hh, x, y_ref) -> dict:
    """The C oracle's compressed H-matvec (decoding on the fly) and its plain FP64 H-matvec over
    the same matrix, on all host cores and on one core, median of 10 products (fewer on one
    core when a product takes seconds)."""
    M, t_enc = c_oracle_matrix(Hh, args.eps)
    nproc = os.cpu_count() or 1
    out = {}
    for plain in (False, True):
        key = "plain_fp64" if plain else "compressed"
        gbs, med, k, y = c_oracle_rate(M, x, plain, nproc, 10, 20.0)
        gbs1, med1, k1, _ = c_oracle_rate(M, x, plain, 1, 10, 20.0)
        out[key] = {"GB/s_all_cores": gbs, "ms_all_cores": med * 1e3, "runs_all_cores": k,
                    "GB/s_one_core": gbs1, "ms_one_core": med1 * 1e3, "runs_one_core": k1}
        if not plain:
            out[key]["rel_diff_vs_gpu_fp64"] = float(np.linalg.norm(y - y_ref) / np.linalg.norm(y_ref))
    M.free()
    c = out["compressed"]
    return {"value": c["GB/s_all_cores"], "unit": UNIT, "cores": nproc, "kind": "oracle",
            "sample": f"C oracle (oracle/cmatvec.c, OpenMP, decodes every unit when used; its own AFL-APLR "
                      f"encoder) over the whole benchmark matrix (n={args.n}, eps={args.eps:g}), median of "
                      f"{c['runs_all_cores']} products on {nproc} threads; encoding took {t_enc:.1f} s (untimed)",
            "one_core": {"value": c["GB/s_one_core"], "runs": c["runs_one_core"]},
            "plain_fp64": out["plain_fp64"], "compressed": c}


def run_reference(args, world: int, rank: int):
    """The reference arm: the C oracle's compressed product over the same workload on the host
    cores (the matrix is built by the library's host builder and encoded by the oracle, both
    untimed); each step is one whole product."""
    if rank != 0:
        return
    import synth
    import paper_2308_10960_gb300 as hg
    prob = synth.laplace_problem(args.n)
    Hh = hg.build_kernel_hmatrix(prob.points, "laplace", args.eps, diag=prob.params["diag"], eta=2.0, leaf_size=64)
    M, t_enc = c_oracle_matrix(Hh, args.eps)
    x = synth.rhs(args.n, 1)
    y = np.zeros(args.n)
    nproc = os.cpu_count() or 1
    for _ in range(args.warmup):
        M.matvec(x, y, threads=nproc)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        M.matvec(x, y, threads=nproc)
    dt = time.perf_counter() - t0
    v = M.algorithmic_bytes() * args.steps / dt / 1e9
    sample = (f"C oracle (oracle/cmatvec.c, OpenMP on {nproc} threads) compressed H-matvec over the whole "
              f"n={args.n}, eps={args.eps:g} matrix; each step one product")
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": workload_config(args, world),
           "cpu_baseline": {"value": v, "unit": UNIT, "cores": nproc, "kind": "oracle", "sample": sample},
           "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
           "gpu_launches": 0}
    M.free()
    Hh.free()
    print(json.dumps(out), flush=True)


# ------------------------------------------------------------------------------------------
# our arm
# ------------------------------------------------------------------------------------------
def time_loop(fn, steps: int, stream):
    import torch
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(steps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / 1e3


def fp64_peak_tflops(dev) -> dict:
    """Dense FP64 rate of this GPU, measured: cuBLAS DGEMM (torch.matmul, 4096^3) best of 5."""
    import torch
    a = torch.randn(4096, 4096, dtype=torch.float64, device=dev)
    b = torch.randn(4096, 4096, dtype=torch.float64, device=dev)
    for _ in range(2):
        a @ b
    best = 1e30
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    for _ in range(5):
        e0.record()
        a @ b
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1) / 1e3)
    return {"tflops": 2.0 * 4096 ** 3 / best / 1e12, "how": "torch.matmul float64 4096^3 (cuBLAS DGEMM), best of 5"}


def kernel_table(A, info, n, stream, calls, step, peak_gbs, eps, acc="fp32", layout=0):
    """Per-kernel CUDA-event times from a separate profiled loop of `calls` products (the timed
    headline loop records no events) and the roofline of the dominant kernel."""
    A.profile_read()
    for _ in range(calls):
        step(True)
    kms, got = A.profile_read()
    tag = "AFL32" if acc == "fp32" else "AFL64"
    names = ["k_permute", f"k_phase1<{tag}>", f"k_phase2<{tag}>", "k_scatter"]
    # algorithmic bytes per launch: x read + two permuted copies written (permute); phase 1 as
    # hlr_info; phase 2 without the y and perm traffic that k_scatter does (8n y read, 8n y
    # written, 8n perm; phase 2 writes its row totals, 8n, which are not algorithmic)
    kb = [16.0 * n, float(info["phase1_bytes"]), float(info["phase2_bytes"]) - 24.0 * n, 24.0 * n]
    avg = [m / max(got, 1) for m in kms]
    dom = int(np.argmax(avg))
    achieved = kb[dom] / (avg[dom] / 1e3) / 1e9
    # the recorded ratio belongs to the default work layout (a tuned layout packs other pieces)
    tr = recorded_traffic(names[dom], kb[dom], eps) if layout == 0 else None
    return {"bound": "hbm", "kernel": names[dom], "achieved": achieved, "peak": peak_gbs["hbm_gbs"], "unit": "GB/s",
            "frac": achieved / peak_gbs["hbm_gbs"], "traffic": tr,
            "peak_source": f"{peak_gbs['source']} copy bandwidth (MEASURED_PEAKS.json hbm_gbs)",
            "algorithmic_bytes_per_launch": kb[dom],
            "kernel_ms_avg": dict(zip(names, avg)), "kernel_share": dict(zip(names, [m / max(sum(avg), 1e-12) for m in avg])),
            "profiled_products": got,
            "kernel_GB/s": {nm: (b / (t / 1e3) / 1e9 if t > 0 else None) for nm, b, t in zip(names, kb, avg)}}


def serve_leg(dev, eps: float) -> dict:
    """A short served run: 6 resident Matern matrices (n 16384 .. 65536), 60 Poisson requests at
    200 requests/s, 30 % CG solves to a relative residual of 1e-8: p50/p99 latency per kind."""
    import torch
    import synth
    import paper_2308_10960_gb300 as hg
    from paper_2308_10960_gb300 import serve
    sizes = [int(round(16384 * 4.0 ** (i / 5))) for i in range(6)]
    host = {}
    for i, n in enumerate(sizes):
        p = synth.matern_problem(n, seed=200 + i)
        host[f"m{i}"] = hg.build_kernel_hmatrix(p.points, "matern15", eps, scale=p.params["scale"], diag=p.params["diag"])
    be = serve.GpuBackend(host)
    names = sorted(host, key=lambda m: int(m[1:]))
    srv = serve.Server(be, budget_bytes=int(150e9), cg_workers=4, max_rhs=32)
    srv.preload(names)
    warm = []
    for i, m in enumerate(names):
        xw = torch.from_numpy(synth.rhs(host[m].n, 9000 + i)).to(dev)
        warm.append(serve.Request(-1 - 2 * i, "matvec", m, xw, arrival=0.0))
        warm.append(serve.Request(-2 - 2 * i, "solve", m, xw, arrival=0.0, rtol=1e-8, maxit=3))
    torch.cuda.synchronize()
    srv.run(warm, realtime=False)
    g = np.random.default_rng(6)
    arr = serve.poisson_arrivals(60, 200.0, 5)
    plan = []
    for i in range(60):
        m = names[int(g.integers(len(names)))]
        plan.append((i, "solve" if g.random() < 0.3 else "matvec", m, arr[i]))
    xs = {i: torch.from_numpy(synth.rhs(host[m].n, 7000 + i)).to(dev) for i, _, m, _ in plan}

    ys = {i: torch.zeros_like(x) for i, x in xs.items()}    # the clients' output buffers

    def requests(kinds):
        return [serve.Request(i, k, m, xs[i], arrival=a, rtol=1e-8, maxit=50000, y=ys[i])
                for i, k, m, a in plan if k in kinds]
    # the same product requests at the same arrival times with no solves running: the latency
    # a product has alone, against which the mixed run's product latency is read
    torch.cuda.synchronize()
    alone = srv.run(requests(("matvec",))).as_dict()["latency_ms"].get("matvec")
    reqs = requests(("matvec", "solve"))
    torch.cuda.synchronize()
    st = srv.run(reqs).as_dict()
    be.close()
    for h in host.values():
        h.free()
    lat = st["latency_ms"]
    prod = lat.get("matvec")
    return {"workload": f"6 resident Matern nu=1.5 matrices n {sizes[0]}..{sizes[-1]}, eps={eps:g}, 60 Poisson "
                        f"requests at 200/s, 30% CG solves to 1e-8",
            "products_ms": prod, "products_alone_ms": alone,
            "products_p99_vs_alone": (prod["p99"] / alone["p99"]) if prod and alone else None,
            "solves_ms": lat.get("solve"), "requests_per_s": st["requests_per_s"],
            "GB/s": st["GB/s"], "failed": st["failed"],
            "cg_true_relres_max": float(max([r.relres for r in reqs if r.kind == "solve"] or [0]))}


def run_ours(args, world: int, rank: int, local: int):
    import torch
    import synth
    import paper_2308_10960_gb300 as hg

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    t_setup = time.perf_counter()
    prob = synth.laplace_problem(args.n)
    Hh = hg.build_kernel_hmatrix(prob.points, "laplace", args.eps, diag=prob.params["diag"], eta=2.0, leaf_size=64)
    t_build = time.perf_counter() - t_setup
    tuned = None
    code = 0
    if args.tune:
        from paper_2308_10960_gb300 import tune
        tt = time.perf_counter()
        res = tune.Autotuner(reps=20).tune(Hh, 1)
        code = hg.tuning_code(*res.best)
        tuned = {"choice (sub, leaf, piece KiB, CTAs/SM)": list(res.best), "tune_s": time.perf_counter() - tt,
                 "ms": {",".join(map(str, k)): round(v, 4) for k, v in res.ms.items()}}
    A = Hh.upload("afl", tuning=code)
    info = A.info
    x = torch.from_numpy(synth.rhs(args.n, 1)).to(dev)
    y = torch.zeros(args.n, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)
    bytes_step = float(info["algorithmic_bytes"])

    def step32(profile=False):
        A.matvec(x, y, acc=args.acc, stream=stream, profile=profile)

    for _ in range(max(3, args.warmup)):
        step32()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    barrier(world)
    el = time_loop(step32, args.steps, stream)       # the headline: no events inside the loop
    barrier(world)
    clk = clocks.stop()
    A.check()
    el_max, total_bytes = aggregate(el, bytes_step * args.steps, world)
    value = total_bytes / el_max / 1e9
    ms_step = el_max / args.steps * 1e3
    peaks = measured_peaks()
    roofline = kernel_table(A, info, args.n, stream, min(200, max(20, args.steps)), step32, peaks, args.eps, args.acc,
                            code)

    extra = {}
    y64 = None
    if not args.quick:
        steps_cmp = max(20, min(200, args.steps // 4))

        def step64(profile=False):
            A.matvec(x, y, acc="fp64", stream=stream, profile=profile)
        for _ in range(3):
            step64()
        el64 = time_loop(step64, steps_cmp, stream)
        A.profile_read()
        for _ in range(10):
            step64(True)
        kms64, c64 = A.profile_read()
        t64 = el64 / steps_cmp
        f64 = fp64_peak_tflops(dev)
        yv = torch.zeros(args.n, dtype=torch.float64, device=dev)
        A.matvec(x, yv, acc="fp64", stream=stream)
        torch.cuda.synchronize()
        y64 = yv.cpu().numpy()
        values = float(info["values"])
        ph2_64 = kms64[2] / max(c64, 1)
        extra["afl_fp64_acc"] = {
            "ms_per_step": t64 * 1e3, "GB/s": bytes_step / t64 / 1e9,
            "kernel_ms_avg": {"k_permute": kms64[0] / max(c64, 1), "k_phase1<AFL64>": kms64[1] / max(c64, 1),
                              "k_phase2<AFL64>": ph2_64},
            "roofline": {"bound": "fp64", "achieved": 2.0 * values / t64 / 1e12, "peak": f64["tflops"],
                         "unit": "TFLOP/s", "frac": 2.0 * values / t64 / 1e12 / f64["tflops"],
                         "peak_source": "measured here: " + f64["how"],
                         "note": "one FP64 multiply-add per decoded value is the product's algorithmic FP64 work",
                         "hbm": {"achieved": bytes_step / t64 / 1e9, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                                 "frac": bytes_step / t64 / 1e9 / peaks["hbm_gbs"]}}}
        Ap = Hh.upload("fp64")
        infp = Ap.info

        def stepp():
            Ap.matvec(x, y, acc="fp64", stream=stream)
        for _ in range(3):
            stepp()
        tp = time_loop(stepp, steps_cmp, stream) / steps_cmp
        Ap.free()
        t32 = el / args.steps
        multi = {}
        for r in (8, 32):
            X = torch.from_numpy(synth.rhs(args.n * r, 2 + r)).to(dev).view(r, args.n)
            Y = torch.zeros((r, args.n), dtype=torch.float64, device=dev)

            def stepm():
                hg.matvec_batched([A], [X], [Y], acc="fp32", stream=stream)
            for _ in range(3):
                stepm()
            km = max(10, steps_cmp // 8)
            tm = time_loop(stepm, km, stream) / km
            bm = multi_rhs_bytes(info, args.n, r)
            multi[str(r)] = {"ms_per_step": tm * 1e3, "GB/s": bm / tm / 1e9, "algorithmic_bytes": bm,
                             "speedup_vs_r_single_products": r * t32 / tm}
            if r == 32:
                # FP64 accumulation of 32 columns: 32 single-RHS FP64 products in one batched launch,
                # beside the floor of any FP64 contraction of the decoded values at the measured
                # DGEMM rate (2 r flops per value)
                def stepm64():
                    hg.matvec_batched([A], [X], [Y], acc="fp64", stream=stream)
                for _ in range(3):
                    stepm64()
                km64 = max(3, km // 4)
                tm64 = time_loop(stepm64, km64, stream) / km64
                floor = 2.0 * r * float(info["values"]) / (f64["tflops"] * 1e12)
                multi["32_fp64"] = {"ms_per_step": tm64 * 1e3, "vs_32_fp64_single_products": r * t64 / tm64,
                                    "vs_fp32_pass": tm64 / tm,
                                    "dgemm_rate_floor_ms": floor * 1e3,
                                    "note": "floor = 2 x 32 x decoded values / measured DGEMM rate: no FP64 "
                                            "contraction of the decoded values runs faster than that rate"}
            del X, Y
        A.check()
        formats = {}
        for fmt in ("aflp", "bfl", "dfl", "mp"):
            Af = Hh.upload(fmt)
            inf_f = Af.info

            def stepf():
                Af.matvec(x, y, acc="fp32", stream=stream)
            for _ in range(3):
                stepf()
            kf = max(20, steps_cmp // 4)
            tf = time_loop(stepf, kf, stream) / kf
            Af.check()
            comp = inf_f["stream_bytes"] + inf_f["header_bytes"] + 8 * inf_f["rank_sum"]
            formats[fmt] = {"ms_per_step": tf * 1e3, "GB/s": inf_f["algorithmic_bytes"] / tf / 1e9,
                            "compressed_bytes": comp, "ratio": comp / inf_f["fp64_bytes"],
                            "speedup_vs_afl": t32 / tf}
            Af.free()
        # GPU encoder (hlr_encode_device) over every unit of the matrix, against the build time
        # (the paper reports compression time relative to construction, Section 5.3)
        vals, off, prec = Hh.unit_arrays("afl")
        v_d = torch.from_numpy(vals).to(dev)
        o_d = torch.from_numpy(off).to(dev)
        u_d = torch.from_numpy(prec).to(dev)
        del vals
        enc = hg.encode_device(v_d, o_d, u_d, "afl", stream=stream)
        torch.cuda.synchronize()
        out_bytes = int(enc[3][-1].item())
        rejected = int((enc[1] < 0).sum().item())
        del enc
        ke = 5
        te = time_loop(lambda: hg.encode_device(v_d, o_d, u_d, "afl", stream=stream), ke, stream) / ke
        in_bytes = v_d.numel() * 8
        encode = {"ms": te * 1e3, "units": int(u_d.numel()), "input_bytes": in_bytes, "output_bytes": out_bytes,
                  "input_GB/s": in_bytes / te / 1e9, "hbm_GB/s_algorithmic": (in_bytes + out_bytes) / te / 1e9,
                  "rejected_units": rejected, "vs_build_time": te / t_build}
        del v_d, o_d, u_d
        torch.cuda.empty_cache()
        # the whole upload (encode, re-place, copy) with the host encoder and with compression on
        # the GPU during the upload (HLR_ENCODE_DEVICE): wall clock, same matrix bytes
        for how, dev_enc in (("host_encode", False), ("device_encode", True)):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            Au = Hh.upload("afl", encode_device=dev_enc)
            torch.cuda.synchronize()
            encode[f"upload_s_{how}"] = time.perf_counter() - t0
            assert Au.info["stream_bytes"] == info["stream_bytes"]
            Au.free()
        extra.update({
            "encode_device": encode,
            "formats": formats,
            "multi_rhs": multi,
            "plain_fp64": {"ms_per_step": tp * 1e3, "GB/s": infp["algorithmic_bytes"] / tp / 1e9,
                           "algorithmic_bytes": infp["algorithmic_bytes"],
                           "pct_hbm": infp["algorithmic_bytes"] / tp / 1e9 / peaks["hbm_gbs"]},
            "speedup_vs_plain_fp64": tp / t32,
            "speedup_fp64acc_vs_plain_fp64": tp / t64,
        })

    # end to end through the C-ABI call with host buffers
    xh = torch.from_numpy(synth.rhs(args.n, 1)).pin_memory()
    yh = torch.zeros(args.n, dtype=torch.float64).pin_memory()
    for _ in range(3):
        A.matvec_host(xh, yh, acc="fp32", stream=stream)
    steps_e2e = max(50, min(500, args.steps // 4))
    t0 = time.perf_counter()
    for _ in range(steps_e2e):
        A.matvec_host(xh, yh, acc="fp32", stream=stream)
    te = (time.perf_counter() - t0) / steps_e2e
    te_max, _ = aggregate(te, 0.0, world)
    e2e = {"value": world * bytes_step / te_max / 1e9, "unit": UNIT, "h2d_bytes_per_step": 16 * args.n,
           "d2h_bytes_per_step": 8 * args.n, "ms_per_step": te_max * 1e3,
           "api": "hlr_matvec_host (pinned host x, y; copies inside the timed region)"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        if y64 is None:
            yv = torch.zeros(args.n, dtype=torch.float64, device=dev)
            A.matvec(x, yv, acc="fp64", stream=stream)
            torch.cuda.synchronize()
            y64 = yv.cpu().numpy()
        cpu = cpu_baseline(args, Hh, x.cpu().numpy(), y64)
    serving = None
    if rank == 0 and not args.quick and not args.no_serve:
        serving = serve_leg(dev, 1e-6)

    if rank == 0:
        out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
               "vs_baseline": None, "dtype": "f32" if args.acc == "fp32" else "f64", "data": "synthetic",
               "config": {**workload_config(args, world),
                          "work_layout": "autotuned " + str(tuned["choice (sub, leaf, piece KiB, CTAs/SM)"]) if tuned
                          else "default (64-row X lanes, 64-row tasks, 16 KiB pieces, resident CTAs/SM)"},
               "pct_hbm_peak": value / world / peaks["hbm_gbs"], "pct_hbm_8tbs_spec": value / world / 8000.0,
               "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clk,
               "gpu_launches": int(info["launches"]) * args.steps,
               "p99_solve_ms": (serving or {}).get("solves_ms", {}) and serving["solves_ms"].get("p99"),
               "serve": serving, "autotuned": tuned,
               "matrix": {"nblocks": info["nblocks"], "rank_sum": info["rank_sum"],
                          "compressed_bytes": info["stream_bytes"] + info["header_bytes"] + 8 * info["rank_sum"],
                          "fp64_bytes": info["fp64_bytes"],
                          "ratio": (info["stream_bytes"] + info["header_bytes"] + 8 * info["rank_sum"]) /
                                   info["fp64_bytes"],
                          "algorithmic_bytes_per_step": bytes_step, "build_s": t_build},
               **extra}
        print(json.dumps(out), flush=True)
    A.free()
    Hh.free()


def run_batch(args, world: int, rank: int, local: int):
    """48 Matern matrices (n log-uniform in [8192, 131072], seed 3; points seed 100 + i), eps from
    --eps, right-hand-side counts from {1, 8, 32} (seed 4), X ~ N(0,1): every step is ONE
    hlr_matvec_batched call over all 48 requests, replayed from a captured CUDA graph.
    value = sum of the requests' algorithmic bytes / time."""
    import torch
    import synth
    import paper_2308_10960_gb300 as hg

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    sizes = synth.batch_sizes(48)
    nrhs = synth.batch_nrhs(48)
    from paper_2308_10960_gb300 import tune
    t0 = time.perf_counter()
    tuner = tune.Autotuner(reps=10)
    tuned, t_tune = {}, 0.0
    mats, Xs, Ys, bytes_step, rhs_single = [], [], [], 0.0, 0.0
    for i, (n, r) in enumerate(zip(sizes, nrhs)):
        p = synth.matern_problem(n, seed=100 + i)
        Hh = hg.build_kernel_hmatrix(p.points, "matern15", args.eps, scale=p.params["scale"], diag=p.params["diag"])
        tt = time.perf_counter()
        code, rc, res = tuner.choose(Hh, r)      # work layout and launch shape per rank class
        t_tune += time.perf_counter() - tt
        if res is not None:
            tuned[f"rank~{rc[0]} x{rc[1]} cols"] = {"choice (sub, leaf, piece KiB, CTAs/SM)": list(res.best),
                                                    "tuned_on_n": n,
                                                    "ms": {",".join(map(str, k)): round(v, 4) for k, v in res.ms.items()}}
        A = Hh.upload("afl", tuning=code)
        Hh.free()
        mats.append(A)
        Xs.append(torch.from_numpy(synth.rhs(n * r, 1000 + i)).to(dev).view(r, n) if r > 1
                  else torch.from_numpy(synth.rhs(n, 1000 + i)).to(dev))
        Ys.append(torch.zeros_like(Xs[-1]))
        bytes_step += multi_rhs_bytes(A.info, n, r) if r > 1 else float(A.info["algorithmic_bytes"])
    t_build = time.perf_counter() - t0
    stream = torch.cuda.Stream(dev)
    stream.wait_stream(torch.cuda.current_stream(dev))
    with torch.cuda.stream(stream):
        for _ in range(max(3, args.warmup)):
            hg.matvec_batched(mats, Xs, Ys, acc="fp32", stream=stream)
    torch.cuda.synchronize()
    eager_el = time_loop(lambda: hg.matvec_batched(mats, Xs, Ys, acc="fp32", stream=stream), args.steps, stream)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        hg.matvec_batched(mats, Xs, Ys, acc="fp32")
    with torch.cuda.stream(stream):
        for _ in range(3):
            g.replay()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    barrier(world)
    def replay():
        with torch.cuda.stream(stream):
            g.replay()
    el = time_loop(replay, args.steps, stream)
    barrier(world)
    clk = clocks.stop()
    for A in mats:
        A.check()
    el_max, total = aggregate(el, bytes_step * args.steps, world)
    peaks = measured_peaks()
    if rank == 0:
        value = total / el_max / 1e9
        # kernels per batched call: per class (single-RHS FP32; wide passes of 32 columns;
        # narrow passes of at most 8) and group of <= 64 products: permute, phase 1, combine,
        # phase 2, and for the single-RHS class the scatter of the row totals (a group never
        # holds one handle's pass twice, which the 48 distinct matrices never ask for)
        n_single = sum(1 for r in nrhs if r == 1)
        n_wide = sum(r // 32 + (1 if r % 32 > 8 else 0) for r in nrhs if r > 1)
        n_narrow = sum(1 for r in nrhs if r > 1 and 0 < r % 32 <= 8)
        n_pass = n_wide + n_narrow
        launches = 5 * ((n_single + 63) // 64) + 4 * ((n_wide + 63) // 64 + (n_narrow + 63) // 64)
        out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": el_max / args.steps * 1e3, "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
               "config": {"workload": f"batch of 48 Matern nu=1.5 matrices, n log-uniform [8192, 131072], "
                                      f"eps={args.eps:g}, 1/8/32 RHS, one batched call per step (CUDA graph)",
                          "sizes": sizes, "nrhs": nrhs, "single_rhs_requests": n_single, "rhs_passes": n_pass,
                          "l2": "inputs larger than L2", "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
               "pct_hbm_peak": value / world / peaks["hbm_gbs"],
               "eager_ms_per_step": eager_el / args.steps * 1e3,
               "autotuned": tuned, "tune_s": t_tune,
               "algorithmic_bytes_per_step": bytes_step, "build_s": t_build, "clocks": clk,
               "gpu_launches": launches * args.steps}
        print(json.dumps(out), flush=True)
    for A in mats:
        A.free()


def run_serve(args, world: int, rank: int, local: int):
    """Serving: --serve-mats Matern matrices (n log-spaced in [--serve-min-n, --serve-max-n],
    points seed 200 + i) resident under an HBM budget; for every arrival rate a Poisson stream
    (seed 5) of --serve-requests requests, CG solves to 1e-8 with probability --serve-solve-frac
    (default 0.3) and products otherwise, over the matrices uniformly (seed 6). value = products'
    and solves' algorithmic bytes / makespan at the highest rate; p50/p99 latency per rate and
    kind."""
    import torch
    import synth
    import paper_2308_10960_gb300 as hg
    from paper_2308_10960_gb300 import serve

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    k = args.serve_mats
    sizes = [int(round(math.exp(math.log(args.serve_min_n) + (math.log(args.serve_max_n) - math.log(args.serve_min_n))
                                * i / max(1, k - 1)))) for i in range(k)]
    t0 = time.perf_counter()
    host = {}
    for i, n in enumerate(sizes):
        p = synth.matern_problem(n, seed=200 + i)
        host[f"m{i}"] = hg.build_kernel_hmatrix(p.points, "matern15", args.eps, scale=p.params["scale"],
                                                diag=p.params["diag"])
    t_build = time.perf_counter() - t0
    # work layout and launch shape per rank class, timed as the server runs products (single
    # columns through the pass kernels)
    from paper_2308_10960_gb300 import tune
    tuner = tune.Autotuner(reps=10, multi=True)
    tunings, tuned = {}, {}
    tt = time.perf_counter()
    for name in sorted(host, key=lambda m: int(m[1:])):
        code, rc, res = tuner.choose(host[name], 1)
        tunings[name] = code
        if res is not None:
            tuned[f"rank~{rc[0]}"] = {"choice (sub, leaf, piece KiB, CTAs/SM)": list(res.best), "tuned_on": name,
                                      "ms": {",".join(map(str, k)): round(v, 4) for k, v in res.ms.items()}}
    t_tune = time.perf_counter() - tt
    be = serve.GpuBackend(host, tunings=tunings)
    budget = int(args.serve_budget_gb * 1e9)
    names = sorted(host, key=lambda m: int(m[1:]))
    rates = [float(r) for r in args.serve_rates.split(",")]
    g = np.random.default_rng(6)
    per_rate = {}
    last = None
    clocks = ClockSampler(local)
    clocks.start()
    for ri, rate in enumerate(rates):
        arr = serve.poisson_arrivals(args.serve_requests, rate, 5 + ri)
        reqs = []
        for i in range(args.serve_requests):
            m = names[int(g.integers(len(names)))]
            kind = "solve" if g.random() < args.serve_solve_frac else "matvec"
            x = torch.from_numpy(synth.rhs(host[m].n, 7000 + 100 * ri + i)).to(dev)
            reqs.append(serve.Request(i, kind, m, x, arrival=arr[i], rtol=1e-8, maxit=50000, y=torch.zeros_like(x)))
        torch.cuda.synchronize()
        srv = serve.Server(be, budget_bytes=budget, cg_workers=4, max_rhs=32)
        srv.preload(names)           # the matrices are resident before the requests arrive
        if ri == 0:
            # warm-up, untimed: every matrix takes one product and a few CG iterations, so that
            # kernels are loaded and per-matrix scratch exists before the first timed request
            warm = []
            for i, m in enumerate(names):
                xw = torch.from_numpy(synth.rhs(host[m].n, 9000 + i)).to(dev)
                warm.append(serve.Request(-1 - 2 * i, "matvec", m, xw, arrival=0.0))
                warm.append(serve.Request(-2 - 2 * i, "solve", m, xw, arrival=0.0, rtol=1e-8, maxit=3))
            torch.cuda.synchronize()
            srv.run(warm, realtime=False)
        torch.cuda.synchronize()
        st = srv.run(reqs)
        d = st.as_dict()
        d["cg_iterations_mean"] = float(np.mean([r.iters for r in reqs if r.kind == "solve"] or [0]))
        d["cg_true_relres_max"] = float(max([r.relres for r in reqs if r.kind == "solve"] or [0]))
        per_rate[str(rate)] = d
        last = d
    clk = clocks.stop()
    if rank == 0:
        peaks = measured_peaks()
        solve_p99 = last["latency_ms"].get("solve", {}).get("p99")
        out = {"metric": METRIC, "value": last["GB/s"] * world, "unit": UNIT, "n_gpus": world,
               "steps": args.serve_requests, "warmup": 0, "ms_per_step": last["makespan_s"] * 1e3 / args.serve_requests,
               "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
               "config": {"workload": f"serving {k} Matern nu=1.5 matrices n {sizes[0]}..{sizes[-1]}, eps={args.eps:g}, "
                                      f"Poisson arrivals, {100 - 100 * args.serve_solve_frac:g}% products / "
                                      f"{100 * args.serve_solve_frac:g}% CG to 1e-8, budget {args.serve_budget_gb:g} GB",
                          "sizes": sizes, "rates": rates, "requests_per_rate": args.serve_requests,
                          "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
               "p99_solve_ms": solve_p99, "per_rate": per_rate, "pct_hbm_peak": last["GB/s"] / peaks["hbm_gbs"],
               "build_s": t_build, "clocks": clk, "autotuned": tuned, "tune_s": t_tune,
               "resident_bytes": {m: be.device_bytes(m) for m in names}}
        print(json.dumps(out), flush=True)
    be.close()


def run_small(args, world: int, rank: int, local: int):
    """n = 4096 points uniform in [0,1]^2 (seed 0), exp(-r/0.2) + 1e-2 I, eps from --eps: the
    whole compressed matrix fits in L2, so L2 is flushed (a 256 MB buffer is written) before
    every product and each product is timed alone with CUDA events; the median latency is
    reported (value = algorithmic bytes / median time)."""
    import torch
    import synth
    import paper_2308_10960_gb300 as hg

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    p = synth.exp2d_problem(4096, seed=0)
    Hh = hg.build_kernel_hmatrix(p.points, "exp2d", args.eps, scale=p.params["scale"], diag=p.params["diag"])
    A = Hh.upload("afl")
    info = A.info
    x = torch.from_numpy(synth.rhs(4096, 1)).to(dev)
    y = torch.zeros(4096, dtype=torch.float64, device=dev)
    flush = torch.empty(256 * 2 ** 20 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    for _ in range(max(3, args.warmup)):
        A.matvec(x, y, acc="fp32", stream=stream)
    times = []
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(local)
    clocks.start()
    for _ in range(args.steps):
        flush.fill_(1.0)
        e0.record(stream)
        A.matvec(x, y, acc="fp32", stream=stream)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1) * 1e3)
    clk = clocks.stop()
    A.check()
    times.sort()
    med = times[len(times) // 2]
    if rank == 0:
        out = {"metric": METRIC, "value": info["algorithmic_bytes"] / (med * 1e-6) / 1e9, "unit": UNIT,
               "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": med / 1e3,
               "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
               "config": {"workload": f"exp2d n=4096 eps={args.eps:g} (fits in L2; L2 flushed by a 256 MB write before "
                                      f"each product, each product timed alone)", "l2": "flushed between products"},
               "latency_us": {"median": med, "min": times[0], "p90": times[int(0.9 * (len(times) - 1))]},
               "matrix": {"algorithmic_bytes": info["algorithmic_bytes"], "nblocks": info["nblocks"]},
               "clocks": clk, "gpu_launches": int(info["launches"]) * args.steps}
        print(json.dumps(out), flush=True)
    A.free()
    Hh.free()


def run_scale(args, world: int, rank: int, local: int):
    """n = 2^21 Fibonacci points on the sphere, 1/(4 pi r) with the mean row sum (1024 sampled
    rows) on the diagonal, eps from --eps: single-column products and 32-column products
    (hlr_matvec_batched). The sampled-row check against direct kernel evaluation is
    tests/test_gpu_scale.py."""
    import torch
    import synth
    import paper_2308_10960_gb300 as hg

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    n = 2 ** 21
    t0 = time.perf_counter()
    p = synth.laplace_problem(n)
    Hh = hg.build_kernel_hmatrix(p.points, "laplace", args.eps, diag=p.params["diag"])
    t_build = time.perf_counter() - t0
    A = Hh.upload("afl")
    Hh.free()
    info = A.info
    stream = torch.cuda.current_stream(dev)
    x = torch.from_numpy(synth.rhs(n, 1)).to(dev)
    y = torch.zeros(n, dtype=torch.float64, device=dev)
    for _ in range(max(3, args.warmup)):
        A.matvec(x, y, acc="fp32", stream=stream)
    clocks = ClockSampler(local)
    clocks.start()
    el = time_loop(lambda: A.matvec(x, y, acc="fp32", stream=stream), args.steps, stream)
    clk = clocks.stop()
    X = torch.from_numpy(synth.rhs(n * 32, 3)).to(dev).view(32, n)
    Y = torch.zeros_like(X)
    for _ in range(2):
        hg.matvec_batched([A], [X], [Y], acc="fp32", stream=stream)
    k32 = max(3, args.steps // 20)
    el32 = time_loop(lambda: hg.matvec_batched([A], [X], [Y], acc="fp32", stream=stream), k32, stream)
    A.check()
    bytes1 = float(info["algorithmic_bytes"])
    b32 = multi_rhs_bytes(info, n, 32)
    t1 = el / args.steps
    t32 = el32 / k32
    peaks = measured_peaks()
    if rank == 0:
        out = {"metric": METRIC, "value": bytes1 / t1 / 1e9 * world, "unit": UNIT, "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": t1 * 1e3, "higher_is_better": True, "scaling": "weak",
               "vs_baseline": None, "dtype": "f32", "data": "synthetic",
               "config": {"workload": f"laplace-sphere n=2097152 eps={args.eps:g} AFL-APLR, single and 32 RHS",
                          "l2": "inputs larger than L2"},
               "pct_hbm_peak": bytes1 / t1 / 1e9 / peaks["hbm_gbs"],
               "rhs32": {"ms_per_step": t32 * 1e3, "GB/s": b32 / t32 / 1e9, "algorithmic_bytes": b32,
                         "speedup_vs_32_single_products": 32 * t1 / t32},
               "matrix": {"nblocks": info["nblocks"], "rank_sum": info["rank_sum"], "algorithmic_bytes": bytes1,
                          "fp64_bytes": info["fp64_bytes"], "device_bytes": info["device_bytes"], "build_s": t_build},
               "clocks": clk, "gpu_launches": int(info["launches"]) * args.steps}
        print(json.dumps(out), flush=True)
    A.free()


def run_multi(args, world: int, rank: int, local: int):
    """Multi-column products on the --n Laplace sphere: one single-column product, then one
    hlr_matvec_batched request of 8 and of 32 columns (narrow and wide passes), with the default
    work lists and with lists made for the passes' 3 CTAs per SM (HLR_CTAS_PER_SM(3)). value =
    algorithmic bytes of the 32-column request / its time with the better shape; --steps timed
    calls each after --warmup."""
    import torch
    import synth
    import paper_2308_10960_gb300 as hg

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    prob = synth.laplace_problem(args.n)
    Hh = hg.build_kernel_hmatrix(prob.points, "laplace", args.eps, diag=prob.params["diag"], eta=2.0, leaf_size=64)
    stream = torch.cuda.current_stream(dev)
    x = torch.from_numpy(synth.rhs(args.n, 1)).to(dev)
    res = {}
    best = None
    for shape in (0, 3):
        A = Hh.upload("afl", tuning=hg.tuning_code(ctas_per_sm=shape))
        info = A.info
        y = torch.zeros(args.n, dtype=torch.float64, device=dev)
        for _ in range(max(3, args.warmup)):
            A.matvec(x, y, acc="fp32", stream=stream)
        t1 = time_loop(lambda: A.matvec(x, y, acc="fp32", stream=stream), args.steps, stream) / args.steps
        row = {"single_ms": t1 * 1e3}
        for r in (8, 32):
            X = torch.from_numpy(synth.rhs(args.n * r, 2 + r)).to(dev).view(r, args.n)
            Y = torch.zeros((r, args.n), dtype=torch.float64, device=dev)
            for _ in range(max(3, args.warmup)):
                hg.matvec_batched([A], [X], [Y], acc="fp32", stream=stream)
            tm = time_loop(lambda: hg.matvec_batched([A], [X], [Y], acc="fp32", stream=stream), args.steps,
                           stream) / args.steps
            bm = multi_rhs_bytes(info, args.n, r)
            row[str(r)] = {"ms": tm * 1e3, "GB/s": bm / tm / 1e9, "vs_one_single": tm / t1,
                           "speedup_vs_r_single_products": r * t1 / tm}
            if r == 32 and (best is None or tm < best[0]):
                best = (tm, bm)
            del X, Y
        A.check()
        A.free()
        res[f"ctas_per_sm={shape or 'default'}"] = row
    if rank == 0:
        out = {"metric": METRIC, "value": best[1] / best[0] / 1e9, "unit": UNIT, "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": best[0] * 1e3, "higher_is_better": True, "scaling": "weak",
               "vs_baseline": None, "dtype": "f32", "data": "synthetic",
               "config": {"workload": f"laplace-sphere n={args.n} eps={args.eps:g}, 32 right-hand sides per request",
                          "n": args.n, "eps": args.eps}, "multi_rhs": res}
        print(json.dumps(out), flush=True)
    Hh.free()


def main():
    args = parse()
    world, rank, local = dist_env()
    if world > 1:
        import torch
        import torch.distributed as dist
        if args.impl == "reference":
            if rank != 0:
                return
        else:
            torch.cuda.set_device(local)
            dist.init_process_group("nccl")
    if args.impl == "reference":
        run_reference(args, world, rank)
        return
    if args.workload == "batch48":
        run_batch(args, world, rank, local)
    elif args.workload == "serve":
        run_serve(args, world, rank, local)
    elif args.workload == "small":
        run_small(args, world, rank, local)
    elif args.workload == "scale":
        run_scale(args, world, rank, local)
    elif args.workload == "multi":
        run_multi(args, world, rank, local)
    else:
        run_ours(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
