#!/usr/bin/env python3
"""Benchmark: randomized PCA of a tall float32 matrix on one GB300 (or N replicas).

Workload (the throughput configuration of the tall-skinny PCA setting):
A is 200000 x 1000 float32, A = U diag(sigma) V^T with Haar factors and
sigma_i = |1/i + 1e-3 xi_i|, centred columns; k = 50, p = 10, q = 2, seeded
Gaussian Omega (1000 x 60) given as input.  One step = one full rsvd() solve
(centring, sketch, q re-orthonormalised power iterations, Rayleigh-Ritz, small
SVD, Ritz vectors) through the C ABI.  A (0.8 GB) is larger than L2 (129 MB),
so no L2 flush is needed between steps.

Metric: rSVD GFLOP/s = algorithmic FLOPs per solve x solves / device time,
with the FLOP count of the paper's randomized PCA step list (Sec. 3.1.2) in the
2-flop multiply-add convention:
    F = 2mnl(2q+2) + 2ml^2(q+1) + 2ml^2 + 2nl^2.

``--impl reference`` times the FP64 CPU oracle (the only reference this
project has) on the host cores on a bounded row sample of the same workload.

``--method block_krylov`` measures the paper's block Krylov method (Sec. 3.1.1)
instead: A 1048576 x 4096 float32 with seeded N(0,1) entries (the Gaussian
matrices of the paper's experiments), blocks of b = 96 columns, i = 2 (W = 288),
k = 256, one step = one rsvd_block_krylov() solve; FLOPs per solve
    F = 2mnb(2i+1) + 2mnW + 2mW^2 + 2nW^2
(the products with A, the QR of the m x W basis, the SVD of T).

``--method gkl`` measures the Golub-Kahan-Lanczos path (HBM-bound): A 1048576 x
2048 float32, sigma_i = exp(-i/200), 150 steps with full reorthogonalisation from
a seeded unit v1, k = 100; metric: algorithmic HBM GB/s of the solve, bytes per
solve = steps r (4mn) + 8(m+n) steps (steps - 1): r reads of A per step (1 for the
float32 one-pass form, 2 with --gkl-two-pass) and the classical Gram-Schmidt
passes over the growing bases, applied twice.

``--method precision --dtype bf16|fp8`` measures the precision form: A 1048576 x
4096 with sigma_i = i^-1.5 (Haar factors built in float32 on the device, a timing
input) stored as bfloat16 or e4m3 with column scales by the library's quantiser;
k = 256, p = 32, q = 3; metric: rSVD GFLOP/s as for the default workload.

``--method gram_grid`` runs the paper's experiment grid (Sec. 4) through the Gram route
(svd_exact, RSVD_EXACT_GRAM, all n triplets, k = n): N(0,1) matrices with 5 row sizes
{2000, ..., 10000} x 12 column sizes {100, ..., 2000}, plus a 60000 x 784 MNIST-shaped
N(0,1) matrix (the dataset is not available); float64 by default (--dtype f32 for the
float32 form).  Metric: solves/s over the grid; every point's time and the paper's
residual delta = ||A - U Sigma V^T||_F / ||A||_F are listed.
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

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "rpca_fp32_200000x1000"
GKL_WORKLOAD = "gkl_fp32_1048576x2048"
PREC_WORKLOAD = "mixed_rsvd_1048576x4096"
BK_WORKLOAD = "block_krylov_fp32_gaussian_1048576x4096"
BK = dict(m=1048576, n=4096, k=256, b=96, iters=2, seed_a=40971, seed_omega=40972)


def alg_flops(m, n, k, p, q):
    l = k + p
    return 2.0 * m * n * l * (2 * q + 2) + 2.0 * m * l * l * (q + 1) + 2.0 * m * l * l + 2.0 * n * l * l


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return d, "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=2)
            except Exception:
                self.proc.kill()
        sm = []
        mx = None
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
                for nm, v in zip(names, r[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(nm)
            except Exception:
                continue
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def traffic_for(kernel_src: str, kernel: str, workload: str = None):
    """DRAM bytes per launch from the committed ncu summary, if it matches the current kernel source
    (captures on a smaller case are stored scaled to a full launch by the rows processed)."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f)
        e = rec[kernel]
        with open(os.path.join(ROOT, "paper_1906_12085_gb300", "csrc", kernel_src), "rb") as f:
            h = hashlib.sha256(f.read()).hexdigest()[:16]
        if e.get("source_sha256_16") != h or e.get("workload") != (workload or WORKLOAD):
            return None
        return float(e["dram_bytes_per_launch"])
    except Exception:
        return None


def slowest_rank_ms(ms: float, world: int, device) -> float:
    """The timed region of the slowest rank (replicas: every rank solves its own matrix)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.barrier()
    return float(t.item())


def job_gflops(world: int, flops_per_solve: float, steps: int, ms_max: float) -> float:
    """Whole-job throughput: every rank's solves over the slowest rank's time (weak scaling)."""
    return world * flops_per_solve * steps / (ms_max * 1e-3) / 1e9


def oracle_sample(A_host32, Om32, k, q, rows):
    """Time the FP64 oracle on the first `rows` rows (centred) of the workload matrix."""
    import numpy as np

    import oracle
    a = np.ascontiguousarray(A_host32[:rows].astype(np.float64))
    om = Om32.astype(np.float64)
    t0 = time.perf_counter()
    ac, mu, fro2 = oracle.center(a)
    oracle.rsvd(ac, om, q=q, k=k)
    return time.perf_counter() - t0


def bk_flops(m, n, b, iters):
    W = (iters + 1) * b
    return 2.0 * m * n * b * (2 * iters + 1) + 2.0 * m * n * W + 2.0 * m * W * W + 2.0 * n * W * W


def run_block_krylov(args):
    """One JSON line for the block Krylov workload (replicas over ranks, like the default)."""
    import torch
    import torch.distributed as dist

    import paper_1906_12085_gb300 as g
    import synth
    from paper_1906_12085_gb300 import build as gbuild

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    gbuild.build()
    m, n, k, b, iters = BK["m"], BK["n"], BK["k"], BK["b"], BK["iters"]
    W = (iters + 1) * b
    A = synth.gaussian(m, n, BK["seed_a"], device=dev, dtype=torch.float32)
    Om = synth.gaussian(n, b, BK["seed_omega"], device=dev, dtype=torch.float32)
    S = torch.zeros(k, dtype=torch.float64, device=dev)
    U = torch.zeros(m, k, dtype=torch.float32, device=dev)
    V = torch.zeros(n, k, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    plan = g.rsvd_plan_create_block_krylov(m, n, k, b, iters, g.RSVD_F32, stream)

    def step():
        g.check(g.rsvd_block_krylov(plan, A, Om, S, U, V), "rsvd_block_krylov")

    for _ in range(max(args.warmup, 0)):
        step()
    g.check(g.rsvd_plan_sync(plan), "warm-up solve status")
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    sampler = ClockSampler(torch.cuda.current_device() if "CUDA_VISIBLE_DEVICES" not in os.environ else local)
    sampler.start()
    launches0 = g.rsvd_launch_count()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    launches = g.rsvd_launch_count() - launches0
    ms = e0.elapsed_time(e1)
    clocks = sampler.stop()
    st = g.rsvd_plan_sync(plan)
    ms_max = slowest_rank_ms(ms, world, dev)
    flops = bk_flops(m, n, b, iters)
    value = job_gflops(world, flops, args.steps, ms_max)

    # per-stage durations (CUDA events on the plan's stream) over the same K steps
    g.rsvd_plan_profile(plan, True)
    g.rsvd_plan_profile_read(plan)
    for _ in range(args.steps):
        step()
    prof = g.rsvd_plan_profile_read(plan)
    g.rsvd_plan_profile(plan, False)
    # The products with A are HBM-bound 3xTF32 passes over A (4mn bytes each): the A X
    # stage makes i + 1 of them (N = b), the A^T X stage i (N = b) plus the Rayleigh-Ritz
    # product at N = W, which runs as ceil(W / 128) column slices, one pass each.
    pk, src = peaks()
    hbm = float(pk.get("hbm_gbs", 6800.0))
    Wp = -(-W // 16) * 16
    passes = {"ax": iters + 1, "atx": iters + -(-Wp // 128)}
    dom = "ax" if prof["ax"][0] >= prof["atx"][0] else "atx"
    per_pass_ms = prof[dom][0] / args.steps / passes[dom]
    achieved = 4.0 * m * n / (per_pass_ms * 1e-3) / 1e9
    roofline = {"bound": "hbm",
                "kernel": "tc_nn_kernel (A X, 3xTF32 tcgen05)" if dom == "ax" else
                          "tc_tn_kernel + sum_chunks_kernel (A^T X, 3xTF32 tcgen05)",  # block Krylov: in-kernel split
                "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                "traffic": None, "algorithmic_bytes_per_launch": 4.0 * m * n,
                "passes_over_A_per_step": passes,
                "peak_source": f"{src} (MEASURED_PEAKS.json hbm_gbs)" if src == "measured" else "fallback 6800 GB/s",
                "stage_ms_per_step": {kk: vv[0] / args.steps for kk, vv in prof.items()},
                "timing": "stage durations from CUDA events around each kernel group over an instrumented "
                          "pass of the same K steps; per pass over A = stage time / passes"}

    e2e = None
    if rank == 0 or world > 1:   # host buffers (pinned), copies inside the timed region
        Ah = A.cpu().pin_memory()
        Omh = Om.cpu().pin_memory()
        Sh = torch.empty_like(S, device="cpu").pin_memory()
        Uh = torch.empty_like(U, device="cpu").pin_memory()
        Vh = torch.empty_like(V, device="cpu").pin_memory()
        n_e2e = max(1, min(args.steps, 3))
        torch.cuda.synchronize(dev)
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        for _ in range(n_e2e):
            A.copy_(Ah, non_blocking=True)
            Om.copy_(Omh, non_blocking=True)
            step()
            Sh.copy_(S, non_blocking=True)
            Uh.copy_(U, non_blocking=True)
            Vh.copy_(V, non_blocking=True)
        f1.record(stream)
        torch.cuda.synchronize(dev)
        ems = f0.elapsed_time(f1)
        e2e = {"value": flops * n_e2e / (ems * 1e-3) / 1e9, "unit": "GFLOP/s",
               "h2d_bytes_per_step": Ah.numel() * 4 + Omh.numel() * 4,
               "d2h_bytes_per_step": Sh.numel() * 8 + Uh.numel() * 4 + Vh.numel() * 4,
               "ms_per_step": ems / n_e2e}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import numpy as np

        import oracle
        rows = args.bk_cpu_rows
        a = np.ascontiguousarray(A[:rows].cpu().numpy().astype(np.float64))
        om = Om.cpu().numpy().astype(np.float64)
        t0 = time.perf_counter()
        oracle.block_krylov(oracle.center(a)[0], om, iters, k)
        tsec = time.perf_counter() - t0
        cpu = {"value": bk_flops(rows, n, b, iters) / tsec / 1e9, "unit": "GFLOP/s", "cores": os.cpu_count(),
               "kind": "oracle",
               "sample": f"first {rows} of {m} rows (same n, b, i, k, Omega); FP64 C oracle, OpenMP, one solve"}

    if rank == 0:
        line = {
            "metric": "block Krylov GFLOP/s", "value": value, "unit": "GFLOP/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": BK_WORKLOAD, "method": "block_krylov", "m": m, "n": n, "k": k, "b": b,
                       "iters": iters, "W": W, "l2": "inputs larger than L2 (A is 17.2 GB), no flush",
                       "parallelism": f"replicas{world}"},
            "solves_per_s": world * args.steps / (ms_max * 1e-3), "status": st,
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": launches, "clocks": clocks, "peaks_source": src,
        }
        print(json.dumps(line), flush=True)
    plan.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


def _timed_solves(step, args, dev, stream, world):
    """Warm-up, then K timed solves between CUDA events with clock sampling (one rank's view)."""
    import torch
    import torch.distributed as dist

    import paper_1906_12085_gb300 as g
    for _ in range(max(args.warmup, 0)):
        step()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    launches0 = g.rsvd_launch_count()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    launches = g.rsvd_launch_count() - launches0
    clocks = sampler.stop()
    return slowest_rank_ms(e0.elapsed_time(e1), world, dev), launches, clocks


def _stage_profile(plan, step, steps):
    """Per-stage CUDA-event durations over `steps` more solves (direct launches)."""
    import paper_1906_12085_gb300 as g
    g.rsvd_plan_profile(plan, True)
    g.rsvd_plan_profile_read(plan)
    for _ in range(steps):
        step()
    prof = g.rsvd_plan_profile_read(plan)
    g.rsvd_plan_profile(plan, False)
    return prof


def _e2e(step, dev, stream, h2d, d2h, reps, work, unit):
    """The same solve through the public API from pinned host buffers, copies inside the timed region."""
    import torch
    pins = [(d, d.cpu().pin_memory()) for d in h2d]
    outs = [(d, torch.empty_like(d, device="cpu").pin_memory()) for d in d2h]
    torch.cuda.synchronize(dev)
    f0 = torch.cuda.Event(enable_timing=True)
    f1 = torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    for _ in range(reps):
        for d, h in pins:
            d.copy_(h, non_blocking=True)
        step()
        for d, h in outs:
            h.copy_(d, non_blocking=True)
    f1.record(stream)
    torch.cuda.synchronize(dev)
    ems = f0.elapsed_time(f1)
    return {"value": work * reps / (ems * 1e-3) / 1e9, "unit": unit,
            "h2d_bytes_per_step": sum(h.numel() * h.element_size() for _, h in pins),
            "d2h_bytes_per_step": sum(h.numel() * h.element_size() for _, h in outs), "ms_per_step": ems / reps}


def gkl_bytes(m, n, steps, reads=2):
    return steps * reads * 4.0 * m * n + 8.0 * (m + n) * steps * (steps - 1)


def run_gkl(args):
    """One JSON line for the Golub-Kahan-Lanczos workload (HBM GB/s)."""
    import numpy as np
    import torch
    import torch.distributed as dist

    import paper_1906_12085_gb300 as g
    import synth
    from paper_1906_12085_gb300 import build as gbuild

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    gbuild.build()
    w = synth.WORKLOADS[GKL_WORKLOAD]
    m, n, k, steps = w["m"], w["n"], w["k"], w["steps"]
    A64, sigma, extras = synth.workload(GKL_WORKLOAD, device=dev)
    A = A64.float().contiguous()
    del A64
    v1 = extras["v1"].to(dev)
    S = torch.zeros(k, dtype=torch.float64, device=dev)
    U = torch.zeros(m, k, dtype=torch.float32, device=dev)
    V = torch.zeros(n, k, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    plan = g.rsvd_plan_create(m, n, k, 0, 0, g.RSVD_F32, stream)
    reads = 2 if args.gkl_two_pass else 1
    if args.gkl_two_pass:
        g.check(g.rsvd_plan_set_flags(plan, g.RSVD_FLAG_GKL_TWO_PASS), "flags")

    def step():
        g.check(g.svd_truncated_krylov(plan, A, v1, steps, S, U, V), "svd_truncated_krylov")

    ms_max, launches, clocks = _timed_solves(step, args, dev, stream, world)
    st = g.rsvd_plan_sync(plan)
    nbytes = gkl_bytes(m, n, steps, reads)
    value = world * nbytes * args.steps / (ms_max * 1e-3) / 1e9
    prof = _stage_profile(plan, step, args.steps)
    pk, src = peaks()
    hbm = float(pk.get("hbm_gbs", 6800.0))
    # dominant GEMV of the step: the one-pass A v and A^T (A v) (ax stage), or with two passes
    # A v (ax) or A^T u (atx); one launch group per step each
    dom = "ax" if prof["ax"][0] >= prof["atx"][0] else "atx"
    per_launch_ms = prof[dom][0] / prof[dom][1]
    achieved = 4.0 * m * n / (per_launch_ms * 1e-3) / 1e9
    kname = ("gemv_nt_kernel (A v and A^T (A v), one read of A)" if reads == 1 else "gemv_n_kernel (A v)") \
        if dom == "ax" else "gemv_t_kernel (A^T u)"
    traffic = traffic_for("k_gkl.cu", "gemv_nt_kernel", GKL_WORKLOAD) if reads == 1 and dom == "ax" else None
    roofline = {"bound": "hbm", "kernel": kname,
                "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm, "traffic": traffic,
                "algorithmic_bytes_per_launch": 4.0 * m * n,
                "solve_algorithmic_bytes": nbytes, "solve_frac": value / world / hbm,
                "peak_source": f"{src} (MEASURED_PEAKS.json hbm_gbs)" if src == "measured" else "fallback 6800 GB/s",
                "stage_ms_per_step": {kk: vv[0] / args.steps for kk, vv in prof.items()},
                "timing": "stage durations from CUDA events around each kernel group over an instrumented pass"}
    e2e = _e2e(step, dev, stream, [A, v1], [S, U, V], 1, nbytes, "GB/s") if rank == 0 or world > 1 else None
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        rows = args.gkl_cpu_rows
        a = np.ascontiguousarray(A[:rows].cpu().numpy().astype(np.float64))
        t0 = time.perf_counter()
        oracle.gkl(oracle.center(a)[0], v1.cpu().numpy().astype(np.float64), steps, k)
        tsec = time.perf_counter() - t0
        cpu = {"value": gkl_bytes(rows, n, steps, reads) / tsec / 1e9, "unit": "GB/s", "cores": os.cpu_count(),
               "kind": "oracle",
               "sample": f"first {rows} of {m} rows (same n, steps, k, v1); FP64 C oracle, OpenMP, one solve"}
    if rank == 0:
        line = {"metric": "GKL HBM GB/s (algorithmic)", "value": value, "unit": "GB/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic",
                "config": {"workload": GKL_WORKLOAD, "method": "gkl", "m": m, "n": n, "k": k, "lanczos_steps": steps,
                           "a_reads_per_step": reads,
                           "l2": "inputs larger than L2 (A is 8.6 GB), no flush", "parallelism": f"replicas{world}"},
                "solves_per_s": world * args.steps / (ms_max * 1e-3), "status": st,
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
                "clocks": clocks, "peaks_source": src}
        print(json.dumps(line), flush=True)
    plan.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


def run_precision(args):
    """One JSON line for the precision form (bfloat16 or e4m3 storage of A)."""
    import numpy as np
    import torch
    import torch.distributed as dist

    import paper_1906_12085_gb300 as g
    import synth
    from paper_1906_12085_gb300 import build as gbuild

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    gbuild.build()
    w = synth.WORKLOADS[PREC_WORKLOAD]
    m, n, k, p, q = w["m"], w["n"], w["k"], w["p"], w["q"]
    l = k + p
    lp = -(-l // 16) * 16
    dt = g.RSVD_BF16 if args.dtype == "bf16" else g.RSVD_FP8_E4M3
    A32, sigma, extras = synth.workload(PREC_WORKLOAD, device=dev, dtype=torch.float32)
    Om = extras["omega"].to(dev).contiguous()
    sc = None
    if dt == g.RSVD_BF16:
        Aq = torch.empty(m, n, dtype=torch.int16, device=dev)
        g.check(g.rsvd_quantize(A32, dt, Aq), "rsvd_quantize")
    else:
        Aq = torch.empty(m, n, dtype=torch.uint8, device=dev)
        sc = torch.empty(n, dtype=torch.float32, device=dev)
        g.check(g.rsvd_quantize(A32, dt, Aq, sc), "rsvd_quantize")
    del A32
    torch.cuda.empty_cache()
    S = torch.zeros(k, dtype=torch.float64, device=dev)
    U = torch.zeros(m, k, dtype=torch.float32, device=dev)
    V = torch.zeros(n, k, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    plan = g.rsvd_plan_create(m, n, k, p, q, dt, stream)

    def step():
        g.check(g.rsvd(plan, Aq, sc, Om, S, U, V), "rsvd")

    ms_max, launches, clocks = _timed_solves(step, args, dev, stream, world)
    st = g.rsvd_plan_sync(plan)
    flops = alg_flops(m, n, k, p, q)
    value = job_gflops(world, flops, args.steps, ms_max)
    prof = _stage_profile(plan, step, args.steps)
    pk, src = peaks()
    hbm = float(pk.get("hbm_gbs", 6800.0))
    # the sketch and power products A Z (ax stage): q + 1 of them, each ceil(lp / 256) column
    # slices of one pass over the stored A (2mn bytes bfloat16, mn e4m3)
    esz = 2 if dt == g.RSVD_BF16 else 1
    passes = (q + 1) * -(-lp // 256)
    per_pass_ms = prof["ax"][0] / args.steps / passes
    achieved = esz * m * n / (per_pass_ms * 1e-3) / 1e9
    nslices = -(-lp // 256)
    slice_n = -(-(-(-lp // nslices)) // 16) * 16   # width of one column slice
    roofline = {"bound": "hbm", "kernel": "tc16_nn_kernel (A Z, kind::f16)" if esz == 2 else
                "tc16_nn_kernel<e4m3> (A Z, kind::f8f6f4)",
                "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm, "traffic": None,
                "algorithmic_bytes_per_launch": esz * float(m) * n, "passes_over_A_per_step_ax": passes,
                "arithmetic_intensity_flop_per_byte": 2.0 * slice_n / esz,
                "tensor": {"achieved_tflops": 2.0 * m * n * slice_n / (per_pass_ms * 1e-3) / 1e12,
                           "peak_bf16_tflops": float(pk.get("bf16_tflops_sustained", pk.get("bf16_tflops", 1900.0)))},
                "peak_source": f"{src} (MEASURED_PEAKS.json hbm_gbs)" if src == "measured" else "fallback 6800 GB/s",
                "stage_ms_per_step": {kk: vv[0] / args.steps for kk, vv in prof.items()},
                "timing": "stage durations from CUDA events around each kernel group over an instrumented pass; "
                          "per pass over A = ax stage time / passes"}
    e2e = None
    if rank == 0 or world > 1:
        e2e = _e2e(step, dev, stream, [Aq, Om] + ([sc] if sc is not None else []), [S, U, V], 1, flops,
                   "GFLOP/s")
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        rows = args.prec_cpu_rows
        codes = Aq[:rows].cpu().numpy()
        a = (oracle.dequantize_bf16(codes.view(np.uint16)) if esz == 2
             else oracle.dequantize_e4m3(codes, sc.cpu().numpy()))
        om = Om.cpu().numpy().astype(np.float64)
        t0 = time.perf_counter()
        oracle.rsvd(oracle.center(a)[0], om, q=q, k=k)
        tsec = time.perf_counter() - t0
        cpu = {"value": alg_flops(rows, n, k, p, q) / tsec / 1e9, "unit": "GFLOP/s", "cores": os.cpu_count(),
               "kind": "oracle",
               "sample": f"first {rows} of {m} rows of the stored matrix, dequantised (same n, k, p, q, Omega); "
                         f"FP64 C oracle, OpenMP, one solve"}
    if rank == 0:
        line = {"metric": "rSVD GFLOP/s", "value": value, "unit": "GFLOP/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": args.dtype, "data": "synthetic",
                "config": {"workload": PREC_WORKLOAD, "method": "precision", "storage": args.dtype, "m": m, "n": n,
                           "k": k, "p": p, "q": q, "l2": f"inputs larger than L2 (A is {esz * m * n / 1e9:.1f} GB), "
                                                          f"no flush", "parallelism": f"replicas{world}"},
                "solves_per_s": world * args.steps / (ms_max * 1e-3), "status": st,
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
                "clocks": clocks, "peaks_source": src}
        print(json.dumps(line), flush=True)
    plan.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


GRID_ROWS = [2000, 4000, 6000, 8000, 10000]
GRID_COLS = [100, 200, 300, 400, 500, 600, 800, 900, 1000, 1200, 1500, 2000]


def run_gram_grid(args):
    """One JSON line for the paper's experiment grid through the Gram route (k = n)."""
    import numpy as np
    import torch

    import paper_1906_12085_gb300 as g
    import synth
    from paper_1906_12085_gb300 import build as gbuild

    if int(os.environ.get("RANK", "0")) != 0:   # replicas are not meaningful for a sweep: rank 0 runs it
        return 0
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    torch.cuda.set_device(dev)
    gbuild.build()
    f64 = args.dtype != "f32"
    dt, tdt = (g.RSVD_F64, torch.float64) if f64 else (g.RSVD_F32, torch.float32)
    stream = torch.cuda.current_stream(dev)
    points = [(m, n) for m in GRID_ROWS for n in GRID_COLS] + [(60000, 784)]
    reps = max(1, args.steps)
    out, total_ms, total = [], 0.0, 0
    launches0 = g.rsvd_launch_count()
    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    for idx, (m, n) in enumerate(points):
        A0 = synth.gaussian(m, n, 40000 + idx, device=dev, dtype=tdt)
        A = A0.clone()
        S = torch.zeros(n, dtype=torch.float64, device=dev)
        U = torch.zeros(m, n, dtype=tdt, device=dev)
        V = torch.zeros(n, n, dtype=tdt, device=dev)
        plan = g.rsvd_plan_create(m, n, 1, 0, 0, dt, stream)
        for _ in range(max(args.warmup, 1)):     # the first call allocates the solver's workspace
            g.check(g.svd_exact(plan, A, g.RSVD_EXACT_GRAM, S, U, V), "svd_exact")
        st = g.rsvd_plan_sync(plan)
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            g.check(g.svd_exact(plan, A, g.RSVD_EXACT_GRAM, S, U, V), "svd_exact")
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1) / reps
        st = g.rsvd_plan_sync(plan) if st == g.RSVD_OK else st
        Ac = A0.double() - A0.double().mean(dim=0, keepdim=True)
        delta = float(torch.linalg.norm(Ac - (U.double() * S) @ V.double().T) / torch.linalg.norm(Ac))
        out.append({"m": m, "n": n, "ms": round(ms, 4), "delta": delta, "status": st})
        total_ms += ms * reps
        total += reps
        plan.close()
        del A0, A, U, V
    clocks = sampler.stop()
    launches = g.rsvd_launch_count() - launches0
    cpu = None
    if not args.no_cpu_baseline:
        import oracle
        sample = [(2000, 100), (2000, 200), (4000, 300), (4000, 500)]
        t0 = time.perf_counter()
        for idx, (m, n) in enumerate(sample):
            a = synth.gaussian(m, n, 50000 + idx).numpy()
            oracle.svd_gram(oracle.center(a)[0])
        tsec = time.perf_counter() - t0
        cpu = {"value": len(sample) / tsec, "unit": "solves/s", "cores": os.cpu_count(), "kind": "oracle",
               "sample": "the grid points " + ", ".join(f"{m}x{n}" for m, n in sample) +
                         " (float64 C oracle: A^T A, cyclic Jacobi, u_i = A v_i / sigma_i), one solve each"}
    big = [p_ for p_ in out if p_["m"] == 10000 and p_["n"] == 2000][0]
    mn = [p_ for p_ in out if p_["m"] == 60000][0]
    line = {"metric": "Gram route (k = n) solves/s over the paper's grid", "value": total / (total_ms * 1e-3),
            "unit": "solves/s", "n_gpus": 1, "steps": reps, "warmup": args.warmup,
            "ms_per_step": total_ms / total, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if f64 else "f32", "data": "synthetic",
            "config": {"workload": "paper_grid_gaussian", "method": "gram_grid", "rows": GRID_ROWS, "cols": GRID_COLS,
                       "extra": "60000x784 N(0,1) (MNIST-shaped)",
                       "l2": "each point solved back to back on the same buffers (A up to 160 MB)"},
            "status": max((p_["status"] for p_ in out), key=abs),
            "max_delta": max(p_["delta"] for p_ in out),
            "point_10000x2000_ms": big["ms"], "point_60000x784_ms": mn["ms"],
            "points": out, "cpu_baseline": cpu, "e2e": None, "gpu_launches": launches, "clocks": clocks}
    print(json.dumps(line), flush=True)
    return 0


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import numpy as np
    import torch

    import synth
    w = synth.WORKLOADS[WORKLOAD]
    m, n, k, p, q = w["m"], w["n"], w["k"], w["p"], w["q"]
    rows = args.sample_rows
    # the sample: the first `rows` rows of the same recipe (same n, k, p, q and Omega)
    A, sigma, extras = synth.workload(WORKLOAD, m=rows)
    A32 = A.float().numpy()
    Om = extras["omega"].numpy()
    flops = alg_flops(rows, n, k, p, q)
    for _ in range(args.warmup):
        oracle_sample(A32, Om, k, q, rows)
    ts = [oracle_sample(A32, Om, k, q, rows) for _ in range(args.steps)]
    total = sum(ts)
    val = flops * len(ts) / total / 1e9
    cores = os.cpu_count()
    line = {
        "impl": "reference", "metric": "rSVD GFLOP/s", "value": val, "unit": "GFLOP/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / len(ts), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "m": m, "n": n, "k": k, "p": p, "q": q, "sample_rows": rows},
        "cpu_baseline": {"value": val, "unit": "GFLOP/s", "cores": cores, "kind": "oracle",
                         "sample": f"first {rows} of {m} rows (same n, k, p, q, Omega); FP64 C oracle, OpenMP"},
        "e2e": {"value": val, "unit": "GFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    del np, torch, sigma
    return 0


def run_ours(args):
    import torch
    import torch.distributed as dist

    import paper_1906_12085_gb300 as g
    import synth
    from paper_1906_12085_gb300 import build as gbuild

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    gbuild.build()

    w = synth.WORKLOADS[WORKLOAD]
    m, n, k, p, q = w["m"], w["n"], w["k"], w["p"], w["q"]
    l = k + p
    A64, sigma, extras = synth.workload(WORKLOAD, device=dev)
    A0 = A64.float().contiguous()           # pristine copy (host source of the end-to-end leg)
    del A64
    Om = extras["omega"].to(dev).contiguous()
    A = A0.clone()
    S = torch.zeros(k, dtype=torch.float64, device=dev)
    U = torch.zeros(m, k, dtype=torch.float32, device=dev)
    V = torch.zeros(n, k, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    plan = g.rsvd_plan_create(m, n, k, p, q, g.RSVD_F32, stream)

    def step():
        g.check(g.rsvd(plan, A, None, Om, S, U, V), "rsvd")

    for _ in range(max(args.warmup, 0)):
        step()
    g.check(g.rsvd_plan_sync(plan), "warm-up solve status")
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    # timed region: the production path (the solve replayed as a captured CUDA graph)
    sampler = ClockSampler(torch.cuda.current_device() if "CUDA_VISIBLE_DEVICES" not in os.environ else local)
    sampler.start()
    launches0 = g.rsvd_launch_count()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    launches = g.rsvd_launch_count() - launches0
    ms = e0.elapsed_time(e1)
    clocks = sampler.stop()
    st = g.rsvd_plan_sync(plan)
    ms_max = slowest_rank_ms(ms, world, dev)
    flops = alg_flops(m, n, k, p, q)
    value = job_gflops(world, flops, args.steps, ms_max)

    # per-kernel durations: the same K steps again with CUDA events recorded on the plan's
    # stream around every kernel group (direct launches, identical kernels)
    g.rsvd_plan_profile(plan, True)
    g.rsvd_plan_profile_read(plan)
    for _ in range(args.steps):
        step()
    prof = g.rsvd_plan_profile_read(plan)
    g.rsvd_plan_profile(plan, False)

    # dominant kernel group and its roofline.  The float32 products run as 3xTF32 on
    # tcgen05: at l = 60 (64 padded) their arithmetic intensity is 2*64 flop / 4 B = 32
    # flop/B, below the 3xTF32 ridge (TF32 dense / 3 / HBM ~ 46 flop/B), so they are
    # HBM-bound; algorithmic bytes per launch = one read of A (4mn).
    pk, src = peaks()
    hbm = float(pk.get("hbm_gbs", 6800.0))
    ax_ms, ax_n = prof["ax"]
    atx_ms, atx_n = prof["atx"]
    if ax_ms >= atx_ms:
        dom, dom_ms, dom_n, dom_kernel = "tc_nn_kernel (Y = A Z, 3xTF32 tcgen05)", ax_ms, ax_n, "tc_nn_kernel"
    else:
        dom, dom_ms, dom_n, dom_kernel = ("tc_tn2_kernel + split_transpose_kernel + sum_chunks_kernel "
                                          "(Z = A^T Q, 3xTF32 tcgen05; the basis split and transposed first)",
                                          atx_ms, atx_n, "tc_tn2_kernel")
    per_launch_bytes = 4.0 * m * n
    achieved = per_launch_bytes / (dom_ms / dom_n * 1e-3) / 1e9 if dom_n else None
    roofline = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": hbm, "unit": "GB/s",
                "frac": (achieved / hbm) if achieved else None,
                "traffic": traffic_for("k_tc.cu", dom_kernel),
                "algorithmic_bytes_per_launch": per_launch_bytes,
                "peak_source": f"{src} (MEASURED_PEAKS.json hbm_gbs)" if src == "measured" else "fallback 6800 GB/s",
                "stage_ms_per_step": {kk: vv[0] / args.steps for kk, vv in prof.items()},
                "timing": "kernel durations from CUDA events around each kernel group over an instrumented "
                          "pass of the same K steps directly after the timed region"}

    # end to end through the public API with host buffers (pinned), copies inside the timed region
    e2e = None
    if rank == 0 or world > 1:
        Ah = A0.cpu().pin_memory()
        Omh = Om.cpu().pin_memory()
        Sh = torch.empty_like(S, device="cpu").pin_memory()
        Uh = torch.empty_like(U, device="cpu").pin_memory()
        Vh = torch.empty_like(V, device="cpu").pin_memory()
        n_e2e = max(1, min(args.steps, 10))
        torch.cuda.synchronize(dev)
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        for _ in range(n_e2e):
            A.copy_(Ah, non_blocking=True)
            Om.copy_(Omh, non_blocking=True)
            step()
            Sh.copy_(S, non_blocking=True)
            Uh.copy_(U, non_blocking=True)
            Vh.copy_(V, non_blocking=True)
        f1.record(stream)
        torch.cuda.synchronize(dev)
        ems = f0.elapsed_time(f1)
        e2e = {"value": flops * n_e2e / (ems * 1e-3) / 1e9, "unit": "GFLOP/s",
               "h2d_bytes_per_step": Ah.numel() * 4 + Omh.numel() * 4,
               "d2h_bytes_per_step": Sh.numel() * 8 + Uh.numel() * 4 + Vh.numel() * 4,
               "ms_per_step": ems / n_e2e}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rows = args.cpu_baseline_rows
        Ah32 = A0[:rows].cpu().numpy()
        Omh = Om.cpu().numpy()
        ts = sorted(oracle_sample(Ah32, Omh, k, q, rows) for _ in range(3))
        tsec = ts[1]  # median of three solves
        cpu = {"value": alg_flops(rows, n, k, p, q) / tsec / 1e9, "unit": "GFLOP/s", "cores": os.cpu_count(),
               "kind": "oracle",
               "sample": f"first {rows} of {m} rows (same n, k, p, q, Omega); FP64 C oracle, OpenMP on all "
                         f"{os.cpu_count()} host threads; median of 3 solves "
                         f"({ts[0]:.2f} / {ts[1]:.2f} / {ts[2]:.2f} s)"}

    if rank == 0:
        line = {
            "metric": "rSVD GFLOP/s", "value": value, "unit": "GFLOP/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "m": m, "n": n, "k": k, "p": p, "q": q,
                       "l2": "inputs larger than L2 (A is 0.8 GB), no flush",
                       "parallelism": f"replicas{world}"},
            "solves_per_s": world * args.steps / (ms_max * 1e-3),
            "status": st,
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": launches, "clocks": clocks, "peaks_source": src,
        }
        print(json.dumps(line), flush=True)
    plan.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--sample-rows", type=int, default=40000, help="rows per reference-arm step")
    ap.add_argument("--cpu-baseline-rows", type=int, default=100000, help="rows of the cpu_baseline sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--method", default="rsvd", choices=["rsvd", "block_krylov", "gkl", "precision", "gram_grid"],
                    help="rsvd: the default workload; block_krylov: the Sec. 3.1.1 workload; gkl: the Lanczos "
                         "workload; precision: the bfloat16 / e4m3 precision form (--dtype)")
    ap.add_argument("--dtype", default=None, choices=["bf16", "fp8", "f32", "f64"],
                    help="storage of --method precision (bf16 | fp8) or gram_grid (f64 | f32)")
    ap.add_argument("--bk-cpu-rows", type=int, default=16384, help="rows of the block Krylov cpu_baseline sample")
    ap.add_argument("--gkl-cpu-rows", type=int, default=16384, help="rows of the Lanczos cpu_baseline sample")
    ap.add_argument("--gkl-two-pass", action="store_true", help="--method gkl: read A twice per step")
    ap.add_argument("--prec-cpu-rows", type=int, default=8192, help="rows of the precision-form cpu_baseline sample")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.method == "block_krylov":
        return run_block_krylov(args)
    if args.method == "gkl":
        return run_gkl(args)
    if args.method == "precision":
        args.dtype = args.dtype or "bf16"
        if args.dtype not in ("bf16", "fp8"):
            ap.error("--method precision takes --dtype bf16 or fp8")
        return run_precision(args)
    if args.method == "gram_grid":
        args.dtype = args.dtype or "f64"
        return run_gram_grid(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
