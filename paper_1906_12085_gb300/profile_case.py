"""One solve of one path at one shape, for kernel profilers.

    python -m paper_1906_12085_gb300.profile_case rsvd --m 200000 --n 1000 --k 50 --p 10 --q 2
    python -m paper_1906_12085_gb300.profile_case gkl  --m 262144 --n 2048 --k 100 --steps 150
    python -m paper_1906_12085_gb300.profile_case exact --m 2000 --n 100 --dtype f64
    python -m paper_1906_12085_gb300.profile_case gram --m 10000 --n 2000 --dtype f32
    python -m paper_1906_12085_gb300.profile_case rsvd --m 1048576 --n 4096 --k 96 --p 16 --q 3 --dtype bf16
    python -m paper_1906_12085_gb300.profile_case rsvd --m 1048576 --n 4096 --k 96 --p 16 --q 3 --dtype fp8
    python -m paper_1906_12085_gb300.profile_case bk --m 1048576 --n 4096 --k 256 --b 96 --iters 2 --repeat 2 --timed 3

`bk` is the block Krylov method (blocks of --b columns, --iters + 1 of them).
The matrix is seeded Gaussian data made on the device (a kernel's DRAM traffic and
its launch shape do not depend on the values), so few launches precede the
library's own.  The solve runs `--repeat` times as direct launches (tracing on,
which disables graph capture); with more than one, the first is a warm-up and the
per-stage times printed are the mean of the others.  The status is checked; the
process exits non-zero on any error.
"""
from __future__ import annotations

import argparse
import sys

import torch

import paper_1906_12085_gb300 as g


def main(argv=None) -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("path", choices=["rsvd", "gkl", "exact", "gram", "bk"])
    ap.add_argument("--m", type=int, default=200000)
    ap.add_argument("--n", type=int, default=1000)
    ap.add_argument("--k", type=int, default=50)
    ap.add_argument("--p", type=int, default=10)
    ap.add_argument("--q", type=int, default=2)
    ap.add_argument("--steps", type=int, default=150)
    ap.add_argument("--b", type=int, default=96, help="block width (bk)")
    ap.add_argument("--iters", type=int, default=2, help="Krylov iterations (bk)")
    ap.add_argument("--dtype", choices=["f32", "f64", "bf16", "fp8"], default="f32")
    ap.add_argument("--repeat", type=int, default=1)
    ap.add_argument("--timed", type=int, default=0,
                    help="then time this many solves (rsvd: graph replays; bk: direct launches)")
    ap.add_argument("--save", default="", help="write the singular values (float64, .npy) to this path")
    a = ap.parse_args(argv)
    dev = torch.device("cuda")
    dt = {"f32": g.RSVD_F32, "f64": g.RSVD_F64, "bf16": g.RSVD_BF16, "fp8": g.RSVD_FP8_E4M3}[a.dtype]
    tdt = torch.float64 if a.dtype == "f64" else torch.float32   # element type of Omega, U, V
    gen = torch.Generator(device=dev)
    gen.manual_seed(12085)
    A = torch.randn(a.m, a.n, generator=gen, device=dev, dtype=tdt)
    sc = None
    if a.dtype == "bf16":  # stored as bfloat16 codes by the library's quantiser
        Aq = torch.empty(a.m, a.n, dtype=torch.int16, device=dev)
        g.check(g.rsvd_quantize(A, g.RSVD_BF16, Aq), "rsvd_quantize")
        del A
        A = Aq
    elif a.dtype == "fp8":  # e4m3 codes and column scales
        Aq = torch.empty(a.m, a.n, dtype=torch.uint8, device=dev)
        sc = torch.empty(a.n, dtype=torch.float32, device=dev)
        g.check(g.rsvd_quantize(A, g.RSVD_FP8_E4M3, Aq, sc), "rsvd_quantize")
        del A
        A = Aq
    k = a.k if a.path not in ("exact", "gram") else a.n
    S = torch.zeros(k, dtype=torch.float64, device=dev)
    if a.path in ("exact", "gram"):
        U = torch.zeros(a.m, a.n, dtype=tdt, device=dev)
        V = torch.zeros(a.n, a.n, dtype=tdt, device=dev)
    else:
        U = torch.zeros(a.m, k, dtype=tdt, device=dev)
        V = torch.zeros(a.n, k, dtype=tdt, device=dev)
    if a.path == "bk":
        plan = g.rsvd_plan_create_block_krylov(a.m, a.n, k, a.b, a.iters, dt)
    else:
        plan = g.rsvd_plan_create(a.m, a.n, 1 if a.path == "gram" else k, a.p if a.path == "rsvd" else 0, a.q, dt)
    with plan:
        g.rsvd_plan_profile(plan, True)
        for rep in range(a.repeat):
            if rep == 1:  # with --repeat > 1 the first solve is a warm-up (module loading, first touch)
                g.check(g.rsvd_plan_sync(plan), "solve status")
                g.rsvd_plan_profile_read(plan)
            if a.path == "rsvd":
                Om = torch.randn(a.n, a.k + a.p, generator=gen, device=dev, dtype=tdt)
                g.check(g.rsvd(plan, A, sc, Om, S, U, V), "rsvd")
            elif a.path == "bk":
                Om = torch.randn(a.n, a.b, generator=gen, device=dev, dtype=tdt)
                g.check(g.rsvd_block_krylov(plan, A, Om, S, U, V), "rsvd_block_krylov")
            elif a.path == "gkl":
                v1 = torch.randn(a.n, generator=gen, device=dev, dtype=tdt)
                v1 /= v1.norm()
                g.check(g.svd_truncated_krylov(plan, A, v1, a.steps, S, U, V), "svd_truncated_krylov")
            elif a.path == "gram":
                g.check(g.svd_exact(plan, A, g.RSVD_EXACT_GRAM, S, U, V), "svd_exact")
            else:
                g.check(g.svd_exact(plan, A, g.RSVD_EXACT_QR_JACOBI, S, U, V), "svd_exact")
        g.check(g.rsvd_plan_sync(plan), "solve status")
        prof = g.rsvd_plan_profile_read(plan)
        if a.timed and a.path in ("rsvd", "bk"):   # CUDA events on the plan's stream (torch's current one)
            g.rsvd_plan_profile(plan, False)
            s0 = torch.cuda.current_stream()

            def solve():
                if a.path == "rsvd":
                    return g.rsvd(plan, A, sc, Om, S, U, V)
                return g.rsvd_block_krylov(plan, A, Om, S, U, V)
            for _ in range(2):
                g.check(solve())
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s0)
            for _ in range(a.timed):
                g.check(solve())
            e1.record(s0)
            torch.cuda.synchronize()
            g.check(g.rsvd_plan_sync(plan), "timed solves status")
            ms = e0.elapsed_time(e1) / a.timed
            if a.path == "rsvd":
                l = a.k + a.p
                flops = 2.0 * a.m * a.n * l * (2 * a.q + 2) + 2.0 * a.m * l * l * (a.q + 2) + 2.0 * a.n * l * l
            else:  # products with A (2 i + 1 of width b, T = A^T Q of width W), QR of the W basis, SVD of T
                W = (a.iters + 1) * a.b
                flops = 2.0 * a.m * a.n * a.b * (2 * a.iters + 1) + 2.0 * a.m * a.n * W + 2.0 * a.m * W * W \
                    + 2.0 * a.n * W * W
            print(f"timed: {ms:.3f} ms per solve, {flops / (ms * 1e-3) / 1e12:.1f} TFLOP/s over {a.timed} solves")
    torch.cuda.synchronize()
    if a.save:
        import numpy as np
        np.save(a.save, S.cpu().numpy())
    traced = max(a.repeat - 1, 1)
    print({kk: round(v[0] / traced, 4) for kk, v in prof.items()}, "ms per traced solve;", "sigma_1 =", float(S[0]))
    return 0


if __name__ == "__main__":
    sys.exit(main())
