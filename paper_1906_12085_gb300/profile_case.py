"""One solve of one path at one shape, for kernel profilers.

    python -m paper_1906_12085_gb300.profile_case rsvd --m 200000 --n 1000 --k 50 --p 10 --q 2
    python -m paper_1906_12085_gb300.profile_case gkl  --m 262144 --n 2048 --k 100 --steps 150
    python -m paper_1906_12085_gb300.profile_case exact --m 2000 --n 100 --dtype f64

The matrix is seeded Gaussian data made on the device (a kernel's DRAM traffic and
its launch shape do not depend on the values), so few launches precede the
library's own.  The solve runs once as direct launches (tracing on, which
disables graph capture), then its status is checked; the process exits non-zero
on any error.
"""
from __future__ import annotations

import argparse
import sys

import torch

import paper_1906_12085_gb300 as g


def main(argv=None) -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("path", choices=["rsvd", "gkl", "exact"])
    ap.add_argument("--m", type=int, default=200000)
    ap.add_argument("--n", type=int, default=1000)
    ap.add_argument("--k", type=int, default=50)
    ap.add_argument("--p", type=int, default=10)
    ap.add_argument("--q", type=int, default=2)
    ap.add_argument("--steps", type=int, default=150)
    ap.add_argument("--dtype", choices=["f32", "f64"], default="f32")
    ap.add_argument("--repeat", type=int, default=1)
    a = ap.parse_args(argv)
    dev = torch.device("cuda")
    dt = g.RSVD_F32 if a.dtype == "f32" else g.RSVD_F64
    tdt = torch.float32 if a.dtype == "f32" else torch.float64
    gen = torch.Generator(device=dev)
    gen.manual_seed(12085)
    A = torch.randn(a.m, a.n, generator=gen, device=dev, dtype=tdt)
    k = a.k if a.path != "exact" else a.n
    S = torch.zeros(k, dtype=torch.float64, device=dev)
    if a.path == "exact":
        U = torch.zeros(a.m, a.n, dtype=tdt, device=dev)
        V = torch.zeros(a.n, a.n, dtype=tdt, device=dev)
    else:
        U = torch.zeros(a.m, k, dtype=tdt, device=dev)
        V = torch.zeros(a.n, k, dtype=tdt, device=dev)
    with g.rsvd_plan_create(a.m, a.n, k, a.p if a.path == "rsvd" else 0, a.q, dt) as plan:
        g.rsvd_plan_profile(plan, True)
        for _ in range(a.repeat):
            if a.path == "rsvd":
                Om = torch.randn(a.n, a.k + a.p, generator=gen, device=dev, dtype=tdt)
                g.check(g.rsvd(plan, A, None, Om, S, U, V), "rsvd")
            elif a.path == "gkl":
                v1 = torch.randn(a.n, generator=gen, device=dev, dtype=tdt)
                v1 /= v1.norm()
                g.check(g.svd_truncated_krylov(plan, A, v1, a.steps, S, U, V), "svd_truncated_krylov")
            else:
                g.check(g.svd_exact(plan, A, g.RSVD_EXACT_QR_JACOBI, S, U, V), "svd_exact")
        g.check(g.rsvd_plan_sync(plan), "solve status")
        prof = g.rsvd_plan_profile_read(plan)
    torch.cuda.synchronize()
    print({kk: round(v[0], 4) for kk, v in prof.items()}, "ms;", "sigma_1 =", float(S[0]))
    return 0


if __name__ == "__main__":
    sys.exit(main())
