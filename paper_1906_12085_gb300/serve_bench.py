"""Poisson stream of randomized PCA requests through the serving loop.

    python -m paper_1906_12085_gb300.serve_bench --requests 4096 --rates 100,500,1000,2000,5000
    python -m paper_1906_12085_gb300.serve_bench --mode sequential ...   # one request at a time

Request mix (q = 2, t = 0.9): n uniform in {64, 128, 256, 512, 1024, 2048},
k uniform in {8, 16, 32, 64, 128}, p = min(8, lmax - k) (at least 0), then k
capped at lmax - p and at n - p (so l = k + p <= min(n, lmax); lmax = 128 by
default, 112 for the bfloat16 / e4m3 forms), m uniform in [max(1000, n),
200000], inter-arrival times exponential at the given rate.
Matrices are materialised before the stream starts: for every n a pool of
`--pool` float32 matrices of 200000 x n, matrix j = G diag(i^-alpha_j) / sqrt(m)
(G seeded Gaussian, alpha_j uniform in [0.5, 2]), stored in the `--dtype`
storage type by rsvd_quantize (e4m3: with its column scales); a request takes
the leading m rows of one of them (its own alpha and seed), so the whole stream
fits in HBM and no generation or conversion runs while it is timed.  Omega
comes from a seeded pool per (n, l).

`server` mode submits each request at its arrival time to rsvd_server_* and
polls (a host backlog feeds it while it holds fewer than 128 requests, so
output buffers stay bounded when the rate exceeds capacity); `sequential` mode solves the requests one at a time in arrival order
with rsvd() on plans carved from one preallocated workspace (the plain GPU
method, no batching, no overlap).  Latency = completion - arrival; prints one
JSON line per rate.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np
import torch

import paper_1906_12085_gb300 as g

NS = (64, 128, 256, 512, 1024, 2048)
KS = (8, 16, 32, 64, 128)
M_MAX = 200000
Q = 2
T = 0.9


def shape(n: int, k: int, lmax: int) -> tuple[int, int]:
    """(k, p) of a drawn (n, k): l = k + p <= min(n, lmax)."""
    p = max(0, min(8, lmax - k))
    return min(k, lmax - p, n - p), p


def store(A, dtype):
    """(stored matrix, column scales or None) of a float32 device matrix."""
    if dtype == g.RSVD_F32:
        return A, None
    if dtype == g.RSVD_BF16:
        Aq = torch.empty(A.shape, dtype=torch.int16, device=A.device)
        g.check(g.rsvd_quantize(A, dtype, Aq), "rsvd_quantize")
        return Aq, None
    Aq = torch.empty(A.shape, dtype=torch.uint8, device=A.device)
    sc = torch.empty(A.shape[1], dtype=torch.float32, device=A.device)
    g.check(g.rsvd_quantize(A, dtype, Aq, sc), "rsvd_quantize")
    return Aq, sc


def make_pool(pool: int, dev, seed: int = 7, dtype: int = g.RSVD_F32, lmax: int = 128):
    gen = torch.Generator(device=dev)
    mats, alphas = {}, {}
    rng = np.random.default_rng(seed)
    for n in NS:
        mats[n], alphas[n] = [], []
        for j in range(pool):
            gen.manual_seed(1_000_000 + 97 * n + j)
            a = float(rng.uniform(0.5, 2.0))
            sig = torch.arange(1, n + 1, device=dev, dtype=torch.float32).pow(-a)
            A = torch.randn(M_MAX, n, generator=gen, device=dev, dtype=torch.float32)
            A.mul_(sig / float(np.sqrt(M_MAX)))
            mats[n].append(store(A, dtype))
            del A
            alphas[n].append(a)
    omegas = {}
    for n in NS:
        for k in KS:
            k, p = shape(n, k, lmax)
            l = k + p
            gen.manual_seed(2_000_000 + 131 * n + l)
            omegas[(n, l)] = torch.randn(n, l, generator=gen, device=dev, dtype=torch.float32)
    return mats, alphas, omegas


def make_requests(count: int, rate: float, pool: int, seed: int, lmax: int = 128):
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, size=count))
    reqs = []
    for i in range(count):
        n = int(rng.choice(NS))
        k = int(rng.choice(KS))
        m = int(rng.integers(max(1000, n), M_MAX + 1))
        k, p = shape(n, k, lmax)
        reqs.append(dict(id=i, t=float(t[i]), m=m, n=n, k=k, p=p, j=int(rng.integers(pool))))
    return reqs


def pct(x, q):
    return float(np.percentile(np.asarray(x), q)) if len(x) else None


def run_server(reqs, mats, omegas, dev, budget, max_batch, max_inflight, max_pending=128, dtype=g.RSVD_F32):
    """Requests arrive on the Poisson clock into a host backlog and are handed to the
    server while it holds fewer than `max_pending`; latency counts from arrival."""
    out = {}
    lat, done = [], []
    srv = g.rsvd_server_create(budget, max_batch=max_batch, max_inflight=max_inflight)
    try:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        offset = None            # server clock - driver clock (ms)
        i = 0
        while len(done) < len(reqs):
            now = time.perf_counter() - t0
            while i < len(reqs) and reqs[i]["t"] <= now and g.rsvd_server_pending(srv) < max_pending:
                r = reqs[i]
                Aj, sc = mats[r["n"]][r["j"]]
                A = Aj[: r["m"]]
                Om = omegas[(r["n"], r["k"] + r["p"])]
                S = torch.empty(r["k"], dtype=torch.float64, device=dev)
                U = torch.empty(r["m"], r["k"], device=dev)
                V = torch.empty(r["n"], r["k"], device=dev)
                out[r["id"]] = (S, U, V, (time.perf_counter() - t0) * 1e3)
                g.check(g.rsvd_server_submit_ex(srv, r["id"], r["k"], r["p"], Q, dtype, T, A, sc, Om, S, U, V),
                        "submit")
                i += 1
            for c in g.rsvd_server_poll(srv, 512):
                S, U, V, sub_drv = out.pop(c["id"])
                if offset is None:
                    offset = c["submit_ms"] - sub_drv
                lat.append(c["done_ms"] - (reqs[c["id"]]["t"] * 1e3 + offset))
                c["arrival_ms"] = reqs[c["id"]]["t"] * 1e3 + offset
                done.append(c)
            if i < len(reqs) and g.rsvd_server_pending(srv) == 0:
                wait = reqs[i]["t"] - (time.perf_counter() - t0)
                if wait > 0:
                    time.sleep(min(wait, 0.001))
        first = min(c["arrival_ms"] for c in done)
        last = max(c["done_ms"] for c in done)
        bad = [c for c in done if c["status"] not in (g.RSVD_OK, g.RSVD_WARN_K_GT_k)]
        return dict(solves_per_s=len(done) / ((last - first) * 1e-3), p50_ms=pct(lat, 50), p99_ms=pct(lat, 99),
                    mean_batch=float(np.mean([c["batch"] for c in done])), failed=len(bad), completed=len(done))
    finally:
        srv.close()


def run_sequential(reqs, mats, omegas, dev, dtype=g.RSVD_F32):
    ws_max = max(g.rsvd_workspace_query(r["m"], r["n"], r["k"], r["p"], Q, dtype)[1] for r in reqs)
    ws = torch.empty(ws_max, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    lat = []
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    first = None
    for r in reqs:
        now = time.perf_counter() - t0
        if r["t"] > now:
            time.sleep(r["t"] - now)
        if first is None:
            first = r["t"]
        Aj, sc = mats[r["n"]][r["j"]]
        A = Aj[: r["m"]]
        Om = omegas[(r["n"], r["k"] + r["p"])]
        S = torch.empty(r["k"], dtype=torch.float64, device=dev)
        U = torch.empty(r["m"], r["k"], device=dev)
        V = torch.empty(r["n"], r["k"], device=dev)
        plan = g.rsvd_plan_create_in(r["m"], r["n"], r["k"], r["p"], Q, dtype, stream, ws)
        g.check(g.rsvd(plan, A, sc, Om, S, U, V), "rsvd")
        st, K = g.pca_threshold(plan, T)   # synchronises: the request is complete
        plan.close()
        end = time.perf_counter() - t0
        lat.append((end - r["t"]) * 1e3)
    total = time.perf_counter() - t0 - first
    return dict(solves_per_s=len(reqs) / total, p50_ms=pct(lat, 50), p99_ms=pct(lat, 99), mean_batch=1.0,
                failed=0, completed=len(reqs))


def main(argv=None) -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("--requests", type=int, default=4096)
    ap.add_argument("--rates", default="100,200,500,1000,2000,5000")
    ap.add_argument("--pool", type=int, default=4)
    ap.add_argument("--mode", choices=["server", "sequential"], default="server")
    ap.add_argument("--budget-gb", type=float, default=48.0)
    ap.add_argument("--max-batch", type=int, default=8)
    ap.add_argument("--max-inflight", type=int, default=8)
    ap.add_argument("--seed", type=int, default=7)
    ap.add_argument("--dtype", choices=["f32", "bf16", "fp8"], default="f32", help="storage type of the matrices")
    ap.add_argument("--lmax", type=int, default=0, help="largest l of the mix (default 128; 112 for bf16 / fp8)")
    ap.add_argument("--autotune", action="store_true",
                    help="tune the product decomposition of every (ceil log2 m, n, l) bucket the stream hits first")
    a = ap.parse_args(argv)
    dev = torch.device("cuda")
    from paper_1906_12085_gb300 import build
    build.build()
    dt = {"f32": g.RSVD_F32, "bf16": g.RSVD_BF16, "fp8": g.RSVD_FP8_E4M3}[a.dtype]
    lmax = a.lmax or (128 if dt == g.RSVD_F32 else 112)
    mats, alphas, omegas = make_pool(a.pool, dev, dtype=dt, lmax=lmax)
    if a.autotune:
        t0 = time.perf_counter()
        seen = {}
        for rate in [float(x) for x in a.rates.split(",")]:
            for r in make_requests(a.requests, rate, a.pool, a.seed, lmax):
                lgm = int(np.ceil(np.log2(r["m"])))
                seen.setdefault((lgm, r["n"], -(-(r["k"] + r["p"]) // 16)), r)
        if dt != g.RSVD_F32:
            raise SystemExit("--autotune tunes the float32 products only")
        for r in seen.values():
            A = mats[r["n"]][r["j"]][0][: r["m"]]
            Om = omegas[(r["n"], r["k"] + r["p"])]
            with g.rsvd_plan_create(r["m"], r["n"], r["k"], r["p"], Q, g.RSVD_F32) as plan:
                g.check(g.rsvd_autotune(plan, A, Om, concurrency=4)[0], "rsvd_autotune")
        print(json.dumps({"autotuned_buckets": len(seen), "seconds": time.perf_counter() - t0}), flush=True)
    warm = make_requests(64, 1e6, a.pool, a.seed + 1, lmax)   # warm-up: kernels loaded, allocator primed
    if a.mode == "server":
        run_server(warm, mats, omegas, dev, int(a.budget_gb * 2**30), a.max_batch, a.max_inflight, dtype=dt)
    else:
        run_sequential(warm[:8], mats, omegas, dev, dt)
    for rate in [float(x) for x in a.rates.split(",")]:
        reqs = make_requests(a.requests, rate, a.pool, a.seed, lmax)
        flops = sum(2.0 * r["m"] * r["n"] * (r["k"] + r["p"]) * (2 * Q + 2) for r in reqs)
        if a.mode == "server":
            res = run_server(reqs, mats, omegas, dev, int(a.budget_gb * 2**30), a.max_batch, a.max_inflight,
                             dtype=dt)
        else:
            res = run_sequential(reqs, mats, omegas, dev, dt)
        res.update(mode=a.mode, dtype=a.dtype, lmax=lmax, rate=rate, requests=a.requests, pool=a.pool,
                   mean_request_gflop=flops / len(reqs) / 1e9,
                   config=dict(budget_gb=a.budget_gb, max_batch=a.max_batch, max_inflight=a.max_inflight))
        print(json.dumps(res), flush=True)
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
