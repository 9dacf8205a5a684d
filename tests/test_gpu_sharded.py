"""GPU: the row-sharded randomized PCA (rsvd_sharded) with two ranks as separate processes
on the one GPU, reducing over gloo on the host (no kernel of one rank waits on the other).

Against the float64 oracle on the whole matrix (same Omega): sigma within the float32
path's 1e-5 sigma_1 (float64: 1e-10 relative); S and V bitwise equal on both ranks; the
assembled U (rank 0's rows, then rank 1's) and V orthonormal; ||A - 1 mu^T||_F^2 to 1e-6
relative; A^T u_i = sigma_i v_i to the same tolerance as sigma.  A rank that leaves before
the solve ends the other's solve with RSVD_ERR_REDUCE (its next reduction fails on the
host)."""
import numpy as np
import pytest
import torch

import oracle
import paper_1906_12085_gb300 as g
from shard_ranks import run_ranks
from shard_worker import matrix

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1906_12085_gb300 import build
    build.build()
    oracle.build()


@pytest.mark.parametrize("m,n,k,p,q,dtype", [
    (20011, 256, 20, 12, 2, "f32"),    # ragged blocks (10006 + 10005 rows)
    (40000, 512, 48, 16, 1, "f32"),
    (6001, 128, 16, 8, 2, "f64"),
])
def test_sharded_rsvd_two_ranks_match_oracle(m, n, k, p, q, dtype, tmp_path):
    seed = 61001
    procs, outs, logs = run_ranks(2, ["solve", str(m), str(n), str(k), str(p), str(q), dtype, str(seed)], tmp_path)
    for pr, log in zip(procs, logs):
        assert pr.returncode == 0, log[-3000:]
    r = [np.load(o) for o in outs]
    for x in r:
        assert int(x["st"]) == g.RSVD_OK and int(x["sync"]) == g.RSVD_OK
    assert np.array_equal(r[0]["S"], r[1]["S"]) and np.array_equal(r[0]["V"], r[1]["V"])
    assert int(r[0]["r1"]) == int(r[1]["r0"]) and int(r[1]["r1"]) == m
    S, V = r[0]["S"], r[0]["V"]
    U = np.concatenate([r[0]["U"], r[1]["U"]])
    A = matrix(m, n, seed).numpy()
    if dtype == "f32":
        A = A.astype(np.float32).astype(np.float64)
    import synth
    Om = synth.gaussian(n, k + p, seed=seed + 3, dtype=torch.float32 if dtype == "f32" else torch.float64)
    Ac, mu, fro2o = oracle.center(A)
    s, Uo, Vo = oracle.rsvd(Ac, Om.double().numpy(), q=q, k=k)
    tol = 1e-5 * s[0] if dtype == "f32" else 1e-10 * s[0]
    err = np.abs(S - s).max()
    print(f"sharded {dtype} {m}x{n} k={k}: max sigma error {err / s[0]:.2e} sigma_1")
    assert err <= tol, err / s[0]
    assert abs(float(r[0]["fro2"]) - fro2o) <= 1e-6 * fro2o
    otol = 1e-5 if dtype == "f32" else 1e-10
    assert np.abs(U.T @ U - np.eye(k)).max() <= otol
    assert np.abs(V.T @ V - np.eye(k)).max() <= otol
    res = np.linalg.norm(Ac.T @ U - V * S[None, :], axis=0).max()   # A^T u_i = sigma_i v_i (A^T Q = B^T)
    assert res <= tol, res / s[0]


def test_rank_leaving_before_the_solve_ends_the_other_with_reduce_error(tmp_path):
    procs, outs, logs = run_ranks(2, ["leave", "20011", "256", "20", "12", "1", "f32", "61011"], tmp_path)
    assert procs[1].returncode == 0
    assert procs[0].returncode == 0, logs[0][-3000:]
    x = np.load(outs[0])
    assert int(x["st"]) == g.RSVD_ERR_REDUCE


def test_sharded_rejects_other_plans_and_sizes():
    dev = torch.device("cuda")
    m, n, k, p = 2000, 64, 8, 8
    A = torch.randn(m, n, device=dev)
    Om = torch.randn(n, k + p, device=dev)
    S = torch.zeros(k, dtype=torch.float64, device=dev)
    U = torch.zeros(m, k, device=dev)
    V = torch.zeros(n, k, device=dev)
    red = lambda buf: None  # noqa: E731  (one rank: the local sums are the totals)
    with g.rsvd_plan_create(m, n, k, p, 1, g.RSVD_F32) as plan:
        assert g.rsvd_sharded(plan, m - 1, A, Om, S, U, V, red) == g.RSVD_ERR_ARG   # m_total < local rows
        assert g.rsvd_sharded(plan, m, A, Om, S, U, V, red) == g.RSVD_OK
        assert g.rsvd_plan_sync(plan) == g.RSVD_OK
        S1 = S.clone()
        g.check(g.rsvd(plan, A, None, Om, S, U, V))
        assert g.rsvd_plan_sync(plan) == g.RSVD_OK
        assert torch.allclose(S1, S, rtol=0, atol=1e-5 * S[0].item())   # one rank = the plain solve

        def boom(_):
            raise RuntimeError("no peers")
        assert g.rsvd_sharded(plan, m, A, Om, S, U, V, boom) == g.RSVD_ERR_REDUCE
        g.rsvd_plan_sync(plan)
    codes = torch.zeros(m, n, dtype=torch.int16, device=dev)
    with g.rsvd_plan_create(m, n, k, p, 1, g.RSVD_BF16) as plan:
        assert g.rsvd_sharded(plan, m, codes, Om, S, U, V, red) == g.RSVD_ERR_UNSUPPORTED
