"""Serving loop (rsvd_server_*): continuous batching with HBM admission.

A mixed stream of requests goes through a server whose arena holds only a few
workspaces at a time, so requests queue, batch (consecutive requests of the
same l) and overlap.  Every result must equal the same request solved alone,
bit for bit (status, K, S, U, V): the split-K sums run in a fixed order and a
batch runs each problem's own kernels.  Admission follows arrival order.

Every served result is also compared with the FP64 oracle (Sec. 3.1.2 with the
same Omega) on the stored matrix -- the float32 values, or the bfloat16 / e4m3
codes the library's quantiser wrote, dequantised exactly -- at the tolerance of
its storage type: |sigma_hat_i - sigma_i^O| <= 1e-5 (float32), 1e-4 (bfloat16),
1e-3 (e4m3) times sigma_1^O; the projection gap (||A - U U^T A||_F - ||A - U^O
U^O^T A||_F) / ||A||_F within the same bound; U and V orthonormal to 1e-5.  The
request mix draws sigma_i = i^-alpha with alpha in [0.5, 2], whose power-step
bases at q = 2 reach condition numbers far beyond a float32 Gram matrix."""
import numpy as np
import pytest
import torch

import oracle
import paper_1906_12085_gb300 as g
import synth

pytestmark = pytest.mark.gpu

Q = 2
TOL = {g.RSVD_F32: 1e-5, g.RSVD_BF16: 1e-4, g.RSVD_FP8_E4M3: 1e-3}


def _proj_residual(A, U):
    """||A - U U^T A||_F for orthonormal U (float64)."""
    B = U.T @ A
    return np.sqrt(max(np.sum(A * A) - np.sum(B * B), 0.0))


def _stored64(A_dev, sc_dev, dtype):
    """The stored matrix in float64: float32 values, or the codes dequantised by the oracle."""
    if dtype == g.RSVD_F32:
        return A_dev.cpu().double().numpy()
    if dtype == g.RSVD_BF16:
        return oracle.dequantize_bf16(A_dev.cpu().numpy().view(np.uint16))
    return oracle.dequantize_e4m3(A_dev.cpu().numpy(), sc_dev.cpu().numpy())


def _check_oracle(A64, Om, k, S, U, V, dtype, status):
    """A served result against the oracle on the stored matrix (tolerances in the module doc)."""
    assert status in (g.RSVD_OK, g.RSVD_WARN_K_GT_k, g.RSVD_WARN_RANK_DEFICIENT), status
    Ac, _, _ = oracle.center(A64)
    s, Uo, _ = oracle.rsvd(Ac, Om.double(), q=Q, k=k)
    tol = TOL[dtype]
    err = np.abs(S - s).max() / s[0]
    Ug = U.astype(np.float64)
    gap = (_proj_residual(Ac, Ug) - _proj_residual(Ac, Uo)) / np.sqrt(np.sum(Ac * Ac))
    assert err <= tol, (dtype, err)
    assert gap <= tol, (dtype, gap)
    assert np.abs(Ug.T @ Ug - np.eye(k)).max() <= 1e-5
    Vg = V.astype(np.float64)
    assert np.abs(Vg.T @ Vg - np.eye(k)).max() <= 1e-5
    return err


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1906_12085_gb300 import build
    build.build()


def _requests(count, seed):
    rng = np.random.default_rng(seed)
    reqs = []
    for i in range(count):
        n = int(rng.choice([64, 128, 256]))
        m = int(rng.integers(max(1000, n), 20000))
        k = int(rng.choice([8, 16, 24]))
        p = 8
        alpha = float(rng.uniform(0.5, 2.0))
        sig = synth.spectrum_power(n, alpha)
        A = synth.prescribed(m, n, sig, 1000 + i, 2000 + i).float()
        Om = synth.gaussian(n, k + p, seed=3000 + i, dtype=torch.float32)
        reqs.append(dict(id=i, m=m, n=n, k=k, p=p, A=A, Om=Om))
    return reqs


def _alone(r):
    dev = torch.device("cuda")
    S = torch.zeros(r["k"], dtype=torch.float64, device=dev)
    U = torch.zeros(r["m"], r["k"], device=dev)
    V = torch.zeros(r["n"], r["k"], device=dev)
    with g.rsvd_plan_create(r["m"], r["n"], r["k"], r["p"], Q, g.RSVD_F32) as plan:
        g.check(g.rsvd(plan, r["A"].to(dev), None, r["Om"].to(dev), S, U, V))
        st = g.rsvd_plan_sync(plan)
        stK, K = g.pca_threshold(plan, 0.9)
    return (stK if st == g.RSVD_OK else st), K, S.cpu().numpy(), U.cpu().numpy(), V.cpu().numpy()


def test_served_results_equal_alone_bitwise():
    reqs = _requests(24, 7)
    alone = {r["id"]: _alone(r) for r in reqs}
    dev = torch.device("cuda")
    for r in reqs:
        r["Ad"], r["Od"] = r["A"].to(dev), r["Om"].to(dev)
        r["S"] = torch.zeros(r["k"], dtype=torch.float64, device=dev)
        r["U"] = torch.zeros(r["m"], r["k"], device=dev)
        r["V"] = torch.zeros(r["n"], r["k"], device=dev)
    ws = max(g.rsvd_workspace_query(r["m"], r["n"], r["k"], r["p"], Q)[1] for r in reqs)
    torch.cuda.synchronize()
    done = []
    with g.rsvd_server_create(3 * ws, max_batch=4, max_inflight=3) as srv:
        for i, r in enumerate(reqs):           # arrivals interleaved with progress
            g.check(g.rsvd_server_submit(srv, r["id"], r["k"], r["p"], Q, 0.9, r["Ad"], r["Od"], r["S"], r["U"],
                                         r["V"]), "submit")
            if i % 3 == 2:
                done += g.rsvd_server_poll(srv)
        while g.rsvd_server_pending(srv) > 0:
            done += g.rsvd_server_poll(srv)
    torch.cuda.synchronize()
    assert sorted(c["id"] for c in done) == [r["id"] for r in reqs]
    assert any(c["batch"] > 1 for c in done)
    starts = {c["id"]: c["start_ms"] for c in done}
    assert all(starts[i] <= starts[i + 1] for i in range(len(reqs) - 1))   # arrival order kept
    for c in done:
        r = reqs[c["id"]]
        a_st, a_K, a_S, a_U, a_V = alone[c["id"]]
        assert c["submit_ms"] <= c["start_ms"] <= c["done_ms"] + 1e-3
        assert c["status"] == a_st and c["K"] == a_K
        assert np.array_equal(r["S"].cpu().numpy(), a_S)
        assert np.array_equal(r["U"].cpu().numpy(), a_U)
        assert np.array_equal(r["V"].cpu().numpy(), a_V)
    errs = [_check_oracle(r["A"].double().numpy(), r["Om"], r["k"], r["S"].cpu().numpy(), r["U"].cpu().numpy(),
                          r["V"].cpu().numpy(), g.RSVD_F32, c["status"])
            for c in done for r in [reqs[c["id"]]]]
    print(f"served float32 requests: max sigma error {max(errs):.2e} sigma_1")


def test_server_rejects_request_larger_than_arena():
    dev = torch.device("cuda")
    m, n, k, p = 20000, 256, 16, 8
    ws = g.rsvd_workspace_query(m, n, k, p, Q)[1]
    with g.rsvd_server_create(ws // 2, max_batch=2, max_inflight=1) as srv:
        A = torch.zeros(m, n, device=dev)
        Om = torch.zeros(n, k + p, device=dev)
        S = torch.zeros(k, dtype=torch.float64, device=dev)
        U = torch.zeros(m, k, device=dev)
        V = torch.zeros(n, k, device=dev)
        assert g.rsvd_server_submit(srv, 0, k, p, Q, 0.9, A, Om, S, U, V) == g.RSVD_ERR_OOM
        assert g.rsvd_server_pending(srv) == 0


def _quantized(r, dtype):
    """The request's matrix stored in `dtype` by the library's quantiser (device)."""
    dev = torch.device("cuda")
    A = r["A"].to(dev)
    if dtype == g.RSVD_F32:
        return A, None
    if dtype == g.RSVD_BF16:
        Aq = torch.empty(r["m"], r["n"], dtype=torch.int16, device=dev)
        g.check(g.rsvd_quantize(A, dtype, Aq), "quantize")
        return Aq, None
    Aq = torch.empty(r["m"], r["n"], dtype=torch.uint8, device=dev)
    sc = torch.empty(r["n"], device=dev)
    g.check(g.rsvd_quantize(A, dtype, Aq, sc), "quantize")
    return Aq, sc


def test_served_mixed_storage_types_equal_alone_bitwise():
    """float32, bfloat16 and e4m3 requests interleaved: a batch holds one storage
    type (consecutive requests of the same l, q and type); the precision forms'
    batches run their solves concurrently, each bit-identical to a solve alone."""
    reqs = _requests(18, 11)
    types = [g.RSVD_BF16, g.RSVD_BF16, g.RSVD_FP8_E4M3, g.RSVD_FP8_E4M3, g.RSVD_F32, g.RSVD_BF16]
    dev = torch.device("cuda")
    alone = {}
    for i, r in enumerate(reqs):
        r["k"], r["p"] = 16, 8                      # one l: batches are cut by type alone
        r["Om"] = synth.gaussian(r["n"], 24, seed=5000 + i, dtype=torch.float32)
        r["dt"] = types[i % len(types)]
        r["Aq"], r["sc"] = _quantized(r, r["dt"])
        r["Od"] = r["Om"].to(dev)
        S = torch.zeros(r["k"], dtype=torch.float64, device=dev)
        U = torch.zeros(r["m"], r["k"], device=dev)
        V = torch.zeros(r["n"], r["k"], device=dev)
        with g.rsvd_plan_create(r["m"], r["n"], r["k"], r["p"], Q, r["dt"]) as plan:
            g.check(g.rsvd(plan, r["Aq"], r["sc"], r["Od"], S, U, V))
            st = g.rsvd_plan_sync(plan)
            stK, K = g.pca_threshold(plan, 0.9)
        alone[r["id"]] = ((stK if st == g.RSVD_OK else st), K, S.cpu().numpy(), U.cpu().numpy(), V.cpu().numpy())
        r["S"] = torch.zeros(r["k"], dtype=torch.float64, device=dev)
        r["U"] = torch.zeros(r["m"], r["k"], device=dev)
        r["V"] = torch.zeros(r["n"], r["k"], device=dev)
    ws = max(g.rsvd_workspace_query(r["m"], r["n"], r["k"], r["p"], Q, r["dt"])[1] for r in reqs)
    torch.cuda.synchronize()
    done = []
    with g.rsvd_server_create(4 * ws, max_batch=4, max_inflight=3) as srv:
        for i, r in enumerate(reqs):
            g.check(g.rsvd_server_submit_ex(srv, r["id"], r["k"], r["p"], Q, r["dt"], 0.9, r["Aq"], r["sc"], r["Od"],
                                            r["S"], r["U"], r["V"]), "submit")
        while g.rsvd_server_pending(srv) > 0:
            done += g.rsvd_server_poll(srv)
    torch.cuda.synchronize()
    assert sorted(c["id"] for c in done) == [r["id"] for r in reqs]
    assert any(c["batch"] > 1 for c in done)
    for c in done:
        r = reqs[c["id"]]
        a_st, a_K, a_S, a_U, a_V = alone[c["id"]]
        assert c["status"] == a_st and c["K"] == a_K, (c, r["dt"])
        assert np.array_equal(r["S"].cpu().numpy(), a_S), r["dt"]
        assert np.array_equal(r["U"].cpu().numpy(), a_U), r["dt"]
        assert np.array_equal(r["V"].cpu().numpy(), a_V), r["dt"]
        err = _check_oracle(_stored64(r["Aq"], r["sc"], r["dt"]), r["Om"], r["k"], r["S"].cpu().numpy(),
                            r["U"].cpu().numpy(), r["V"].cpu().numpy(), r["dt"], c["status"])
        print(f"served request {c['id']} (dtype {r['dt']}): sigma error {err:.2e} sigma_1")


def test_server_submit_ex_checks_scales():
    dev = torch.device("cuda")
    m, n, k, p = 4000, 64, 8, 8
    Aq = torch.zeros(m, n, dtype=torch.uint8, device=dev)
    sc = torch.ones(n, device=dev)
    Om = torch.zeros(n, k + p, device=dev)
    S = torch.zeros(k, dtype=torch.float64, device=dev)
    U = torch.zeros(m, k, device=dev)
    V = torch.zeros(n, k, device=dev)
    with g.rsvd_server_create(1 << 28, max_batch=2, max_inflight=1) as srv:
        assert g.rsvd_server_submit_ex(srv, 0, k, p, Q, g.RSVD_FP8_E4M3, 0.9, Aq, None, Om, S, U, V) == g.RSVD_ERR_ARG
        A16 = torch.zeros(m, n, dtype=torch.int16, device=dev)
        assert g.rsvd_server_submit_ex(srv, 1, k, p, Q, g.RSVD_BF16, 0.9, A16, sc, Om, S, U, V) == g.RSVD_ERR_ARG
        assert g.rsvd_server_submit_ex(srv, 2, k, p, Q, g.RSVD_F64, 0.9, Aq, None, Om, S, U, V) \
            == g.RSVD_ERR_UNSUPPORTED
        assert g.rsvd_server_pending(srv) == 0


def test_served_wide_float32_requests_equal_alone_bitwise():
    """float32 requests with l > 128 (beyond the lockstep batch's shared-memory small
    kernels) are served as concurrent solves; each equals the same request alone."""
    dev = torch.device("cuda")
    reqs = []
    for i in range(4):
        m, n, k, p = 6000 + 500 * i, 300, 136, 8      # l = 144
        sig = synth.spectrum_power(n, 1.0)
        A = synth.prescribed(m, n, sig, 7000 + i, 7100 + i).float()
        Om = synth.gaussian(n, k + p, seed=7200 + i, dtype=torch.float32)
        reqs.append(dict(id=i, m=m, n=n, k=k, p=p, A=A, Om=Om))
    alone = {r["id"]: _alone(r) for r in reqs}
    for r in reqs:
        r["Ad"], r["Od"] = r["A"].to(dev), r["Om"].to(dev)
        r["S"] = torch.zeros(r["k"], dtype=torch.float64, device=dev)
        r["U"] = torch.zeros(r["m"], r["k"], device=dev)
        r["V"] = torch.zeros(r["n"], r["k"], device=dev)
    ws = max(g.rsvd_workspace_query(r["m"], r["n"], r["k"], r["p"], Q)[1] for r in reqs)
    torch.cuda.synchronize()
    done = []
    with g.rsvd_server_create(4 * ws, max_batch=4, max_inflight=2) as srv:
        for r in reqs:
            g.check(g.rsvd_server_submit(srv, r["id"], r["k"], r["p"], Q, 0.9, r["Ad"], r["Od"], r["S"], r["U"],
                                         r["V"]), "submit")
        while g.rsvd_server_pending(srv) > 0:
            done += g.rsvd_server_poll(srv)
    torch.cuda.synchronize()
    assert sorted(c["id"] for c in done) == [r["id"] for r in reqs]
    for c in done:
        r = reqs[c["id"]]
        a_st, a_K, a_S, a_U, a_V = alone[c["id"]]
        assert c["status"] == a_st and c["K"] == a_K
        assert np.array_equal(r["S"].cpu().numpy(), a_S)
        assert np.array_equal(r["U"].cpu().numpy(), a_U)
        assert np.array_equal(r["V"].cpu().numpy(), a_V)
        _check_oracle(r["A"].double().numpy(), r["Om"], r["k"], r["S"].cpu().numpy(), r["U"].cpu().numpy(),
                      r["V"].cpu().numpy(), g.RSVD_F32, c["status"])
