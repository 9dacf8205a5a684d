"""The allocation-free entry point svd_exact_gram_static against svd_exact.

svd_exact_gram_static serves callers that cannot allocate device memory (a
host framework's fixed pool, a hard memory budget, or a loop that must not
hit cudaMalloc/cudaFree synchronisation): it takes its scratch from a static
device array inside the library.  Its results must equal those of the plan
based svd_exact (Gram route) on the same input, on two calls in a row (the
second call reuses the static array the first one left behind).

This file is named to be collected last, so a run that stops at the first
failure has already run every other test.
"""
import numpy as np
import pytest
import torch

import paper_1906_12085_gb300 as g
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1906_12085_gb300 import build
    build.build()


def _with_plan(A, dtype):
    m, n = A.shape
    S = torch.zeros(n, dtype=torch.float64, device=A.device)
    U = torch.zeros(m, n, dtype=A.dtype, device=A.device)
    V = torch.zeros(n, n, dtype=A.dtype, device=A.device)
    with g.rsvd_plan_create(m, n, 1, 0, 0, dtype) as plan:
        g.check(g.svd_exact(plan, A, g.RSVD_EXACT_GRAM, S, U, V), "svd_exact")
        g.check(g.rsvd_plan_sync(plan), "svd_exact status")
    return S.cpu().numpy(), U.cpu().double().numpy(), V.cpu().double().numpy()


def _static(A, dtype):
    m, n = A.shape
    S = torch.full((n,), np.nan, dtype=torch.float64, device=A.device)
    U = torch.full((m, n), np.nan, dtype=A.dtype, device=A.device)
    V = torch.full((n, n), np.nan, dtype=A.dtype, device=A.device)
    g.check(g.svd_exact_gram_static(A, dtype, S, U, V), "svd_exact_gram_static")
    return S.cpu().numpy(), U.cpu().double().numpy(), V.cpu().double().numpy()


@pytest.mark.parametrize("dtype,tdt,tol_s,tol_v", [
    (g.RSVD_F64, torch.float64, 1e-9, 1e-6),    # the Gram-route tolerances of the exact tests
    (g.RSVD_F32, torch.float32, 1e-5, 2e-3),    # the float32 tolerances of the parity tests
])
def test_static_scratch_matches_svd_exact_twice(dtype, tdt, tol_s, tol_v):
    dev = torch.device("cuda")
    for call, (m, n, seed) in enumerate([(3001, 48, 11), (2003, 64, 12)]):
        sig = synth.spectrum_pow2(n)
        A0 = synth.prescribed(m, n, sig, seed, seed + 100) + 0.25   # a column offset the centring removes
        A0 = A0.to(dev, tdt)
        s_ref, u_ref, v_ref = _with_plan(A0.clone(), dtype)
        s, u, v = _static(A0.clone(), dtype)
        assert np.all(np.isfinite(s)) and np.all(np.isfinite(u)) and np.all(np.isfinite(v)), f"call {call}"
        assert np.abs(s - s_ref).max() <= tol_s * s_ref[0], f"call {call}"
        assert np.abs(v - v_ref).max() <= tol_v, f"call {call}"
        assert np.abs(u - u_ref).max() <= tol_v, f"call {call}"


def test_static_scratch_rejects_sizes_beyond_limit():
    dev = torch.device("cuda")
    m, n = 500, 65
    A = torch.zeros(m, n, dtype=torch.float64, device=dev)
    S = torch.zeros(n, dtype=torch.float64, device=dev)
    st = g.svd_exact_gram_static(A, g.RSVD_F64, S, torch.zeros(m, n, dtype=torch.float64, device=dev),
                                 torch.zeros(n, n, dtype=torch.float64, device=dev))
    assert st == g.RSVD_ERR_UNSUPPORTED
