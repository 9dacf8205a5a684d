"""GPU parity: exact SVD routes (Sec. 2.1 definition; Sec. 2.3 / 3.1.3 Gram route).

Workload: the exact-SVD recipe 2000 x 100, sigma_i = 2^(-i/10), Haar factors,
centred columns (full size: the oracle finishes it in well under a second).

Tolerances:
* QR_JACOBI (float64): max_i |sigma_hat_i - sigma_i| / sigma_i <= 1e-10 against
  the prescribed spectrum and against the oracle's Householder SVD.
* GRAM (float64): forming A^T A squares cond(A) = 2^(9.9) ~ 955, so the
  attainable relative error of sigma_100 is ~ u * cond(A)^2 ~ 1e-10; the test
  bound is 1e-9 (the value reached is printed by the bench, not asserted tighter).
* vectors: sign-convention-aligned entrywise agreement with the oracle's
  Householder SVD to 1e-8 (QR_JACOBI) / 1e-6 (GRAM).
* K(t = 0.95) = 22 from the closed-form geometric sum of the prescribed spectrum.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_1906_12085_gb300 as g
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1906_12085_gb300 import build
    build.build()


def _solve(A_host, method, dtype=g.RSVD_F64):
    tdt = torch.float64 if dtype == g.RSVD_F64 else torch.float32
    m, n = A_host.shape
    dev = torch.device("cuda")
    A = A_host.to(dev, tdt).contiguous()
    S = torch.zeros(n, dtype=torch.float64, device=dev)
    U = torch.zeros(m, n, dtype=tdt, device=dev)
    V = torch.zeros(n, n, dtype=tdt, device=dev)
    with g.rsvd_plan_create(m, n, 1, 0, 0, dtype) as plan:
        g.check(g.svd_exact(plan, A, method, S, U, V), "svd_exact")
        st = g.rsvd_plan_sync(plan)
        stK, K = g.pca_threshold(plan, 0.95)
        fro2 = g.rsvd_plan_fro2(plan)
    return st, S.cpu().numpy(), U.cpu().double().numpy(), V.cpu().double().numpy(), K, stK, fro2


@pytest.fixture(scope="module")
def exact_case():
    A, sigma, _ = synth.workload("exact_fp64_2000x100")
    A = A + torch.linspace(1.0, -1.0, 100, dtype=torch.float64).unsqueeze(0)  # removed by centring
    Ac, mu, fro2 = oracle.center(A)
    s, U, V = oracle.svd(Ac)
    U, V = oracle.sign_normalize(U, V)   # the library's sign convention (largest |v_i| entry positive)
    return A, sigma.numpy(), Ac, s, U, V, fro2


@pytest.mark.parametrize("method,tol_s,tol_v", [(g.RSVD_EXACT_QR_JACOBI, 1e-10, 1e-8), (g.RSVD_EXACT_GRAM, 1e-9, 1e-6)])
def test_exact_f64_workload(exact_case, method, tol_s, tol_v):
    A, sigma, Ac, s_o, U_o, V_o, fro2 = exact_case
    st, S, U, V, K, stK, fro2_g = _solve(A, method)
    assert st == g.RSVD_OK
    assert (np.abs(S - sigma) / sigma).max() <= tol_s
    assert (np.abs(S - s_o) / s_o).max() <= tol_s
    assert np.abs(V - V_o).max() <= tol_v
    assert np.abs(U - U_o).max() <= tol_v
    assert np.abs(V.T @ V - np.eye(100)).max() <= tol_v
    assert np.abs(U.T @ U - np.eye(100)).max() <= tol_v
    # delta of Sec. 4 on the centred matrix
    delta = np.linalg.norm(Ac - (U * S) @ V.T) / np.linalg.norm(Ac)
    assert delta <= 10 * tol_v
    assert abs(fro2_g - fro2) <= 1e-12 * fro2
    assert K == 22 and stK == g.RSVD_OK


@pytest.mark.parametrize("method", [g.RSVD_EXACT_QR_JACOBI, g.RSVD_EXACT_GRAM])
def test_exact_f32(method):
    """float32 storage: sigma within 1e-5 * sigma_1 of the oracle on the stored values."""
    A, sigma, _ = synth.workload("exact_fp64_2000x100", m=3001, n=57)
    A32 = A.float()
    st, S, U, V, K, stK, fro2 = _solve(A32, method, g.RSVD_F32)
    Ac, mu, _ = oracle.center(A32.double())
    s = oracle.svd(Ac, vectors=False)
    assert np.abs(S - s).max() <= 1e-5 * s[0]


@pytest.mark.parametrize("m,n", [(130, 1), (257, 2), (1000, 33), (65, 64)])
def test_exact_small_and_square(m, n):
    rng = np.random.default_rng(m + n)
    A = torch.from_numpy(rng.standard_normal((m, n)))
    for method in (g.RSVD_EXACT_QR_JACOBI, g.RSVD_EXACT_GRAM):
        st, S, U, V, K, stK, fro2 = _solve(A, method)
        Ac, _, _ = oracle.center(A)
        s = oracle.svd(Ac, vectors=False)
        tol = 1e-10 if method == g.RSVD_EXACT_QR_JACOBI else 1e-8
        assert np.abs(S - s).max() <= tol * s[0]
        assert np.abs(Ac @ V - U * S).max() <= 1e-8 * s[0]


def test_exact_size_limits():
    """Beyond the one-CTA limit (n > 112) only the Gram route runs (up to n = 4096)."""
    m, n = 5000, 200
    dev = torch.device("cuda")
    A = torch.zeros(m, n, dtype=torch.float64, device=dev)
    with g.rsvd_plan_create(m, n, 4, 2, 0, g.RSVD_F64) as plan:
        S = torch.zeros(n, dtype=torch.float64, device=dev)
        st = g.svd_exact(plan, A, g.RSVD_EXACT_QR_JACOBI, S, torch.zeros(m, n, dtype=torch.float64, device=dev),
                         torch.zeros(n, n, dtype=torch.float64, device=dev))
        assert st == g.RSVD_ERR_UNSUPPORTED
        assert g.svd_exact(plan, A, 7, S, A, A) == g.RSVD_ERR_ARG
    m, n = 4200, 4097
    A = torch.zeros(m, n, dtype=torch.float32, device=dev)
    with g.rsvd_plan_create(m, n, 4, 2, 0, g.RSVD_F32) as plan:
        S = torch.zeros(n, dtype=torch.float64, device=dev)
        assert g.svd_exact(plan, A, g.RSVD_EXACT_GRAM, S, A, A) == g.RSVD_ERR_UNSUPPORTED
