"""GPU parity: the Gram route (Sec. 2.3 and the step list of Sec. 3.1.3) beyond one CTA,
112 < n <= 4096 -- the k = n regime of the paper's experiments (Sec. 4), where it argues the
Gram route is the fastest -- through svd_exact(RSVD_EXACT_GRAM).

The n x n eigen-decomposition runs in float64 on the whole GPU (Householder
tridiagonalisation, bisection, inverse iteration, back-transformation).  Checks:
* against the FP64 oracle's Gram route (cyclic Jacobi on A^T A) on the same stored values:
  float64 plans |sigma_hat_i - sigma_i^O| <= 1e-10 sigma_i^O + 1e-12 sigma_1^O (forming A^T A
  squares cond(A); these matrices have cond(A) < 10), vectors of well-separated values
  entrywise to 1e-8; float32 plans (float32 Gram matrix) within 1e-5 sigma_1^O;
* at the paper's sizes (10000 x 2000, and 60000 x 784 for the MNIST-shaped case), against
  the prescribed spectrum of A = U diag(sigma) V^T, with V^T V = I, U^T U = I on the
  non-zero values, and the paper's accuracy measure delta = ||A - U Sigma V^T||_F / ||A||_F;
* an exactly rank-deficient input (rank 50 of 300): the zero eigenvalues form one cluster
  whose vectors are orthonormalised, the 50 values are exact, the status warns, and every
  u_i of a sigma_i below sqrt(n eps) sigma_1 (zero to the resolution of A^T A) is zero.
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


def _solve(A_host, dtype):
    tdt = torch.float64 if dtype == g.RSVD_F64 else torch.float32
    m, n = A_host.shape
    dev = torch.device("cuda")
    A = A_host.to(dev, tdt).contiguous()
    S = torch.zeros(n, dtype=torch.float64, device=dev)
    U = torch.zeros(m, n, dtype=tdt, device=dev)
    V = torch.zeros(n, n, dtype=tdt, device=dev)
    with g.rsvd_plan_create(m, n, 1, 0, 0, dtype) as plan:
        g.check(g.svd_exact(plan, A, g.RSVD_EXACT_GRAM, S, U, V), "svd_exact")
        st = g.rsvd_plan_sync(plan)
    return st, S.cpu().numpy(), U.cpu().double().numpy(), V.cpu().double().numpy()


def _gaps(s):
    gap = np.full(s.shape, np.inf)
    d = np.abs(np.diff(s)) / s[0]
    gap[:-1] = np.minimum(gap[:-1], d)
    gap[1:] = np.minimum(gap[1:], d)
    return gap


@pytest.mark.parametrize("m,n,dtype", [
    (3000, 300, g.RSVD_F64),
    (5001, 513, g.RSVD_F64),     # ragged n: the tridiagonalisation's last steps, odd tiles
    (4000, 400, g.RSVD_F32),     # float32 Gram matrix on the tensor cores (n % 16 == 0)
    (4000, 301, g.RSVD_F32),     # float32 Gram matrix on the CUDA cores
])
def test_gram_large_matches_oracle(m, n, dtype):
    sig = torch.linspace(3.0, 1.0, n, dtype=torch.float64) ** 2 / 3.0   # cond(A) = 3
    A = synth.prescribed(m, n, sig, 7001 + n, 7002 + n)
    A = A + torch.linspace(-1.0, 1.0, n, dtype=torch.float64).unsqueeze(0)   # removed by the centring
    if dtype == g.RSVD_F32:
        A = A.float().double()
    st, S, U, V = _solve(A, dtype)
    assert st == g.RSVD_OK
    Ac, _, _ = oracle.center(A)
    s, Uo, Vo = oracle.svd_gram(Ac)
    Uo, Vo = oracle.sign_normalize(Uo, Vo)
    if dtype == g.RSVD_F64:
        assert (np.abs(S - s) <= 1e-10 * s + 1e-12 * s[0]).all()
        sep = _gaps(s) >= 1e-3
        assert np.abs(V[:, sep] - Vo[:, sep]).max() <= 1e-8
        assert np.abs(U[:, sep] - Uo[:, sep]).max() <= 1e-8
        assert np.abs(V.T @ V - np.eye(n)).max() <= 1e-12
    else:
        assert np.abs(S - s).max() <= 1e-5 * s[0]
        assert np.abs(V.T @ V - np.eye(n)).max() <= 1e-5
        assert np.abs(U.T @ U - np.eye(n)).max() <= 1e-4


@pytest.mark.parametrize("m,n,dtype", [
    (10000, 2000, g.RSVD_F64),   # the paper's widest grid point (m = 10000, n = 2000)
    (10000, 2000, g.RSVD_F32),
    (60000, 784, g.RSVD_F32),    # MNIST-shaped (the dataset itself is not available)
])
def test_gram_large_paper_sizes_prescribed_spectrum(m, n, dtype):
    i = torch.arange(1, n + 1, dtype=torch.float64)
    sig = 1.0 + 1.0 / i            # distinct values, cond(A) = 2
    A = synth.prescribed(m, n, sig, 7101 + n, 7102 + n)
    if dtype == g.RSVD_F32:
        A = A.float().double()
    st, S, U, V = _solve(A, dtype)
    assert st == g.RSVD_OK
    An = A.numpy()
    delta = np.linalg.norm(An - (U * S) @ V.T) / np.linalg.norm(An)
    orth_v = np.abs(V.T @ V - np.eye(n)).max()
    orth_u = np.abs(U.T @ U - np.eye(n)).max()
    err = np.abs(S - sig.numpy()).max() / sig[0].item()
    print(f"{m}x{n} dtype {dtype}: max sigma error {err:.2e} sigma_1, delta {delta:.2e}, "
          f"|V^T V - I| {orth_v:.1e}, |U^T U - I| {orth_u:.1e}")
    if dtype == g.RSVD_F64:
        assert err <= 1e-12 and delta <= 1e-12 and orth_v <= 1e-12 and orth_u <= 1e-11
    else:
        assert err <= 1e-5 and delta <= 1e-5 and orth_v <= 1e-6 and orth_u <= 1e-5


def test_gram_large_rank_deficient():
    m, n, r = 3000, 300, 50
    sig = torch.zeros(n, dtype=torch.float64)
    sig[:r] = torch.linspace(2.0, 1.0, r, dtype=torch.float64)
    A = synth.prescribed(m, n, sig, 7201, 7202)
    st, S, U, V = _solve(A, g.RSVD_F64)
    assert st == g.RSVD_WARN_RANK_DEFICIENT
    assert np.abs(S[:r] - sig[:r].numpy()).max() <= 1e-12 * 2.0
    assert np.abs(S[r:]).max() <= 1e-6           # sqrt of eigenvalues at the rounding level of A^T A
    assert np.abs(V.T @ V - np.eye(n)).max() <= 1e-12
    assert np.abs(U[:, :r].T @ U[:, :r] - np.eye(r)).max() <= 1e-12
    assert np.abs(U[:, r:]).max() == 0.0          # u_i of a zero sigma_i is the zero vector
