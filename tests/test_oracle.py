"""Pins of the FP64 CPU oracle against facts fixed by the paper and by mathematics.

None of these compare the oracle with itself: each check uses a closed form, a
prescribed spectrum, an invariant the paper states, brute force on tiny
integer inputs, or an independent library (numpy.linalg).
"""
import math
import os

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _int_mats():
    mats = []
    with open(os.path.join(GOLDEN, "int4x3.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            rows = [[float(x) for x in r.split()] for r in line.split(";")]
            mats.append(np.array(rows))
    return mats


def _eig3_closed_form(G):
    """Eigenvalues of a symmetric 3x3 matrix by the trigonometric cubic solution (descending)."""
    p1 = G[0, 1] ** 2 + G[0, 2] ** 2 + G[1, 2] ** 2
    if p1 == 0.0:
        return np.sort(np.diag(G))[::-1]
    q = np.trace(G) / 3.0
    p2 = (G[0, 0] - q) ** 2 + (G[1, 1] - q) ** 2 + (G[2, 2] - q) ** 2 + 2.0 * p1
    p = math.sqrt(p2 / 6.0)
    B = (G - q * np.eye(3)) / p
    r = np.linalg.det(B) / 2.0
    r = min(1.0, max(-1.0, r))
    phi = math.acos(r) / 3.0
    l1 = q + 2.0 * p * math.cos(phi)
    l3 = q + 2.0 * p * math.cos(phi + 2.0 * math.pi / 3.0)
    l2 = 3.0 * q - l1 - l3
    return np.array([l1, l2, l3])


def _orth_err(X):
    return np.abs(X.T @ X - np.eye(X.shape[1])).max()


# ------------------------------------------------------------------ brute force

@pytest.mark.parametrize("idx", range(6))
def test_int4x3_svd_matches_closed_form_cubic(idx):
    """sigma_i^2 = lambda_i(A^T A) (Sec. 2.1, Eqs. AB and LambdaSigma) on 4x3 integer inputs."""
    A = _int_mats()[idx]
    lam = _eig3_closed_form(A.T @ A)
    scale = max(lam[0], 1.0)
    s, U, V = oracle.svd(A)
    assert np.abs(s ** 2 - lam).max() <= 1e-13 * scale
    sg, Ug, Vg = oracle.svd_gram(A)
    assert np.abs(sg ** 2 - lam).max() <= 1e-13 * scale
    lj, Vj, _ = oracle.eig_jacobi(A.T @ A)
    assert np.abs(lj - lam).max() <= 1e-13 * scale
    # A = U Sigma V^T and A v_i = sigma_i u_i (Eq. AV)
    assert np.abs(U @ np.diag(s) @ V.T - A).max() <= 1e-13 * scale
    assert np.abs(A @ V - U * s).max() <= 1e-13 * scale
    assert _orth_err(U) < 1e-14 and _orth_err(V) < 1e-14


# ------------------------------------------------------------ prescribed spectra

def test_exact_svd_recovers_prescribed_spectrum():
    """Exact-SVD workload recipe (2000 x 100, sigma_i = 2^(-i/10)); Householder route and Gram route."""
    A, sigma, _ = synth.workload("exact_fp64_2000x100")
    A = A.numpy()
    sig = sigma.numpy()
    s, U, V = oracle.svd(A)
    assert np.abs(s - sig).max() / sig.max() < 1e-14
    assert (np.abs(s - sig) / sig).max() < 1e-12  # relative, every sigma
    assert _orth_err(U) < 1e-13 and _orth_err(V) < 1e-13
    # delta = ||A - U S V^T||_F / ||A||_F (Sec. 4)
    delta = np.linalg.norm(A - (U * s) @ V.T) / np.linalg.norm(A)
    assert delta < 1e-14
    # Gram route: squares the condition number (cond(A) ~ 955), relative error ~ u * cond^2
    sg, Ug, Vg = oracle.svd_gram(A)
    assert (np.abs(sg - sig) / sig).max() < 1e-9
    assert np.abs(sg - sig).max() < 1e-13


def test_cov_of_projection_is_sigma_squared():
    """Sec. 2.2: rows are examples, Y = A V has Y^T Y = Sigma^2 (no 1/(m-1))."""
    A, sigma, _ = synth.workload("exact_fp64_2000x100", m=600, n=40)
    A = A.numpy()
    s, U, V = oracle.svd(A)
    Y = A @ V
    assert np.abs(Y.T @ Y - np.diag(s ** 2)).max() < 1e-14 * s[0] ** 2 * 10


def test_trace_identity_and_centering():
    """Eq. (sumeigen): sum lambda_i = ||A||_F^2; centring recovers a known column shift."""
    A, sigma, _ = synth.workload("exact_fp64_2000x100", m=500, n=30)
    A = A.numpy()
    mu = np.linspace(-3.0, 5.0, 30)
    Ac, mu_hat, fro2 = oracle.center(A + mu[None, :])
    assert np.abs(mu_hat - mu).max() < 1e-13
    assert np.abs(Ac - A).max() < 1e-13
    assert abs(fro2 - float((sigma.numpy() ** 2).sum())) < 1e-12 * fro2
    lam, _, _ = oracle.eig_jacobi(Ac.T @ Ac)
    assert abs(lam.sum() - fro2) < 1e-12 * fro2


# ----------------------------------------------------------------- special cases

def test_special_cases():
    rng = np.random.default_rng(1)
    # diagonal matrix (stacked on zeros): singular values are |d| sorted
    d = np.array([3.0, -7.0, 0.5, 2.0])
    A = np.vstack([np.diag(d), np.zeros((3, 4))])
    s = oracle.svd(A, vectors=False)
    assert np.allclose(s, np.sort(np.abs(d))[::-1], rtol=0, atol=1e-15)
    # rank 1: one singular value ||x|| ||y||, the rest zero
    x, y = rng.standard_normal(30), rng.standard_normal(8)
    s = oracle.svd(np.outer(x, y), vectors=False)
    assert abs(s[0] - np.linalg.norm(x) * np.linalg.norm(y)) < 1e-13 * s[0]
    assert np.abs(s[1:]).max() < 1e-13 * s[0]
    # orthonormal columns: all singular values 1
    Q = synth.haar(40, 12, seed=5).numpy()
    assert np.abs(oracle.svd(Q, vectors=False) - 1.0).max() < 1e-14
    # zero matrix
    s, U, V = oracle.svd(np.zeros((6, 3)))
    assert np.all(s == 0.0)


def test_library_crosscheck_numpy():
    """Independent library: numpy.linalg.svd and eigh on Gaussian inputs (Sec. 4 distribution)."""
    rng = np.random.default_rng(2)
    for m, n in [(50, 20), (333, 97), (64, 64)]:
        A = rng.standard_normal((m, n))
        s_np = np.linalg.svd(A, compute_uv=False)
        s, U, V = oracle.svd(A)
        assert np.abs(s - s_np).max() < 1e-13 * s_np[0]
        lam_np = np.linalg.eigvalsh(A.T @ A)[::-1]
        lam, Vj, sweeps = oracle.eig_jacobi(A.T @ A)
        assert np.abs(lam - lam_np).max() < 1e-13 * lam_np[0]
        assert np.abs((A.T @ A) @ Vj - Vj * lam).max() < 1e-12 * lam_np[0]
        assert sweeps < 20


def test_qr_positive_diagonal():
    rng = np.random.default_rng(3)
    Y = rng.standard_normal((200, 17))
    Q, R = oracle.qr(Y)
    assert _orth_err(Q) < 1e-14
    assert np.allclose(np.tril(R, -1), 0.0)
    assert np.all(np.diag(R) > 0)
    assert np.abs(Q @ R - Y).max() < 1e-13
    qn, rn = np.linalg.qr(Y)
    sg = np.sign(np.diag(rn))
    assert np.abs(Q - qn * sg).max() < 1e-12


# ----------------------------------------------------------------- randomized PCA

def test_rsvd_exact_when_rank_at_most_l():
    """Sec. 3.1.2: if rank(A) <= l the range finder captures range(A) exactly."""
    rng = np.random.default_rng(4)
    m, n, r, l, k = 400, 60, 12, 16, 10
    sig = np.linspace(5.0, 1.0, r)
    U0 = synth.haar(m, r, seed=11).numpy()
    V0 = synth.haar(n, r, seed=12).numpy()
    A = (U0 * sig) @ V0.T
    Om = rng.standard_normal((n, l))
    for q in (0, 1, 2):
        s, U, V = oracle.rsvd(A, Om, q=q, k=k)
        assert np.abs(s - sig[:k]).max() < 1e-13 * sig[0]
        # singular vectors match up to the sign convention
        assert np.abs(np.abs(np.sum(V * V0[:, :k], axis=0)) - 1.0).max() < 1e-12
        assert np.abs(A @ V - U * s).max() < 1e-12 * sig[0]


def test_rsvd_equals_unorthonormalised_power_scheme():
    """Sec. 3.1.2 as printed: H = A (A^T A)^q G without intermediate orthonormalisation.

    In exact arithmetic range(H) equals the oracle's re-orthonormalised range,
    so the Ritz values sigma(Q^T A) agree; computed here independently with numpy.
    """
    rng = np.random.default_rng(5)
    m, n, l, k = 300, 40, 8, 6
    A = rng.standard_normal((m, n)) @ np.diag(np.linspace(3.0, 0.2, n))
    Om = rng.standard_normal((n, l))
    for q in (0, 1):
        H = A @ Om
        for _ in range(q):
            H = A @ (A.T @ H)
        Qn, _ = np.linalg.qr(H)
        s_ref = np.linalg.svd(Qn.T @ A, compute_uv=False)[:k]
        s, U, V = oracle.rsvd(A, Om, q=q, k=k)
        assert np.abs(s - s_ref).max() < 1e-12 * s_ref[0]
        # U = Q W lies in range(H)
        assert np.abs(U - Qn @ (Qn.T @ U)).max() < 1e-12


def test_rsvd_converges_with_power_iterations():
    A, sigma, _ = synth.workload("rpca_fp32_200000x1000", m=3000, n=120)
    A = A.numpy()
    rng = np.random.default_rng(6)
    Om = rng.standard_normal((120, 30))
    s, U, V = oracle.rsvd(A, Om, q=6, k=10)
    assert np.abs(s - sigma.numpy()[:10]).max() < 1e-8


def test_rsvd_argument_checks():
    A = np.zeros((10, 4))
    with pytest.raises(oracle.OracleError):
        oracle.rsvd(A, np.zeros((4, 5)), q=1, k=2)  # l > n


# ------------------------------------------------------------------------- GKL

def test_gkl_full_steps_reproduces_all_sigma():
    """n Lanczos steps with full reorthogonalisation span R^n: every sigma is exact."""
    rng = np.random.default_rng(7)
    A = rng.standard_normal((150, 30))
    s_np = np.linalg.svd(A, compute_uv=False)
    s, U, V, al, be = oracle.gkl(A, rng.standard_normal(30), steps=30, k=30)
    assert np.abs(s - s_np).max() < 1e-12 * s_np[0]
    assert np.abs(A @ V - U * s).max() < 1e-11 * s_np[0]
    assert _orth_err(U) < 1e-12 and _orth_err(V) < 1e-12


def test_gkl_ritz_values_are_krylov_projection():
    """Ritz values after s steps = sigma(A P) with P the orthogonal basis of K_s(A^T A, v1)."""
    rng = np.random.default_rng(8)
    A = rng.standard_normal((200, 25)) @ np.diag(np.exp(-np.arange(25) / 4.0))
    v1 = rng.standard_normal(25)
    for s_steps in (1, 3, 5):
        K = [v1 / np.linalg.norm(v1)]
        for _ in range(s_steps - 1):
            w = A.T @ (A @ K[-1])
            K.append(w / np.linalg.norm(w))
        P, _ = np.linalg.qr(np.stack(K, axis=1))
        s_ref = np.linalg.svd(A @ P, compute_uv=False)
        s, U, V, al, be = oracle.gkl(A, v1, steps=s_steps, k=s_steps)
        assert np.abs(s - s_ref).max() < 1e-11 * s_ref[0]
        # the first alpha is ||A v1|| / ||v1||
        assert abs(al[0] - np.linalg.norm(A @ v1) / np.linalg.norm(v1)) < 1e-13 * al[0]


# ---------------------------------------------------------------------- K choice

def _k_geometric(r, n, t):
    """Minimal K with (1 - r^K) / (1 - r^n) >= t for lambda_i = r^i (closed form)."""
    return math.ceil(math.log(1.0 - t * (1.0 - r ** n)) / math.log(r))


def test_pca_threshold_closed_forms():
    """Sec. 2.4 criterion with denominator ||A||_F^2 (Eq. sumeigen)."""
    # exact-SVD workload: sigma_i = 2^(-i/10) -> lambda_i = r^i, r = 2^(-1/5), t = 0.95
    sig = synth.spectrum_pow2(100).numpy()
    fro2 = float((sig ** 2).sum())
    K, ok = oracle.pca_threshold(sig, fro2, 0.95)
    assert ok and K == _k_geometric(2.0 ** -0.2, 100, 0.95) == 22
    # Lanczos workload spectrum sigma_i = exp(-i/200): lambda_i = r^i, r = exp(-1/100), n = 2048
    sig = synth.spectrum_exp(2048).numpy()
    fro2 = float((sig ** 2).sum())
    K, ok = oracle.pca_threshold(sig, fro2, 0.9)
    assert ok and K == _k_geometric(math.exp(-0.01), 2048, 0.9) == 231
    # only the first 100 known: threshold not reached within count -> warning, K = count
    K, ok = oracle.pca_threshold(sig[:100], fro2, 0.9)
    assert (not ok) and K == 100
    # harmonic spectrum sigma_i = 1/i (noiseless) with n = 1000 and t = 0.9
    i = np.arange(1, 1001, dtype=np.float64)
    sig = 1.0 / i
    fro2 = float((sig ** 2).sum())
    K, ok = oracle.pca_threshold(sig, fro2, 0.9)
    partial = np.cumsum(sig ** 2)
    assert ok and K == 6 and partial[K - 1] >= 0.9 * fro2 > partial[K - 2]
    # equality counts as reached (>= in Sec. 2.4)
    K, ok = oracle.pca_threshold(np.array([1.0, 1.0]), 2.0, 0.5)
    assert ok and K == 1


@pytest.mark.parametrize("m,n", [(2000, 100), (4000, 300)])
def test_gram_route_on_the_papers_gaussian_matrices(m, n):
    """Sec. 4's experiment: A with N(0,1) entries, all n triplets by the Gram route
    ("truncated SVD" at k = n).  The residual delta = ||A - U S V^T||_F / ||A||_F is at
    rounding level (cond(A) is about (sqrt m + sqrt n) / (sqrt m - sqrt n) < 2, so forming
    A^T A loses nothing), and the extreme singular values sit at the Marchenko-Pastur
    edges sqrt(m) +- sqrt(n) (to a few percent at these sizes)."""
    A = synth.gaussian(m, n, seed=1906 + n).numpy()
    s, U, V = oracle.svd_gram(A)
    delta = np.linalg.norm(A - (U * s) @ V.T) / np.linalg.norm(A)
    assert delta < 1e-13
    assert 0.97 < s[0] / (math.sqrt(m) + math.sqrt(n)) < 1.03
    assert 0.95 < s[-1] / (math.sqrt(m) - math.sqrt(n)) < 1.05
