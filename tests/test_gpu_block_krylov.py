"""GPU parity: the block Krylov method (Sec. 3.1.1) through the C ABI against the FP64 oracle.

The oracle follows the step list (power blocks re-orthonormalised, Householder QR of
their concatenation); the library builds an orthonormal basis of the same Krylov
space block by block.  Both Ritz value sets are those of one subspace in exact
arithmetic, so they are compared element by element.  Tolerances:
* float32: |sigma_hat_i - sigma_i^O| <= 1e-5 * sigma_1^O (i <= k); U, V orthonormal
  to 1e-5; vectors of well-separated values (relative gap >= 2e-2) entrywise to 2e-3.
* float64: relative sigma error <= 1e-10; vectors to 1e-8.
The method's own inequalities hold at any size: Ritz values do not exceed the
singular values, and (the Krylov space containing the randomized method's basis
for q = i) are not below the randomized method's values on the same Omega.
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


def _matrix(m, n, sig, seed=0, shift=True):
    A = synth.prescribed(m, n, sig, 19061 + seed, 19062 + seed)
    if shift:  # a known column offset, removed by the centring
        A = A + torch.linspace(-2.0, 3.0, n, dtype=torch.float64).unsqueeze(0)
    return A


def _gaps(s):
    s = np.asarray(s)
    gap = np.full(s.shape, np.inf)
    d = np.abs(np.diff(s)) / s[0]
    gap[:-1] = np.minimum(gap[:-1], d)
    gap[1:] = np.minimum(gap[1:], d)
    return gap


def _run_bk(A_host, Om_host, k, b, iters, dtype, flags=0, t=0.9):
    tdt = torch.float32 if dtype == g.RSVD_F32 else torch.float64
    m, n = A_host.shape
    dev = torch.device("cuda")
    A = A_host.to(dev, tdt).contiguous()
    Om = Om_host.to(dev, tdt).contiguous()
    S = torch.zeros(k, dtype=torch.float64, device=dev)
    U = torch.zeros(m, k, dtype=tdt, device=dev)
    V = torch.zeros(n, k, dtype=tdt, device=dev)
    with g.rsvd_plan_create_block_krylov(m, n, k, b, iters, dtype) as plan:
        g.check(g.rsvd_plan_set_flags(plan, flags), "flags")
        g.check(g.rsvd_block_krylov(plan, A, Om, S, U, V), "rsvd_block_krylov")
        st = g.rsvd_plan_sync(plan)
        fro2 = g.rsvd_plan_fro2(plan)
        stK, K = g.pca_threshold(plan, t)
        # a block Krylov plan does not run the randomized method
        assert g.rsvd(plan, A, None, Om, S, U, V) == g.RSVD_ERR_ARG
    return dict(S=S.cpu().numpy(), U=U.cpu().double().numpy(), V=V.cpu().double().numpy(),
                A=A.cpu().double().numpy(), status=st, fro2=fro2, K=K, stK=stK)


@pytest.mark.parametrize("m,n,k,b,iters", [
    (5037, 301, 20, 24, 2),     # several row tiles, ragged m and n, b padded to 32 (W = 72)
    (4000, 200, 40, 40, 3),     # four blocks, W = 160
    (6000, 300, 64, 96, 2),     # W = 288: products on column slices, cluster Cholesky and Jacobi
    (3000, 120, 30, 112, 0),    # one block: the randomized method with q = 0
])
def test_block_krylov_f32_matches_oracle(m, n, k, b, iters):
    A32 = _matrix(m, n, synth.spectrum_harmonic_noise(n, 7)).float()
    Om = synth.gaussian(n, b, seed=19063, dtype=torch.float32)
    r = _run_bk(A32, Om, k, b, iters, g.RSVD_F32)
    assert r["status"] == g.RSVD_OK
    assert np.array_equal(r["A"], A32.double().numpy())           # read only
    Ac, mu, fro2 = oracle.center(A32.double())
    assert abs(r["fro2"] - fro2) <= 1e-5 * fro2
    s, U, V = oracle.block_krylov(Ac, Om.double(), iters, k)
    assert np.abs(r["S"] - s).max() <= 1e-5 * s[0]
    assert np.abs(r["U"].T @ r["U"] - np.eye(k)).max() <= 1e-5
    assert np.abs(r["V"].T @ r["V"] - np.eye(k)).max() <= 1e-5
    sep = _gaps(s) >= 2e-2
    assert np.abs(r["V"][:, sep] - V[:, sep]).max() <= 2e-3
    assert np.abs(r["U"][:, sep] - U[:, sep]).max() <= 2e-3
    Ko, reached = oracle.pca_threshold(s, fro2, 0.9)
    assert r["K"] == Ko
    assert r["stK"] == (g.RSVD_OK if reached else g.RSVD_WARN_K_GT_k)


def test_block_krylov_f32_one_block_is_randomized_q0():
    """With i = 0 the Krylov space is range(A Omega): the randomized method with q = 0."""
    m, n, b = 2500, 150, 40
    A32 = _matrix(m, n, synth.spectrum_harmonic_noise(n, 8), seed=4).float()
    Om = synth.gaussian(n, b, seed=19064, dtype=torch.float32)
    r = _run_bk(A32, Om, b, b, 0, g.RSVD_F32)
    Ac, _, _ = oracle.center(A32.double())
    s, _, _ = oracle.rsvd(Ac, Om.double(), q=0, k=b)
    assert np.abs(r["S"] - s).max() <= 1e-5 * s[0]


@pytest.mark.parametrize("name", ["pow3", "exp5", "rank20", "step"])
def test_block_krylov_f32_hard_spectra(name):
    """Fast decay, exact rank deficiency and a spectral step: the blocks become
    numerically rank deficient in float32; the basis stays orthonormal and the Ritz
    values still agree with the FP64 oracle."""
    m, n, b, iters = 8000, 1024, 48, 4
    i = torch.arange(1, n + 1, dtype=torch.float64)
    sig = {"pow3": i ** -3.0, "exp5": torch.exp(-i / 5),
           "rank20": torch.where(i <= 20, 1.0 / i, torch.zeros_like(i)),
           "step": torch.where(i <= 40, torch.ones_like(i), 1e-4 * torch.ones_like(i))}[name]
    A32 = _matrix(m, n, sig, seed=5, shift=False).float()
    Om = synth.gaussian(n, b, seed=19065, dtype=torch.float32)
    k = 32
    r = _run_bk(A32, Om, k, b, iters, g.RSVD_F32, flags=g.RSVD_FLAG_NO_CENTER)
    assert r["status"] in ((g.RSVD_OK, g.RSVD_WARN_RANK_DEFICIENT) if name == "rank20" else (g.RSVD_OK,))
    A64 = A32.double().numpy()
    s, _, _ = oracle.block_krylov(A64, Om.double(), iters, k)
    assert np.abs(r["S"] - s).max() <= 1e-5 * s[0]
    assert np.abs(r["U"].T @ r["U"] - np.eye(k)).max() <= 1e-5
    assert np.abs(r["V"].T @ r["V"] - np.eye(k)).max() <= 1e-5
    # Rayleigh-Ritz from the left: A^T u_i = sigma_i v_i
    res = A64.T @ r["U"] - r["V"] * r["S"][None, :]
    assert np.abs(res).max() <= 1e-5 * s[0]


def test_block_krylov_f32_method_inequalities():
    """sigma_i(randomized, q = i) - tol <= sigma_hat_i <= sigma_i + tol (Sec. 3.1.1 vs 3.1.2)."""
    m, n, b, iters, k = 6000, 400, 32, 2, 32
    sig = synth.spectrum_power(n, 1.0)
    A32 = _matrix(m, n, sig, seed=6, shift=False).float()
    Om = synth.gaussian(n, b, seed=19066, dtype=torch.float32)
    r = _run_bk(A32, Om, k, b, iters, g.RSVD_F32, flags=g.RSVD_FLAG_NO_CENTER)
    A64 = A32.double().numpy()
    true = oracle.svd(A64, vectors=False)[:k]
    s_pow, _, _ = oracle.rsvd(A64, Om.double(), q=iters, k=k)
    tol = 1e-5 * true[0]
    assert (r["S"] <= true + tol).all()
    assert (r["S"] >= s_pow - tol).all()
    # and the Krylov space does strictly better somewhere on this slowly decaying spectrum
    assert (r["S"] - s_pow).max() > 10 * tol


@pytest.mark.parametrize("m,n,k,b,iters", [(2021, 97, 16, 16, 2), (1500, 100, 20, 30, 2)])
def test_block_krylov_f64_matches_oracle(m, n, k, b, iters):
    A0 = _matrix(m, n, synth.spectrum_harmonic_noise(n, 9), seed=7)
    Om = synth.gaussian(n, b, seed=19067, dtype=torch.float64)
    r = _run_bk(A0, Om, k, b, iters, g.RSVD_F64)
    assert r["status"] == g.RSVD_OK
    Ac, _, fro2 = oracle.center(A0)
    assert abs(r["fro2"] - fro2) <= 1e-12 * fro2
    s, U, V = oracle.block_krylov(Ac, Om, iters, k)
    assert (np.abs(r["S"] - s) / s).max() <= 1e-10
    sep = _gaps(s) >= 1e-3
    assert np.abs(r["V"][:, sep] - V[:, sep]).max() <= 1e-8
    assert np.abs(r["U"][:, sep] - U[:, sep]).max() <= 1e-8


def test_block_krylov_plan_rules():
    dev = torch.device("cuda")
    m, n = 500, 64
    A = torch.randn(m, n, device=dev)
    Om = torch.randn(n, 16, device=dev)
    S = torch.zeros(16, dtype=torch.float64, device=dev)
    U = torch.zeros(m, 16, device=dev)
    V = torch.zeros(n, 16, device=dev)
    with g.rsvd_plan_create(m, n, 8, 8, 1, g.RSVD_F32) as plan:   # an ordinary plan
        assert g.rsvd_block_krylov(plan, A, Om, S, U, V) == g.RSVD_ERR_ARG
    with g.rsvd_plan_create_block_krylov(m, n, 16, 16, 1, g.RSVD_F32) as plan:
        assert g.rsvd_block_krylov(plan, A, None, S, U, V) == g.RSVD_ERR_ARG
        assert g.rsvd_autotune(plan, A, Om, 1)[0] == g.RSVD_ERR_ARG
        g.check(g.rsvd_block_krylov(plan, A, Om, S, U, V), "rsvd_block_krylov")
        assert g.rsvd_plan_sync(plan) == g.RSVD_OK


def test_block_krylov_f32_power15_spectrum_w288():
    """sigma_i = i^-1.5 (the precision-form workload's spectrum), b = 96, i = 2, k = 256."""
    m, n, k, b, iters = 20000, 2048, 256, 96, 2
    A32 = synth.prescribed(m, n, synth.spectrum_power(n, 1.5), 40961, 40962).float()
    Om = synth.gaussian(n, b, seed=40965, dtype=torch.float32)
    r = _run_bk(A32, Om, k, b, iters, g.RSVD_F32)
    assert r["status"] == g.RSVD_OK
    Ac, _, _ = oracle.center(A32.double())
    s, _, _ = oracle.block_krylov(Ac, Om.double(), iters, k)
    assert np.abs(r["S"] - s).max() <= 1e-5 * s[0]
