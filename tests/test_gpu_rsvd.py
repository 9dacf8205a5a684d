"""GPU parity: randomized PCA (Sec. 3.1.2) through the C ABI against the FP64 oracle.

Tolerances (stated per dtype):
* float32 path: |sigma_hat_i - sigma_i^O| <= 1e-5 * sigma_1^O for i <= k; vectors
  of well-separated singular values (relative gap >= 2e-2) agree entrywise to
  2e-3 after the common sign convention; U and V orthonormal to 1e-5.
* float64 path: relative sigma error <= 1e-10; vectors to 1e-8.
The oracle runs on the same stored values (the float32 matrix widened to
float64) with the same Gaussian test matrix Omega.
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


def _matrix(m, n, seed=0, shift=True):
    sig = synth.spectrum_harmonic_noise(n, 12087 + seed)
    A = synth.prescribed(m, n, sig, 12085 + seed, 12086 + seed)
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


def _run_rsvd(A_host, Om_host, k, p, q, dtype):
    tdt = torch.float32 if dtype == g.RSVD_F32 else torch.float64
    m, n = A_host.shape
    dev = torch.device("cuda")
    A = A_host.to(dev, tdt).contiguous()
    Om = Om_host.to(dev, tdt).contiguous()
    S = torch.zeros(k, dtype=torch.float64, device=dev)
    U = torch.zeros(m, k, dtype=tdt, device=dev)
    V = torch.zeros(n, k, dtype=tdt, device=dev)
    with g.rsvd_plan_create(m, n, k, p, q, dtype) as plan:
        g.check(g.rsvd(plan, A, None, Om, S, U, V), "rsvd")
        st = g.rsvd_plan_sync(plan)
        fro2 = g.rsvd_plan_fro2(plan)
        stK, K = g.pca_threshold(plan, 0.9)
    return dict(S=S.cpu().numpy(), U=U.cpu().double().numpy(), V=V.cpu().double().numpy(),
                A=A.cpu().double().numpy(), status=st, fro2=fro2, K=K, stK=stK)


@pytest.mark.parametrize("m,n,k,p,q", [
    (5037, 301, 20, 8, 2),     # several row tiles, ragged m, n and l
    (4096, 256, 50, 10, 2),    # the workload's k, p, q at reduced size
    (777, 64, 10, 6, 0),       # no power iteration
    (3000, 40, 30, 10, 1),     # l = n (full width)
    (6000, 300, 120, 8, 1),    # l = 128, the largest float32 batched / lockstep-served sketch
    (6000, 300, 136, 8, 1),    # l = 144: products on two column slices
    (6000, 300, 160, 16, 1),   # l = 176: Cholesky and Jacobi blocks in the global scratch
    (8000, 400, 256, 32, 1),   # l = 288, the largest single solve
])
def test_rsvd_f32_matches_oracle(m, n, k, p, q):
    A0 = _matrix(m, n)
    A32 = A0.float()
    Om = synth.gaussian(n, k + p, seed=12088, dtype=torch.float32)
    r = _run_rsvd(A32, Om, k, p, q, g.RSVD_F32)
    assert r["status"] == g.RSVD_OK
    Ac, mu, fro2 = oracle.center(A32.double())
    # A is read only (the means are subtracted inside the products); ||A - 1 mu^T||_F^2 (Eq. sumeigen)
    assert np.array_equal(r["A"], A32.double().numpy())
    assert abs(r["fro2"] - fro2) <= 1e-5 * fro2
    s, U, V = oracle.rsvd(Ac, Om.double(), q=q, k=k)
    assert np.abs(r["S"] - s).max() <= 1e-5 * s[0]
    assert np.abs(r["U"].T @ r["U"] - np.eye(k)).max() <= 1e-5
    assert np.abs(r["V"].T @ r["V"] - np.eye(k)).max() <= 1e-5
    sep = _gaps(s) >= 2e-2
    assert np.abs(r["V"][:, sep] - V[:, sep]).max() <= 2e-3
    assert np.abs(r["U"][:, sep] - U[:, sep]).max() <= 2e-3
    # K of Sec. 2.4 over the returned values
    Ko, reached = oracle.pca_threshold(s, fro2, 0.9)
    assert r["K"] == Ko
    assert r["stK"] == (g.RSVD_OK if reached else g.RSVD_WARN_K_GT_k)


@pytest.mark.parametrize("m,n,k,p,q", [(2021, 97, 12, 5, 2), (600, 33, 33, 0, 1)])
def test_rsvd_f64_matches_oracle(m, n, k, p, q):
    A0 = _matrix(m, n, seed=3)
    Om = synth.gaussian(n, k + p, seed=5, dtype=torch.float64)
    r = _run_rsvd(A0, Om, k, p, q, g.RSVD_F64)
    assert r["status"] == g.RSVD_OK
    Ac, mu, fro2 = oracle.center(A0)
    assert abs(r["fro2"] - fro2) <= 1e-12 * fro2
    s, U, V = oracle.rsvd(Ac, Om, q=q, k=k)
    assert (np.abs(r["S"] - s) / s).max() <= 1e-10
    sep = _gaps(s) >= 1e-3
    assert np.abs(r["V"][:, sep] - V[:, sep]).max() <= 1e-8
    assert np.abs(r["U"][:, sep] - U[:, sep]).max() <= 1e-8


def test_rsvd_rank_deficient_tail_exact():
    """rank(A) <= l: the sketch captures range(A); sigma equal the prescribed values."""
    m, n, r_, k, p = 3001, 120, 10, 8, 4
    sig = torch.linspace(4.0, 1.0, r_, dtype=torch.float64)
    A = synth.prescribed(m, n, sig, 7, 8)
    Om = synth.gaussian(n, k + p, seed=9, dtype=torch.float64)
    r = _run_rsvd(A, Om, k, p, 1, g.RSVD_F64)
    assert np.abs(r["S"] - sig.numpy()[:k]).max() <= 1e-12 * 4.0


def test_rsvd_single_column():
    m, n = 1000, 1
    A = synth.gaussian(m, 1, seed=1)
    Om = torch.ones(1, 1, dtype=torch.float32)
    r = _run_rsvd(A.float(), Om, 1, 0, 1, g.RSVD_F32)
    Ac = A.numpy() - A.numpy().mean(0)
    assert abs(r["S"][0] - np.linalg.norm(Ac)) <= 1e-5 * np.linalg.norm(Ac)
    assert abs(abs(r["V"][0, 0]) - 1.0) < 1e-6 and r["V"][0, 0] > 0


def test_rsvd_zero_matrix_reports_breakdown():
    """A = 0 after centring: the Gram matrix is zero, CholeskyQR cannot proceed."""
    m, n = 500, 20
    A = torch.ones(m, n, dtype=torch.float64) * 3.0   # constant columns centre to zero
    Om = synth.gaussian(n, 6, seed=2, dtype=torch.float32)
    r = _run_rsvd(A.float(), Om, 4, 2, 1, g.RSVD_F32)
    assert r["status"] == g.RSVD_ERR_CHOL
    assert r["fro2"] == 0.0
    assert np.all(np.isfinite(r["S"]))


def test_rsvd_no_center_flag_keeps_input():
    m, n, k, p = 1500, 50, 5, 3
    A0 = _matrix(m, n, shift=False).float()
    Om = synth.gaussian(n, k + p, seed=4, dtype=torch.float32)
    dev = torch.device("cuda")
    A = A0.to(dev).contiguous()
    A_before = A.clone()
    S = torch.zeros(k, dtype=torch.float64, device=dev)
    U = torch.zeros(m, k, device=dev)
    V = torch.zeros(n, k, device=dev)
    with g.rsvd_plan_create(m, n, k, p, 1, g.RSVD_F32) as plan:
        assert g.rsvd_plan_set_flags(plan, g.RSVD_FLAG_NO_CENTER) == g.RSVD_OK
        g.check(g.rsvd(plan, A, None, Om.to(dev), S, U, V))
        assert g.rsvd_plan_sync(plan) == g.RSVD_OK
    assert torch.equal(A, A_before)
    s, _, _ = oracle.rsvd(A0.double(), Om.double(), q=1, k=k)
    assert np.abs(S.cpu().numpy() - s).max() <= 1e-5 * s[0]


def test_rsvd_rejects_col_scales_for_f32():
    m, n = 100, 10
    dev = torch.device("cuda")
    A = torch.randn(m, n, device=dev)
    with g.rsvd_plan_create(m, n, 2, 1, 0, g.RSVD_F32) as plan:
        sc = torch.ones(n, device=dev)
        st = g.rsvd(plan, A, sc, torch.randn(n, 3, device=dev), torch.zeros(2, dtype=torch.float64, device=dev),
                    torch.zeros(m, 2, device=dev), torch.zeros(n, 2, device=dev))
        assert st == g.RSVD_ERR_ARG


def test_rsvd_repeatable_bitwise():
    """Split-K partials are summed in a fixed order: two solves give identical bits."""
    m, n, k, p = 20000, 200, 16, 8
    A0 = _matrix(m, n, shift=False).float()
    Om = synth.gaussian(n, k + p, seed=4, dtype=torch.float32)
    r1 = _run_rsvd(A0, Om, k, p, 2, g.RSVD_F32)
    r2 = _run_rsvd(A0, Om, k, p, 2, g.RSVD_F32)
    assert np.array_equal(r1["S"], r2["S"]) and np.array_equal(r1["U"], r2["U"])


@pytest.mark.slow
def test_rsvd_f32_full_workload_matches_oracle():
    """The benchmark's workload at full size (200000 x 1000, k = 50, p = 10, q = 2),
    solved as bench.py times it (captured graph on a user stream), against the FP64
    oracle on the same stored float32 matrix and Omega."""
    dev = torch.device("cuda")
    A64, sigma, ex = synth.workload("rpca_fp32_200000x1000", device=dev)
    A = A64.float().contiguous()
    del A64
    Om = ex["omega"].to(dev).contiguous()
    m, n = A.shape
    k, p, q = 50, 10, 2
    S = torch.zeros(k, dtype=torch.float64, device=dev)
    U = torch.zeros(m, k, device=dev)
    V = torch.zeros(n, k, device=dev)
    stream = torch.cuda.Stream()
    torch.cuda.synchronize()                       # inputs were made on the default stream
    with torch.cuda.stream(stream):
        with g.rsvd_plan_create(m, n, k, p, q, g.RSVD_F32, stream) as plan:
            for _ in range(2):                     # capture, then replay
                g.check(g.rsvd(plan, A, None, Om, S, U, V))
            assert g.rsvd_plan_sync(plan) == g.RSVD_OK
            stK, K = g.pca_threshold(plan, 0.9)
    torch.cuda.synchronize()
    Ah = A.cpu().double().numpy()
    Ac, mu, fro2 = oracle.center(Ah)
    s, Uo, Vo = oracle.rsvd(Ac, Om.cpu().double(), q=q, k=k)
    Sg = S.cpu().numpy()
    assert np.abs(Sg - s).max() <= 1e-5 * s[0]
    Vg = V.cpu().double().numpy()
    assert np.abs(Vg.T @ Vg - np.eye(k)).max() <= 1e-5
    sep = _gaps(s) >= 2e-2
    assert np.abs(Vg[:, sep] - Vo[:, sep]).max() <= 2e-3
    assert K == oracle.pca_threshold(s, fro2, 0.9)[0]


@pytest.mark.parametrize("q", [1, 3])
def test_rsvd_f32_power15_spectrum_l288(q):
    """The precision-form workload's spectrum sigma_i = i^-1.5 at l = 288 (reduced m, n): the
    float32 path's CholeskyQR2 of T still resolves it (cond(T) ~ 288^1.5)."""
    m, n, k, p = 20000, 2048, 256, 32
    A32 = synth.prescribed(m, n, synth.spectrum_power(n, 1.5), 40961, 40962).float()
    Om = synth.gaussian(n, k + p, seed=40964, dtype=torch.float32)
    r = _run_rsvd(A32, Om, k, p, q, g.RSVD_F32)
    assert r["status"] == g.RSVD_OK
    Ac, _, _ = oracle.center(A32.double())
    s, _, _ = oracle.rsvd(Ac, Om.double(), q=q, k=k)
    assert np.abs(r["S"] - s).max() <= 1e-5 * s[0]
