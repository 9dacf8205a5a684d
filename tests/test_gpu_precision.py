"""Precision form: randomized PCA of a bfloat16- or e4m3-stored matrix
against the FP64 oracle run on the same stored matrix (the oracle's own
bfloat16 encoding of the float32 matrix, dequantised exactly) and the same
Omega.  The sketch and power products round their small operand to bfloat16,
which perturbs only the basis; the Rayleigh-Ritz product is float32-accurate.
Reported and bounded (tolerances stated here, derived in the design notes;
||A - 1 mu^T||_F^2 to 1e-6 relative):
  sigma: |s_i - s_i^O| <= 1e-4 sigma_1^O for i <= k;
  gap:   (||A - U U^T A||_F - ||A - U^O U^O^T A||_F) / ||A||_F <= 1e-4;
  U, V orthonormal to 1e-5."""
import os

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
    oracle.build()


def _stored(m, n, seed, shift=True):
    sig = synth.spectrum_power(n, 1.5)
    A = synth.prescribed(m, n, sig, 40961 + seed, 40962 + seed)
    if shift:
        A = A + torch.linspace(-0.05, 0.1, n, dtype=torch.float64).unsqueeze(0)
    A32 = A.float().numpy()
    codes = oracle.quantize_bf16(A32)
    return codes, oracle.dequantize_bf16(codes)


def _proj_residual(A, U):
    """||A - U U^T A||_F for orthonormal U (float64)."""
    B = U.T @ A
    return np.sqrt(max(np.sum(A * A) - np.sum(B * B), 0.0))


@pytest.mark.parametrize("m,n,k,p,q,shift", [
    (60000, 512, 48, 16, 3, True),
    (20011, 256, 20, 12, 2, True),     # ragged m
    (30000, 1024, 40, 8, 1, False),    # data centred, NO_CENTER
    (20011, 512, 256, 32, 2, True),    # l = 288 (k = 256, p = 32: the precision form's widest sketch)
])
def test_bf16_rsvd_matches_oracle_on_stored_matrix(m, n, k, p, q, shift):
    codes, Ad = _stored(m, n, m % 97, shift)
    Om = synth.gaussian(n, k + p, seed=40964, dtype=torch.float32)
    dev = torch.device("cuda")
    A = torch.from_numpy(codes.view(np.int16)).to(dev)
    S = torch.zeros(k, dtype=torch.float64, device=dev)
    U = torch.zeros(m, k, device=dev)
    V = torch.zeros(n, k, device=dev)
    with g.rsvd_plan_create(m, n, k, p, q, g.RSVD_BF16) as plan:
        if not shift:
            g.check(g.rsvd_plan_set_flags(plan, g.RSVD_FLAG_NO_CENTER))
        g.check(g.rsvd(plan, A, None, Om.to(dev), S, U, V), "rsvd bf16")
        assert g.rsvd_plan_sync(plan) == g.RSVD_OK
        fro2 = g.rsvd_plan_fro2(plan)
        stK, K = g.pca_threshold(plan, 0.9)
    torch.cuda.synchronize()
    Ac, mu, fro2o = oracle.center(Ad) if shift else (Ad, None, float(np.sum(Ad * Ad)))
    # squares summed in float32 over 32-row groups, then float64; sum a^2 - m mu^2 cancels by (mu / std)^2
    assert abs(fro2 - fro2o) <= 1e-6 * fro2o
    s, Uo, Vo = oracle.rsvd(Ac, Om.double(), q=q, k=k)
    Sg, Ug, Vg = S.cpu().numpy(), U.cpu().double().numpy(), V.cpu().double().numpy()
    err = np.abs(Sg - s).max() / s[0]
    assert err <= 1e-4, err
    assert np.abs(Ug.T @ Ug - np.eye(k)).max() <= 1e-5
    assert np.abs(Vg.T @ Vg - np.eye(k)).max() <= 1e-5
    gap = (_proj_residual(Ac, Ug) - _proj_residual(Ac, Uo)) / np.sqrt(np.sum(Ac * Ac))
    assert gap <= 1e-4, gap
    print(f"bf16 rsvd {m}x{n} k={k}: max sigma error {err:.2e} sigma_1, projection gap {gap:.2e} ||A||_F")
    Ko, reached = oracle.pca_threshold(s, fro2o, 0.9)
    assert K == Ko


def test_bf16_plan_rejects_unsupported_paths():
    dev = torch.device("cuda")
    with g.rsvd_plan_create(1000, 64, 8, 8, 1, g.RSVD_BF16) as plan:
        A = torch.zeros(1000, 64, dtype=torch.int16, device=dev)
        S = torch.zeros(64, dtype=torch.float64, device=dev)
        assert g.svd_exact(plan, A, g.RSVD_EXACT_GRAM, S, S, S) == g.RSVD_ERR_UNSUPPORTED
        v1 = torch.ones(64, device=dev)
        assert g.svd_truncated_krylov(plan, A, v1, 16, S, S, S) == g.RSVD_ERR_UNSUPPORTED
        with pytest.raises(g.RsvdError):
            g.rsvd_batch_create([plan])


def _stored8(m, n, seed, shift=True):
    sig = synth.spectrum_power(n, 1.5)
    A = synth.prescribed(m, n, sig, 40963 + seed, 40964 + seed)
    if shift:
        A = A + torch.linspace(-0.05, 0.1, n, dtype=torch.float64).unsqueeze(0)
    codes, scales = oracle.quantize_e4m3(A.float().numpy())
    return codes, scales, oracle.dequantize_e4m3(codes, scales)


@pytest.mark.parametrize("m,n,k,p,q,shift", [
    (60000, 512, 48, 16, 3, True),
    (20011, 256, 20, 12, 2, True),
    (30000, 1024, 40, 8, 1, False),
    (20011, 512, 256, 32, 2, True),    # l = 288
])
def test_e4m3_rsvd_matches_oracle_on_stored_matrix(m, n, k, p, q, shift):
    """e4m3 storage: the sketch and power operands are quantised to e4m3 (3 mantissa
    bits), which perturbs the basis by up to 2^-4 relative per step; the
    Rayleigh-Ritz product is float32-accurate.  Bounds: sigma within 1e-3 sigma_1,
    projection gap within 1e-3 ||A||_F (both stated, not derived tight)."""
    codes, scales, Ad = _stored8(m, n, m % 89, shift)
    Om = synth.gaussian(n, k + p, seed=40965, dtype=torch.float32)
    dev = torch.device("cuda")
    A = torch.from_numpy(codes).to(dev)
    sc = torch.from_numpy(scales).to(dev)
    S = torch.zeros(k, dtype=torch.float64, device=dev)
    U = torch.zeros(m, k, device=dev)
    V = torch.zeros(n, k, device=dev)
    with g.rsvd_plan_create(m, n, k, p, q, g.RSVD_FP8_E4M3) as plan:
        if not shift:
            g.check(g.rsvd_plan_set_flags(plan, g.RSVD_FLAG_NO_CENTER))
        assert g.rsvd(plan, A, None, Om.to(dev), S, U, V) == g.RSVD_ERR_ARG    # the scales are required
        g.check(g.rsvd(plan, A, sc, Om.to(dev), S, U, V), "rsvd e4m3")
        assert g.rsvd_plan_sync(plan) == g.RSVD_OK
        fro2 = g.rsvd_plan_fro2(plan)
        stK, K = g.pca_threshold(plan, 0.9)
    torch.cuda.synchronize()
    Ac, mu, fro2o = oracle.center(Ad) if shift else (Ad, None, float(np.sum(Ad * Ad)))
    assert abs(fro2 - fro2o) <= 1e-6 * fro2o
    s, Uo, Vo = oracle.rsvd(Ac, Om.double(), q=q, k=k)
    Sg, Ug, Vg = S.cpu().numpy(), U.cpu().double().numpy(), V.cpu().double().numpy()
    err = np.abs(Sg - s).max() / s[0]
    gap = (_proj_residual(Ac, Ug) - _proj_residual(Ac, Uo)) / np.sqrt(np.sum(Ac * Ac))
    print(f"e4m3 rsvd {m}x{n} k={k}: max sigma error {err:.2e} sigma_1, projection gap {gap:.2e} ||A||_F")
    assert err <= 1e-3, err
    assert gap <= 1e-3, gap
    assert np.abs(Ug.T @ Ug - np.eye(k)).max() <= 1e-5
    assert np.abs(Vg.T @ Vg - np.eye(k)).max() <= 1e-5


@pytest.fixture(scope="module")
def mixed_262144x4096():
    """The precision form's workload with a quarter of its rows: 262144 x 4096, sigma_i = i^-1.5,
    Haar factors (built in float64 on the device), rounded to float32; Omega 4096 x 288."""
    A, sig, ex = synth.workload("mixed_rsvd_1048576x4096", m=262144, device="cuda")
    A32 = A.float().cpu().numpy()
    del A
    torch.cuda.empty_cache()
    return A32, ex["omega"].cpu()


@pytest.mark.slow
@pytest.mark.skipif(os.environ.get("RSVD_TEST_FULL") != "1",
                    reason="about 6 minutes of float64 oracle time per case; set RSVD_TEST_FULL=1")
@pytest.mark.parametrize("dtype", ["bf16", "fp8"])
def test_precision_form_at_262144x4096_l288_matches_oracle(mixed_262144x4096, dtype):
    """k = 256, p = 32, q = 3 on the stored matrix; the oracle runs in float64 on the decoded
    matrix.  Bounds as in the smaller cases: sigma within 1e-4 (BF16) / 1e-3 (e4m3) of
    sigma_1, the same for the projection gap relative to ||A||_F; U, V orthonormal to 1e-5."""
    A32, Om = mixed_262144x4096
    m, n = A32.shape
    k, p, q = 256, 32, 3
    dev = torch.device("cuda")
    if dtype == "bf16":
        codes = oracle.quantize_bf16(A32)
        Ad = oracle.dequantize_bf16(codes)
        A, sc, dt, tol = torch.from_numpy(codes.view(np.int16)).to(dev), None, g.RSVD_BF16, 1e-4
    else:
        codes, scales = oracle.quantize_e4m3(A32)
        Ad = oracle.dequantize_e4m3(codes, scales)
        A, sc, dt, tol = torch.from_numpy(codes).to(dev), torch.from_numpy(scales).to(dev), g.RSVD_FP8_E4M3, 1e-3
    del codes
    S = torch.zeros(k, dtype=torch.float64, device=dev)
    U = torch.zeros(m, k, device=dev)
    V = torch.zeros(n, k, device=dev)
    with g.rsvd_plan_create(m, n, k, p, q, dt) as plan:
        g.check(g.rsvd(plan, A, sc, Om.to(dev), S, U, V), "rsvd " + dtype)
        assert g.rsvd_plan_sync(plan) == g.RSVD_OK
        fro2 = g.rsvd_plan_fro2(plan)
    torch.cuda.synchronize()
    del A
    Ac, mu, fro2o = oracle.center(Ad)
    del Ad
    assert abs(fro2 - fro2o) <= 1e-6 * fro2o
    s, Uo, Vo = oracle.rsvd(Ac, Om.double(), q=q, k=k)
    Sg, Ug, Vg = S.cpu().numpy(), U.cpu().double().numpy(), V.cpu().double().numpy()
    err = np.abs(Sg - s).max() / s[0]
    gap = (_proj_residual(Ac, Ug) - _proj_residual(Ac, Uo)) / np.sqrt(fro2o)
    print(f"{dtype} rsvd {m}x{n} k={k} p={p} q={q}: max sigma error {err:.2e} sigma_1, "
          f"projection gap {gap:.2e} ||A||_F")
    assert err <= tol, err
    assert gap <= tol, gap
    assert np.abs(Ug.T @ Ug - np.eye(k)).max() <= 1e-5
    assert np.abs(Vg.T @ Vg - np.eye(k)).max() <= 1e-5
