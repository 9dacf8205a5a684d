"""GPU parity: Golub-Kahan-Lanczos with full reorthogonalisation (svd_truncated_krylov)
against the FP64 oracle GKL run from the same start vector v1.

Tolerances: float32 |sigma_hat_i - sigma_i^O| <= 1e-5 * sigma_1^O (i <= k);
float64 relative 1e-10.  Ritz pairs satisfy A v_i = sigma_i u_i exactly in exact
arithmetic (A V_s = U_s B), checked to 1e-5 * sigma_1 (float32) at every size,
including the full 1048576 x 2048 Lanczos workload.
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


def _run(A_dev, v1_dev, k, steps, dtype, flags=0):
    m, n = A_dev.shape
    S = torch.zeros(k, dtype=torch.float64, device=A_dev.device)
    U = torch.zeros(m, k, dtype=A_dev.dtype, device=A_dev.device)
    V = torch.zeros(n, k, dtype=A_dev.dtype, device=A_dev.device)
    with g.rsvd_plan_create(m, n, k, 0, 0, dtype) as plan:
        g.check(g.rsvd_plan_set_flags(plan, flags), "flags")
        g.check(g.svd_truncated_krylov(plan, A_dev, v1_dev, steps, S, U, V), "svd_truncated_krylov")
        st = g.rsvd_plan_sync(plan)
    return st, S, U, V


def _check_f32(A32, v1, k, steps, S, U, V, tag=""):
    Ac, _, _ = oracle.center(A32.double())
    s, Uo, Vo, al, be = oracle.gkl(Ac, v1.double(), steps=steps, k=k)
    S = S.cpu().numpy()
    err = np.abs(S - s).max() / s[0]
    print(f"{tag}: max sigma error {err:.2e} sigma_1")
    assert err <= 1e-5
    Ud, Vd = U.cpu().double().numpy(), V.cpu().double().numpy()
    assert np.abs(Ud.T @ Ud - np.eye(k)).max() <= 1e-5
    assert np.abs(Vd.T @ Vd - np.eye(k)).max() <= 1e-5
    assert np.abs(Ac @ Vd - Ud * S).max() <= 1e-5 * s[0]


@pytest.mark.parametrize("scale", [200.0, 10.0])
def test_gkl_f32_one_pass_and_two_pass_match_oracle(scale):
    """float32 plans read A once per step (A^T u_j recovered by linearity); on the steep
    exp(-i/10) spectrum the recovery's bound sends steps to the second read of A.  Both
    forms and the forced two-pass form agree with the oracle from the same v1."""
    m, n, k, steps = 20011, 512, 40, 120
    i = torch.arange(1, n + 1, dtype=torch.float64)
    A = synth.prescribed(m, n, torch.exp(-i / scale), 20481, 20482)
    A32 = A.float()
    v1 = synth.unit_vector(n, 20483, dtype=torch.float32)
    dev = torch.device("cuda")
    for flags, tag in [(0, "one pass"), (g.RSVD_FLAG_GKL_TWO_PASS, "two passes")]:
        st, S, U, V = _run(A32.to(dev), v1.to(dev), k, steps, g.RSVD_F32, flags)
        assert st == g.RSVD_OK
        _check_f32(A32, v1, k, steps, S, U, V, f"exp(-i/{scale:g}) {tag}")


@pytest.mark.slow
def test_gkl_f32_lanczos_width_matches_oracle():
    """The Lanczos workload's columns, steps and k (2048, 150, 100) at 262144 rows, from its v1."""
    m, n, k, steps = 262144, 2048, 100, 150
    dev = torch.device("cuda")
    A, sigma, ex = synth.workload("gkl_fp32_1048576x2048", m=m, device=dev)
    A32 = A.float()
    del A
    v1 = ex["v1"]
    st, S, U, V = _run(A32, v1.to(dev), k, steps, g.RSVD_F32)
    assert st == g.RSVD_OK
    _check_f32(A32.cpu(), v1.cpu(), k, steps, S, U, V, "262144 x 2048, 150 steps")


@pytest.mark.parametrize("m,n,k,steps", [(20011, 301, 20, 60), (5000, 130, 10, 40)])
def test_gkl_f32_matches_oracle(m, n, k, steps):
    A, sigma, ex = synth.workload("gkl_fp32_1048576x2048", m=m, n=n)
    A32 = A.float()
    v1 = synth.unit_vector(n, 20483, dtype=torch.float32)
    dev = torch.device("cuda")
    st, S, U, V = _run(A32.to(dev), v1.to(dev), k, steps, g.RSVD_F32)
    assert st == g.RSVD_OK
    Ac, _, _ = oracle.center(A32.double())
    s, Uo, Vo, al, be = oracle.gkl(Ac, v1.double(), steps=steps, k=k)
    S = S.cpu().numpy()
    assert np.abs(S - s).max() <= 1e-5 * s[0]
    Ud, Vd = U.cpu().double().numpy(), V.cpu().double().numpy()
    assert np.abs(Ud.T @ Ud - np.eye(k)).max() <= 1e-5
    assert np.abs(Vd.T @ Vd - np.eye(k)).max() <= 1e-5
    assert np.abs(Ac @ Vd - Ud * S).max() <= 1e-5 * s[0]


def test_gkl_f64_matches_oracle():
    m, n, k, steps = 3001, 90, 12, 50
    A, sigma, ex = synth.workload("gkl_fp32_1048576x2048", m=m, n=n)
    v1 = synth.unit_vector(n, 7)
    dev = torch.device("cuda")
    st, S, U, V = _run(A.to(dev), v1.to(dev), k, steps, g.RSVD_F64)
    assert st == g.RSVD_OK
    Ac, _, _ = oracle.center(A)
    s, Uo, Vo, al, be = oracle.gkl(Ac, v1, steps=steps, k=k)
    S = S.cpu().numpy()
    assert (np.abs(S - s) / s).max() <= 1e-10
    Vd = V.cpu().numpy()
    assert np.abs(np.abs(np.sum(Vd * Vo, axis=0)) - 1).max() <= 1e-8


def test_gkl_full_steps_reproduces_spectrum():
    """steps = n spans R^n: every singular value is exact (prescribed spectrum)."""
    m, n = 4000, 40
    sig = torch.linspace(3.0, 0.5, n, dtype=torch.float64)
    A = synth.prescribed(m, n, sig, 3, 4)
    v1 = synth.unit_vector(n, 5)
    dev = torch.device("cuda")
    st, S, U, V = _run(A.to(dev), v1.to(dev), n, n, g.RSVD_F64)
    assert np.abs(S.cpu().numpy() - sig.numpy()).max() <= 1e-12 * 3.0


def test_gkl_rejects_bad_steps():
    dev = torch.device("cuda")
    m, n = 1000, 50
    A = torch.randn(m, n, device=dev)
    v1 = torch.randn(n, device=dev)
    S = torch.zeros(10, dtype=torch.float64, device=dev)
    with g.rsvd_plan_create(m, n, 10, 0, 0, g.RSVD_F32) as plan:
        U = torch.zeros(m, 10, device=dev)
        V = torch.zeros(n, 10, device=dev)
        assert g.svd_truncated_krylov(plan, A, v1, 5, S, U, V) == g.RSVD_ERR_ARG     # steps < k
        assert g.svd_truncated_krylov(plan, A, v1, 51, S, U, V) == g.RSVD_ERR_ARG    # steps > n


@pytest.mark.slow
def test_gkl_full_size_workload_properties():
    """1048576 x 2048 float32, sigma_i = exp(-i/200), 150 steps, k = 100 (full size)."""
    dev = torch.device("cuda")
    name = "gkl_fp32_1048576x2048"
    A64, sigma, ex = synth.workload(name, device=dev)
    A = A64.float()
    del A64
    v1 = ex["v1"].to(dev)
    st, S, U, V = _run(A, v1, 100, 150, g.RSVD_F32)
    assert st == g.RSVD_OK
    S64 = S.double()
    # Ritz values are ordered and bounded by the true singular values (sigma(A V_s) <= sigma(A)),
    # up to the float32 tolerance 1e-5 * sigma_1
    sig = sigma.to(dev)
    assert torch.all(S64[:-1] >= S64[1:])
    assert float((S64 - sig[:100]).max()) <= 1e-5 * float(sig[0])
    # the leading Ritz values have converged to the prescribed spectrum
    assert torch.abs(S64[:5] - sig[:5]).max() <= 1e-5 * sig[0]
    assert torch.abs(U.T @ U - torch.eye(100, device=dev)).max() <= 1e-4
    assert torch.abs(V.T @ V - torch.eye(100, device=dev)).max() <= 1e-4
    R = A @ V - U * S.float()
    assert R.abs().max() <= 1e-5 * float(sig[0])
