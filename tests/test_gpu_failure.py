"""Failure detection without a GPU fault: each failure is made on purpose in a way that
leaves the context usable, and the status that reports it is checked.

* Jacobi non-convergence: the process-wide sweep cap set to one sweep makes the one-sided
  SVD of R (randomized PCA) and the two-sided eigen-decomposition (Gram route) stop
  before a sweep without rotations: RSVD_ERR_NOCONV.  With the default cap restored the
  same solves succeed.
* Bounded device waits: a standalone kernel (tests/native/mbar_timeout.cu) runs the
  product kernels' mbarrier wait with a short cap on a barrier nothing arrives at; the
  wait gives up and reports the timeout status bit, and a barrier that is completed is
  still waited on successfully.  No TMA copy, MMA or tensor-memory allocation is in
  flight in that kernel (the product kernels' own waits are not shortened).
"""
import os
import shutil
import subprocess

import numpy as np
import pytest
import torch

import oracle
import paper_1906_12085_gb300 as g
import synth

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
ST_TIMEOUT = 16  # the device status bit of a wait that gave up (maps to RSVD_ERR_TIMEOUT)


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1906_12085_gb300 import build
    build.build()
    yield
    g.rsvd_set_jacobi_sweep_cap(0)


def _rsvd(A, Om, k, p, q):
    dev = torch.device("cuda")
    m, n = A.shape
    S = torch.zeros(k, dtype=torch.float64, device=dev)
    U = torch.zeros(m, k, device=dev)
    V = torch.zeros(n, k, device=dev)
    with g.rsvd_plan_create(m, n, k, p, q, g.RSVD_F32) as plan:
        g.check(g.rsvd(plan, A.to(dev), None, Om.to(dev), S, U, V), "rsvd")
        return g.rsvd_plan_sync(plan), S.cpu().numpy()


def _gram(A):
    dev = torch.device("cuda")
    m, n = A.shape
    Ad = A.to(dev).clone()
    S = torch.zeros(n, dtype=torch.float64, device=dev)
    U = torch.zeros(m, n, dtype=torch.float64, device=dev)
    V = torch.zeros(n, n, dtype=torch.float64, device=dev)
    with g.rsvd_plan_create(m, n, 1, 0, 0, g.RSVD_F64) as plan:
        g.check(g.svd_exact(plan, Ad, g.RSVD_EXACT_GRAM, S, U, V), "svd_exact")
        return g.rsvd_plan_sync(plan), S.cpu().numpy()


def test_jacobi_sweep_cap_reports_noconv():
    m, n, k, p, q = 3000, 200, 20, 8, 1
    A = synth.prescribed(m, n, synth.spectrum_power(n, 1.0), 31, 32).float()
    Om = synth.gaussian(n, k + p, seed=33, dtype=torch.float32)
    A64 = synth.prescribed(2000, 100, synth.spectrum_pow2(100), 34, 35)
    assert g.rsvd_set_jacobi_sweep_cap(-1) == g.RSVD_ERR_ARG
    try:
        assert g.rsvd_set_jacobi_sweep_cap(1) == g.RSVD_OK
        st, _ = _rsvd(A, Om, k, p, q)
        assert st == g.RSVD_ERR_NOCONV
        st, _ = _gram(A64)
        assert st == g.RSVD_ERR_NOCONV
    finally:
        g.rsvd_set_jacobi_sweep_cap(0)
    st, S = _rsvd(A, Om, k, p, q)
    assert st == g.RSVD_OK
    s, _, _ = oracle.rsvd(oracle.center(A.double())[0], Om.double(), q=q, k=k)
    assert np.abs(S - s).max() <= 1e-5 * s[0]
    st, S = _gram(A64)
    assert st == g.RSVD_OK
    assert np.abs(S - synth.spectrum_pow2(100).numpy()).max() <= 1e-9


def test_bounded_mbarrier_wait_gives_up():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    exe = os.path.join(ROOT, "paper_1906_12085_gb300", "_build", "mbar_timeout")
    os.makedirs(os.path.dirname(exe), exist_ok=True)
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-std=c++17", "-O2",
                    "-I", os.path.join(ROOT, "include"), "-I", os.path.join(ROOT, "paper_1906_12085_gb300", "csrc"),
                    os.path.join(HERE, "native", "mbar_timeout.cu"), "-o", exe], check=True)
    out = subprocess.run([exe, "256"], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0, out.stdout + out.stderr
    err, status, completed, ns = (int(x) for x in out.stdout.split())
    assert err == 0
    assert status == ST_TIMEOUT
    assert completed == 1
    print(f"abandoned wait: 256 polls in {ns / 1e3:.1f} us")
