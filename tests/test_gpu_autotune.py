"""Autotuner of the tensor-core products' launch shape (rsvd_autotune): the
choice is one of the candidates, it is recorded for the plan's bucket and
picked up by plans created afterwards, and since only the number of
persistent CTAs changes (not the tiles or their summation order) a solve with
the tuned shape is bitwise the solve with the default one, which in turn meets
the float32 tolerance against the FP64 oracle (1e-5 sigma_1)."""
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
    yield
    g.rsvd_tune_clear()


def test_autotune_records_and_applies_choice():
    m, n, k, p, q = 40000, 512, 24, 8, 2
    dev = torch.device("cuda")
    sig = synth.spectrum_power(n, 1.0)
    A = synth.prescribed(m, n, sig, 41, 42).float()
    Om = synth.gaussian(n, k + p, seed=43, dtype=torch.float32)
    Ad, Od = A.to(dev), Om.to(dev)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    g.rsvd_tune_clear()
    with g.rsvd_plan_create(m, n, k, p, q, g.RSVD_F32) as plan:
        st, nn, tn = g.rsvd_autotune(plan, Ad, Od, concurrency=3)
        assert st == g.RSVD_OK
    assert (nn, tn) in {(0, 0), (sms // 2, sms // 2), (sms // 4, sms // 4), (sms // 2, 0), (0, sms // 2)}
    assert g.rsvd_tune_lookup(m, n, k, p) == (g.RSVD_OK, nn, tn)
    assert g.rsvd_tune_lookup(m + 1, n, k, p)[0] == g.RSVD_OK          # same ceil(log2 m) bucket

    def solve():
        S = torch.zeros(k, dtype=torch.float64, device=dev)
        U = torch.zeros(m, k, device=dev)
        V = torch.zeros(n, k, device=dev)
        with g.rsvd_plan_create(m, n, k, p, q, g.RSVD_F32) as plan:
            g.check(g.rsvd(plan, Ad, None, Od, S, U, V))
            assert g.rsvd_plan_sync(plan) == g.RSVD_OK
        return S.cpu().numpy(), U.cpu().numpy(), V.cpu().numpy()

    tuned = solve()
    g.rsvd_tune_clear()
    assert g.rsvd_tune_lookup(m, n, k, p)[0] == g.RSVD_ERR_ARG
    default = solve()
    for a, b in zip(tuned, default):
        assert np.array_equal(a, b)
    Ac, mu, fro2 = oracle.center(A.double())
    s, _, _ = oracle.rsvd(Ac, Om.double(), q=q, k=k)
    assert np.abs(default[0] - s).max() <= 1e-5 * s[0]
