"""rsvd_quantize (precision-form storage) against the oracle's encoders, code
for code (byte / index work: bit-exact), on matrices that exercise exact ties,
subnormal quotients, saturation, signed zeros and an all-zero column."""
import numpy as np
import pytest
import torch

import oracle
import paper_1906_12085_gb300 as g

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1906_12085_gb300 import build
    build.build()
    oracle.build()


def _matrix(m, n, seed):
    rng = np.random.default_rng(seed)
    A = rng.normal(0, 1, (m, n)).astype(np.float32) * np.float32(10.0) ** rng.integers(-6, 6, n).astype(np.float32)
    if n > 3:
        A[:, 1] = 0.0                                    # all-zero column
        A[0, 2] = -0.0
        A[1, 3] = np.float32(1e-30)                      # quotient far below the smallest e4m3 subnormal
    bits = A.view(np.uint32)
    bits[2::7, 0] = (bits[2::7, 0] & 0xFFFF0000) | 0x8000   # bfloat16 ties
    return A


@pytest.mark.parametrize("m,n", [(1000, 37), (4097, 256), (3, 1)])
def test_bf16_codes_bit_exact(m, n):
    A = _matrix(m, n, m + n)
    dev = torch.device("cuda")
    Aq = torch.empty(m, n, dtype=torch.int16, device=dev)
    g.check(g.rsvd_quantize(torch.from_numpy(A).to(dev), g.RSVD_BF16, Aq))
    torch.cuda.synchronize()
    got = Aq.cpu().numpy().view(np.uint16)
    assert np.array_equal(got, oracle.quantize_bf16(A))


@pytest.mark.parametrize("m,n", [(1000, 37), (4097, 256), (3, 1), (20000, 64)])
def test_e4m3_codes_and_scales_bit_exact(m, n):
    A = _matrix(m, n, 10 * m + n)
    dev = torch.device("cuda")
    Aq = torch.empty(m, n, dtype=torch.uint8, device=dev)
    sc = torch.empty(n, dtype=torch.float32, device=dev)
    g.check(g.rsvd_quantize(torch.from_numpy(A).to(dev), g.RSVD_FP8_E4M3, Aq, sc))
    torch.cuda.synchronize()
    codes, scales = oracle.quantize_e4m3(A)
    assert np.array_equal(sc.cpu().numpy().view(np.uint32), scales.view(np.uint32))
    assert np.array_equal(Aq.cpu().numpy(), codes)


def test_quantize_argument_errors():
    dev = torch.device("cuda")
    A = torch.zeros(10, 4, device=dev)
    Aq = torch.empty(10, 4, dtype=torch.uint8, device=dev)
    assert g.rsvd_quantize(A, g.RSVD_FP8_E4M3, Aq, None) == g.RSVD_ERR_ARG
    assert g.rsvd_quantize(A, g.RSVD_F32, Aq, None) == g.RSVD_ERR_UNSUPPORTED
