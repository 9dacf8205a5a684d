"""Pins of the oracle's storage-format encoders (precision form: BF16
round-to-nearest-even, e4m3 with per-column scales): values fixed by the format definitions (bfloat16: 8 exponent
and 7 mantissa bits; OCP e4m3: bias 7, 3 mantissa bits, largest finite 448,
no infinities), exact ties resolved to the even code, saturation, subnormals,
round trips over every code, and torch's own converters as an independent
library on many random and constructed-tie inputs."""
import numpy as np
import pytest
import torch

import oracle


@pytest.fixture(scope="module", autouse=True)
def built():
    oracle.build()


@pytest.mark.parametrize("x,code", [
    (1.0, 0x3F80), (-2.0, 0xC000), (0.0, 0x0000), (-0.0, 0x8000),
    (1.0 + 2.0 ** -8, 0x3F80),                  # tie between 1 and 1 + 2^-7: even mantissa
    (1.0 + 3 * 2.0 ** -8, 0x3F82),              # tie between 1 + 2^-7 (odd) and 1 + 2^-6 (even)
    (1.0 + 2.0 ** -8 + 2.0 ** -20, 0x3F81),     # just above the tie
    (3.0e38, 0x7F62), (np.finfo(np.float32).max, 0x7F80),   # rounds up to +inf
    (2.0 ** -149, 0x0000), (2.0 ** -126, 0x0080),
])
def test_bf16_definition_values(x, code):
    assert oracle.bf16_encode(x) == code


def test_bf16_matches_torch_on_random_and_ties():
    rng = np.random.default_rng(0)
    bits = rng.integers(0, 2 ** 32, size=200000, dtype=np.uint64).astype(np.uint32)
    bits[:50000] = (bits[:50000] & 0xFFFF0000) | 0x8000          # exact ties
    bits[50000:60000] = (bits[50000:60000] & 0xFFFF0000) | 0x7FFF
    x = bits.view(np.float32)
    x = x[np.isfinite(x)]
    ours = oracle.quantize_bf16(x.reshape(-1, 1)).ravel()
    ref = torch.from_numpy(x).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    assert np.array_equal(ours, ref)


@pytest.mark.parametrize("x,code", [
    (448.0, 0x7E), (1000.0, 0x7E), (-448.0, 0xFE), (464.0, 0x7E),   # saturation (480 is not a value)
    (1.0, 0x38), (0.5, 0x30), (-1.5, 0xBC),
    (2.0 ** -6, 0x08),                          # smallest normal
    (2.0 ** -9, 0x01),                          # smallest subnormal
    (2.0 ** -10, 0x00),                         # tie between 0 and 2^-9: even code 0
    (3 * 2.0 ** -10, 0x02),                     # tie between codes 1 and 2: even
    (1.0625, 0x38), (1.1875, 0x3A),             # ties between 1, 1.125 and 1.125, 1.25
    (0.0, 0x00), (-0.0, 0x80),
])
def test_e4m3_definition_values(x, code):
    assert oracle.e4m3_encode(x) == code


def test_e4m3_round_trip_every_code():
    for c in range(256):
        v = oracle.e4m3_decode(c)
        if np.isnan(v):
            assert c & 0x7F == 0x7F
            continue
        assert oracle.e4m3_encode(v) == c or (v == 0.0 and c in (0x00, 0x80))
    finite = sorted({oracle.e4m3_decode(c) for c in range(0x7F)})
    assert finite[-1] == 448.0 and len(finite) == 127


def test_e4m3_matches_torch_in_range():
    rng = np.random.default_rng(1)
    x = np.concatenate([rng.uniform(-448, 448, 20000), rng.normal(0, 1e-2, 20000),
                        rng.normal(0, 3, 20000)]).astype(np.float32)
    # exact ties: midpoints of consecutive finite values
    vals = np.array(sorted({oracle.e4m3_decode(c) for c in range(0x7F)}))
    mids = ((vals[:-1] + vals[1:]) / 2).astype(np.float32)
    x = np.concatenate([x, mids, -mids])
    ours = np.array([oracle.e4m3_encode(v) for v in x], dtype=np.uint8)
    ref = torch.from_numpy(x).to(torch.float8_e4m3fn).view(torch.uint8).numpy()
    assert np.array_equal(ours, ref)


def test_e4m3_matrix_scales_and_error_bound():
    rng = np.random.default_rng(2)
    A = (rng.normal(0, 1, (300, 7)) * np.array([1e-3, 1, 50, 1e4, 1, 0, 3])).astype(np.float32)
    A[5, 4] = 0.0
    codes, sc = oracle.quantize_e4m3(A)
    amax = np.abs(A).max(axis=0)
    want = np.where(amax > 0, (amax / np.float32(448)).astype(np.float32), np.float32(1))
    assert np.array_equal(sc, want)
    assert np.all(codes[:, 5] & 0x7F == 0)             # all-zero column: scale 1, codes +-0
    deq = oracle.dequantize_e4m3(codes, sc)
    q = A.astype(np.float64) / sc.astype(np.float64)
    # nearest-value rounding: half a spacing (2^-4 relative for normals, 2^-10 absolute below 2^-6)
    bound = np.maximum(np.abs(q) * 2.0 ** -4, 2.0 ** -10) * sc + 1e-30
    assert np.all(np.abs(deq - A) <= bound * (1 + 1e-6))
    assert np.all(np.abs(deq).max(axis=0) <= 448.0 * sc * (1 + 1e-7))


def test_bf16_matrix_dequantizes_within_half_ulp():
    rng = np.random.default_rng(3)
    A = rng.normal(0, 1, (100, 50)).astype(np.float32)
    deq = oracle.dequantize_bf16(oracle.quantize_bf16(A))
    assert np.all(np.abs(deq - A) <= np.abs(A) * 2.0 ** -8)
