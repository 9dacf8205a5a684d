"""FP64 CPU oracle for the tall-skinny SVD / PCA methods (arXiv:1906.12085).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by ``__graft_entry__.smoke()``
and by the CPU-baseline leg of ``bench.py``; never by the library.  The C
source (``oracle.c``) is plain float64 loops written from the paper's
definitions and step lists; this module only marshals numpy arrays into it.

Functions and the passages they follow:

* ``center``        -- Sec. 1 zero-mean assumption, Eq. (sumeigen) for ||A||_F^2
* ``svd``           -- Sec. 2.1 definition A = U Sigma V^T (Golub-Reinsch)
* ``eig_jacobi``    -- eigen-decomposition used by the Gram route
* ``svd_gram``      -- Sec. 2.3 / Sec. 3.1.3 "Truncated SVD" (A^T A, eig, sqrt, A v / sigma)
* ``rsvd``          -- Sec. 3.1.2 randomized PCA with a given Gaussian test matrix
* ``block_krylov``  -- Sec. 3.1.1 block Krylov method with a given Gaussian test matrix
* ``gkl``           -- Golub-Kahan-Lanczos with full reorthogonalisation
* ``pca_threshold`` -- Sec. 2.4 cumulative explained-variance criterion
* ``qr``            -- Householder QR (orthonormalisation inside ``rsvd``)
* ``quantize_bf16``, ``quantize_e4m3`` and the encoders / decoders -- the
  storage formats of the precision form (bfloat16 round-to-nearest-even; OCP
  e4m3 with per-column scales amax/448, round-to-nearest-even, saturating)

Parity status: every function is pinned by ``tests/test_oracle_*.py`` against
closed forms, prescribed spectra, invariants, brute force on 4x3 integer
inputs and an independent library (numpy.linalg).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_SRC = os.path.join(_HERE, "oracle.c")

OK, ERR_ARG, ERR_OOM, ERR_NOCONV, ERR_BREAKDOWN, WARN_K_GT_COUNT = 0, -1, -2, -4, -7, 1


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so with gcc (float64, no FMA contraction)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
               "-o", _SO + ".tmp", _SRC, "-lm"]
        subprocess.check_call(cmd, cwd=_HERE)
        os.replace(_SO + ".tmp", _SO)
    return _SO


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_SO)
        P = ctypes.POINTER(ctypes.c_double)
        i64 = ctypes.c_int64
        L.orc_center.argtypes = [i64, i64, P, P, P]
        L.orc_qr.argtypes = [i64, i64, P, P, P]
        L.orc_svd.argtypes = [i64, i64, P, P, P, P]
        L.orc_eig_jacobi.argtypes = [i64, P, P, P, ctypes.POINTER(ctypes.c_int)]
        L.orc_svd_gram.argtypes = [i64, i64, P, P, P, P]
        L.orc_rsvd.argtypes = [i64, i64, P, i64, ctypes.c_int, P, i64, P, P, P]
        L.orc_gkl.argtypes = [i64, i64, P, P, ctypes.c_int, i64, P, P, P, P, P]
        L.orc_block_krylov.argtypes = [i64, i64, P, i64, ctypes.c_int, P, i64, P, P, P]
        L.orc_pca_threshold.argtypes = [i64, P, ctypes.c_double, ctypes.c_double, ctypes.POINTER(i64)]
        L.orc_sign_normalize.argtypes = [i64, i64, i64, P, P]
        L.orc_bf16_encode.argtypes = [ctypes.c_float]
        L.orc_bf16_encode.restype = ctypes.c_uint16
        L.orc_bf16_decode.argtypes = [ctypes.c_uint16]
        L.orc_bf16_decode.restype = ctypes.c_double
        L.orc_e4m3_encode.argtypes = [ctypes.c_float]
        L.orc_e4m3_encode.restype = ctypes.c_uint8
        L.orc_e4m3_decode.argtypes = [ctypes.c_uint8]
        L.orc_e4m3_decode.restype = ctypes.c_double
        L.orc_quantize_bf16.argtypes = [i64, i64, ctypes.c_void_p, i64, ctypes.c_void_p]
        L.orc_quantize_e4m3.argtypes = [i64, i64, ctypes.c_void_p, i64, ctypes.c_void_p, ctypes.c_void_p]
        for f in ("orc_center", "orc_qr", "orc_svd", "orc_eig_jacobi", "orc_svd_gram", "orc_rsvd",
                  "orc_gkl", "orc_pca_threshold", "orc_block_krylov"):
            getattr(L, f).restype = ctypes.c_int
        L.orc_sign_normalize.restype = None
        _lib = L
    return _lib


def _f64(x) -> np.ndarray:
    if hasattr(x, "detach"):
        x = x.detach().cpu().numpy()
    return np.ascontiguousarray(np.asarray(x, dtype=np.float64))


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


class OracleError(RuntimeError):
    pass


def _check(st: int, name: str, allow=(OK,)):
    if st not in allow:
        raise OracleError(f"{name} returned status {st}")
    return st


def center(A):
    """Returns (centred copy of A, column means mu, ||A_centred||_F^2)."""
    a = _f64(A).copy()
    m, n = a.shape
    mu = np.zeros(n)
    f = ctypes.c_double(0.0)
    _check(lib().orc_center(m, n, _p(a), _p(mu), ctypes.byref(f)), "orc_center")
    return a, mu, f.value


def qr(Y):
    y = _f64(Y)
    m, n = y.shape
    q = np.zeros((m, n))
    r = np.zeros((n, n))
    _check(lib().orc_qr(m, n, _p(y), _p(q), _p(r)), "orc_qr")
    return q, r


def svd(A, vectors: bool = True):
    a = _f64(A)
    m, n = a.shape
    s = np.zeros(n)
    u = np.zeros((m, n)) if vectors else None
    v = np.zeros((n, n)) if vectors else None
    _check(lib().orc_svd(m, n, _p(a), _p(s), _p(u) if vectors else None, _p(v) if vectors else None), "orc_svd")
    return (s, u, v) if vectors else s


def eig_jacobi(G):
    g = _f64(G)
    n = g.shape[0]
    lam = np.zeros(n)
    v = np.zeros((n, n))
    sw = ctypes.c_int(0)
    _check(lib().orc_eig_jacobi(n, _p(g), _p(lam), _p(v), ctypes.byref(sw)), "orc_eig_jacobi")
    return lam, v, sw.value


def svd_gram(A):
    a = _f64(A)
    m, n = a.shape
    s = np.zeros(n)
    u = np.zeros((m, n))
    v = np.zeros((n, n))
    _check(lib().orc_svd_gram(m, n, _p(a), _p(s), _p(u), _p(v)), "orc_svd_gram")
    return s, u, v


def rsvd(A, Omega, q: int, k: int):
    a = _f64(A)
    om = _f64(Omega)
    m, n = a.shape
    l = om.shape[1]
    s = np.zeros(k)
    u = np.zeros((m, k))
    v = np.zeros((n, k))
    _check(lib().orc_rsvd(m, n, _p(a), l, int(q), _p(om), k, _p(s), _p(u), _p(v)), "orc_rsvd")
    return s, u, v


def block_krylov(A, Omega, iters: int, k: int):
    """Sec. 3.1.1 block Krylov method with the given Omega (n x l): (S, U, V) of the
    leading k triplets from the basis of [H(0) | ... | H(iters)]."""
    a = _f64(A)
    om = _f64(Omega)
    m, n = a.shape
    l = om.shape[1]
    s = np.zeros(k)
    u = np.zeros((m, k))
    v = np.zeros((n, k))
    _check(lib().orc_block_krylov(m, n, _p(a), l, int(iters), _p(om), k, _p(s), _p(u), _p(v)),
           "orc_block_krylov")
    return s, u, v


def gkl(A, v1, steps: int, k: int):
    a = _f64(A)
    x = _f64(v1).reshape(-1)
    m, n = a.shape
    s = np.zeros(k)
    u = np.zeros((m, k))
    v = np.zeros((n, k))
    al = np.zeros(steps)
    be = np.zeros(steps)
    _check(lib().orc_gkl(m, n, _p(a), _p(x), int(steps), k, _p(s), _p(u), _p(v), _p(al), _p(be)), "orc_gkl")
    return s, u, v, al, be


def pca_threshold(sigma, fro2: float, t: float):
    """Returns (K, reached): minimal K with sum_{i<=K} sigma_i^2 >= t * fro2."""
    s = _f64(sigma).reshape(-1)
    K = ctypes.c_int64(0)
    st = _check(lib().orc_pca_threshold(s.size, _p(s), float(fro2), float(t), ctypes.byref(K)),
                "orc_pca_threshold", allow=(OK, WARN_K_GT_COUNT))
    return int(K.value), st == OK


def sign_normalize(U, V):
    u = _f64(U).copy()
    v = _f64(V).copy()
    lib().orc_sign_normalize(u.shape[0], v.shape[0], v.shape[1], _p(u), _p(v))
    return u, v


# ------------------------------------------------------------ storage formats
def bf16_encode(x: float) -> int:
    return int(lib().orc_bf16_encode(float(np.float32(x))))


def bf16_decode(b: int) -> float:
    return float(lib().orc_bf16_decode(int(b)))


def e4m3_encode(x: float) -> int:
    return int(lib().orc_e4m3_encode(float(np.float32(x))))


def e4m3_decode(c: int) -> float:
    return float(lib().orc_e4m3_decode(int(c)))


def _f32(x) -> np.ndarray:
    if hasattr(x, "detach"):
        x = x.detach().cpu().numpy()
    return np.ascontiguousarray(np.asarray(x, dtype=np.float32))


def quantize_bf16(A) -> np.ndarray:
    """bfloat16 codes (uint16, m x n) of the float32 matrix A."""
    a = _f32(A)
    m, n = a.shape
    out = np.empty((m, n), dtype=np.uint16)
    lib().orc_quantize_bf16(m, n, a.ctypes.data, n, out.ctypes.data)
    return out


def quantize_e4m3(A):
    """(e4m3 codes uint8 m x n, float32 column scales n) of the float32 matrix A."""
    a = _f32(A)
    m, n = a.shape
    out = np.empty((m, n), dtype=np.uint8)
    sc = np.empty(n, dtype=np.float32)
    lib().orc_quantize_e4m3(m, n, a.ctypes.data, n, out.ctypes.data, sc.ctypes.data)
    return out, sc


_BF16_LUT = None
_E4M3_LUT = None


def dequantize_bf16(codes) -> np.ndarray:
    """float64 values of bfloat16 codes (exact)."""
    global _BF16_LUT
    if _BF16_LUT is None:
        _BF16_LUT = np.array([bf16_decode(i) for i in range(65536)], dtype=np.float64)
    return _BF16_LUT[np.asarray(codes, dtype=np.uint16)]


def dequantize_e4m3(codes, scales) -> np.ndarray:
    """float64 values code * scale (exact: 4 significant bits times a float32)."""
    global _E4M3_LUT
    if _E4M3_LUT is None:
        _E4M3_LUT = np.array([e4m3_decode(i) for i in range(256)], dtype=np.float64)
    return _E4M3_LUT[np.asarray(codes, dtype=np.uint8)] * np.asarray(scales, dtype=np.float64)[None, :]
