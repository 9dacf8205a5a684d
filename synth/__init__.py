"""Seeded synthetic inputs shared by the tests, the oracle checks and the benchmark.

This module only draws random numbers and assembles test matrices with a
prescribed spectrum.  It contains none of the arithmetic of the SVD / PCA
methods themselves: neither the CPU oracle nor the CUDA library imports it,
and it imports neither of them.

Construction (the workloads of the tall-skinny PCA setting, Sec. 2 and Sec. 4
of arXiv:1906.12085):

* ``haar(rows, cols, seed, center)``: a Haar-distributed matrix with
  orthonormal columns, obtained from the QR factorisation of a seeded
  Gaussian matrix with the signs fixed so that diag(R) > 0 (Mezzadri 2007).
  With ``center=True`` every Gaussian column is first projected onto the
  complement of the all-ones vector, so the orthonormal columns are
  orthogonal to 1 and the assembled matrix already has zero column means
  while keeping its prescribed singular values exactly.
* ``prescribed(m, n, sigma, seed_u, seed_v)``: A = U diag(sigma) V^T.
* spectra used by the five workloads (index base i = 1..n).

Generation runs in float64 with torch on the requested device (CPU for the
small cases, CUDA for the multi-GB ones); results are deterministic for a
given (seed, device).  ``prescribed(..., dtype=torch.float32)`` draws and
factors in float32 (orthonormal to ~1e-6): a timing input of the largest
workloads, whose float64 QR would take minutes of float64 arithmetic.
"""
from __future__ import annotations

import torch

__all__ = [
    "gaussian",
    "haar",
    "prescribed",
    "spectrum_pow2",
    "spectrum_harmonic_noise",
    "spectrum_exp",
    "spectrum_power",
    "workload",
    "WORKLOADS",
]


def _gen(seed: int, device) -> torch.Generator:
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    return g


def gaussian(rows: int, cols: int, seed: int, device="cpu", dtype=torch.float64) -> torch.Tensor:
    """Seeded N(0,1) matrix, rows x cols, row-major."""
    g = _gen(seed, device)
    return torch.randn(rows, cols, generator=g, device=device, dtype=dtype)


def unit_vector(n: int, seed: int, device="cpu", dtype=torch.float64) -> torch.Tensor:
    """Seeded Gaussian vector scaled to unit 2-norm (start vector of a Krylov run)."""
    v = gaussian(n, 1, seed, device, torch.float64)[:, 0]
    v = v / torch.linalg.vector_norm(v)
    return v.to(dtype)


def haar(rows: int, cols: int, seed: int, center: bool = False, device="cpu",
         dtype=torch.float64) -> torch.Tensor:
    """rows x cols matrix with orthonormal columns, Haar distributed (float64 unless dtype says)."""
    assert rows >= cols
    g = gaussian(rows, cols, seed, device, dtype)
    if center:
        g = g - g.mean(dim=0, keepdim=True)
    q, r = torch.linalg.qr(g, mode="reduced")
    s = torch.sign(torch.diagonal(r))
    s[s == 0] = 1.0
    return q * s.unsqueeze(0)


def prescribed(m: int, n: int, sigma: torch.Tensor, seed_u: int, seed_v: int,
               center: bool = True, device="cpu", dtype=torch.float64) -> torch.Tensor:
    """A = U diag(sigma) V^T with Haar U (m x r, orthogonal to 1 if center) and V (n x r)."""
    sigma = sigma.to(device=device, dtype=dtype)
    r = sigma.numel()
    u = haar(m, r, seed_u, center=center, device=device, dtype=dtype)
    v = haar(n, r, seed_v, center=False, device=device, dtype=dtype)
    return (u * sigma.unsqueeze(0)) @ v.T


def spectrum_pow2(n: int) -> torch.Tensor:
    """sigma_i = 2^(-i/10), i = 1..n (exact-SVD workload)."""
    i = torch.arange(1, n + 1, dtype=torch.float64)
    return torch.pow(2.0, -i / 10.0)


def spectrum_harmonic_noise(n: int, seed: int, noise: float = 1e-3) -> torch.Tensor:
    """sigma_i = |1/i + noise * xi_i|, xi ~ N(0,1) seeded, sorted descending."""
    i = torch.arange(1, n + 1, dtype=torch.float64)
    xi = gaussian(n, 1, seed)[:, 0]
    s = torch.abs(1.0 / i + noise * xi)
    return torch.sort(s, descending=True).values


def spectrum_exp(n: int, scale: float = 200.0) -> torch.Tensor:
    """sigma_i = exp(-i/scale), i = 1..n (Lanczos workload)."""
    i = torch.arange(1, n + 1, dtype=torch.float64)
    return torch.exp(-i / scale)


def spectrum_power(n: int, alpha: float) -> torch.Tensor:
    """sigma_i = i^(-alpha), i = 1..n."""
    i = torch.arange(1, n + 1, dtype=torch.float64)
    return torch.pow(i, -float(alpha))


# The five workloads of the tall-skinny PCA setting: name -> parameters.
WORKLOADS = {
    "exact_fp64_2000x100": dict(m=2000, n=100, spectrum="pow2", t=0.95, seeds=(19061, 19062)),
    "rpca_fp32_200000x1000": dict(m=200000, n=1000, k=50, p=10, q=2, t=0.9, spectrum="harmonic_noise",
                                  seeds=(12085, 12086, 12087, 12088)),
    "gkl_fp32_1048576x2048": dict(m=1048576, n=2048, k=100, steps=150, spectrum="exp",
                                  seeds=(20481, 20482, 20483)),
    "mixed_rsvd_1048576x4096": dict(m=1048576, n=4096, k=256, p=32, q=3, spectrum="power1.5",
                                    seeds=(40961, 40962, 40963, 40964)),
}


def workload(name: str, m: int | None = None, n: int | None = None, device="cpu", dtype=torch.float64):
    """Build (A, sigma, extras) for a named workload, optionally at a reduced size (A in
    float64 unless dtype says otherwise; see prescribed).

    The spectrum is always evaluated at the (possibly reduced) n; the
    recipe is otherwise the one of the named workload.
    """
    w = dict(WORKLOADS[name])
    m = m or w["m"]
    n = n or w["n"]
    seeds = w["seeds"]
    sp = w["spectrum"]
    if sp == "pow2":
        sigma = spectrum_pow2(n)
    elif sp == "harmonic_noise":
        sigma = spectrum_harmonic_noise(n, seeds[2])
    elif sp == "exp":
        sigma = spectrum_exp(n)
    elif sp == "power1.5":
        sigma = spectrum_power(n, 1.5)
    else:
        raise ValueError(sp)
    a = prescribed(m, n, sigma, seeds[0], seeds[1], center=True, device=device, dtype=dtype)
    extras = {}
    if "p" in w:
        l = w["k"] + w["p"]
        extras["omega"] = gaussian(n, l, seeds[3], device=device, dtype=torch.float32)
    if name.startswith("gkl"):
        extras["v1"] = unit_vector(n, seeds[2], device=device, dtype=torch.float32)
    return a, sigma, extras


def poisson_arrivals(count: int, rate: float, seed: int) -> list[float]:
    """Arrival times (seconds) of a Poisson stream: exponential inter-arrivals."""
    g = _gen(seed, "cpu")
    u = torch.rand(count, generator=g, dtype=torch.float64)
    gaps = -torch.log1p(-u) / rate
    return torch.cumsum(gaps, 0).tolist()
