"""Pins of the oracle's Sec. 3.1.1 block Krylov method (oracle.block_krylov).

Each check is fixed by mathematics, not by re-running the oracle's own steps:
  * with no iteration the method is the randomized range finder of Sec. 3.1.2
    with q = 0 (the separately pinned oracle.rsvd);
  * the Krylov basis span{A G, (A A^T) A G, ..., (A A^T)^i A G} contains the
    range of the power scheme (A A^T)^i A G, so its Rayleigh-Ritz singular
    values are at least those of the randomized method with q = i, and at most
    the true ones (interlacing);
  * when rank(A) <= l the first block already spans range(A) (exact result);
  * the Rayleigh-Ritz identity A^T u_i = sigma_i v_i holds for the returned
    triplets, and U, V have orthonormal columns;
  * the paper's chain printed without re-orthonormalisation spans the same space
    (numpy, small i where it is still well conditioned);
  * a prescribed spectrum is recovered with few iterations;
  * the block-by-block basis the library builds (each block A A^T applied to the
    previous orthonormalised block, projected against the earlier blocks, then
    orthonormalised) spans the same Krylov space, so its Ritz values agree with
    the step list's (float64 restatement, well-conditioned sizes)."""
import numpy as np
import pytest

import oracle
import synth


def _matrix(m, n, sig, seed):
    U0 = synth.haar(m, len(sig), seed=seed).numpy()
    V0 = synth.haar(n, len(sig), seed=seed + 1).numpy()
    return (U0 * sig) @ V0.T


def test_no_iteration_is_the_range_finder():
    rng = np.random.default_rng(21)
    A = rng.standard_normal((300, 50)) @ np.diag(np.linspace(4.0, 0.1, 50))
    Om = rng.standard_normal((50, 12))
    s, U, V = oracle.block_krylov(A, Om, iters=0, k=8)
    s0, U0, V0 = oracle.rsvd(A, Om, q=0, k=8)
    assert np.abs(s - s0).max() < 1e-12 * s0[0]
    assert np.abs(U - U0).max() < 1e-10 and np.abs(V - V0).max() < 1e-10


@pytest.mark.parametrize("iters", [1, 2, 3])
def test_dominates_power_scheme_and_interlaces(iters):
    n = 80
    sig = 1.0 / np.arange(1, n + 1)
    A = _matrix(600, n, sig, 31)
    rng = np.random.default_rng(22)
    Om = rng.standard_normal((n, 10))
    k = 8
    s, U, V = oracle.block_krylov(A, Om, iters=iters, k=k)
    s_pow, _, _ = oracle.rsvd(A, Om, q=iters, k=k)
    assert np.all(s >= s_pow - 1e-12 * sig[0])      # the Krylov space contains the power scheme's range
    assert np.all(s <= sig[:k] + 1e-12 * sig[0])     # Ritz values never exceed the singular values
    assert np.abs(U.T @ U - np.eye(k)).max() < 1e-12
    assert np.abs(V.T @ V - np.eye(k)).max() < 1e-12
    assert np.abs(A.T @ U - V * s).max() < 1e-12 * sig[0]


def test_exact_when_rank_at_most_l():
    m, n, r, l, k = 400, 60, 9, 12, 9
    sig = np.linspace(6.0, 1.0, r)
    A = _matrix(m, n, sig, 41)
    Om = np.random.default_rng(23).standard_normal((n, l))
    for iters in (0, 1, 2):
        s, U, V = oracle.block_krylov(A, Om, iters=iters, k=k)
        assert np.abs(s - sig).max() < 1e-12 * sig[0]
        assert np.abs(A @ V - U * s).max() < 1e-12 * sig[0]


def test_same_span_as_unorthonormalised_chain():
    """Sec. 3.1.1 as printed: H = [A G | A A^T A G] without intermediate
    orthonormalisation spans the same space (numpy QR of the concatenation)."""
    rng = np.random.default_rng(24)
    m, n, l, k = 300, 40, 6, 5
    A = rng.standard_normal((m, n)) @ np.diag(np.linspace(2.0, 0.5, n))
    Om = rng.standard_normal((n, l))
    H0 = A @ Om
    H = np.hstack([H0, A @ (A.T @ H0)])
    Qn, _ = np.linalg.qr(H)
    s_ref = np.linalg.svd(Qn.T @ A, compute_uv=False)[:k]
    s, U, V = oracle.block_krylov(A, Om, iters=1, k=k)
    assert np.abs(s - s_ref).max() < 1e-11 * s_ref[0]
    assert np.abs(U - Qn @ (Qn.T @ U)).max() < 1e-11


def test_recovers_prescribed_spectrum_with_few_iterations():
    n = 120
    sig = np.exp(-np.arange(n) / 10.0)
    A = _matrix(2000, n, sig, 51)
    Om = np.random.default_rng(25).standard_normal((n, 16))
    s3, _, _ = oracle.block_krylov(A, Om, iters=3, k=10)
    s0, _, _ = oracle.block_krylov(A, Om, iters=0, k=10)
    assert np.abs(s3 - sig[:10]).max() < 1e-10
    assert np.abs(s0 - sig[:10]).max() > 1e-6     # one block alone does not resolve the spectrum


def test_argument_checks():
    A = np.zeros((50, 20))
    with pytest.raises(oracle.OracleError):
        oracle.block_krylov(A, np.zeros((20, 8)), iters=2, k=4)   # (iters + 1) l = 24 > n
    with pytest.raises(oracle.OracleError):
        oracle.block_krylov(A, np.zeros((20, 4)), iters=1, k=9)   # k > (iters + 1) l


@pytest.mark.parametrize("iters,b", [(1, 6), (2, 8), (3, 5)])
def test_block_by_block_basis_spans_the_same_space(iters, b):
    """span{Q_0, ..., Q_j} = span{H(0), ..., H(j)} with Q_j the part of A A^T Q_{j-1}
    orthogonal to Q_0..Q_{j-1}: by induction, since A A^T maps the first j blocks'
    span into the first j + 1 blocks' span.  The Ritz values of the two bases agree."""
    rng = np.random.default_rng(40 + iters)
    m, n = 400, 60
    A = _matrix(m, n, 1.0 / np.arange(1, n + 1) ** 0.7, seed=31 + iters)
    Om = rng.standard_normal((n, b))
    k = (iters + 1) * b
    s_or, _, _ = oracle.block_krylov(A, Om, iters, k)
    Q = [np.linalg.qr(A @ Om)[0]]
    for _ in range(iters):
        H = np.concatenate(Q, axis=1)
        X = A @ (A.T @ Q[-1])
        for _ in range(2):                       # block classical Gram-Schmidt, twice
            X = X - H @ (H.T @ X)
        Q.append(np.linalg.qr(X)[0])
    H = np.concatenate(Q, axis=1)
    assert np.abs(H.T @ H - np.eye(k)).max() < 1e-12
    s_bb = np.linalg.svd(A.T @ H, compute_uv=False)
    assert np.abs(s_bb - s_or).max() < 1e-10 * s_or[0]
