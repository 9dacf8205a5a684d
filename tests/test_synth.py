"""The seeded input generators (synth/): the properties every test and benchmark input
relies on, checked on CPU against their definitions."""
import math

import numpy as np
import pytest
import torch

import synth


@pytest.mark.parametrize("center", [False, True])
def test_haar_columns_are_orthonormal(center):
    Q = synth.haar(300, 40, seed=11, center=center).numpy()
    assert np.abs(Q.T @ Q - np.eye(40)).max() < 1e-13
    if center:   # orthogonal to the all-ones vector: zero column means
        assert np.abs(Q.sum(axis=0)).max() < 1e-12


def test_prescribed_matrix_has_the_prescribed_spectrum_and_zero_means():
    sig = synth.spectrum_power(30, 1.5)
    A = synth.prescribed(500, 30, sig, 3, 4).numpy()
    s = np.linalg.svd(A, compute_uv=False)          # an independent library
    assert np.abs(s - sig.numpy()).max() < 1e-13
    assert np.abs(A.mean(axis=0)).max() < 1e-15 * 500


def test_generators_are_deterministic_in_the_seed():
    a = synth.gaussian(64, 8, seed=7)
    assert torch.equal(a, synth.gaussian(64, 8, seed=7))
    assert not torch.equal(a, synth.gaussian(64, 8, seed=8))
    v = synth.unit_vector(100, seed=5)
    assert abs(float(torch.linalg.vector_norm(v)) - 1.0) < 1e-15


def test_spectra_follow_their_formulas():
    n = 50
    i = np.arange(1, n + 1, dtype=np.float64)
    assert np.allclose(synth.spectrum_pow2(n).numpy(), 2.0 ** (-i / 10.0), rtol=1e-15, atol=0)
    assert np.allclose(synth.spectrum_exp(n, 200.0).numpy(), np.exp(-i / 200.0), rtol=1e-15, atol=0)
    assert np.allclose(synth.spectrum_power(n, 1.5).numpy(), i ** -1.5, rtol=1e-15, atol=0)
    s = synth.spectrum_harmonic_noise(n, 12087).numpy()
    assert (s > 0).all() and (np.diff(s) <= 0).all()          # |1/i + 1e-3 xi|, sorted descending
    assert np.abs(np.sort(np.abs(1.0 / i + 1e-3 * synth.gaussian(n, 1, 12087)[:, 0].numpy()))[::-1] - s).max() == 0


def test_workload_shapes_and_test_matrix():
    A, sigma, extras = synth.workload("rpca_fp32_200000x1000", m=2000, n=100)
    assert A.shape == (2000, 100) and sigma.shape == (100,)
    om = extras["omega"]
    assert om.shape == (100, 60) and om.dtype == torch.float32
    A, sigma, extras = synth.workload("gkl_fp32_1048576x2048", m=3000, n=64)
    assert extras["v1"].shape == (64,)


def test_poisson_stream_rate():
    t = np.asarray(synth.poisson_arrivals(4096, 500.0, seed=7))
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert (gaps > 0).all()
    # mean inter-arrival 1 / rate; the sample mean of 4096 exponentials is within 5% (> 3 sigma)
    assert abs(gaps.mean() * 500.0 - 1.0) < 0.05
    # exponential: the coefficient of variation is 1
    assert abs(gaps.std() / gaps.mean() - 1.0) < 0.08
    assert math.isclose(t[-1], gaps.sum())
