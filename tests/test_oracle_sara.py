"""Pins of the oracle's SARA dictionary (Section 2.2, Section 5.1)."""
import math

import numpy as np
import pytest

from oracle import sara


def test_db1_is_haar_and_db2_closed_form():
    assert np.allclose(sara.daubechies(1), [1 / math.sqrt(2)] * 2, rtol=0, atol=1e-16)
    s3 = math.sqrt(3.0)
    expect = np.array([1 + s3, 3 + s3, 3 - s3, 1 - s3]) / (4 * math.sqrt(2.0))
    assert np.abs(sara.daubechies(2) - expect).max() <= 1e-15


@pytest.mark.parametrize("p", range(1, 9))
def test_daubechies_filter_identities(p):
    h = sara.daubechies(p)
    g = sara.highpass(h)
    assert h.shape == (2 * p,)
    assert abs(h.sum() - math.sqrt(2)) <= 1e-14
    assert abs((h * h).sum() - 1.0) <= 1e-14
    for m in range(1, p):
        assert abs(np.dot(h[: 2 * p - 2 * m], h[2 * m:])) <= 1e-14
    k = np.arange(2 * p, dtype=np.float64)
    for mom in range(p):       # p vanishing moments of the wavelet
        scale = np.sum(np.abs(g) * k ** mom)
        assert abs(np.sum(g * k ** mom)) <= 1e-12 * scale
    # first moment of the low-pass is nonzero (not a wavelet)
    assert abs(h.sum()) > 1.0


def test_haar_one_level_layout_by_hand():
    a, b, c, d = 1.0, 2.0, 5.0, 11.0
    out = sara.dwt2(np.array([[a, b], [c, d]]), sara.daubechies(1), levels=1)
    expect = np.array([[(a + b + c + d) / 2, (a - b + c - d) / 2],
                       [(a + b - c - d) / 2, (a - b - c + d) / 2]])
    assert np.abs(out - expect).max() <= 1e-14


@pytest.mark.parametrize("p,L", [(8, 16), (8, 4), (3, 6), (5, 32)])
def test_1d_analysis_matrix_is_orthogonal(p, L):
    h = sara.daubechies(p)
    W = np.stack([sara.analysis_1d(e, h, 0) for e in np.eye(L)], axis=1)
    assert np.abs(W @ W.T - np.eye(L)).max() <= 1e-14
    # synthesis is the transpose
    S = np.stack([sara.synthesis_1d(e, h, 0) for e in np.eye(L)], axis=1)
    assert np.abs(S - W.T).max() <= 1e-15


def test_perfect_reconstruction_and_isometry():
    rng = np.random.default_rng(2)
    x = rng.normal(size=(32, 48))
    for h in sara.filters():
        c = sara.dwt2(x, h, 4)
        assert abs(np.linalg.norm(c) - np.linalg.norm(x)) <= 1e-13 * np.linalg.norm(x)
        assert np.abs(sara.idwt2(c, h, 4) - x).max() <= 1e-13
    u = sara.psi_adjoint(x)
    assert u.shape == (9, 32, 48)
    assert np.abs(sara.psi(u) - x).max() <= 1e-13


def test_psi_is_adjoint_of_psi_dagger():
    rng = np.random.default_rng(4)
    x = rng.normal(size=(32, 32))
    u = rng.normal(size=(9, 32, 32))
    lhs = float(np.sum(sara.psi_adjoint(x) * u))
    rhs = float(np.sum(x * sara.psi(u)))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_psi_spectral_norm_is_one():
    rng = np.random.default_rng(6)
    x = rng.normal(size=(16, 16))
    for _ in range(30):
        y = sara.psi(sara.psi_adjoint(x))
        lam = np.linalg.norm(y) / np.linalg.norm(x)
        x = y / np.linalg.norm(y)
    assert abs(lam - 1.0) <= 1e-12


def test_dirac_basis_is_the_scaled_image():
    x = np.arange(256, dtype=np.float64).reshape(16, 16)
    assert np.allclose(sara.psi_adjoint(x)[0], x / 3.0, rtol=1e-15, atol=0)
