"""Pins of the oracle's measurement operator against definitions it does not use.

Phi = Theta G F Z (Section 2) must reach the exact discrete measurement
equation within the Kaiser-Bessel interpolation error; the pins below use a
brute-force NUDFT, a direct DFT matrix, numerical quadrature of the kernel's
Fourier transform and brute-force loops for the binning.
"""
import math

import numpy as np
import pytest
from scipy import integrate

from oracle import nufft


def _rng(s=0):
    return np.random.default_rng(s)


def test_kb_transform_matches_quadrature():
    J, beta = 8, nufft.kb_beta(8)
    for f in (0.0, 0.05, 0.13, 0.25):
        num, _ = integrate.quad(lambda d: float(nufft.kb_kernel(d, J, beta)) * math.cos(2 * math.pi * f * d),
                                -J / 2, J / 2, epsabs=1e-14, epsrel=1e-13, limit=200)
        assert abs(float(nufft.kb_transform(f, J, beta)) - num) <= 1e-11 * abs(num)


def test_kb_kernel_support_and_peak():
    assert float(nufft.kb_kernel(0.0)) == 1.0
    assert float(nufft.kb_kernel(4.0001)) == 0.0
    assert float(nufft.kb_kernel(-4.0)) > 0.0
    # symmetric
    d = np.linspace(-4, 4, 33)
    assert np.allclose(nufft.kb_kernel(d), nufft.kb_kernel(-d), rtol=0, atol=0)


def test_numpy_fft2_is_the_unnormalised_forward_dft():
    rng = _rng(1)
    for K in (8, 16, 32):
        z = rng.normal(size=(K, K)) + 1j * rng.normal(size=(K, K))
        n = np.arange(K)
        F = np.exp(-2j * np.pi * np.outer(n, n) / K)
        assert np.abs(np.fft.fft2(z) - F @ z @ F.T).max() <= 1e-13 * np.abs(z).sum()


@pytest.mark.parametrize("L,M", [(16, 120), (32, 400), (16, 500)])
def test_phi_matches_brute_force_nudft(L, M):
    rng = _rng(L + M)
    om = rng.uniform(-np.pi, np.pi, size=(M, 2))
    om[:4] = [[-np.pi, -np.pi], [np.pi - 1e-12, 0.0], [0.0, 0.0], [1e-13, -1e-13]]
    x = rng.random((L, L))
    P = nufft.Plan(om, L)
    y = nufft.phi(x, P)
    ye = nufft.nudft(x, om)
    assert np.linalg.norm(y - ye) <= 1e-5 * np.linalg.norm(ye)


def test_phi_adjoint_matches_nudft_adjoint():
    rng = _rng(7)
    L, M = 16, 200
    om = rng.uniform(-np.pi, np.pi, size=(M, 2))
    v = rng.normal(size=M) + 1j * rng.normal(size=M)
    P = nufft.Plan(om, L)
    n = np.arange(L) - L / 2
    exact = np.zeros((L, L))
    for m in range(M):
        e = np.exp(1j * (om[m, 0] * n[:, None] + om[m, 1] * n[None, :]))
        exact += (e * v[m]).real
    got = nufft.phi_adjoint(v, P)
    assert np.linalg.norm(got - exact) <= 1e-5 * np.linalg.norm(exact)


@pytest.mark.parametrize("L", [16, 32])
def test_adjoint_identity(L):
    rng = _rng(3 * L)
    M = 300
    om = rng.uniform(-np.pi, np.pi, size=(M, 2))
    th = rng.uniform(0.5, 2.0, size=M)
    P = nufft.Plan(om, L, theta=th)
    x = rng.normal(size=(L, L))
    y = rng.normal(size=M) + 1j * rng.normal(size=M)
    lhs = float(np.vdot(nufft.phi(x, P), y).real)
    rhs = float(np.sum(x * nufft.phi_adjoint(y, P)))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_theta_is_a_diagonal_whitening():
    rng = _rng(11)
    L, M = 16, 64
    om = rng.uniform(-np.pi, np.pi, size=(M, 2))
    th = rng.uniform(0.5, 2.0, size=M)
    x = rng.random((L, L))
    a = nufft.phi(x, nufft.Plan(om, L, theta=th))
    b = nufft.phi(x, nufft.Plan(om, L))
    assert np.allclose(a, th * b, rtol=1e-14, atol=0)


def test_kappa_and_taps_brute_force():
    rng = _rng(5)
    K = 64
    om = rng.uniform(-np.pi, np.pi, size=50)
    kap = nufft.kappa(om, K)
    for w, k in zip(om, kap):
        assert k == (float(w) * float(K)) * 0.15915494309189535
    b0, b1, f0, f1 = nufft.base_cells(np.stack([om, om[::-1]], 1), K, K)
    for m in range(50):
        k = (float(om[m]) * K) * 0.15915494309189535
        assert b0[m] == (math.floor(k) - 3) % K
        assert f0[m] == k - math.floor(k)


def test_uniform_weights_brute_force():
    rng = _rng(9)
    K = 32
    om = rng.normal(0, 0.3, size=(400, 2)).clip(-np.pi, np.pi - 1e-9)
    U, cnt = nufft.uniform_weights(om, K, K)
    cells = []
    for w0, w1 in om:
        c0 = math.floor((float(w0) * K) * 0.15915494309189535 + 0.5) % K
        c1 = math.floor((float(w1) * K) * 0.15915494309189535 + 0.5) % K
        cells.append((c0, c1))
    for m, c in enumerate(cells):
        n = sum(1 for d in cells if d == c)
        assert cnt[m] == n and U[m] == 1.0 / n


def test_visibility_order_brute_force():
    rng = _rng(13)
    K, T = 64, 16
    om = rng.normal(0, 0.8, size=(300, 2)).clip(-np.pi, np.pi - 1e-9)
    blk = rng.integers(0, 3, size=300)
    perm, tile, cb0, cb1 = nufft.visibility_order(om, blk, K, K, T)
    keys = []
    for m in range(300):
        k0 = (float(om[m, 0]) * K) * 0.15915494309189535
        k1 = (float(om[m, 1]) * K) * 0.15915494309189535
        c0 = (math.floor(k0) - 3 + K // 2) % K
        c1 = (math.floor(k1) - 3 + K // 2) % K
        keys.append(((c0 // T) * (K // T) + c1 // T, int(blk[m]), c0, c1, m))
    expect = [k[-1] for k in sorted(keys)]
    assert list(perm) == expect
