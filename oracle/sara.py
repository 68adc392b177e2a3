"""SARA dictionary Psi = [Dirac, db1, ..., db8] (FP64, plain).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Paper passages: the analysis prior ||Psi^dagger x||_1 with the SARA
dictionary (Section 2.2), split into b bases Psi_i (Section 3, Eq.
"split-min-problem"), and its content: a Dirac basis concatenated with the
first eight Daubechies wavelets (Section 5.1).  Readings where the paper is
silent: 4 decomposition levels, periodic boundaries, separable 2-D
transform (rows, then columns) with the Mallat quadrant layout per level,
and every basis scaled by 1/3 = 1/sqrt(9) so that Psi Psi^dagger = I and
||Psi||_S = 1 (hence zeta = 1 and the clip level kappa ||Psi||^2 = kappa).

Daubechies filters are obtained by the minimum-phase spectral factorisation
of Daubechies (1988): |m0|^2 = cos^{2p}(xi/2) P(sin^2(xi/2)) with
P(y) = sum_{k<p} C(p-1+k, k) y^k; the roots of P are mapped to z through
sin^2(xi/2) = (2 - z - 1/z)/4, the root inside the unit circle is kept,
and h is the coefficient list of (1+z)^p prod (z - z_r), scaled to sum sqrt(2).
"""
from __future__ import annotations

import math

import numpy as np

N_BASES = 9
SCALE = 1.0 / 3.0


def daubechies(p: int) -> np.ndarray:
    """Low-pass filter h of db_p (2p taps, sum sqrt(2), sum of squares 1)."""
    if p == 1:
        return np.array([1.0, 1.0]) / math.sqrt(2.0)
    coeffs = [math.comb(p - 1 + k, k) for k in range(p)]     # ascending powers
    yroots = np.roots(coeffs[::-1])
    poly = np.array([1.0 + 0j])
    for _ in range(p):
        poly = np.convolve(poly, [1.0, 1.0])
    for yr in yroots:
        a = 1.0 - 2.0 * yr
        disc = np.sqrt(a * a - 1.0 + 0j)
        z1, z2 = a + disc, a - disc
        zr = z1 if abs(z1) < abs(z2) else z2
        poly = np.convolve(poly, [1.0, -zr])
    h = np.real(poly)
    h = h * (math.sqrt(2.0) / h.sum())
    # orientation: largest early taps first (Daubechies' tables)
    if abs(h[0]) < abs(h[-1]):
        h = h[::-1]
    return h


def highpass(h: np.ndarray) -> np.ndarray:
    """g[k] = (-1)^k h[Lf-1-k]."""
    Lf = h.shape[0]
    return np.array([(-1.0) ** k * h[Lf - 1 - k] for k in range(Lf)])


def analysis_1d(x: np.ndarray, h: np.ndarray, axis: int) -> np.ndarray:
    """a[n] = sum_k h[k] x[(2n+k) mod L], d[n] = sum_k g[k] x[(2n+k) mod L]; output [a | d]."""
    x = np.moveaxis(x, axis, 0)
    L = x.shape[0]
    g = highpass(h)
    n = np.arange(L // 2)
    a = np.zeros((L // 2,) + x.shape[1:])
    d = np.zeros_like(a)
    for k in range(h.shape[0]):
        xs = x[np.mod(2 * n + k, L)]
        a += h[k] * xs
        d += g[k] * xs
    return np.moveaxis(np.concatenate([a, d], axis=0), 0, axis)


def synthesis_1d(c: np.ndarray, h: np.ndarray, axis: int) -> np.ndarray:
    """Adjoint (= inverse) of analysis_1d: x[(2n+k) mod L] += h[k] a[n] + g[k] d[n]."""
    c = np.moveaxis(c, axis, 0)
    L = c.shape[0]
    g = highpass(h)
    a, d = c[: L // 2], c[L // 2:]
    n = np.arange(L // 2)
    x = np.zeros_like(c)
    for k in range(h.shape[0]):
        # for a fixed tap k the targets (2n+k) mod L are distinct
        x[np.mod(2 * n + k, L)] += h[k] * a + g[k] * d
    return np.moveaxis(x, 0, axis)


def dwt2(x: np.ndarray, h: np.ndarray, levels: int = 4) -> np.ndarray:
    """Multi-level periodic 2-D DWT, Mallat layout (rows then columns per level)."""
    c = np.array(x, dtype=np.float64, copy=True)
    n0, n1 = c.shape
    for _ in range(levels):
        blk = c[:n0, :n1]
        blk = analysis_1d(blk, h, axis=1)
        blk = analysis_1d(blk, h, axis=0)
        c[:n0, :n1] = blk
        n0 //= 2
        n1 //= 2
    return c


def idwt2(c: np.ndarray, h: np.ndarray, levels: int = 4) -> np.ndarray:
    """Inverse of dwt2 (columns then rows per level, coarsest level first)."""
    x = np.array(c, dtype=np.float64, copy=True)
    L0, L1 = x.shape
    for lev in range(levels - 1, -1, -1):
        n0, n1 = L0 >> lev, L1 >> lev
        blk = x[:n0, :n1]
        blk = synthesis_1d(blk, h, axis=0)
        blk = synthesis_1d(blk, h, axis=1)
        x[:n0, :n1] = blk
    return x


def filters():
    """The eight Daubechies low-pass filters db1..db8."""
    return [daubechies(p) for p in range(1, 9)]


def psi_adjoint(x: np.ndarray, levels: int = 4, hs=None) -> np.ndarray:
    """Psi^dagger x = (1/3) [x; W_db1 x; ...; W_db8 x], shape (9, L0, L1)."""
    hs = filters() if hs is None else hs
    out = np.empty((N_BASES,) + x.shape)
    out[0] = SCALE * x
    for i, h in enumerate(hs):
        out[i + 1] = SCALE * dwt2(x, h, levels)
    return out


def psi(u: np.ndarray, levels: int = 4, hs=None) -> np.ndarray:
    """Psi u = (1/3) (u_0 + sum_i W_dbi^T u_i)."""
    hs = filters() if hs is None else hs
    x = np.array(u[0], dtype=np.float64, copy=True)
    for i, h in enumerate(hs):
        x += idwt2(u[i + 1], h, levels)
    return SCALE * x
