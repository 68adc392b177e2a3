"""Measurement operator Phi = Theta G F Z and related set-up (FP64, plain).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Paper passages: the discrete measurement model y = Phi x + n with
Phi = Theta G F Z (Section 2, Eq. "inverse-problem"); n = 4 total
oversampling, 8x8 Kaiser-Bessel interpolation and uniform-weighting
preconditioner (Section 5, "Simulations and results").  The paper leaves the
interpolation details to Fessler & Sutton (2003); the readings used here are:

* frequencies omega in [-pi, pi)^2 (Section 5: normalised coverages), pixel
  origin at the image centre: the exact operator is
  y_m = sum_n x[n] exp(-i <omega_m, n - L/2>);
* oversampled grid K = 2L per axis (2 x 2 = n = 4);
* Kaiser-Bessel kernel psi(d) = I0(beta sqrt(1 - (2d/J)^2)) / I0(beta) for
  |d| <= J/2, J = 8, beta = 2.34 J, evaluated at the 8 grid points
  k_j = floor(kappa) - 3 + j (j = 0..7) around kappa = omega K / (2 pi);
* Z scales pixel n by 1 / psi_hat((n - L/2)/K), psi_hat the continuous
  Fourier transform of psi, and places it at grid index (n - L/2) mod K;
* F is the unnormalised forward DFT (exp(-2 pi i k n / K));
* Theta = diag(1/sigma_e) (natural weighting, Section 2).
"""
from __future__ import annotations

import math

import numpy as np

# The double nearest to 1/(2 pi); kappa = (omega * K) * INV_TWO_PI, evaluated
# left to right with two correctly rounded multiplies.
INV_TWO_PI = 0.15915494309189535
KB_J = 8


def kb_beta(J: int = KB_J) -> float:
    """Kaiser-Bessel shape for 2x oversampling (Fessler & Sutton choice)."""
    return 2.34 * J


def kb_kernel(d, J: int = KB_J, beta: float | None = None):
    """psi(d) = I0(beta sqrt(1-(2d/J)^2)) / I0(beta) on |d| <= J/2, else 0."""
    beta = kb_beta(J) if beta is None else beta
    d = np.asarray(d, dtype=np.float64)
    t = 1.0 - (2.0 * d / J) ** 2
    out = np.where(t >= 0.0, np.i0(beta * np.sqrt(np.maximum(t, 0.0))) / np.i0(beta), 0.0)
    return out


def kb_transform(f, J: int = KB_J, beta: float | None = None):
    """Continuous Fourier transform of psi at frequency f (cycles per grid cell).

    psi_hat(f) = (J / I0(beta)) sinh(s) / s, s = sqrt(beta^2 - (pi J f)^2);
    only the sinh branch is needed because |f| <= 1/4 and pi J / 4 < beta.
    """
    beta = kb_beta(J) if beta is None else beta
    f = np.asarray(f, dtype=np.float64)
    s = np.sqrt(beta * beta - (math.pi * J * f) ** 2)
    return (J / np.i0(beta)) * np.sinh(s) / s


def deapodisation(L: int, K: int, J: int = KB_J, beta: float | None = None):
    """Z's scaling s(n) = 1 / psi_hat((n - L/2) / K), n = 0..L-1."""
    n = np.arange(L, dtype=np.float64)
    return 1.0 / kb_transform((n - L / 2) / K, J, beta)


def nudft(x: np.ndarray, omega: np.ndarray) -> np.ndarray:
    """Exact operator: y_m = sum_n x[n0,n1] exp(-i(w0 (n0-L0/2) + w1 (n1-L1/2))).

    Direct O(M N) sum (the discretised measurement equation, Section 2);
    used only as ground truth on small inputs.
    """
    L0, L1 = x.shape
    n0 = np.arange(L0) - L0 / 2
    n1 = np.arange(L1) - L1 / 2
    y = np.empty(omega.shape[0], dtype=np.complex128)
    for m in range(omega.shape[0]):
        e0 = np.exp(-1j * omega[m, 0] * n0)
        e1 = np.exp(-1j * omega[m, 1] * n1)
        y[m] = e0 @ x @ e1
    return y


def kappa(omega_axis: np.ndarray, K: int) -> np.ndarray:
    """Grid coordinate kappa = (omega * K) * (1/(2 pi)) in FP64."""
    return (np.asarray(omega_axis, dtype=np.float64) * float(K)) * INV_TWO_PI


class Plan:
    """Interpolation taps of G for one coverage (8 taps per axis per visibility)."""

    def __init__(self, omega: np.ndarray, L0: int, L1: int | None = None,
                 theta: np.ndarray | None = None, J: int = KB_J,
                 beta: float | None = None):
        L1 = L0 if L1 is None else L1
        self.L0, self.L1 = int(L0), int(L1)
        self.K0, self.K1 = 2 * self.L0, 2 * self.L1
        self.J = J
        self.beta = kb_beta(J) if beta is None else beta
        self.omega = np.asarray(omega, dtype=np.float64)
        self.M = self.omega.shape[0]
        self.theta = np.ones(self.M) if theta is None else np.asarray(theta, np.float64)
        self.idx = []   # per axis (M, J) grid indices mod K
        self.w = []     # per axis (M, J) kernel weights
        for ax, K in ((0, self.K0), (1, self.K1)):
            kap = kappa(self.omega[:, ax], K)
            f = np.floor(kap)
            k = f[:, None] + (np.arange(J) - (J // 2 - 1))[None, :]
            self.w.append(kb_kernel(kap[:, None] - k, J, self.beta))
            self.idx.append(np.mod(k.astype(np.int64), K))
        self.s0 = deapodisation(self.L0, self.K0, J, self.beta)
        self.s1 = deapodisation(self.L1, self.K1, J, self.beta)
        self.rows = np.mod(np.arange(self.L0) - self.L0 // 2, self.K0)
        self.cols = np.mod(np.arange(self.L1) - self.L1 // 2, self.K1)


def zero_pad_scale(x: np.ndarray, P: Plan) -> np.ndarray:
    """Z: scale by s0(n0) s1(n1) and place at ((n - L/2) mod K) on the K0 x K1 grid."""
    z = np.zeros((P.K0, P.K1), dtype=np.complex128)
    z[np.ix_(P.rows, P.cols)] = P.s0[:, None] * P.s1[None, :] * x
    return z


def interpolate(grid: np.ndarray, P: Plan) -> np.ndarray:
    """G: y_m = sum_{a,b} w0[m,a] w1[m,b] grid[idx0[m,a], idx1[m,b]]."""
    y = np.zeros(P.M, dtype=np.complex128)
    for a in range(P.J):
        for b in range(P.J):
            y += P.w[0][:, a] * P.w[1][:, b] * grid[P.idx[0][:, a], P.idx[1][:, b]]
    return y


def interpolate_adjoint(v: np.ndarray, P: Plan) -> np.ndarray:
    """G^H: scatter-add w0 w1 v onto the grid (the weights are real).

    The 8 taps along axis 1 of one axis-0 tap go through one bincount (the
    scatter of all (m, b) pairs for that a), so the K0 x K1 histogram is
    built 2 J times rather than 2 J^2 times.
    """
    K0, K1 = P.K0, P.K1
    re = np.zeros(K0 * K1)
    im = np.zeros(K0 * K1)
    for a in range(P.J):
        c = (P.w[0][:, a] * v)[:, None] * P.w[1]                 # (M, J): w0[m,a] w1[m,b] v[m]
        lin = (P.idx[0][:, a] * K1)[:, None] + P.idx[1]          # (M, J) linear cells
        re += np.bincount(lin.ravel(), weights=c.real.ravel(), minlength=K0 * K1)
        im += np.bincount(lin.ravel(), weights=c.imag.ravel(), minlength=K0 * K1)
    return (re + 1j * im).reshape(K0, K1)


def phi(x: np.ndarray, P: Plan) -> np.ndarray:
    """Phi x = Theta G F Z x (Section 2)."""
    grid = np.fft.fft2(zero_pad_scale(x, P))
    return P.theta * interpolate(grid, P)


def phi_adjoint(y: np.ndarray, P: Plan) -> np.ndarray:
    """Phi^dagger y = Re(Z^T F^H G^H Theta y); F^H is the unnormalised inverse DFT."""
    grid = interpolate_adjoint(P.theta * y, P)
    img = np.fft.ifft2(grid) * (P.K0 * P.K1)
    crop = img[np.ix_(P.rows, P.cols)]
    return (P.s0[:, None] * P.s1[None, :] * crop).real


# --------------------------------------------------------------------------
# Binning, preconditioner and visibility ordering.
# --------------------------------------------------------------------------

def nearest_cells(omega: np.ndarray, K0: int, K1: int):
    """Nearest grid cell of each visibility: floor(kappa + 0.5) mod K per axis."""
    c0 = np.mod(np.floor(kappa(omega[:, 0], K0) + 0.5).astype(np.int64), K0)
    c1 = np.mod(np.floor(kappa(omega[:, 1], K1) + 0.5).astype(np.int64), K1)
    return c0, c1


def uniform_weights(omega: np.ndarray, K0: int, K1: int):
    """Preconditioner U_e = 1 / (number of visibilities in e's grid cell).

    Section 4.3: U holds the inverse of the sampling density in the vicinity
    of each visibility ("uniform weighting"); Section 5: the density is the
    visibility count per cell of the oversampled grid, over the whole
    coverage (all blocks).  Returns (U, counts_per_visibility).
    """
    c0, c1 = nearest_cells(omega, K0, K1)
    lin = c0 * K1 + c1
    counts = np.bincount(lin, minlength=K0 * K1)
    cnt = counts[lin]
    return 1.0 / cnt.astype(np.float64), cnt


def base_cells(omega: np.ndarray, K0: int, K1: int):
    """First interpolation tap (floor(kappa) - 3) mod K per axis, and frac = kappa - floor(kappa)."""
    out = []
    for ax, K in ((0, K0), (1, K1)):
        kap = kappa(omega[:, ax], K)
        f = np.floor(kap)
        out.append((np.mod(f.astype(np.int64) - 3, K), kap - f))
    return out[0][0], out[1][0], out[0][1], out[1][1]


def visibility_order(omega: np.ndarray, block: np.ndarray, K0: int, K1: int,
                     T: int):
    """Processing order of the visibilities in the CUDA library (bit-exact contract).

    The library stores its grid with the zero frequency at the centre: a
    plain grid index k lives at (k + K/2) mod K.  A visibility's tile is the
    T x T tile of that centred grid holding its first tap; the order is
    ascending (tile row-major, block, centred base row, centred base
    column, original index) — a stable sort.
    Returns (perm, tile_id, centred_base0, centred_base1).
    """
    b0, b1, _, _ = base_cells(omega, K0, K1)
    cb0 = np.mod(b0 + K0 // 2, K0)
    cb1 = np.mod(b1 + K1 // 2, K1)
    ntile1 = K1 // T
    tile = (cb0 // T) * ntile1 + (cb1 // T)
    idx = np.arange(omega.shape[0])
    perm = np.lexsort((idx, cb1, cb0, np.asarray(block, np.int64), tile))
    return perm, tile, cb0, cb1
