"""Re-weighted l1 (Algorithm 1, Eq. "reweighting") in plain FP64.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Paper passages: the re-weighted l1 scheme of Section 3.2 (Algorithm 1):
the weights W_i are diagonal, with e-th entry omega / (omega + |Psi_i^dagger x|_e)
computed from the previous solution (Eq. "reweighting"); every PPD run is
warm-started from the previous primal and dual variables; inside Algorithm 3
the prior step becomes u_i <- (I - S_{kappa ||Psi W||_S^2})(u_i + W_i Psi_i^dagger xt)
and ut_i = Psi_i W_i u_i; the schedule omega^(k) = 0.25^k omega^(0),
omega^(0) = 1e-2, one re-weight every 1024 iterations (Section 5.1, real
data).

Readings (the paper is silent or inconsistent):

* Indexing: Algorithm 1 runs PPD (giving x^(k)), then lowers omega, then
  sets W^(k); Eq. "reweighting" writes x^(k-1).  Read as: after the k-th run,
  W = omega^(k) / (omega^(k) + |Psi^dagger x|) with x the solution of that run
  and omega^(k) = factor^k omega^(0).  With x^(0) = 0 the same formula gives
  W^(0) = I, the unweighted first run.
* Psi_i^dagger is the scaled analysis of the SARA oracle (each basis times
  1/3), so the weights see the coefficients the prior step clips.
* zeta = 1/||Psi W||_S^2 (the convergence condition with the weighted
  dictionary) and the clip level kappa ||Psi W||_S^2, both recomputed at
  every re-weight; ||Psi W||_S^2 by power iteration on Psi W^2 Psi^dagger
  from the all-ones image, stopped at relative change < 1e-10 or 1000 steps.
* The driver runs n_reweights + 1 PPD runs of `iters` iterations each, with
  a re-weight between consecutive runs.
"""
from __future__ import annotations

import numpy as np

from . import ppd, sara


def weights(x: np.ndarray, omega: float, levels: int = 4, hs=None) -> np.ndarray:
    """W_i diagonals (9, L, L): omega / (omega + |Psi_i^dagger x|) (Eq. "reweighting")."""
    c = sara.psi_adjoint(np.asarray(x, dtype=np.float64), levels, hs)
    return omega / (omega + np.abs(c))


def psiw_norm_sq(W: np.ndarray, levels: int = 4, max_iter: int = 1000, tol: float = 1e-10, hs=None):
    """||Psi W||_S^2 by power iteration on Psi W^2 Psi^dagger. Returns (value, iterations)."""
    L0, L1 = W.shape[1], W.shape[2]
    x = np.ones((L0, L1)) / np.sqrt(L0 * L1)
    W2 = W * W
    val = 0.0
    for it in range(1, max_iter + 1):
        y = sara.psi(W2 * sara.psi_adjoint(x, levels, hs), levels, hs)
        new = float(np.linalg.norm(y))
        x = y / new
        if abs(new - val) <= tol * new:
            return new, it
        val = new
    return val, max_iter


def set_weights(S: ppd.Setup, W, max_iter: int = 1000, tol: float = 1e-10) -> float:
    """Install W (None = identity) in the setup, with its ||Psi W||_S^2."""
    if W is None:
        S.W, S.psiw_sq = None, 1.0
    else:
        S.W = np.asarray(W, dtype=np.float64)
        S.psiw_sq = psiw_norm_sq(S.W, S.levels, max_iter, tol, S.hs)[0]
    return S.psiw_sq


def reweight(st: ppd.State, S: ppd.Setup, omega: float, max_iter: int = 1000, tol: float = 1e-10) -> float:
    """One re-weight of Algorithm 1 from the current primal iterate x."""
    return set_weights(S, weights(st.x, omega, S.levels, S.hs), max_iter, tol)


def run(S: ppd.Setup, n_reweights: int, iters: int, omega0: float = 1e-2, factor: float = 0.25,
        st: ppd.State | None = None, power_iters: int = 1000):
    """Algorithm 1: PPD runs of `iters` iterations, warm-started, re-weighting between them."""
    st = ppd.init_state(S) if st is None else st
    hist = []
    for k in range(n_reweights + 1):
        if k > 0:
            reweight(st, S, omega0 * factor ** k, max_iter=power_iters)
        st, h = ppd.run(S, iters, st)
        hist.extend(h)
    return st, hist


def weighted_l1(x: np.ndarray, W: np.ndarray, levels: int = 4) -> float:
    """||W Psi^dagger x||_1, the objective of the weighted problem."""
    return float(np.sum(np.abs(W * sara.psi_adjoint(x, levels))))
