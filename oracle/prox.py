"""Proximity operators of PPD (FP64, plain).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Section 3.3: projection onto the positive orthant (Eq. "proj-plus"),
soft-thresholding (Eq. "prox-L1"), projection onto the l2 ball
(Eq. "proj-L2").  Section 4.1: the generalised proximity operator in the
metric U (Eq. "generalised-proximity-operator"), its ellipsoid form
(Eqs. "elip-proj-1", "elip-proj-2") and the forward-backward iteration that
computes it (Algorithm 2, step mu <= 1/||U||_S^2 with ||U||_S = max_e U_e).
"""
from __future__ import annotations

import numpy as np


def proj_positive(z):
    """(P_C z)_e = Re(z_e) if Re(z_e) > 0 else 0."""
    r = np.real(z)
    return np.where(r > 0.0, r, 0.0)


def soft(z, alpha: float):
    """(S_alpha z)_e = z_e {|z_e| - alpha}_+ / |z_e|, and 0 where z_e = 0."""
    z = np.asarray(z)
    mag = np.abs(z)
    safe = np.where(mag > 0.0, mag, 1.0)
    return np.where(mag > 0.0, z * np.maximum(mag - alpha, 0.0) / safe, 0.0)


def clip_complement(z, alpha: float):
    """(I - S_alpha) z; for real z this is min(max(z, -alpha), alpha)."""
    return z - soft(z, alpha)


def proj_l2ball(z, y, eps: float):
    """P_B(z): y + eps (z - y)/||z - y|| if ||z - y|| > eps, else z."""
    r = z - y
    n = float(np.sqrt(np.sum(np.abs(r) ** 2)))
    if n > eps:
        return y + (eps / n) * r
    return np.array(z, copy=True)


def _inner_converged(cur, prev, tol: float) -> bool:
    """Algorithm 2's stopping test (the paper says only "until convergence";
    reading): ||zbar^t - zbar^(t-1)||_2 <= tol ||zbar^t||_2, in FP64."""
    return float(np.linalg.norm(cur - prev)) <= tol * float(np.linalg.norm(cur))


def ellipsoid_prox_fb(z, y, eps: float, U, n_itr: int, start=None, mu=None, tol: float = 0.0,
                      info: dict | None = None):
    """Algorithm 2: zbar <- P_B(zbar - mu U (zbar - z)), at most n_itr times.

    Computes prox^U_h(z) = argmin_{||p - y|| <= eps} (z-p)^H U (z-p) / 2.
    start is zbar^(0) (defaults to z); mu defaults to 1/max(U)^2.  tol > 0
    stops after the first step t with ||zbar^t - zbar^(t-1)|| <= tol
    ||zbar^t||; tol = 0 runs all n_itr steps.  info, if given, receives
    info["steps"] = the number of steps taken.
    """
    U = np.asarray(U, dtype=np.float64)
    mu = 1.0 / float(np.max(U)) ** 2 if mu is None else mu
    zb = np.array(z if start is None else start, dtype=np.complex128, copy=True)
    steps = 0
    for _ in range(n_itr):
        nxt = proj_l2ball(zb - mu * U * (zb - z), y, eps)
        steps += 1
        done = tol > 0.0 and _inner_converged(nxt, zb, tol)
        zb = nxt
        if done:
            break
    if info is not None:
        info["steps"] = steps
    return zb


def ellipsoid_prox_fista(z, y, eps: float, U, n_itr: int, start=None, mu=None, tol: float = 0.0,
                         info: dict | None = None):
    """Accelerated Algorithm 2 (Section 4.1 points to faster proximal gradient
    methods, Tseng 2008): the same projected gradient step on
    (zbar - z)^H U (zbar - z) / 2 taken at an extrapolated point,
        zbar_k = P_B(q_k - mu U (q_k - z)),
        t_{k+1} = (1 + sqrt(1 + 4 t_k^2)) / 2,  t_1 = 1,
        q_{k+1} = zbar_k + ((t_k - 1) / t_{k+1}) (zbar_k - zbar_{k-1}),
    with q_1 = zbar_0 = start (FISTA, Beck & Teboulle 2009).  The first two
    steps coincide with Algorithm 2 (t_1 = 1 gives no extrapolation).  tol
    and info as in ellipsoid_prox_fb (the test compares zbar_k with zbar_{k-1}).
    """
    U = np.asarray(U, dtype=np.float64)
    mu = 1.0 / float(np.max(U)) ** 2 if mu is None else mu
    prev = np.array(z if start is None else start, dtype=np.complex128, copy=True)
    q = prev.copy()
    t = 1.0
    steps = 0
    for _ in range(n_itr):
        cur = proj_l2ball(q - mu * U * (q - z), y, eps)
        steps += 1
        done = tol > 0.0 and _inner_converged(cur, prev, tol)
        t_next = 0.5 * (1.0 + np.sqrt(1.0 + 4.0 * t * t))
        q = cur + ((t - 1.0) / t_next) * (cur - prev)
        prev, t = cur, t_next
        if done:
            break
    if info is not None:
        info["steps"] = steps
    return prev


def ellipsoid_prox_exact(z, y, eps: float, U, tol: float = 1e-15):
    """Exact prox^U_h(z) through its optimality conditions (used to pin Algorithm 2).

    If ||z - y|| <= eps the answer is z.  Otherwise p = (U z + lam y)/(U + lam)
    with lam > 0 the root of sum_e U_e^2 |z_e - y_e|^2 / (U_e + lam)^2 = eps^2,
    found by bisection in FP64.  Returns (p, lam).
    """
    U = np.asarray(U, dtype=np.float64)
    r2 = np.abs(z - y) ** 2
    if np.sqrt(r2.sum()) <= eps:
        return np.array(z, dtype=np.complex128, copy=True), 0.0

    def g(lam):
        return float(np.sum(U * U * r2 / (U + lam) ** 2)) - eps * eps

    lo, hi = 0.0, 1.0
    while g(hi) > 0.0:
        hi *= 2.0
    for _ in range(2000):
        mid = 0.5 * (lo + hi)
        if g(mid) > 0.0:
            lo = mid
        else:
            hi = mid
        if hi - lo <= tol * max(hi, 1e-300):
            break
    lam = 0.5 * (lo + hi)
    return (U * z + lam * y) / (U + lam), lam
