"""Preconditioned primal-dual iteration (Algorithm 3) in plain FP64.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Paper passages: Algorithm 3 (Section 4) with lambda = 1 and no randomised
active sets (Section 5.1); the dual data step through the generalised Moreau
identity (Eq. "generalised-proximity-operator-decomposition") and the
ellipsoid prox (Section 4.1, Algorithm 2); the prior step (I - S_k) with
threshold kappa ||Psi W||_S^2 (Section 4.2); parameters tau = 0.49,
zeta = 1/||Psi||_S^2, eta = 1/||U^{1/2} Phi||_S^2, kappa = 1e-4 (Section 5.1);
eps^2 two standard deviations above the chi^2 mean (Section 5.1);
the convergence condition (Eq. "convergence-req-explicit-pd").

Readings (the paper is silent or its printed step is garbled):

* Dual step (Algorithm 3, data update): with z = U^{-1} v + Theta G a the
  update is vbar = U (z - p), p = prox^U_h(z) computed by Algorithm 2; this
  is the generalised Moreau identity with alpha = 1 after the rescaling
  v <- v/eta that puts eta in the primal step.
* Algorithm 2 starts from the previous iteration's p (warm start) and, on
  the first iteration, from P_B(z); optionally from z itself every
  iteration ("current").  n_itr fixed (default 1).  Optionally its
  accelerated (FISTA) form, which Section 4.1 points to (Tseng 2008).
* mu_j = 1/max_e(U_j,e)^2 (Algorithm 2, as printed).
* Per-block bound eps_j^2 = M_j + 2 sqrt(M_j) in whitened units (the
  chi^2 rule applied per block; y whitened as Theta y).
* Initial state x = xt = 0, u = 0, v = 0.
* Power iteration for ||U^{1/2} Phi||_S^2 on Phi^dagger U Phi from the
  all-ones vector, stopped at relative change < 1e-10 or 1000 steps.
* Algorithm 2's "until convergence": optionally stop at the first step t
  with ||zbar^t - zbar^(t-1)||_2 <= inner_tol ||zbar^t||_2 (FP64, per
  block), capped at n_itr steps; inner_tol = 0 keeps the fixed n_itr.
* Algorithm 3's "until convergence": optionally stop once the relative
  variation ||x^t - x^(t-1)|| / ||x^t|| is below a tolerance and every block
  residual is within 1.005 eps_j (``converged`` / ``run_until``).

Prior weights W (Algorithm 1) enter the prior step as printed in Algorithm
3; ``oracle/reweight.py`` sets them.

Randomised active sets (Algorithm 3, "generate sets P and D"; Section 4.4:
nonzero probabilities, independent and identical draws along the
iterations): the draws are inputs (``paper_1701_01748_gb300.synth.active_sets``
makes seeded Bernoulli masks).  A data block j outside D keeps v_j (so its
gridded contribution is unchanged) and its Algorithm 2 warm start p_j; a
basis i outside P keeps u_i (so Psi_i u_i is unchanged).  Reading (the paper
is silent): a block that has never been active starts Algorithm 2 from
P_B(z), as every block does on the first iteration.

Parity: the invariants of the whole iteration (feasibility, positivity,
PPD and PD reaching the same minimiser, U = I reducing to PD) are pinned by
tests; the trajectory itself is "parity unpinned" beyond them.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

from . import nufft, prox, sara


def eps_chi2(block: np.ndarray, n_blocks: int) -> np.ndarray:
    """eps_j = sqrt(M_j + 2 sqrt(M_j)) (whitened noise: ||n_j||^2 ~ chi^2 with mean M_j, std sqrt(M_j))."""
    Mj = np.bincount(np.asarray(block, np.int64), minlength=n_blocks).astype(np.float64)
    return np.sqrt(Mj + 2.0 * np.sqrt(Mj))


def op_norm_sq(P: nufft.Plan, U: np.ndarray, max_iter: int = 1000, tol: float = 1e-10,
               start: np.ndarray | None = None):
    """||U^{1/2} Phi||_S^2 by power iteration on Phi^dagger U Phi. Returns (value, iterations)."""
    x = np.ones((P.L0, P.L1)) if start is None else np.array(start, dtype=np.float64)
    x /= np.linalg.norm(x)
    val = 0.0
    for it in range(1, max_iter + 1):
        y = nufft.phi_adjoint(U * nufft.phi(x, P), P)
        new = float(np.linalg.norm(y))
        x = y / new
        if abs(new - val) <= tol * new:
            return new, it
        val = new
    return val, max_iter


def op_norm_sq_lanczos(P: nufft.Plan, U: np.ndarray, tol: float = 1e-8, ncv: int = 12):
    """||U^{1/2} Phi||_S^2 as the largest eigenvalue of Phi^dagger U Phi by
    implicitly restarted Lanczos (ARPACK through scipy's eigsh) from the
    all-ones vector.  The same quantity as op_norm_sq; used where the
    power iteration converges too slowly for a CPU run (strongly
    non-uniform coverages, where the two largest eigenvalues are close).
    Returns (value, operator applications)."""
    from scipy.sparse.linalg import LinearOperator, eigsh
    n = P.L0 * P.L1
    count = [0]

    def matvec(v):
        count[0] += 1
        return nufft.phi_adjoint(U * nufft.phi(np.reshape(v, (P.L0, P.L1)), P), P).ravel()

    A = LinearOperator((n, n), matvec=matvec, dtype=np.float64)
    w = eigsh(A, k=1, which="LA", tol=tol, v0=np.ones(n), ncv=min(ncv, n - 1),
              return_eigenvectors=False)
    return float(w[0]), count[0]


@dataclasses.dataclass
class Setup:
    P: nufft.Plan
    yw: np.ndarray          # whitened data Theta y
    U: np.ndarray           # preconditioner diagonal
    block: np.ndarray
    n_blocks: int
    eps: np.ndarray         # per block
    mu: np.ndarray          # per block
    eta: float
    zeta: float = 1.0
    tau: float = 0.49
    kappa: float = 1e-4
    n_itr: int = 1
    levels: int = 4
    x_true: np.ndarray | None = None
    inner_init: str = "warm"    # Algorithm 2 start: "warm" (previous p) or "current" (z)
    inner_solver: str = "fb"     # "fb": Algorithm 2; "fista": its accelerated form (Section 4.1)
    W: np.ndarray | None = None  # prior weights (9, L0, L1) of Algorithm 1; None = identity
    psiw_sq: float = 1.0         # ||Psi W||_S^2 (1 for W = I)
    inner_tol: float = 0.0       # Algorithm 2 stop: ||zbar^t - zbar^(t-1)|| <= inner_tol ||zbar^t|| (0: n_itr steps)

    def __post_init__(self):
        self.members = [np.flatnonzero(self.block == j) for j in range(self.n_blocks)]
        self.hs = sara.filters()


def make_setup(omega, y, theta, block, n_blocks, L, *, precond: bool = True,
               eta: float | None = None, eps=None, U=None, n_itr: int = 1,
               tau: float = 0.49, kappa: float = 1e-4, x_true=None,
               power_iters: int = 1000, inner_init: str = "warm", inner_solver: str = "fb",
               inner_tol: float = 0.0, L1: int | None = None) -> Setup:
    """The solver's inputs and parameters for an L x L1 image (L1 = L by default)."""
    P = nufft.Plan(omega, L, L if L1 is None else L1, theta=theta)
    if U is None:
        U = nufft.uniform_weights(omega, P.K0, P.K1)[0] if precond else np.ones(P.M)
    U = np.asarray(U, dtype=np.float64)
    block = np.asarray(block, np.int64)
    eps = eps_chi2(block, n_blocks) if eps is None else np.asarray(eps, np.float64)
    mu = np.ones(n_blocks)
    for j in range(n_blocks):
        sel = block == j
        if np.any(sel):
            mu[j] = 1.0 / float(np.max(U[sel])) ** 2
    if eta is None:
        eta = 1.0 / op_norm_sq(P, U, max_iter=power_iters)[0]
    return Setup(P=P, yw=np.asarray(theta) * np.asarray(y), U=U, block=block,
                 n_blocks=n_blocks, eps=eps, mu=mu, eta=float(eta), tau=tau, kappa=kappa,
                 n_itr=n_itr, x_true=x_true, inner_init=inner_init, inner_solver=inner_solver,
                 inner_tol=float(inner_tol))


def convergence_lhs(S: Setup, psi_norm_sq: float | None = None, phi_norm_sq: float | None = None):
    """tau zeta_eff ||Psi W||^2 + tau eta ||U^{1/2} Phi||^2 (must be < 1)."""
    if phi_norm_sq is None:
        phi_norm_sq = 1.0 / S.eta
    if psi_norm_sq is None:
        psi_norm_sq = S.psiw_sq
    return S.tau * (S.zeta / S.psiw_sq) * psi_norm_sq + S.tau * S.eta * phi_norm_sq


@dataclasses.dataclass
class State:
    x: np.ndarray
    xt: np.ndarray
    u: np.ndarray
    v: np.ndarray
    p: np.ndarray            # Algorithm 2 output of each block's last active iteration
    seen: np.ndarray         # per block: has been active (p_j holds a prox output)
    t: int = 0


def init_state(S: Setup) -> State:
    L0, L1 = S.P.L0, S.P.L1
    return State(x=np.zeros((L0, L1)), xt=np.zeros((L0, L1)),
                 u=np.zeros((sara.N_BASES, L0, L1)), v=np.zeros(S.P.M, np.complex128),
                 p=np.zeros(S.P.M, np.complex128), seen=np.zeros(S.n_blocks, dtype=bool))


def iterate(st: State, S: Setup, active_blocks=None, active_bases=None) -> dict:
    """One iteration of Algorithm 3 (lambda = 1).

    active_blocks (d booleans, the set D) and active_bases (9 booleans, the
    set P, Dirac first) select the dual variables updated this iteration;
    None means all (no randomisation, Section 5.1).
    """
    P = S.P
    act_d = np.ones(S.n_blocks, bool) if active_blocks is None else np.asarray(active_blocks, bool)
    act_p = np.ones(sara.N_BASES, bool) if active_bases is None else np.asarray(active_bases, bool)
    # forward: a = F Z xt, Theta G a
    phix = P.theta * nufft.interpolate(np.fft.fft2(nufft.zero_pad_scale(st.xt, P)), P)
    res = np.array([np.linalg.norm(phix[m] - S.yw[m]) for m in S.members])
    # dual data step (Algorithm 2 inside the Moreau identity) for the blocks in D;
    # the others keep v_j and p_j
    z = st.v / S.U + phix
    v = st.v.copy()
    p = st.p.copy()
    inner_steps = np.zeros(S.n_blocks, np.int64)
    for j, m in enumerate(S.members):
        if m.size == 0 or not act_d[j]:
            continue
        if S.inner_init == "current":
            start = z[m]
        elif not st.seen[j]:
            start = prox.proj_l2ball(z[m], S.yw[m], S.eps[j])
        else:
            start = st.p[m]
        solve = prox.ellipsoid_prox_fista if S.inner_solver == "fista" else prox.ellipsoid_prox_fb
        info = {}
        p[m] = solve(z[m], S.yw[m], S.eps[j], S.U[m], S.n_itr, start=start, mu=S.mu[j], tol=S.inner_tol,
                     info=info)
        inner_steps[j] = info["steps"]
        v[m] = S.U[m] * (z[m] - p[m])
    g = nufft.phi_adjoint(v, P)
    # prior step for the bases in P: clip (I - S_{kappa ||Psi W||^2}) of
    # u + W Psi^dagger xt; the others keep u_i; then the synthesis of W u;
    # zeta = 1/||Psi W||^2 (W = I: ||Psi|| = 1)
    c = sara.psi_adjoint(st.xt, S.levels, S.hs)
    if S.W is not None:
        c = S.W * c
    u = prox.clip_complement(st.u + c, S.kappa * S.psiw_sq)
    if not act_p.all():
        u = np.where(act_p[:, None, None], u, st.u)
    ut = sara.psi(u if S.W is None else S.W * u, S.levels, S.hs)
    zeta = S.zeta / S.psiw_sq
    # primal step
    xbar = prox.proj_positive(st.x - S.tau * (S.eta * g + zeta * ut))
    dx = float(np.linalg.norm(xbar - st.x))
    nx = float(np.linalg.norm(xbar))
    xt = 2.0 * xbar - st.x
    st.x, st.xt, st.u, st.v, st.p = xbar, xt, u, v, p
    st.seen = st.seen | act_d
    st.t += 1
    stats = dict(residual=res, rel_var=dx / nx if nx > 0 else float("inf"), inner_steps=inner_steps)
    if S.x_true is not None:
        stats["snr"] = snr(S.x_true, xbar)
    return stats


def run(S: Setup, n_iters: int, st: State | None = None):
    """n_iters iterations of Algorithm 3 from st (warm start) or from zero."""
    st = init_state(S) if st is None else st
    hist = []
    for _ in range(n_iters):
        hist.append(iterate(st, S))
    return st, hist


def converged(S: Setup, stats: dict, rel_var_tol: float, eps_factor: float = 1.005) -> bool:
    """Global stopping rule of Algorithm 3 ("until convergence"; reading, the
    paper gives no test): the relative variation of x is below rel_var_tol and
    every block residual ||Phi_j xt - y_j|| of the iteration's data step is
    within eps_factor eps_j."""
    return stats["rel_var"] < rel_var_tol and bool(np.all(stats["residual"] <= eps_factor * S.eps))


def run_until(S: Setup, max_iters: int, rel_var_tol: float, eps_factor: float = 1.005,
              check_every: int = 1, st: State | None = None):
    """Algorithm 3 until the global stopping rule holds (tested after every
    check_every-th iteration) or max_iters iterations.  Returns (state,
    history, stopped)."""
    st = init_state(S) if st is None else st
    hist = []
    for t in range(1, max_iters + 1):
        hist.append(iterate(st, S))
        if t % check_every == 0 and converged(S, hist[-1], rel_var_tol, eps_factor):
            return st, hist, True
    return st, hist, False


def snr(x_true: np.ndarray, x: np.ndarray) -> float:
    """SNR = 20 log10(||x_true|| / ||x_true - x||) (Section 5)."""
    den = float(np.linalg.norm(x_true - x))
    return 20.0 * math.log10(float(np.linalg.norm(x_true)) / den) if den > 0 else float("inf")


def l1_objective(x: np.ndarray, levels: int = 4) -> float:
    """||Psi^dagger x||_1, the objective of the minimisation problem."""
    return float(np.sum(np.abs(sara.psi_adjoint(x, levels))))
