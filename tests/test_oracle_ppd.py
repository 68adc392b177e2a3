"""Pins of the oracle's PPD iteration (Algorithm 3) and its parameters.

The trajectory itself has no closed form; what the paper fixes is pinned:
the chi^2 noise bound, the operator norm behind eta, the Moreau-identity
reading of the dual step, the U = I reduction to PD, the convergence
condition, and that PPD and PD reach the same feasible, positive minimiser.
"""
import math

import numpy as np
import pytest
from scipy import optimize

from oracle import nufft, ppd, prox
from paper_1701_01748_gb300 import synth


def test_chi2_bound_matches_noise_statistics():
    rng = np.random.default_rng(0)
    Mj, trials = 400, 4000
    n = (rng.normal(size=(trials, Mj)) + 1j * rng.normal(size=(trials, Mj))) / math.sqrt(2.0)
    s = np.sum(np.abs(n) ** 2, axis=1)
    assert abs(s.mean() - Mj) < 4 * math.sqrt(Mj / trials) * 1.0 + 0.5
    assert abs(s.std() - math.sqrt(Mj)) < 0.05 * math.sqrt(Mj)
    eps = ppd.eps_chi2(np.zeros(Mj, np.int64), 1)[0]
    assert abs(eps ** 2 - (s.mean() + 2 * s.std())) < 0.1 * math.sqrt(Mj) + 0.05 * Mj ** 0.5 * 2


def test_power_iteration_matches_dense_spectral_norm():
    rng = np.random.default_rng(1)
    L, M = 16, 80
    om = rng.uniform(-np.pi, np.pi, size=(M, 2))
    P = nufft.Plan(om, L, theta=rng.uniform(0.5, 2, size=M))
    U = rng.uniform(0.1, 1.0, size=M)
    cols = []
    for i in range(L * L):
        e = np.zeros(L * L)
        e[i] = 1.0
        y = np.sqrt(U) * nufft.phi(e.reshape(L, L), P)
        cols.append(np.concatenate([y.real, y.imag]))
    A = np.stack(cols, axis=1)
    dense = np.linalg.norm(A, 2) ** 2
    got, it = ppd.op_norm_sq(P, U, max_iter=5000, tol=1e-13)
    assert abs(got - dense) <= 1e-8 * dense
    lz, _ = ppd.op_norm_sq_lanczos(P, U, tol=1e-12)
    assert abs(lz - dense) <= 1e-9 * dense


def test_dual_step_is_the_conjugate_prox_in_metric_U_inverse():
    """vbar = U(z - prox^U_h(z)), z = U^{-1} w, equals prox^{U^{-1}}_{h*}(w) (generalised Moreau)."""
    rng = np.random.default_rng(2)
    m = 5
    y = rng.normal(size=m) + 1j * rng.normal(size=m)
    w = 4.0 * (rng.normal(size=m) + 1j * rng.normal(size=m))
    U = rng.uniform(0.2, 1.0, size=m)
    eps = 0.7
    z = w / U
    p, _ = prox.ellipsoid_prox_exact(z, y, eps, U)
    vbar = U * (z - p)

    def obj(q):   # h*(v) = Re<y, v> + eps ||v||  (support function of the ball)
        v = q[:m] + 1j * q[m:]
        return (float(np.vdot(y, v).real) + eps * float(np.linalg.norm(v))
                + 0.5 * float(np.sum(np.abs(w - v) ** 2 / U)))
    q0 = np.concatenate([vbar.real, vbar.imag]) + 0.3
    res = optimize.minimize(obj, q0, method="Nelder-Mead",
                            options=dict(xatol=1e-12, fatol=1e-14, maxiter=200000, maxfev=200000))
    res = optimize.minimize(obj, res.x, method="BFGS", options=dict(gtol=1e-12))
    got = res.x[:m] + 1j * res.x[m:]
    assert np.abs(got - vbar).max() <= 1e-5 * np.abs(vbar).max()


def _tiny(seed=5, M=600, n_blocks=2):
    return synth.make_problem("tiny", L=16, M=M, n_blocks=n_blocks, uv_sigma=0.2, seed=seed,
                              n_points=4, n_blobs=1)


def test_identity_metric_is_pd():
    """With U = I every PPD dual step is z - P_B(z) (Onose 2016 PD)."""
    p = _tiny(seed=6, M=200)
    S = ppd.make_setup(p.omega, p.y, p.theta, p.block, p.n_blocks, p.L, precond=False,
                       power_iters=200)
    st = ppd.init_state(S)
    x_ref = np.zeros((16, 16))
    xt_ref = np.zeros((16, 16))
    u_ref = np.zeros((9, 16, 16))
    v_ref = np.zeros(S.P.M, np.complex128)
    from oracle import sara
    for _ in range(5):
        ppd.iterate(st, S)
        z = v_ref + nufft.phi(xt_ref, S.P)
        vb = np.empty_like(z)
        for j, m in enumerate(S.members):
            vb[m] = z[m] - prox.proj_l2ball(z[m], S.yw[m], S.eps[j])
        v_ref = vb
        u_ref = prox.clip_complement(u_ref + sara.psi_adjoint(xt_ref), S.kappa)
        xb = prox.proj_positive(x_ref - S.tau * (S.eta * nufft.phi_adjoint(v_ref, S.P) + sara.psi(u_ref)))
        xt_ref, x_ref = 2 * xb - x_ref, xb
    assert np.abs(st.x - x_ref).max() <= 1e-12 * max(np.abs(x_ref).max(), 1e-30)
    assert np.abs(st.v - v_ref).max() <= 1e-12 * np.abs(v_ref).max()


def test_convergence_condition_holds():
    p = _tiny(seed=7, M=200)
    S = ppd.make_setup(p.omega, p.y, p.theta, p.block, p.n_blocks, p.L, power_iters=300)
    lhs = ppd.convergence_lhs(S)
    assert lhs < 1.0 and abs(lhs - 0.98) < 1e-9


def test_ppd_and_pd_reach_the_same_feasible_minimiser():
    p = _tiny()
    xs, objs = [], []
    for precond in (True, False):
        S = ppd.make_setup(p.omega, p.y, p.theta, p.block, p.n_blocks, p.L, precond=precond,
                           x_true=p.x_true, power_iters=300)
        st, hist = ppd.run(S, 1500)
        assert st.x.min() >= 0.0
        assert np.all(hist[-1]["residual"] <= 1.01 * S.eps)
        xs.append(st.x)
        objs.append(ppd.l1_objective(st.x))
    assert np.linalg.norm(xs[0] - xs[1]) <= 1e-2 * np.linalg.norm(xs[0])
    assert abs(objs[0] - objs[1]) <= 2e-3 * objs[0]


def test_more_subiterations_approach_the_exact_prox():
    """Algorithm 2 with many sub-iterations equals the exact ellipsoid prox inside one PPD step."""
    p = _tiny(seed=8, M=150, n_blocks=1)
    S = ppd.make_setup(p.omega, p.y, p.theta, p.block, 1, p.L, power_iters=200, n_itr=20000)
    st = ppd.init_state(S)
    ppd.iterate(st, S)
    z = np.zeros(S.P.M, np.complex128)   # at t=1 xt = 0 and v = 0, so z = 0
    p_exact, _ = prox.ellipsoid_prox_exact(z, S.yw, S.eps[0], S.U)
    assert np.abs(st.p - p_exact).max() <= 1e-8 * np.abs(p_exact).max()


def test_accelerated_inner_solver_in_the_iteration():
    """With one or two sub-iterations the accelerated inner solver is Algorithm 2;
    with many, both give the exact prox, so the iterates agree."""
    p = _tiny(seed=9, M=300, n_blocks=2)
    runs = {}
    for solver in ("fb", "fista"):
        for n_itr in (2, 400):
            S = ppd.make_setup(p.omega, p.y, p.theta, p.block, p.n_blocks, p.L, power_iters=200,
                               n_itr=n_itr, inner_solver=solver)
            st, _ = ppd.run(S, 4)
            runs[(solver, n_itr)] = st.x
    assert np.array_equal(runs[("fb", 2)], runs[("fista", 2)])
    assert np.abs(runs[("fb", 400)] - runs[("fista", 400)]).max() <= 1e-8 * np.abs(runs[("fb", 400)]).max()


def test_inner_stopping_test_in_the_iteration():
    """Algorithm 2 stopped by its test inside PPD: per-block step counts lie in
    [1, n_itr]; with a tight test and a high cap each block's prox is the exact
    one (so the iterates equal those of a run to convergence), and a looser test
    takes fewer steps."""
    p = _tiny(seed=10, M=300, n_blocks=3)
    kw = dict(power_iters=200, n_itr=20000)
    S_exact = ppd.make_setup(p.omega, p.y, p.theta, p.block, p.n_blocks, p.L, **kw)
    S_tol = ppd.make_setup(p.omega, p.y, p.theta, p.block, p.n_blocks, p.L, inner_tol=1e-11, **kw)
    S_loose = ppd.make_setup(p.omega, p.y, p.theta, p.block, p.n_blocks, p.L, inner_tol=1e-3, **kw)
    st_e, st_t, st_l = ppd.init_state(S_exact), ppd.init_state(S_tol), ppd.init_state(S_loose)
    for _ in range(3):
        he = ppd.iterate(st_e, S_exact)
        ht = ppd.iterate(st_t, S_tol)
        hl = ppd.iterate(st_l, S_loose)
        assert np.all(he["inner_steps"] == 20000)
        assert np.all((ht["inner_steps"] >= 1) & (ht["inner_steps"] < 20000))
        assert np.all(hl["inner_steps"] <= ht["inner_steps"])
    assert np.abs(st_t.x - st_e.x).max() <= 1e-7 * np.abs(st_e.x).max()


def test_global_stopping_rule_stops_near_the_minimiser():
    """Algorithm 3 stopped by the rule (relative variation below tol, every block
    residual within 1.005 eps_j): the rule holds where it stopped, a looser
    tolerance stops no later, and the stopped image is close to the minimiser of
    a long run."""
    p = _tiny()
    S = ppd.make_setup(p.omega, p.y, p.theta, p.block, p.n_blocks, p.L, x_true=p.x_true, power_iters=300)
    x_min, _ = ppd.run(S, 1500)
    stops = []
    for tol in (1e-2, 1e-3, 1e-4):
        st, hist, stopped = ppd.run_until(S, 1500, tol)
        assert stopped
        assert hist[-1]["rel_var"] < tol and np.all(hist[-1]["residual"] <= 1.005 * S.eps)
        stops.append(len(hist))
    assert stops == sorted(stops) and stops[0] < stops[-1]
    assert np.linalg.norm(st.x - x_min.x) <= 5e-2 * np.linalg.norm(x_min.x)
    # checked every 5th iteration only: stops at a multiple of 5, no earlier than every-iteration checks
    _, hist5, stopped5 = ppd.run_until(S, 1500, 1e-3, check_every=5)
    assert stopped5 and len(hist5) % 5 == 0 and len(hist5) >= stops[1]
