"""Pins of the oracle's proximity operators (Section 3.3, Section 4.1, Algorithm 2)."""
import numpy as np
import pytest
from scipy import optimize

from oracle import prox


def test_positive_projection_by_hand():
    z = np.array([1.5 + 2j, -0.5 + 1j, 0.0, 3.0 - 7j])
    assert np.array_equal(prox.proj_positive(z), [1.5, 0.0, 0.0, 3.0])


def test_soft_threshold_by_hand():
    z = np.array([3.0, -0.5, 0.0, -2.0, 3 + 4j])
    out = prox.soft(z, 1.0)
    assert np.allclose(out, [2.0, 0.0, 0.0, -1.0, (3 + 4j) * 4 / 5], rtol=0, atol=1e-15)
    # (I - S_alpha) is the clip for real input
    r = np.array([3.0, -0.5, 0.0, -2.0, 0.99])
    assert np.array_equal(prox.clip_complement(r, 1.0), np.clip(r, -1.0, 1.0))


def test_l2_ball_projection_by_hand():
    y = np.array([1.0 + 0j, 0.0])
    z = np.array([4.0 + 0j, 4.0j])           # ||z - y|| = 5
    p = prox.proj_l2ball(z, y, 2.5)
    assert np.allclose(p, [1.0 + 1.5, 2.0j], rtol=0, atol=1e-15)
    inside = np.array([1.1 + 0j, 0.1j])
    assert np.array_equal(prox.proj_l2ball(inside, y, 2.5), inside)


def _block(seed, m=12, cond=4.0):
    rng = np.random.default_rng(seed)
    y = rng.normal(size=m) + 1j * rng.normal(size=m)
    z = y + 3.0 * (rng.normal(size=m) + 1j * rng.normal(size=m))
    U = rng.uniform(1.0 / cond, 1.0, size=m)
    return z, y, U


def test_exact_ellipsoid_prox_matches_generic_solver():
    z, y, U = _block(1, m=6)
    eps = 1.5
    p, lam = prox.ellipsoid_prox_exact(z, y, eps, U)
    # independent: SLSQP on the real-packed problem
    def obj(q):
        pc = q[:6] + 1j * q[6:]
        return 0.5 * float(np.sum(U * np.abs(z - pc) ** 2))
    cons = {"type": "ineq", "fun": lambda q: eps ** 2 - float(np.sum(np.abs(q[:6] + 1j * q[6:] - y) ** 2))}
    q0 = np.concatenate([y.real, y.imag])
    res = optimize.minimize(obj, q0, constraints=[cons], method="SLSQP",
                            options=dict(ftol=1e-15, maxiter=500))
    pq = res.x[:6] + 1j * res.x[6:]
    assert np.abs(pq - p).max() <= 1e-5


@pytest.mark.parametrize("seed", [2, 3, 4])
def test_exact_ellipsoid_prox_kkt(seed):
    z, y, U = _block(seed, m=20)
    eps = 2.0
    p, lam = prox.ellipsoid_prox_exact(z, y, eps, U)
    assert lam > 0
    assert abs(np.linalg.norm(p - y) - eps) <= 1e-12 * eps
    assert np.abs(U * (z - p) - lam * (p - y)).max() <= 1e-12 * np.abs(U * (z - p)).max()


@pytest.mark.parametrize("seed", [5, 6, 7])
def test_algorithm2_converges_to_exact_prox(seed):
    z, y, U = _block(seed, m=64, cond=3.0)
    eps = 4.0
    p_exact, _ = prox.ellipsoid_prox_exact(z, y, eps, U)
    p_fb = prox.ellipsoid_prox_fb(z, y, eps, U, n_itr=5000)
    assert np.abs(p_fb - p_exact).max() <= 1e-8 * np.abs(p_exact).max()


def test_identity_metric_reduces_to_ball_projection():
    z, y, _ = _block(8, m=16)
    U = np.ones(16)
    start = y + 100.0        # any start: one step with mu = 1 lands on P_B(z)
    p = prox.ellipsoid_prox_fb(z, y, 1.0, U, n_itr=1, start=start)
    assert np.allclose(p, prox.proj_l2ball(z, y, 1.0), rtol=0, atol=1e-14)
    p_exact, _ = prox.ellipsoid_prox_exact(z, y, 1.0, U)
    assert np.allclose(p_exact, prox.proj_l2ball(z, y, 1.0), rtol=0, atol=1e-12)


def test_inside_the_ball_the_prox_is_the_point():
    z, y, U = _block(9, m=8)
    z = y + 1e-3
    p = prox.ellipsoid_prox_fb(z, y, 1.0, U, n_itr=3, start=z)
    assert np.array_equal(p, z)
    p2 = prox.ellipsoid_prox_fb(z, y, 1.0, U, n_itr=4000, start=y)
    assert np.abs(p2 - z).max() <= 1e-12


# ----------------------------------------------------------------- accelerated Algorithm 2
def _weak_block(seed, m=64, cond=3.0, out=1.05, eps=4.0):
    """z just outside the ball (small Lagrange multiplier) and U spread over
    `cond` decades: the regime where the plain step is slow."""
    rng = np.random.default_rng(seed)
    y = rng.normal(size=m) + 1j * rng.normal(size=m)
    d = rng.normal(size=m) + 1j * rng.normal(size=m)
    z = y + out * eps * d / np.linalg.norm(d)
    U = 10.0 ** (-cond * rng.random(m))
    U[0] = 1.0
    return z, y, U, eps


def test_fista_first_two_steps_are_algorithm2():
    z, y, U = _block(8, m=32, cond=3.0)
    for n in (1, 2):
        assert np.array_equal(prox.ellipsoid_prox_fista(z, y, 4.0, U, n_itr=n, start=y),
                              prox.ellipsoid_prox_fb(z, y, 4.0, U, n_itr=n, start=y))


@pytest.mark.parametrize("seed", [5, 6, 7])
def test_fista_converges_to_exact_prox(seed):
    z, y, U = _block(seed, m=64, cond=3.0)
    p_exact, _ = prox.ellipsoid_prox_exact(z, y, 4.0, U)
    p = prox.ellipsoid_prox_fista(z, y, 4.0, U, n_itr=5000)
    assert np.abs(p - p_exact).max() <= 1e-8 * np.abs(p_exact).max()
    z, y, U, eps = _weak_block(seed)
    p_exact, _ = prox.ellipsoid_prox_exact(z, y, eps, U)
    p = prox.ellipsoid_prox_fista(z, y, eps, U, n_itr=20000)
    assert np.abs(p - p_exact).max() <= 1e-8 * np.abs(p_exact).max()


@pytest.mark.parametrize("seed", [5, 6])
def test_fista_is_faster_when_the_constraint_is_weakly_active(seed):
    """O(1/k^2) against O(1/k): after 100 steps the accelerated iterate is
    several times closer to the exact prox than Algorithm 2's."""
    z, y, U, eps = _weak_block(seed)
    p_exact, _ = prox.ellipsoid_prox_exact(z, y, eps, U)
    err = lambda p: np.abs(p - p_exact).max() / np.abs(p_exact).max()
    e_fb = err(prox.ellipsoid_prox_fb(z, y, eps, U, n_itr=100))
    e_fa = err(prox.ellipsoid_prox_fista(z, y, eps, U, n_itr=100))
    assert e_fa <= 0.2 * e_fb, (e_fa, e_fb)


# ----------------------------------------------------------------- Algorithm 2 stopping test
def test_stopping_test_with_identity_metric_stops_at_the_second_step():
    """U = I, mu = 1: every step lands on P_B(z) (the textbook l2-ball projection),
    so zbar^2 = zbar^1 and the test ||zbar^t - zbar^(t-1)|| <= tol ||zbar^t|| first
    holds at t = 2 from any other start, at t = 1 from P_B(z) itself."""
    z, y, _ = _block(8, m=16)
    U = np.ones(16)
    ball = prox.proj_l2ball(z, y, 1.0)
    for solve in (prox.ellipsoid_prox_fb, prox.ellipsoid_prox_fista):
        info = {}
        p = solve(z, y, 1.0, U, n_itr=50, start=y + 100.0, tol=1e-12, info=info)
        assert info["steps"] == 2 and np.allclose(p, ball, rtol=0, atol=1e-14)
        info = {}
        solve(z, y, 1.0, U, n_itr=50, start=ball, tol=1e-12, info=info)
        assert info["steps"] == 1
        info = {}
        solve(z, y, 1.0, U, n_itr=7, start=y + 100.0, tol=0.0, info=info)
        assert info["steps"] == 7          # tol = 0: the fixed number of steps


@pytest.mark.parametrize("seed", [11, 12, 13])
def test_stopping_test_bounds_the_distance_to_the_exact_prox(seed):
    """With max U = 1 and mu = 1 the step zbar -> P_B(zbar - U (zbar - z)) is a
    contraction of factor q = 1 - min U (P_B is non-expansive), so at the stop
    ||zbar^t - p*|| <= q/(1-q) ||zbar^t - zbar^(t-1)|| <= q/(1-q) tol ||zbar^t||
    (the a-posteriori bound of Banach's fixed-point theorem), p* the exact prox."""
    rng = np.random.default_rng(seed)
    m = 48
    y = rng.normal(size=m) + 1j * rng.normal(size=m)
    z = y + 6.0 * (rng.normal(size=m) + 1j * rng.normal(size=m)) / np.sqrt(m)
    U = rng.uniform(0.2, 1.0, size=m)
    U[0] = 1.0
    q = 1.0 - U.min()
    p_exact, lam = prox.ellipsoid_prox_exact(z, y, 2.0, U)
    assert lam > 0
    steps = []
    for tol in (1e-3, 1e-5, 1e-7, 1e-9):
        info = {}
        p = prox.ellipsoid_prox_fb(z, y, 2.0, U, n_itr=100000, start=y, tol=tol, info=info)
        bound = q / (1.0 - q) * tol * np.linalg.norm(p)
        assert np.linalg.norm(p - p_exact) <= bound * (1 + 1e-6) + 1e-13 * np.linalg.norm(p)
        assert info["steps"] < 100000
        steps.append(info["steps"])
    assert steps == sorted(steps) and steps[0] < steps[-1]   # tighter tolerance, more steps
