"""Pins of the oracle's re-weighted l1 (Algorithm 1, Eq. "reweighting").

What the paper and the mathematics fix: the weight formula on coefficients
known in closed form, ||Psi W||_S^2 for weights with a known answer and
against a dense singular value, W = I reducing to plain PPD, and that the
weighted problem's minimiser is feasible, positive and has a weighted l1
norm no larger than the unweighted minimiser's.
"""
import math

import numpy as np
import pytest

from oracle import ppd, reweight, sara
from paper_1701_01748_gb300 import synth


def test_weights_of_zero_image_are_identity():
    W = reweight.weights(np.zeros((16, 16)), 1e-2)
    assert W.shape == (9, 16, 16)
    assert np.all(W == 1.0)


def test_weights_of_a_point_source_closed_form():
    """A point of flux a at pixel (1, 1): the Dirac coefficient is a/3; the level-1
    Haar (db1) coefficients at quadrant position (0, 0) are +-a/2 times 1/3."""
    L, a, om = 16, 0.6, 0.05
    x = np.zeros((L, L))
    x[1, 1] = a
    W = reweight.weights(x, om)
    h = L // 2
    assert W[0, 1, 1] == pytest.approx(om / (om + a / 3), rel=1e-14)
    assert W[0, 0, 0] == 1.0 and W[0, 2, 1] == 1.0
    haar = W[1]
    for (r, c) in [(h, h), (0, h), (h, 0)]:     # HH, LH (cols high), HL (rows high): |c| = a/2/3
        assert haar[r, c] == pytest.approx(om / (om + a / 6), rel=1e-13)
    # the signed coefficient of the column-high quadrant is negative: the weight takes |.|
    c = sara.psi_adjoint(x)
    assert c[1, 0, h] < 0


@pytest.mark.parametrize("scale", [1.0, 0.37])
def test_norm_of_uniform_weights(scale):
    W = np.full((9, 16, 16), scale)
    val, _ = reweight.psiw_norm_sq(W)
    assert val == pytest.approx(scale ** 2, rel=1e-12)


def test_norm_of_one_basis():
    """Each basis is orthonormal times 1/3: ||Psi_i||_S^2 = 1/9."""
    W = np.zeros((9, 16, 16))
    W[4] = 1.0
    val, _ = reweight.psiw_norm_sq(W)
    assert val == pytest.approx(1.0 / 9.0, rel=1e-12)


def test_norm_matches_dense_singular_value():
    rng = np.random.default_rng(11)
    L = 16
    W = rng.uniform(0.05, 1.0, size=(9, L, L))
    cols = []
    for i in range(9 * L * L):
        e = np.zeros(9 * L * L)
        e[i] = W.reshape(-1)[i]
        cols.append(sara.psi(e.reshape(9, L, L)).reshape(-1))
    A = np.stack(cols, axis=1)                 # Psi W, N x 9N
    dense = float(np.linalg.eigvalsh(A @ A.T)[-1])
    got, it = reweight.psiw_norm_sq(W, max_iter=20000, tol=1e-15)
    assert abs(got - dense) <= 1e-9 * dense


def _tiny(seed=21, M=500, n_blocks=2):
    return synth.make_problem("tiny", L=16, M=M, n_blocks=n_blocks, uv_sigma=0.2, seed=seed,
                              n_points=4, n_blobs=1)


def test_unit_weights_reproduce_plain_ppd():
    p = _tiny(seed=22, M=200)
    runs = []
    for weighted in (False, True):
        S = ppd.make_setup(p.omega, p.y, p.theta, p.block, p.n_blocks, p.L, power_iters=200)
        if weighted:
            reweight.set_weights(S, np.ones((9, 16, 16)))
            assert S.psiw_sq == pytest.approx(1.0, rel=1e-12)
        st, _ = ppd.run(S, 20)
        runs.append(st.x)
    assert np.abs(runs[0] - runs[1]).max() <= 1e-10 * np.abs(runs[0]).max()


def test_weighted_minimiser_is_feasible_and_lowers_the_weighted_norm():
    """Algorithm 1's second run, warm-started from the first run's variables, reaches a
    feasible positive point whose weighted l1 norm is no larger than the first run's
    (unweighted) minimiser's, which is feasible too."""
    p = _tiny(M=300, n_blocks=1)
    S = ppd.make_setup(p.omega, p.y, p.theta, p.block, p.n_blocks, p.L, power_iters=300)
    st, hist = ppd.run(S, 1000)
    assert np.all(hist[-1]["residual"] <= 1.01 * S.eps)
    x_u = st.x.copy()
    W = reweight.weights(x_u, 1e-2)
    reweight.set_weights(S, W)
    assert ppd.convergence_lhs(S) == pytest.approx(0.98, abs=1e-9)
    st, hist = ppd.run(S, 1500, st)
    assert st.x.min() >= 0.0
    assert np.all(hist[-1]["residual"] <= 1.01 * S.eps)
    assert hist[-1]["rel_var"] < 1e-4
    assert reweight.weighted_l1(st.x, W) <= reweight.weighted_l1(x_u, W) * (1 + 1e-3)


def test_schedule_runs_warm_started_with_decreasing_omega():
    p = _tiny(seed=23, M=300)
    S = ppd.make_setup(p.omega, p.y, p.theta, p.block, p.n_blocks, p.L, power_iters=200)
    st, hist = reweight.run(S, 2, 30, omega0=1e-2, factor=0.25, power_iters=300)
    assert len(hist) == 90 and st.t == 90
    # weights in (0, 1] give ||Psi W|| <= ||Psi|| = 1
    assert S.W is not None and 0.0 < S.psiw_sq <= 1.0 + 1e-12
    assert np.all(S.W <= 1.0) and np.all(S.W > 0.0) and S.W.min() < 1.0
    assert math.isfinite(S.psiw_sq)
