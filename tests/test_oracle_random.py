"""Pins of the oracle's randomised active sets (Algorithm 3, sets P and D).

What the paper fixes: dual variables outside the active sets keep their
values (the "set" steps of Algorithm 3 for j outside D and i outside P),
active ones are updated exactly as in the full iteration, all-active sets
are the plain iteration, and with nonzero activation probabilities drawn
i.i.d. along the iterations the method still converges to the minimiser
(Section 4.4, convergence requirements).
"""
import copy

import numpy as np

from oracle import ppd
from paper_1701_01748_gb300 import synth


def _tiny(seed=5, M=600, n_blocks=4):
    p = synth.make_problem("tiny", L=16, M=M, n_blocks=n_blocks, uv_sigma=0.2, seed=seed,
                           n_points=4, n_blobs=1)
    S = ppd.make_setup(p.omega, p.y, p.theta, p.block, p.n_blocks, p.L, x_true=p.x_true, power_iters=300)
    return p, S


def test_active_set_draws_are_bernoulli_and_seeded():
    B, P = synth.active_sets(4000, 16, 0.3, 0.8, seed=1)
    assert B.shape == (4000, 16) and P.shape == (4000, 9)
    assert abs(B.mean() - 0.3) < 0.01 and abs(P.mean() - 0.8) < 0.01
    B2, P2 = synth.active_sets(4000, 16, 0.3, 0.8, seed=1)
    assert np.array_equal(B, B2) and np.array_equal(P, P2)
    # independence across iterations: lag-1 correlation of a block's indicator is ~0
    b = B[:, 3].astype(float) - B[:, 3].mean()
    assert abs(np.dot(b[1:], b[:-1]) / np.dot(b, b)) < 0.05


def test_all_active_sets_are_the_plain_iteration():
    p, S = _tiny(M=300, n_blocks=3)
    a, b = ppd.init_state(S), ppd.init_state(S)
    for _ in range(6):
        ppd.iterate(a, S)
        ppd.iterate(b, S, np.ones(3, bool), np.ones(9, bool))
    for f in ("x", "xt", "u", "v", "p"):
        assert np.array_equal(getattr(a, f), getattr(b, f)), f


def test_inactive_duals_keep_their_values_and_active_ones_update_as_in_full_iteration():
    p, S = _tiny(M=400, n_blocks=4)
    st = ppd.init_state(S)
    for _ in range(4):
        ppd.iterate(st, S)
    full, part = copy.deepcopy(st), copy.deepcopy(st)
    ppd.iterate(full, S)
    act_d = np.array([True, False, True, False])
    act_p = np.array([False, True, True, False, True, False, False, True, True])
    ppd.iterate(part, S, act_d, act_p)
    for j, m in enumerate(S.members):
        if act_d[j]:
            assert np.array_equal(part.v[m], full.v[m]) and np.array_equal(part.p[m], full.p[m])
        else:
            assert np.array_equal(part.v[m], st.v[m]) and np.array_equal(part.p[m], st.p[m])
    for i in range(9):
        assert np.array_equal(part.u[i], full.u[i] if act_p[i] else st.u[i]), i
    # the primal step used the mixed duals: it differs from the full one
    assert not np.array_equal(part.x, full.x)


def test_a_block_first_active_later_starts_from_the_ball_projection():
    """A block outside D at t = 1 starts Algorithm 2 from P_B(z) when it first becomes active."""
    p, S = _tiny(M=300, n_blocks=2)
    a = ppd.init_state(S)
    ppd.iterate(a, S, np.array([True, False]), np.ones(9, bool))
    assert a.seen.tolist() == [True, False]
    m1 = S.members[1]
    assert not np.any(a.v[m1]) and not np.any(a.p[m1])
    # block 1 joins at t = 2: same p as a run whose block 1 state is fresh and
    # whose Algorithm 2 starts at P_B(z) (inner start "current" plus one step)
    b = copy.deepcopy(a)
    ppd.iterate(a, S, np.array([False, True]), np.ones(9, bool))
    S1 = copy.copy(S)
    S1.n_itr = S.n_itr + 1
    S1.inner_init = "current"
    ppd.iterate(b, S1, np.array([False, True]), np.ones(9, bool))
    assert np.allclose(a.p[m1], b.p[m1], rtol=1e-12, atol=0)


def test_randomised_ppd_reaches_the_same_minimiser():
    p, S = _tiny(M=600, n_blocks=4)
    det, hist = ppd.run(S, 1200)
    B, P = synth.active_sets(1600, p.n_blocks, 0.7, 0.7, seed=3)
    st = ppd.init_state(S)
    for t in range(1600):
        h = ppd.iterate(st, S, B[t], P[t])
    assert st.x.min() >= 0.0
    assert np.all(h["residual"] <= 1.01 * S.eps)
    assert np.linalg.norm(st.x - det.x) <= 5e-3 * np.linalg.norm(det.x)
    assert abs(ppd.l1_objective(st.x) - ppd.l1_objective(det.x)) <= 2e-3 * ppd.l1_objective(det.x)
