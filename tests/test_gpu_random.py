"""Randomised active sets (Algorithm 3, sets P and D) and the accelerated
inner solver through the C ABI, against the FP64 oracle fed the same seeded
draws.

Tolerances as in test_gpu_parity: image after a fixed number of iterations
<= 1e-4 relative l2 in FP32, <= 1e-8 in FP64; grouped and solo runs
bit-identical.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import ppd as oppd  # noqa: E402
from paper_1701_01748_gb300 import build, ppd, synth  # noqa: E402

pytestmark = pytest.mark.gpu

F32, F64 = ppd.PPD_FP32_FP64NORMS, ppd.PPD_FP64_PLAIN
TOL = {F32: 1e-4, F64: 1e-8}
SMALL = dict(L=32, M=3000, n_blocks=3, uv_sigma=0.3, seed=11, n_points=6, n_blobs=1)


@pytest.fixture(scope="module", autouse=True)
def lib():
    build.build()
    assert torch.cuda.is_available()
    return ppd._lib()


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def draws(n, d, seed):
    B, P = synth.active_sets(n, d, 0.5, 0.6, seed=seed)
    B[0, 1] = 0          # block 1 first becomes active after t = 1
    B[0, 0] = 1
    return B, P


@pytest.mark.parametrize("prec", [F32, F64])
@pytest.mark.parametrize("n_itr,solver", [(1, "fb"), (3, "fb"), (4, "fista")])
def test_active_sets_match_the_oracle(prec, n_itr, solver):
    p = synth.make_problem("small", **SMALL)
    S = oppd.make_setup(p.omega, p.y, p.theta, p.block, p.n_blocks, p.L, power_iters=300, x_true=p.x_true,
                        n_itr=n_itr, inner_solver=solver)
    B, P = draws(30, p.n_blocks, seed=21)
    st = oppd.init_state(S)
    for t in range(30):
        oppd.iterate(st, S, B[t], P[t])
    for _ in range(5):                       # queue used up: full sets again
        oppd.iterate(st, S)
    s = ppd.Solver(p.L, p.n_blocks, precision=prec, eta=S.eta, n_itr=n_itr,
                   inner_solver=ppd.PPD_INNER_FISTA if solver == "fista" else ppd.PPD_INNER_FB)
    s.set_problem(p.omega, p.y, p.block, theta=p.theta, x_true=p.x_true)
    ppd.ppd_set_active_sets(s.ctx, B, P)
    s.iterate(12)
    s.iterate(18)
    s.iterate(5)
    assert rel(s.image(), st.x) <= TOL[prec], rel(s.image(), st.x)
    s.close()


def test_switching_the_sets_off_returns_to_the_plain_iteration():
    p = synth.make_problem("small", **SMALL)
    S = oppd.make_setup(p.omega, p.y, p.theta, p.block, p.n_blocks, p.L, power_iters=300)
    B, P = draws(10, p.n_blocks, seed=22)
    st = oppd.init_state(S)
    for t in range(10):
        oppd.iterate(st, S, B[t], P[t])
    for _ in range(10):
        oppd.iterate(st, S)
    s = ppd.Solver(p.L, p.n_blocks, precision=F32, eta=S.eta)
    s.set_problem(p.omega, p.y, p.block, theta=p.theta)
    ppd.ppd_set_active_sets(s.ctx, B, P)
    s.iterate(10, stats=False)
    ppd.ppd_set_active_sets(s.ctx, n_iters=0)
    s.iterate(10, stats=False)
    assert rel(s.image(), st.x) <= TOL[F32]
    # an operator call between iterations overwrites the gridding's partial
    # tiles; the inactive blocks' contributions are then recomputed
    B2, P2 = draws(6, p.n_blocks, seed=23)
    for t in range(6):
        oppd.iterate(st, S, B2[t], P2[t])
    ppd.ppd_set_active_sets(s.ctx, B2, P2)
    s.iterate(3, stats=False)
    yd = torch.zeros((p.M, 2), dtype=torch.float32, device="cuda")
    xd = torch.empty((p.L, p.L), dtype=torch.float32, device="cuda")
    ppd.ppd_op_adjoint(s.ctx, yd.data_ptr(), xd.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    s.iterate(3, stats=False)
    assert rel(s.image(), st.x) <= TOL[F32]
    s.close()


def test_group_with_active_sets_matches_solo_runs():
    probs = [synth.make_problem("grp", L=L, M=M, n_blocks=d, uv_sigma=0.15, seed=60 + i, n_points=6, n_blobs=1)
             for i, (L, M, d) in enumerate([(32, 3000, 2), (64, 9000, 4)])]
    solo, grouped = [], []
    for i, p in enumerate(probs):
        B, P = draws(9, p.n_blocks, seed=30 + i)
        for dest in (solo, grouped):
            s = ppd.Solver(p.L, p.n_blocks, precision=F32, eta=1e-3)
            s.set_problem(p.omega, p.y, p.block, theta=p.theta)
            ppd.ppd_set_active_sets(s.ctx, B, P)
            dest.append(s)
    for s in solo:
        s.iterate(12, stats=False)
    g = ppd.ppd_group_create([s.ctx for s in grouped])
    ppd.ppd_group_iterate(g, 4)
    ppd.ppd_group_iterate(g, 8)
    ppd.ppd_group_destroy(g)
    for a, b in zip(solo, grouped):
        assert np.array_equal(a.image(), b.image())
        a.close()
        b.close()


def test_state_resume_with_active_sets_is_bit_identical():
    p = synth.make_problem("small", **SMALL)
    B, P = draws(20, p.n_blocks, seed=24)
    s = ppd.Solver(p.L, p.n_blocks, precision=F32, eta=1e-3)
    s.set_problem(p.omega, p.y, p.block, theta=p.theta)
    ppd.ppd_set_active_sets(s.ctx, B[:8], P[:8])
    s.iterate(8, stats=False)
    blob = ppd.ppd_get_state(s.ctx)
    ppd.ppd_set_active_sets(s.ctx, B[8:], P[8:])
    s.iterate(12, stats=False)
    x_run = s.image()
    ppd.ppd_set_state(s.ctx, blob)
    ppd.ppd_set_active_sets(s.ctx, B[8:], P[8:])
    s.iterate(12, stats=False)
    assert np.array_equal(s.image(), x_run)
    s.close()


def test_active_sets_errors():
    p = synth.make_problem("small", **SMALL)
    s = ppd.Solver(p.L, p.n_blocks, precision=F32)
    with pytest.raises(ppd.PPDError) as e:
        ppd.ppd_set_active_sets(s.ctx, n_iters=-1)
    assert e.value.status == ppd.PPD_ERR_INVALID_ARG
    s.close()
