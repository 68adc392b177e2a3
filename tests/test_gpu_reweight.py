"""Re-weighted l1 (Algorithm 1, Eq. "reweighting"): CUDA path vs the FP64 oracle.

The weights W = omega / (omega + |Psi^dagger x|) computed on the device from
the device iterate, ||Psi W||_S^2 from the device power iteration, and the
weighted PPD trajectory are compared with the oracle on the same inputs.
Tolerances as in test_gpu_parity: weights and images <= 1e-4 relative l2
in FP32 (<= 1e-8 in FP64), ||Psi W||^2 <= 1e-5 (<= 1e-9).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import ppd as oppd, reweight as orw  # noqa: E402
from paper_1701_01748_gb300 import build, ppd, synth  # noqa: E402

pytestmark = pytest.mark.gpu

F32, F64 = ppd.PPD_FP32_FP64NORMS, ppd.PPD_FP64_PLAIN
TOL = {F32: dict(w=1e-4, img=1e-4, nrm=1e-5), F64: dict(w=1e-8, img=1e-8, nrm=1e-9)}
POWER = 300     # power-iteration steps for ||Psi W||^2 on both sides (same start and stop rule)


@pytest.fixture(scope="module", autouse=True)
def lib():
    build.build()
    assert torch.cuda.is_available()
    return ppd._lib()


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def small():
    return synth.make_problem("rw", L=32, M=3000, n_blocks=3, uv_sigma=0.3, seed=31, n_points=6, n_blobs=1)


def both(p, prec, **kw):
    S = oppd.make_setup(p.omega, p.y, p.theta, p.block, p.n_blocks, p.L, power_iters=400, x_true=p.x_true)
    s = ppd.Solver(p.L, p.n_blocks, precision=prec, eta=S.eta, power_iters=POWER, **kw)
    s.set_problem(p.omega, p.y, p.block, theta=p.theta, x_true=p.x_true)
    return S, oppd.init_state(S), s


@pytest.mark.parametrize("prec", [F32, F64])
def test_reweight_from_the_iterate(prec):
    p = small()
    S, st, s = both(p, prec)
    oppd.run(S, 30, st)
    s.iterate(30, stats=False)
    omega = 1e-2 * 0.25
    orw.reweight(st, S, omega, max_iter=POWER)
    ppd.ppd_reweight(s.ctx, omega)
    Wg = ppd.ppd_get_prior_weights(s.ctx, p.L, p.L)
    assert rel(Wg, S.W) <= TOL[prec]["w"], rel(Wg, S.W)
    prm = s.params()
    assert abs(prm["psiw_norm_sq"] - S.psiw_sq) <= TOL[prec]["nrm"] * S.psiw_sq
    assert abs(prm["alpha"] - S.kappa * S.psiw_sq) <= TOL[prec]["nrm"] * S.kappa
    assert abs(prm["zeta"] - S.zeta / S.psiw_sq) <= TOL[prec]["nrm"] * prm["zeta"]
    assert prm["convergence_lhs"] < 1.0
    # warm-started weighted iterations (Algorithm 1)
    for _ in range(20):
        hist = oppd.iterate(st, S)
    stats = s.iterate(20)
    assert rel(s.image(), st.x) <= TOL[prec]["img"], rel(s.image(), st.x)
    assert abs(stats["snr_db"] - hist["snr"]) <= 1e-3
    s.close()


@pytest.mark.parametrize("prec", [F32, F64])
def test_given_weights(prec):
    p = small()
    S, st, s = both(p, prec, use_graph=0 if prec == F32 else 1)
    W = np.random.default_rng(5).uniform(0.05, 1.0, size=(9, p.L, p.L))
    orw.set_weights(S, W, max_iter=POWER)
    ppd.ppd_set_prior_weights(s.ctx, W)
    back = ppd.ppd_get_prior_weights(s.ctx, p.L, p.L)
    assert rel(back, W) <= (1e-7 if prec == F32 else 0.0)
    assert abs(s.params()["psiw_norm_sq"] - S.psiw_sq) <= TOL[prec]["nrm"] * S.psiw_sq
    oppd.run(S, 25, st)
    s.iterate(25, stats=False)
    assert rel(s.image(), st.x) <= TOL[prec]["img"], rel(s.image(), st.x)
    # W = I again: back to the plain prior step
    ppd.ppd_set_prior_weights(s.ctx, None)
    orw.set_weights(S, None)
    assert s.params()["psiw_norm_sq"] == 1.0
    assert np.all(ppd.ppd_get_prior_weights(s.ctx, p.L, p.L) == 1.0)
    oppd.run(S, 10, st)
    s.iterate(10, stats=False)
    assert rel(s.image(), st.x) <= TOL[prec]["img"], rel(s.image(), st.x)
    s.close()


def test_reweighted_schedule_matches_oracle():
    p = small()
    S, st, s = both(p, F32)
    st, _ = orw.run(S, 2, 15, omega0=1e-2, factor=0.25, st=st, power_iters=POWER)
    s.reweighted(2, 15, omega0=1e-2, factor=0.25)
    assert s.iterate(0)["iters_done"] == 45
    assert rel(s.image(), st.x) <= TOL[F32]["img"], rel(s.image(), st.x)
    s.close()


def test_group_recaptures_after_reweight():
    probs = [synth.make_problem("grw", L=L, M=M, n_blocks=d, uv_sigma=0.15, seed=60 + i, n_points=6, n_blobs=1)
             for i, (L, M, d) in enumerate([(32, 3000, 2), (64, 9000, 4)])]
    solo, grouped = [], []
    for p in probs:
        for dest in (solo, grouped):
            s = ppd.Solver(p.L, p.n_blocks, precision=F32, eta=1e-3, power_iters=50)
            s.set_problem(p.omega, p.y, p.block, theta=p.theta)
            dest.append(s)
    for s in solo:
        s.iterate(6, stats=False)
    ppd.ppd_reweight(solo[1].ctx, 1e-3)
    for s in solo:
        s.iterate(5, stats=False)
    g = ppd.ppd_group_create([s.ctx for s in grouped])
    ppd.ppd_group_iterate(g, 6)
    ppd.ppd_reweight(grouped[1].ctx, 1e-3)
    ppd.ppd_group_iterate(g, 5)
    ppd.ppd_group_destroy(g)
    for a, b in zip(solo, grouped):
        assert np.array_equal(a.image(), b.image())
        a.close()
        b.close()


def test_reweight_errors():
    p = small()
    s = ppd.Solver(p.L, p.n_blocks, precision=F32, eta=1e-3)
    s.set_problem(p.omega, p.y, p.block, theta=p.theta)
    for bad in (0.0, -1.0, float("nan"), float("inf")):
        with pytest.raises(ppd.PPDError) as e:
            ppd.ppd_reweight(s.ctx, bad)
        assert e.value.status == ppd.PPD_ERR_INVALID_ARG
    with pytest.raises(ppd.PPDError) as e:
        ppd.ppd_set_prior_weights(s.ctx, np.ones((9, p.L, p.L - 1)))
    assert e.value.status == ppd.PPD_ERR_INVALID_ARG
    w = np.ones((9, p.L, p.L))
    w[3, 1, 2] = -0.5
    with pytest.raises(ppd.PPDError) as e:
        ppd.ppd_set_prior_weights(s.ctx, w)
    assert e.value.status == ppd.PPD_ERR_INVALID_ARG
    with pytest.raises(ppd.PPDError) as e:     # ||Psi W|| = 0: refused, context left unweighted
        ppd.ppd_set_prior_weights(s.ctx, np.zeros((9, p.L, p.L)))
    assert e.value.status == ppd.PPD_ERR_NONFINITE
    assert s.params()["psiw_norm_sq"] == 1.0
    s.iterate(3, stats=False)
    s.close()
