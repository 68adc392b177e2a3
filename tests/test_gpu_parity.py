"""CUDA path vs the FP64 oracle, element by element, through the C ABI.

Tolerances (relative l2 unless stated): bins, sort order and cell counts
bit-exact; Phi, Phi^dagger, Psi, Psi^dagger <= 1e-5 in FP32 (<= 1e-10 in
FP64); image after a fixed number of PPD iterations <= 1e-4 in FP32 (<= 1e-8
in FP64); gradients of 1/2 ||y - Phi x||^2 <= 1e-3 against finite
differences.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import nufft, ppd as oppd, sara  # noqa: E402
from paper_1701_01748_gb300 import build, ppd, synth  # noqa: E402

pytestmark = pytest.mark.gpu

F32, F64 = ppd.PPD_FP32_FP64NORMS, ppd.PPD_FP64_PLAIN
TOL = {F32: dict(op=1e-5, img=1e-4), F64: dict(op=1e-10, img=1e-8)}


@pytest.fixture(scope="session", autouse=True)
def lib():
    build.build()
    assert torch.cuda.is_available()
    return ppd._lib()


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def tdtype(prec):
    return torch.float32 if prec == F32 else torch.float64


def solver(p, prec, **cfg):
    s = ppd.Solver(p.L, p.n_blocks, precision=prec, **cfg)
    s.set_problem(p.omega, p.y, p.block, theta=p.theta, x_true=p.x_true)
    return s


def stream():
    return torch.cuda.current_stream().cuda_stream


def op_forward(s, x, prec):
    xd = torch.tensor(x, dtype=tdtype(prec), device="cuda")
    yd = torch.empty((s.M, 2), dtype=tdtype(prec), device="cuda")
    ppd.ppd_op_forward(s.ctx, xd.data_ptr(), yd.data_ptr(), stream())
    torch.cuda.synchronize()
    return yd.cpu().double().numpy() @ np.array([1.0, 1j])


def op_adjoint(s, y, prec):
    yd = torch.tensor(np.stack([y.real, y.imag], 1), dtype=tdtype(prec), device="cuda")
    xd = torch.empty((s.L, s.L), dtype=tdtype(prec), device="cuda")
    ppd.ppd_op_adjoint(s.ctx, yd.data_ptr(), xd.data_ptr(), stream())
    torch.cuda.synchronize()
    return xd.cpu().double().numpy()


SMALL = dict(L=32, M=3000, n_blocks=3, uv_sigma=0.3, seed=11, n_points=6, n_blobs=1)
_cache = {}


def problem(name, **kw):
    key = (name, tuple(sorted(kw.items())))
    if key not in _cache:
        _cache[key] = synth.make_problem(name, **kw)
    return _cache[key]


# ----------------------------------------------------------------- binning
@pytest.mark.parametrize("which", ["small", "c1", "edges"])
def test_bins_and_order_bit_exact(which):
    if which == "small":
        p = problem("small", **SMALL)
        om, blk, L, d = p.omega, p.block, p.L, p.n_blocks
    elif which == "c1":
        p = problem("c1_128")
        om, blk, L, d = p.omega, p.block, p.L, p.n_blocks
    else:
        L, d = 64, 2
        rng = np.random.default_rng(3)
        om = rng.uniform(-np.pi, np.pi, size=(500, 2))
        om[:8] = [[-np.pi, -np.pi], [np.pi, np.pi], [0.0, -0.0], [-1e-300, 1e-300],
                  [-5e-17, 3.0], [np.nextafter(-np.pi, 0), 0.1], [1.5, -1.5], [1.5, -1.5]]
        blk = rng.integers(0, d, size=500).astype(np.int32)
    s = ppd.Solver(L, d, precision=F32)
    y = np.zeros(om.shape[0], np.complex128) + 1.0
    ppd.ppd_set_visibilities(s.ctx, om, y, blk)
    perm, b0, b1, cnt = ppd.ppd_get_bins(s.ctx, om.shape[0])
    K = 2 * L
    ob0, ob1, _, _ = nufft.base_cells(om, K, K)
    _, ocnt = nufft.uniform_weights(om, K, K)
    T = 16
    operm, _, _, _ = nufft.visibility_order(om, blk, K, K, T)
    assert np.array_equal(b0, ob0) and np.array_equal(b1, ob1)
    assert np.array_equal(cnt, ocnt)
    assert np.array_equal(perm, operm)
    s.close()


# ----------------------------------------------------------------- operators
@pytest.mark.parametrize("prec", [F32, F64])
@pytest.mark.parametrize("name", ["small", "c1_128"])
def test_phi_and_adjoint(prec, name):
    p = problem("small", **SMALL) if name == "small" else problem(name)
    s = solver(p, prec, eta=1.0)
    P = nufft.Plan(p.omega, p.L, theta=p.theta)
    rng = np.random.default_rng(5)
    x = rng.random((p.L, p.L))
    assert rel(op_forward(s, x, prec), nufft.phi(x, P)) <= TOL[prec]["op"]
    yv = rng.normal(size=p.M) + 1j * rng.normal(size=p.M)
    assert rel(op_adjoint(s, yv, prec), nufft.phi_adjoint(yv, P)) <= TOL[prec]["op"]
    # adjoint identity of the GPU operators themselves
    a = float(np.vdot(op_forward(s, x, prec), yv).real)
    b = float(np.sum(x * op_adjoint(s, yv, prec)))
    assert abs(a - b) <= TOL[prec]["op"] * abs(a)
    s.close()


def test_phi_full_size_c2():
    p = problem("c2_512")
    s = solver(p, F32, eta=1.0)
    P = nufft.Plan(p.omega, p.L, theta=p.theta)
    x = p.x_true
    assert rel(op_forward(s, x, F32), nufft.phi(x, P)) <= 1e-5
    yv = np.random.default_rng(2).normal(size=p.M) * (1 + 0j)
    assert rel(op_adjoint(s, yv, F32), nufft.phi_adjoint(yv, P)) <= 1e-5
    s.close()


@pytest.mark.parametrize("prec", [F32, F64])
def test_psi_analysis_synthesis(prec):
    p = problem("small", **SMALL)
    s = solver(p, prec, eta=1.0)
    x = np.random.default_rng(8).normal(size=(p.L, p.L))
    xd = torch.tensor(x, dtype=tdtype(prec), device="cuda")
    cd = torch.empty((9, p.L, p.L), dtype=tdtype(prec), device="cuda")
    ppd.ppd_psi_analysis(s.ctx, xd.data_ptr(), cd.data_ptr(), stream())
    torch.cuda.synchronize()
    ref = sara.psi_adjoint(x)
    assert rel(cd.cpu().double().numpy(), ref) <= TOL[prec]["op"]
    u = np.random.default_rng(9).normal(size=(9, p.L, p.L))
    ud = torch.tensor(u, dtype=tdtype(prec), device="cuda")
    ppd.ppd_psi_synthesis(s.ctx, ud.data_ptr(), xd.data_ptr(), stream())
    torch.cuda.synchronize()
    assert rel(xd.cpu().double().numpy(), sara.psi(u)) <= TOL[prec]["op"]
    s.close()


@pytest.mark.parametrize("prec", [F32, F64])
@pytest.mark.parametrize("method", ["lanczos", "power"])
def test_eta_operator_norm(prec, method):
    """||U^{1/2} Phi||_S^2 by the library's Lanczos process (default) or power
    iteration, against the oracle's routine of the same name."""
    p = problem("small", **SMALL)
    P = nufft.Plan(p.omega, p.L, theta=p.theta)
    U = nufft.uniform_weights(p.omega, 2 * p.L, 2 * p.L)[0]
    if method == "power":
        ref, _ = oppd.op_norm_sq(P, U, max_iter=1000, tol=1e-10)
        s = solver(p, prec, norm_method=ppd.PPD_NORM_POWER)
    else:
        ref, _ = oppd.op_norm_sq_lanczos(P, U, tol=1e-12)
        s = solver(p, prec)
    got = s.params()
    assert abs(got["op_norm_sq"] - ref) <= (1e-5 if prec == F32 else 1e-8) * ref
    assert got["convergence_lhs"] < 1.0
    if method == "lanczos":
        assert got["power_iters_done"] < 200
    s.close()


def test_lanczos_gets_the_norm_the_power_iteration_misses():
    """The 512^2 workload (strongly non-uniform coverage): the library's
    Lanczos estimate equals the oracle's stored Lanczos value, which 20 power
    steps underestimate by >10 %."""
    import json
    import os
    p = problem("c2_512")
    rec = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "op_norms.json")))["c2_512"]
    assert rec["seed"] == p.seed and rec["M"] == p.M
    s = solver(p, F32)
    got = s.params()
    assert abs(got["op_norm_sq"] - rec["op_norm_sq"]) <= 1e-4 * rec["op_norm_sq"]
    assert got["power_iters_done"] < 300
    s.close()


# ----------------------------------------------------------------- PPD
def run_both(p, prec, n_iter, **kw):
    n_itr = kw.pop("n_itr", 1)
    precond = kw.pop("precond", 1)
    init = kw.pop("inner_init", ppd.PPD_INNER_WARM)
    solver_kind = kw.pop("inner_solver", ppd.PPD_INNER_FB)
    S = oppd.make_setup(p.omega, p.y, p.theta, p.block, p.n_blocks, p.L, precond=bool(precond),
                        n_itr=n_itr, power_iters=400, x_true=p.x_true,
                        inner_init="current" if init == ppd.PPD_INNER_CURRENT else "warm",
                        inner_solver="fista" if solver_kind == ppd.PPD_INNER_FISTA else "fb")
    s = ppd.Solver(p.L, p.n_blocks, precision=prec, eta=S.eta, n_itr=n_itr, precond=precond,
                   inner_init=init, inner_solver=solver_kind, **kw)
    s.set_problem(p.omega, p.y, p.block, theta=p.theta, x_true=p.x_true)
    st = oppd.init_state(S)
    for _ in range(n_iter):
        hist = oppd.iterate(st, S)
    stats = s.iterate(n_iter)
    xg = s.image()
    s.close()
    return xg, st, hist, stats, S


@pytest.mark.parametrize("prec", [F32, F64])
def test_ppd_c1_fixed_iterations(prec):
    p = problem("c1_128")
    n = 200 if prec == F64 else 200
    xg, st, hist, stats, S = run_both(p, prec, n)
    assert rel(xg, st.x) <= TOL[prec]["img"], rel(xg, st.x)
    assert abs(stats["snr_db"] - hist["snr"]) <= 1e-3
    assert abs(stats["rel_var"] - hist["rel_var"]) <= 1e-2 * hist["rel_var"] + 1e-9
    assert np.allclose(stats["block_residual"], hist["residual"], rtol=1e-4)


@pytest.mark.parametrize("prec", [F32, F64])
def test_ppd_multiblock_subiterations_weights(prec):
    p = problem("small", **SMALL)
    p2 = synth.Problem(**{**p.__dict__})
    p2.theta = p.theta * np.random.default_rng(4).uniform(0.5, 2.0, size=p.M)   # non-uniform Theta
    xg, st, hist, stats, S = run_both(p2, prec, 30, n_itr=3)
    assert rel(xg, st.x) <= TOL[prec]["img"], rel(xg, st.x)


@pytest.mark.parametrize("prec", [F32, F64])
def test_inner_start_at_z(prec):
    p = problem("small", **SMALL)
    xg, st, hist, stats, S = run_both(p, prec, 20, n_itr=3, inner_init=ppd.PPD_INNER_CURRENT)
    assert rel(xg, st.x) <= TOL[prec]["img"], rel(xg, st.x)


@pytest.mark.parametrize("prec", [F32, F64])
@pytest.mark.parametrize("init", ["warm", "current"])
def test_accelerated_inner_solver(prec, init):
    """Accelerated Algorithm 2 (FISTA t-sequence) with 6 sub-iterations."""
    p = problem("small", **SMALL)
    xg, st, hist, stats, S = run_both(p, prec, 20, n_itr=6, inner_solver=ppd.PPD_INNER_FISTA,
                                      inner_init=ppd.PPD_INNER_CURRENT if init == "current" else ppd.PPD_INNER_WARM)
    assert rel(xg, st.x) <= TOL[prec]["img"], rel(xg, st.x)


@pytest.mark.parametrize("prec", [F32, F64])
def test_pd_special_case_and_graph_off(prec):
    p = problem("small", **SMALL)
    xg, st, hist, stats, S = run_both(p, prec, 25, precond=0, use_graph=0)
    assert rel(xg, st.x) <= TOL[prec]["img"], rel(xg, st.x)


def test_ppd_c2_fixed_iterations():
    p = problem("c2_512")
    P = nufft.Plan(p.omega, p.L, theta=p.theta)
    U = nufft.uniform_weights(p.omega, 2 * p.L, 2 * p.L)[0]
    eta = 1.0 / oppd.op_norm_sq(P, U, max_iter=8, tol=1e-3)[0]
    S = oppd.make_setup(p.omega, p.y, p.theta, p.block, p.n_blocks, p.L, eta=eta, x_true=p.x_true)
    st = oppd.init_state(S)
    for _ in range(5):
        hist = oppd.iterate(st, S)
    s = ppd.Solver(p.L, p.n_blocks, precision=F32, eta=eta)
    s.set_problem(p.omega, p.y, p.block, theta=p.theta, x_true=p.x_true)
    stats = s.iterate(5)
    assert rel(s.image(), st.x) <= 1e-4
    assert np.allclose(stats["block_residual"], hist["residual"], rtol=1e-4)
    s.close()


# ----------------------------------------------------------------- autograd
@pytest.mark.parametrize("prec", [F32, F64])
def test_phi_autograd_gradient(prec):
    from paper_1701_01748_gb300 import torch_ops
    p = problem("small", **SMALL)
    s = solver(p, prec, eta=1.0)
    P = nufft.Plan(p.omega, p.L, theta=p.theta)
    x0 = p.x_true
    yw = p.theta * p.y
    x = torch.tensor(x0, dtype=tdtype(prec), device="cuda", requires_grad=True)
    yt = torch.tensor(yw, dtype=torch.complex64 if prec == F32 else torch.complex128, device="cuda")
    loss = 0.5 * (torch_ops.phi(x, s) - yt).abs().pow(2).sum()
    loss.backward()
    g = x.grad.cpu().double().numpy()
    g_ref = nufft.phi_adjoint(nufft.phi(x0, P) - yw, P)
    assert rel(g, g_ref) <= (1e-5 if prec == F32 else 1e-10)
    # central finite differences of the oracle loss along random directions
    rng = np.random.default_rng(3)
    f = lambda z: 0.5 * float(np.sum(np.abs(nufft.phi(z, P) - yw) ** 2))
    for _ in range(3):
        dvec = rng.normal(size=x0.shape)
        h = 1e-4
        fd = (f(x0 + h * dvec) - f(x0 - h * dvec)) / (2 * h)
        assert abs(fd - float(np.sum(g * dvec))) <= 1e-3 * abs(fd)
    s.close()


# ----------------------------------------------------------------- errors
def test_error_codes():
    p = problem("small", **SMALL)
    s = ppd.Solver(p.L, p.n_blocks, precision=F32)
    with pytest.raises(ppd.PPDError) as e:
        ppd.ppd_set_weights(s.ctx)
    assert e.value.status == ppd.PPD_ERR_NOT_READY
    with pytest.raises(ppd.PPDError) as e:
        ppd.ppd_iterate(s.ctx, 1)
    assert e.value.status == ppd.PPD_ERR_NOT_READY
    bad = p.omega.copy()
    bad[3, 0] = 4.0
    with pytest.raises(ppd.PPDError) as e:
        ppd.ppd_set_visibilities(s.ctx, bad, p.y, p.block)
    assert e.value.status == ppd.PPD_ERR_INVALID_ARG
    ynan = p.y.copy()
    ynan[5] = np.nan
    with pytest.raises(ppd.PPDError) as e:
        ppd.ppd_set_visibilities(s.ctx, p.omega, ynan, p.block)
    assert e.value.status == ppd.PPD_ERR_INVALID_ARG
    blk = p.block.copy()
    blk[0] = p.n_blocks
    with pytest.raises(ppd.PPDError) as e:
        ppd.ppd_set_visibilities(s.ctx, p.omega, p.y, blk)
    assert e.value.status == ppd.PPD_ERR_INVALID_ARG
    ppd.ppd_set_visibilities(s.ctx, p.omega, p.y, p.block)
    with pytest.raises(ppd.PPDError) as e:
        ppd.ppd_set_weights(s.ctx, theta=-np.ones(p.M))
    assert e.value.status == ppd.PPD_ERR_INVALID_ARG
    ppd.ppd_set_weights(s.ctx, theta=p.theta)
    out = s.iterate(2)
    assert out["iters_done"] == 2 and math.isfinite(out["rel_var"])
    s.close()


# ----------------------------------------------------------------- checkpoint / resume
@pytest.mark.parametrize("prec", [F32, F64])
def test_state_resume_is_bit_identical(prec):
    p = problem("small", **SMALL)
    s = solver(p, prec)                      # eta by the library's power iteration
    s.iterate(7)
    blob = ppd.ppd_get_state(s.ctx)
    s.iterate(9)
    x_run = s.image()
    ppd.ppd_set_state(s.ctx, blob)
    out = s.iterate(9)
    assert out["iters_done"] == 16
    assert np.array_equal(s.image(), x_run)
    # a blob for another configuration is refused
    s2 = solver(problem("c1_128"), prec, eta=1.0)
    with pytest.raises(ppd.PPDError) as e:
        ppd.ppd_set_state(s2.ctx, blob)
    assert e.value.status == ppd.PPD_ERR_INVALID_ARG
    s2.close()
    s.close()


# ----------------------------------------------------------------- autotuner
def test_autotune_picks_a_candidate_and_keeps_parity():
    p = problem("small", **SMALL)
    S = oppd.make_setup(p.omega, p.y, p.theta, p.block, p.n_blocks, p.L, power_iters=400, x_true=p.x_true)
    s = ppd.Solver(p.L, p.n_blocks, precision=F32, eta=S.eta)
    s.set_problem(p.omega, p.y, p.block, theta=p.theta, x_true=p.x_true)
    tile, chunk = ppd.ppd_autotune(s.ctx, 3)
    prm = s.params()
    assert tile in (16, 32) and chunk in (512, 1024, 2048)
    assert prm["grid_warps"] in (4, 8) and prm["degrid_threads"] in (128, 256)
    assert prm["tile"] == tile and prm["chunk"] == chunk and abs(prm["eta"] - S.eta) <= 1e-12 * S.eta
    st = oppd.init_state(S)
    for _ in range(10):
        oppd.iterate(st, S)
    s.iterate(10)
    assert rel(s.image(), st.x) <= 1e-4
    perm, _, _, _ = ppd.ppd_get_bins(s.ctx, p.M)
    assert np.array_equal(perm, nufft.visibility_order(p.omega, p.block, 2 * p.L, 2 * p.L, tile)[0])
    s.close()


@pytest.mark.parametrize("warps,dthreads", [(4, 128), (8, 256), (4, 256), (8, 128)])
@pytest.mark.parametrize("tile", [16, 32])
def test_gridding_and_degridding_cta_shapes(warps, dthreads, tile):
    """Four or eight warps per gridding CTA (each warp a slice of the chunk),
    128 or 256 threads per degridding CTA: the same operators and iterates as
    the oracle."""
    p = problem("small", **SMALL)
    S = oppd.make_setup(p.omega, p.y, p.theta, p.block, p.n_blocks, p.L, power_iters=400, x_true=p.x_true)
    s = solver(p, F32, eta=S.eta, grid_warps=warps, degrid_threads=dthreads, tile=tile, chunk=512)
    assert s.params()["grid_warps"] == warps and s.params()["degrid_threads"] == dthreads
    P = nufft.Plan(p.omega, p.L, theta=p.theta)
    x = np.random.default_rng(11).random((p.L, p.L))
    assert rel(op_forward(s, x, F32), nufft.phi(x, P)) <= TOL[F32]["op"]
    yv = np.random.default_rng(12).normal(size=p.M) + 1j * np.random.default_rng(13).normal(size=p.M)
    assert rel(op_adjoint(s, yv, F32), nufft.phi_adjoint(yv, P)) <= TOL[F32]["op"]
    st = oppd.init_state(S)
    for _ in range(8):
        oppd.iterate(st, S)
    s.iterate(8)
    assert rel(s.image(), st.x) <= TOL[F32]["img"]
    s.close()


def test_cta_shape_values_are_checked():
    for prec, kw in ((F32, dict(grid_warps=6)), (F64, dict(grid_warps=8)), (F32, dict(grid_warps=-4)),
                     (F32, dict(degrid_threads=64)), (F64, dict(degrid_threads=128))):
        with pytest.raises(ppd.PPDError) as e:
            ppd.Solver(32, 1, precision=prec, **kw)
        assert e.value.status == ppd.PPD_ERR_INVALID_ARG


# ----------------------------------------------------------------- batched group
def test_group_matches_individual_runs():
    probs = [synth.make_problem("grp", L=L, M=M, n_blocks=d, uv_sigma=0.15, seed=40 + i, n_points=6, n_blobs=1)
             for i, (L, M, d) in enumerate([(32, 3000, 2), (64, 9000, 4), (32, 2000, 3)])]
    solo, grouped = [], []
    for p in probs:
        a = ppd.Solver(p.L, p.n_blocks, precision=F32)   # eta by power iteration, shared below
        a.set_problem(p.omega, p.y, p.block, theta=p.theta)
        eta = a.params()["eta"]
        a.close()
        for dest in (solo, grouped):
            s = ppd.Solver(p.L, p.n_blocks, precision=F32, eta=eta)
            s.set_problem(p.omega, p.y, p.block, theta=p.theta)
            dest.append(s)
    for s in solo:
        s.iterate(12, stats=False)
    g = ppd.ppd_group_create([s.ctx for s in grouped])
    ppd.ppd_group_iterate(g, 5)
    ppd.ppd_group_iterate(g, 7)
    ppd.ppd_group_destroy(g)
    for a, b in zip(solo, grouped):
        assert b.iterate(0)["iters_done"] == 12
        assert np.array_equal(a.image(), b.image())
        a.close()
        b.close()
