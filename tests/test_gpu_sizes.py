"""Image sizes beyond square powers of two: any sides n0, n1 that are
multiples of 16 whose oversampled grid sides 2 n0, 2 n1 have no prime factor
above 5 (the mixed-radix FFT passes), square or not.  CUDA path against the
FP64 oracle through the C ABI, with the tolerances of the other parity tests
(relative l2: operators 1e-5 FP32 / 1e-10 FP64, image after a fixed number
of iterations 1e-4 / 1e-8; binning and order bit-exact)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import nufft, ppd as oppd, sara  # noqa: E402
from paper_1701_01748_gb300 import build, ppd, synth  # noqa: E402

pytestmark = pytest.mark.gpu

F32, F64 = ppd.PPD_FP32_FP64NORMS, ppd.PPD_FP64_PLAIN
TOL = {F32: dict(op=1e-5, img=1e-4), F64: dict(op=1e-10, img=1e-8)}
# (rows, columns): K = 96 x 160 (2^5 3, 2^5 5), a non-square power-of-two grid,
# 480^2 (K = 960 = 2^6 3 5, several tiles and strips), 16 x 240 (one SARA
# tile along the rows, 3 x 5 x 32 along the columns)
SIZES = [(48, 80), (64, 128), (480, 480), (16, 240)]


@pytest.fixture(scope="session", autouse=True)
def lib():
    build.build()
    assert torch.cuda.is_available()
    return ppd._lib()


_cache = {}


def problem(L0, L1, M=None, n_blocks=3):
    key = (L0, L1, M, n_blocks)
    if key not in _cache:
        M = M or min(4 * L0 * L1, 200000)
        _cache[key] = synth.make_problem("sizes", L=L0, L1=L1, M=M, n_blocks=n_blocks, uv_sigma=0.2,
                                         seed=21 + L0 + 7 * L1, n_points=6, n_blobs=1)
    return _cache[key]


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def tdtype(prec):
    return torch.float32 if prec == F32 else torch.float64


def solver(p, prec, **cfg):
    s = ppd.Solver(p.L, p.n_blocks, precision=prec, L1=p.L1, **cfg)
    s.set_problem(p.omega, p.y, p.block, theta=p.theta, x_true=p.x_true)
    return s


def stream():
    return torch.cuda.current_stream().cuda_stream


@pytest.mark.parametrize("shape", SIZES)
def test_bins_and_order_bit_exact(shape):
    p = problem(*shape)
    s = ppd.Solver(p.L, p.n_blocks, precision=F32, L1=p.L1)
    ppd.ppd_set_visibilities(s.ctx, p.omega, p.y, p.block)
    perm, b0, b1, cnt = ppd.ppd_get_bins(s.ctx, p.M)
    K0, K1 = 2 * p.L, 2 * p.L1
    ob0, ob1, _, _ = nufft.base_cells(p.omega, K0, K1)
    _, ocnt = nufft.uniform_weights(p.omega, K0, K1)
    assert np.array_equal(b0, ob0) and np.array_equal(b1, ob1) and np.array_equal(cnt, ocnt)
    assert np.array_equal(perm, nufft.visibility_order(p.omega, p.block, K0, K1, 16)[0])
    s.close()


@pytest.mark.parametrize("prec", [F32, F64])
@pytest.mark.parametrize("shape", SIZES)
def test_phi_adjoint_and_psi(prec, shape):
    p = problem(*shape)
    s = solver(p, prec, eta=1.0)
    P = nufft.Plan(p.omega, p.L, p.L1, theta=p.theta)
    rng = np.random.default_rng(5)
    x = rng.random((p.L, p.L1))
    xd = torch.tensor(x, dtype=tdtype(prec), device="cuda")
    yd = torch.empty((p.M, 2), dtype=tdtype(prec), device="cuda")
    ppd.ppd_op_forward(s.ctx, xd.data_ptr(), yd.data_ptr(), stream())
    torch.cuda.synchronize()
    y_gpu = yd.cpu().double().numpy() @ np.array([1.0, 1j])
    assert rel(y_gpu, nufft.phi(x, P)) <= TOL[prec]["op"]
    yv = rng.normal(size=p.M) + 1j * rng.normal(size=p.M)
    yd = torch.tensor(np.stack([yv.real, yv.imag], 1), dtype=tdtype(prec), device="cuda")
    gd = torch.empty((p.L, p.L1), dtype=tdtype(prec), device="cuda")
    ppd.ppd_op_adjoint(s.ctx, yd.data_ptr(), gd.data_ptr(), stream())
    torch.cuda.synchronize()
    g = gd.cpu().double().numpy()
    assert rel(g, nufft.phi_adjoint(yv, P)) <= TOL[prec]["op"]
    a, b = float(np.vdot(y_gpu, yv).real), float(np.sum(x * g))
    assert abs(a - b) <= TOL[prec]["op"] * abs(a)          # adjoint identity of the GPU operators
    # SARA analysis and synthesis
    cd = torch.empty((9, p.L, p.L1), dtype=tdtype(prec), device="cuda")
    ppd.ppd_psi_analysis(s.ctx, xd.data_ptr(), cd.data_ptr(), stream())
    torch.cuda.synchronize()
    assert rel(cd.cpu().double().numpy(), sara.psi_adjoint(x)) <= TOL[prec]["op"]
    u = rng.normal(size=(9, p.L, p.L1))
    ud = torch.tensor(u, dtype=tdtype(prec), device="cuda")
    ppd.ppd_psi_synthesis(s.ctx, ud.data_ptr(), xd.data_ptr(), stream())
    torch.cuda.synchronize()
    assert rel(xd.cpu().double().numpy(), sara.psi(u)) <= TOL[prec]["op"]
    s.close()


@pytest.mark.parametrize("prec", [F32, F64])
@pytest.mark.parametrize("shape,iters", [((48, 80), 30), ((16, 240), 20), ((480, 480), 5)])
def test_ppd_trajectory(prec, shape, iters):
    p = problem(*shape)
    S = oppd.make_setup(p.omega, p.y, p.theta, p.block, p.n_blocks, p.L, L1=p.L1, power_iters=60,
                        x_true=p.x_true, n_itr=2)
    s = solver(p, prec, eta=S.eta, n_itr=2)
    st = oppd.init_state(S)
    for _ in range(iters):
        h = oppd.iterate(st, S)
    out = s.iterate(iters)
    assert rel(s.image(), st.x) <= TOL[prec]["img"], rel(s.image(), st.x)
    assert np.allclose(out["block_residual"], h["residual"], rtol=1e-4)
    s.close()


def test_unsupported_sizes_are_refused():
    for n0, n1 in ((112, 112), (64, 56), (40, 64), (4112, 64)):   # 2 x 112 = 2^5 7; 56, 40 not multiples of 16
        cfg = ppd.ppd_config_default(n0=n0, n1=n1)
        with pytest.raises(ppd.PPDError) as e:
            ppd.ppd_create(cfg)
        assert e.value.status == ppd.PPD_ERR_UNSUPPORTED


def test_contexts_of_different_sizes_share_the_mixed_radix_kernels():
    """Two contexts whose row passes take the mixed-radix kernels with more
    than 48 KB of shared memory each (K1 = 3840, then 3200): the second
    context's set-up must not lower the limit the first one's launches need
    (the shared-memory attribute is one value per kernel)."""
    big = problem(16, 1920, M=3000, n_blocks=2)
    small = problem(16, 1600, M=3000, n_blocks=2)
    a = solver(big, F32, eta=1.0)
    b = solver(small, F32, eta=1.0)
    for s, p in ((a, big), (b, small), (a, big)):
        P = nufft.Plan(p.omega, p.L, p.L1, theta=p.theta)
        rng = np.random.default_rng(6)
        x = rng.random((p.L, p.L1))
        xd = torch.tensor(x, dtype=torch.float32, device="cuda")
        yd = torch.empty((p.M, 2), dtype=torch.float32, device="cuda")
        ppd.ppd_op_forward(s.ctx, xd.data_ptr(), yd.data_ptr(), stream())
        torch.cuda.synchronize()
        y = yd.cpu().double().numpy() @ np.array([1.0, 1j])
        assert rel(y, nufft.phi(x, P)) <= TOL[F32]["op"]
        yv = rng.normal(size=p.M) + 1j * rng.normal(size=p.M)
        yd = torch.tensor(np.stack([yv.real, yv.imag], 1), dtype=torch.float32, device="cuda")
        gd = torch.empty((p.L, p.L1), dtype=torch.float32, device="cuda")
        ppd.ppd_op_adjoint(s.ctx, yd.data_ptr(), gd.data_ptr(), stream())
        torch.cuda.synchronize()
        assert rel(gd.cpu().double().numpy(), nufft.phi_adjoint(yv, P)) <= TOL[F32]["op"]
    a.close()
    b.close()
