"""ppd_op_adjoint_noalloc: Phi^dagger for callers that cannot let the library
allocate device memory during a call (fixed memory budgets reserved at
start-up, real-time loops that must not block on the allocator).  Its output
must match ppd_op_adjoint on consecutive calls; problems whose gridding
scratch exceeds the fixed array are refused with a clear error.

This file is collected last so that a run stopping at the first failure has
already run every other test; it also passes alone in a fresh process.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1701_01748_gb300 import build, ppd, synth  # noqa: E402

pytestmark = pytest.mark.gpu

TOL = {ppd.PPD_FP32_FP64NORMS: 1e-5, ppd.PPD_FP64_PLAIN: 1e-10}


@pytest.fixture(scope="module", autouse=True)
def lib():
    build.build()
    assert torch.cuda.is_available()
    return ppd._lib()


def _adjoint(fn, s, y, dt):
    yd = torch.tensor(np.stack([y.real, y.imag], 1), dtype=dt, device="cuda")
    xd = torch.empty((s.L, s.L), dtype=dt, device="cuda")
    fn(s.ctx, yd.data_ptr(), xd.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return xd.cpu().double().numpy()


@pytest.mark.parametrize("prec", [ppd.PPD_FP32_FP64NORMS, ppd.PPD_FP64_PLAIN])
def test_noalloc_adjoint_matches_adjoint_on_two_calls(prec):
    p = synth.make_problem("noalloc", L=64, M=20000, n_blocks=4, uv_sigma=0.2, seed=21, n_points=8, n_blobs=2)
    s = ppd.Solver(p.L, p.n_blocks, precision=prec, eta=1.0)
    s.set_problem(p.omega, p.y, p.block, theta=p.theta)
    dt = torch.float32 if prec == ppd.PPD_FP32_FP64NORMS else torch.float64
    rng = np.random.default_rng(5)
    for call in range(2):
        y = rng.normal(size=p.M) + 1j * rng.normal(size=p.M)
        got = _adjoint(ppd.ppd_op_adjoint_noalloc, s, y, dt)
        ref = _adjoint(ppd.ppd_op_adjoint, s, y, dt)
        err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert err <= TOL[prec], (call, err)
    s.close()


def test_noalloc_refuses_problems_beyond_its_scratch():
    p = synth.make_problem("noalloc_big", L=64, M=60000, n_blocks=1, uv_sigma=0.2, seed=22, n_points=4, n_blobs=1)
    s = ppd.Solver(p.L, 1, precision=ppd.PPD_FP32_FP64NORMS, eta=1.0, chunk=16, tile=32)
    s.set_problem(p.omega, p.y, p.block, theta=p.theta)
    E = s.params()["tile"] + 8
    assert s.params()["n_chunks"] * E * E * 8 > 32 * 2 ** 20
    y = np.ones(p.M, np.complex128)
    with pytest.raises(ppd.PPDError) as e:
        _adjoint(ppd.ppd_op_adjoint_noalloc, s, y, torch.float32)
    assert e.value.status == ppd.PPD_ERR_UNSUPPORTED
    assert "scratch" in ppd.ppd_last_error()
    s.close()
