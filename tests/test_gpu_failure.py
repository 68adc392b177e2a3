"""Failure detection of the bounded device waits, without a GPU fault.

The degridding kernel's wait for each TMA tile copy is bounded.  The test
shortens the first wait of every tile to zero polls (ppd_set_wait_limit), so
that wait runs out while the copy is still in flight; the kernel records the
timeout in the device error word, waits for its copies under the normal bound
and leaves.  The host must report PPD_ERR_TIMEOUT, and the context must give
the same results as a fresh one once the limit is back to its default.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1701_01748_gb300 import build, ppd, synth  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="session", autouse=True)
def lib():
    build.build()
    assert torch.cuda.is_available()
    return ppd._lib()


def test_bounded_tma_wait_reports_a_timeout_and_the_context_recovers():
    p = synth.make_problem("wait", L=64, M=8000, n_blocks=2, uv_sigma=0.2, seed=31, n_points=5, n_blobs=1)
    ref = ppd.Solver(p.L, p.n_blocks, precision=ppd.PPD_FP32_FP64NORMS)
    ref.set_problem(p.omega, p.y, p.block, theta=p.theta)
    eta = ref.params()["eta"]
    assert ref.params()["K0"] == 128   # 16 x 16 tiles with 24 x 24 TMA boxes: most tiles are interior
    ref.iterate(5, stats=False)
    s = ppd.Solver(p.L, p.n_blocks, precision=ppd.PPD_FP32_FP64NORMS, eta=eta)
    s.set_problem(p.omega, p.y, p.block, theta=p.theta)
    zero = ppd.ppd_get_state(s.ctx)
    ppd.ppd_set_wait_limit(s.ctx, 0)
    with pytest.raises(ppd.PPDError) as e:
        s.iterate(2)
    assert e.value.status == ppd.PPD_ERR_TIMEOUT
    ppd.ppd_set_wait_limit(s.ctx, ppd.PPD_WAIT_LIMIT_DEFAULT)
    ppd.ppd_set_state(s.ctx, zero)
    out = s.iterate(5)                  # no error, same trajectory as the fresh context
    assert out["iters_done"] == 5
    assert np.array_equal(s.image(), ref.image())
    with pytest.raises(ppd.PPDError) as e:
        ppd.ppd_set_wait_limit(s.ctx, -1)
    assert e.value.status == ppd.PPD_ERR_INVALID_ARG
    s.close()
    ref.close()
