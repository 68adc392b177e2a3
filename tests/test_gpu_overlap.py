"""Overlapped launches change no result.

With launch_overlap = 1 a kernel of the iteration may start while the
kernel before it in its stream drains (programmatic dependent launch); with
launch_overlap = 0 (the default) every kernel waits for its predecessor.  The
arithmetic is the same, so the iterates, the statistics, the operators and
the SARA transforms must be bit-identical both ways, in the captured graph
and without it, on the power-of-two and on the mixed-radix FFT path.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1701_01748_gb300 import build, ppd, synth  # noqa: E402

pytestmark = pytest.mark.gpu

F32, F64 = ppd.PPD_FP32_FP64NORMS, ppd.PPD_FP64_PLAIN
CASES = {
    "pow2": dict(L=128, M=60000, n_blocks=6, uv_sigma=0.2, seed=21, n_points=10, n_blobs=2),
    "mixed": dict(L=48, L1=80, M=9000, n_blocks=3, uv_sigma=0.3, seed=22, n_points=6, n_blobs=1),
}


@pytest.fixture(scope="session", autouse=True)
def lib():
    build.build()
    assert torch.cuda.is_available()
    return ppd._lib()


def tdtype(prec):
    return torch.float32 if prec == F32 else torch.float64


def run(p, prec, overlap, graph):
    s = ppd.Solver(p.L, p.n_blocks, precision=prec, L1=p.L1, n_itr=3, use_graph=graph,
                   launch_overlap=overlap)
    s.set_problem(p.omega, p.y, p.block, theta=p.theta, x_true=p.x_true)
    eta = s.params()["eta"]
    hist = [s.iterate(4) for _ in range(3)]
    img = s.image()
    dev = torch.cuda.current_stream().cuda_stream
    rng = np.random.default_rng(3)
    x = torch.tensor(rng.random((p.L, p.L1)), dtype=tdtype(prec), device="cuda")
    y = torch.empty((s.M, 2), dtype=tdtype(prec), device="cuda")
    ppd.ppd_op_forward(s.ctx, x.data_ptr(), y.data_ptr(), dev)
    g = torch.empty_like(x)
    ppd.ppd_op_adjoint(s.ctx, y.data_ptr(), g.data_ptr(), dev)
    c = torch.empty((9, p.L, p.L1), dtype=tdtype(prec), device="cuda")
    ppd.ppd_psi_analysis(s.ctx, x.data_ptr(), c.data_ptr(), dev)
    xs = torch.empty_like(x)
    ppd.ppd_psi_synthesis(s.ctx, c.data_ptr(), xs.data_ptr(), dev)
    torch.cuda.synchronize()
    out = dict(eta=eta, hist=hist, img=img, y=y.cpu().numpy(), g=g.cpu().numpy(), c=c.cpu().numpy(),
               xs=xs.cpu().numpy())
    s.close()
    return out


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("graph", [1, 0])
@pytest.mark.parametrize("prec", [F32, F64])
def test_overlapped_launches_are_bit_identical(case, graph, prec):
    p = synth.make_problem(case, **CASES[case])
    a = run(p, prec, overlap=0, graph=graph)
    b = run(p, prec, overlap=1, graph=graph)
    assert a["eta"] == b["eta"]
    for key in ("img", "y", "g", "c", "xs"):
        assert np.array_equal(a[key], b[key]), key
    for ha, hb in zip(a["hist"], b["hist"]):
        for k in ha:
            assert np.array_equal(np.asarray(ha[k]), np.asarray(hb[k])), k


def test_launch_overlap_flag_is_checked():
    with pytest.raises(ppd.PPDError):
        ppd.Solver(32, 1, launch_overlap=2)
