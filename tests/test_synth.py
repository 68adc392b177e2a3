"""The seeded input generator: shapes, seeds and the u-v samplers."""
import math

import numpy as np

from paper_1701_01748_gb300 import synth


def test_problem_is_reproducible_and_well_formed():
    a = synth.make_problem("t", L=32, M=500, n_blocks=3, uv_sigma=0.2, seed=3, n_points=4, n_blobs=1)
    b = synth.make_problem("t", L=32, M=500, n_blocks=3, uv_sigma=0.2, seed=3, n_points=4, n_blobs=1)
    assert np.array_equal(a.y, b.y) and np.array_equal(a.omega, b.omega)
    assert a.x_true.min() >= 0 and a.omega.shape == (500, 2)
    assert np.all((a.omega >= -math.pi) & (a.omega < math.pi))
    assert set(np.unique(a.block)) <= {0, 1, 2}


def test_exact_visibilities_match_a_direct_sum():
    rng = np.random.default_rng(1)
    pts, blob = synth.sky_image(16, rng, n_points=3, n_blobs=1)
    x = blob.copy()
    for p0, p1, f in pts:
        x[p0, p1] += f
    om = rng.uniform(-math.pi, math.pi, size=(40, 2))
    n = np.arange(16) - 8
    direct = np.array([np.sum(x * np.exp(-1j * (w0 * n[:, None] + w1 * n[None, :]))) for w0, w1 in om])
    assert np.abs(synth.exact_visibilities(pts, blob, om) - direct).max() <= 1e-12 * np.abs(direct).max()


def test_ggd_sampler_shape():
    rng = np.random.default_rng(2)
    g2 = synth.sample_uv_ggd(100000, 2.0, 0.15, rng)
    assert abs(g2.std() / math.pi - 0.15) < 0.005          # beta = 2 is the Gaussian of that std
    centre = [np.mean(np.abs(synth.sample_uv_ggd(50000, b, 0.15, rng)) < 0.05 * math.pi) for b in (2.0, 0.5, 0.25)]
    assert centre[0] < centre[1] < centre[2]                # smaller beta: denser centre


def test_compact_blobs_analytic_spectra_match_the_exact_sum():
    """For compact blobs (L >= 256) the analytic Gaussian spectra equal the exact
    pixel sum (truncated SVD route) to ~1e-8."""
    rng = np.random.default_rng(77)
    L = 256
    params = []
    points, blob = synth.sky_image(L, rng, n_points=3, n_blobs=3, compact=True, params_out=params)
    omega = rng.uniform(-np.pi, np.pi, size=(1500, 2))
    exact = synth.exact_visibilities(points, blob, omega)
    fast = synth.point_visibilities(points, omega, L) + synth.gaussian_visibilities(params, omega, L)
    assert np.linalg.norm(fast - exact) <= 1e-8 * np.linalg.norm(exact)


def test_batch_shapes_stay_in_their_ranges():
    probs = synth.make_batch(6, seed=9, sides=(16, 32), ratio=(2.0, 8.0), blocks=(2, 5))
    assert {p.L for p in probs} <= {16, 32}
    for p in probs:
        assert 2.0 * p.L ** 2 - 1 <= p.M <= 8.0 * p.L ** 2 + 1
        assert 2 <= p.n_blocks <= 5 and p.block.max() < p.n_blocks


def test_splitmix64_published_outputs_and_power_start():
    """SplitMix64 from state 0 gives 0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4
    (the generator's published first outputs); power_start draws in [0.5, 1.5)
    before normalisation and is all ones for seed 0."""
    import numpy as np
    g = np.uint64(0x9E3779B97F4A7C15)
    with np.errstate(over="ignore"):
        out = synth.splitmix64(np.array([g, g * np.uint64(2)], dtype=np.uint64))
    assert [int(v) for v in out] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4]
    x = synth.power_start(8, 6, 1234)
    assert x.shape == (8, 6) and abs(np.linalg.norm(x) - 1.0) < 1e-15
    r = x / x.max()
    assert r.min() > 0.5 / 1.5 - 1e-12
    assert np.array_equal(synth.power_start(4, 4, 0), np.full((4, 4), 0.25))


def test_batch_sides_are_five_smooth_multiples_of_16():
    """The batched workload's sides: log-uniform draws rounded to the nearest
    16 * 2^a 3^b 5^c, so every oversampled grid side 2 L is 5-smooth."""
    assert synth.smooth_sides(256, 1024) == [256, 288, 320, 384, 400, 432, 480, 512, 576, 640, 720, 768, 800,
                                             864, 960, 1024]
    probs = synth.make_batch(5, seed=3, side_range=(16, 96), ratio=(2.0, 3.0), blocks=(2, 3))
    for p in probs:
        assert p.L in synth.smooth_sides(16, 96) and p.x_true.shape == (p.L, p.L)
        assert 2 * p.L * p.L <= p.M <= 3 * p.L * p.L + 1


def test_rectangular_problem_data_are_the_exact_measurement():
    """An L x L1 problem: noise-free data equal the direct DTFT of the pixel sky."""
    import numpy as np
    from oracle import nufft
    p = synth.make_problem("rect", L=32, L1=48, M=300, n_blocks=2, uv_sigma=0.3, seed=4, isnr_db=300.0)
    assert p.x_true.shape == (32, 48) and p.L1 == 48
    y = nufft.nudft(p.x_true, p.omega)
    assert np.abs(p.y - y).max() <= 1e-9 * np.abs(y).max()
