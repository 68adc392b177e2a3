"""Seeded synthetic radio-interferometric problems.

This module makes the *inputs* of the imaging problem and nothing else: a
positive sky image, the u-v sampling, the data-block split, the noisy
visibilities and the noise level.  It holds none of the solver's arithmetic
(no interpolation kernel, no oversampled FFT, no preconditioner, no bound on
the noise norm), so the FP64 oracle and the CUDA library can both be fed from
it without sharing any of the method.

Visibilities are the exact measurement of the pixelised sky,
``y_m = sum_n x[n] exp(-i <omega_m, n - L/2>)`` (the discretised measurement
equation of Section 2, with DDEs ignored as in the paper's simulations),
plus circular complex Gaussian noise whose power is set from the noise-free
signal power for a given input SNR (Section 5, "iSNR").  The sum is evaluated
exactly: point sources one by one, the smooth Gaussian blobs through a
truncated SVD of their pixel image (the DTFT is separable per rank-one term).

The shapes stand in for the paper's workloads (its images and coverages are
not available): point sources plus elliptical Gaussian blobs for the sky, a
Gaussian u-v density (the paper's generalised Gaussian with shape 2) whose
width sets how non-uniform the sampling is, and radial u-v bands as uneven
data blocks.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = ["Problem", "CONFIGS", "make_problem", "make_batch", "make_batch32", "sky_image", "sample_uv",
           "sample_uv_ggd", "radial_blocks", "exact_visibilities", "gaussian_visibilities",
           "point_visibilities", "active_sets", "power_start", "splitmix64", "smooth_sides"]


@dataclasses.dataclass
class Problem:
    """One synthetic imaging problem (all arrays FP64 / int32, host)."""
    name: str
    L: int                    # image rows (an L x L1 image)
    x_true: np.ndarray        # (L, L1) float64, >= 0
    omega: np.ndarray         # (M, 2) float64 in [-pi, pi); col 0 -> image rows
    y: np.ndarray             # (M,) complex128, raw (un-whitened) visibilities
    sigma: float              # noise standard deviation of each complex visibility
    theta: np.ndarray         # (M,) float64 natural weights 1/sigma_e
    block: np.ndarray         # (M,) int32 data-block id in [0, n_blocks)
    n_blocks: int
    isnr_db: float
    seed: int
    L1: int | None = None     # image columns (None: square, L1 = L)

    def __post_init__(self):
        if self.L1 is None:
            self.L1 = self.L

    @property
    def M(self) -> int:
        return int(self.omega.shape[0])


# Workload shapes.  uv_sigma is the std of omega per axis in units of pi.
CONFIGS = {
    # 128x128, 8192 visibilities, one block, broad Gaussian coverage
    "c1_128": dict(L=128, M=8192, n_blocks=1, uv_sigma=0.25, seed=1701),
    # 512x512, 524288 visibilities, strongly non-uniform, 16 radial blocks
    "c2_512": dict(L=512, M=524288, n_blocks=16, uv_sigma=0.1, seed=1702),
    # 1024x1024, 4M visibilities, 64 radial blocks
    "c3_1024": dict(L=1024, M=4194304, n_blocks=64, uv_sigma=0.1, seed=1703),
    # 4096x4096, 64M visibilities, 256 radial blocks (compact blobs, analytic blob spectra)
    "c5_4096": dict(L=4096, M=67108864, n_blocks=256, uv_sigma=0.1, seed=1705, compact=True),
    # the 4096x4096 image with 8M visibilities: the 4096^2 workload at a size a
    # multi-pass profiler capture can replay (visibility-side traffic scales with M)
    "c5m8_4096": dict(L=4096, M=8388608, n_blocks=256, uv_sigma=0.1, seed=1705, compact=True),
}


def sky_image(L: int, rng: np.random.Generator, n_points: int = 20,
              n_blobs: int = 3, compact: bool = False, params_out: list | None = None,
              L1: int | None = None):
    """Positive test sky: point sources plus elliptical Gaussian blobs.

    Returns (points, blob_image): points is a list of (row, col, flux) with
    integer pixel positions (collisions add), blob_image is (L, L) float64.
    Point fluxes are log-uniform in [1e-3, 1]; blob centres uniform in the
    central half, major-axis std uniform in [0.02L, 0.08L], axis ratio uniform
    in [0.3, 1], position angle uniform in [0, pi), peak log-uniform in
    [1e-2, 1e-1].  compact=True keeps every blob at least 6 standard
    deviations inside the image (centres in [0.3L, 0.7L], major-axis std in
    [0.03L, 0.05L]) so that its spectrum is the analytic Gaussian one to
    ~1e-8 (see gaussian_visibilities); the draws are the same.  L1 (default
    L) gives an L x L1 image: positions and centres scale with each axis,
    blob widths with the shorter side.  params_out,
    if given, receives (c0, c1, smaj, smin, angle, peak) per blob.
    """
    L1 = L if L1 is None else L1
    if L1 == L:
        pos = rng.integers(0, L, size=(n_points, 2))
    else:
        pos = np.stack([rng.integers(0, L, size=n_points), rng.integers(0, L1, size=n_points)], axis=1)
    flux = 10.0 ** rng.uniform(-3.0, 0.0, size=n_points)
    points = [(int(p[0]), int(p[1]), float(f)) for p, f in zip(pos, flux)]
    R0, R1 = np.meshgrid(np.arange(L, dtype=np.float64), np.arange(L1, dtype=np.float64), indexing="ij")
    blob = np.zeros((L, L1))
    Ls = min(L, L1)
    clo, chi = (0.3 * L, 0.7 * L) if compact else (L / 4, 3 * L / 4)
    slo, shi = (0.03 * Ls, 0.05 * Ls) if compact else (0.02 * Ls, 0.08 * Ls)
    for _ in range(n_blobs):
        if L1 == L:
            c0, c1 = rng.uniform(clo, chi, size=2)
        else:
            f0, f1 = (0.3, 0.7) if compact else (0.25, 0.75)
            c0, c1 = rng.uniform(f0, f1, size=2) * np.array([L, L1], dtype=np.float64)
        smaj = rng.uniform(slo, shi)
        smin = smaj * rng.uniform(0.3, 1.0)
        ang = rng.uniform(0.0, math.pi)
        peak = 10.0 ** rng.uniform(-2.0, -1.0)
        if params_out is not None:
            params_out.append((c0, c1, smaj, smin, ang, peak))
        ca, sa = math.cos(ang), math.sin(ang)
        d0, d1 = R0 - c0, R1 - c1
        a = ca * d0 + sa * d1
        b = -sa * d0 + ca * d1
        blob += peak * np.exp(-0.5 * ((a / smaj) ** 2 + (b / smin) ** 2))
    return points, blob


def sample_uv(M: int, uv_sigma: float, rng: np.random.Generator) -> np.ndarray:
    """omega ~ N(0, (uv_sigma*pi)^2) per axis, redrawn until inside [-pi, pi)^2."""
    out = np.empty((0, 2))
    while out.shape[0] < M:
        need = M - out.shape[0]
        s = rng.normal(0.0, uv_sigma * math.pi, size=(need + need // 8 + 16, 2))
        ok = np.all((s >= -math.pi) & (s < math.pi), axis=1)
        out = np.concatenate([out, s[ok]], axis=0)
    return np.ascontiguousarray(out[:M])


def sample_uv_ggd(M: int, beta: float, std: float, rng: np.random.Generator) -> np.ndarray:
    """omega per axis from a zero-mean generalised Gaussian, density ~ exp(-|w/a|^beta),
    scaled to standard deviation std*pi (Section 5's GGD coverages; beta = 2 is
    Gaussian, smaller beta concentrates the samples at the centre), redrawn
    until inside [-pi, pi)^2.  |w/a|^beta ~ Gamma(1/beta) with a random sign."""
    a = std * math.pi * math.sqrt(math.gamma(1.0 / beta) / math.gamma(3.0 / beta))
    out = np.empty((0, 2))
    while out.shape[0] < M:
        need = M - out.shape[0] + 16
        g = rng.gamma(1.0 / beta, 1.0, size=(need, 2)) ** (1.0 / beta)
        sgn = np.where(rng.random(size=(need, 2)) < 0.5, -1.0, 1.0)
        w = a * sgn * g
        ok = np.all((w >= -math.pi) & (w < math.pi), axis=1)
        out = np.concatenate([out, w[ok]], axis=0)
    return np.ascontiguousarray(out[:M])


def radial_blocks(omega: np.ndarray, n_blocks: int) -> np.ndarray:
    """Uneven data blocks: equal-width radial bands of |omega| (FP64)."""
    r = np.hypot(omega[:, 0], omega[:, 1])
    rmax = float(r.max()) if r.size else 1.0
    b = np.floor(n_blocks * r / rmax).astype(np.int64)
    return np.minimum(b, n_blocks - 1).astype(np.int32)


def _phase_rows(w: np.ndarray, L: int) -> np.ndarray:
    """exp(-i w (n - L/2)) for n = 0..L-1, as an (m, L) array.

    Built as an outer product of a coarse and a fine factor (n = S*a + b) so
    that only m*(L/S + S) complex exponentials are evaluated.
    """
    S = 32 if L % 32 == 0 else 1
    a = np.arange(L // S, dtype=np.float64) * S
    b = np.arange(S, dtype=np.float64)
    A = np.exp(-1j * w[:, None] * (a[None, :] - L / 2))
    B = np.exp(-1j * w[:, None] * b[None, :])
    return (A[:, :, None] * B[:, None, :]).reshape(w.shape[0], L)


def exact_visibilities(points, blob: np.ndarray, omega: np.ndarray,
                       chunk: int = 8192) -> np.ndarray:
    """Exact y_m = sum_n x[n] exp(-i <omega_m, n - L/2>) of the pixel sky (L = (L0, L1))."""
    L0, L1 = blob.shape
    M = omega.shape[0]
    y = np.zeros(M, dtype=np.complex128)
    for (p0, p1, f) in points:
        y += f * np.exp(-1j * (omega[:, 0] * (p0 - L0 / 2) + omega[:, 1] * (p1 - L1 / 2)))
    if np.any(blob):
        U, s, Vt = np.linalg.svd(blob)
        r = int(np.sum(s > s[0] * 1e-15))
        Us = U[:, :r] * s[None, :r]
        V = Vt[:r, :].T
        for i in range(0, M, chunk):
            w = omega[i:i + chunk]
            e0 = _phase_rows(w[:, 0], L0) @ Us
            e1 = _phase_rows(w[:, 1], L1) @ V
            y[i:i + chunk] += np.sum(e0 * e1, axis=1)
    return y


def gaussian_visibilities(params, omega: np.ndarray, L: int, chunk: int = 1 << 22,
                          L1: int | None = None) -> np.ndarray:
    """Spectra of the Gaussian blobs at omega (sign and origin of exact_visibilities):
    for a blob A exp(-(a^2/smaj^2 + b^2/smin^2)/2) centred at c, the sum over the
    integer lattice is A 2 pi smaj smin exp(-omega^T S omega / 2) exp(-i <omega, c - L/2>)
    with omega^T S omega = smaj^2 (cos t w0 + sin t w1)^2 + smin^2 (-sin t w0 + cos t w1)^2
    (Poisson summation; the aliased terms and the part of the blob outside
    the image are below 1e-8 for compact blobs)."""
    L1 = L if L1 is None else L1
    M = omega.shape[0]
    y = np.zeros(M, dtype=np.complex128)
    for i in range(0, M, chunk):
        w0, w1 = omega[i:i + chunk, 0], omega[i:i + chunk, 1]
        for (c0, c1, smaj, smin, ang, peak) in params:
            ca, sa = math.cos(ang), math.sin(ang)
            q = (smaj * (ca * w0 + sa * w1)) ** 2 + (smin * (-sa * w0 + ca * w1)) ** 2
            amp = peak * 2.0 * math.pi * smaj * smin * np.exp(-0.5 * q)
            y[i:i + chunk] += amp * np.exp(-1j * (w0 * (c0 - L / 2) + w1 * (c1 - L1 / 2)))
    return y


def point_visibilities(points, omega: np.ndarray, L: int, chunk: int = 1 << 22,
                       L1: int | None = None) -> np.ndarray:
    """Exact spectra of the point sources (chunked)."""
    L1 = L if L1 is None else L1
    M = omega.shape[0]
    y = np.zeros(M, dtype=np.complex128)
    for i in range(0, M, chunk):
        w0, w1 = omega[i:i + chunk, 0], omega[i:i + chunk, 1]
        for (p0, p1, f) in points:
            y[i:i + chunk] += f * np.exp(-1j * (w0 * (p0 - L / 2) + w1 * (p1 - L1 / 2)))
    return y


def smooth_sides(lo: int, hi: int) -> list:
    """Image sides 16 * 2^a 3^b 5^c in [lo, hi]: multiples of 16 whose
    oversampled grid side 2 L has no prime factor above 5."""
    out = []
    for L in range(16 * ((lo + 15) // 16), hi + 1, 16):
        m = L // 16
        for f in (2, 3, 5):
            while m % f == 0:
                m //= f
        if m == 1:
            out.append(L)
    return out


def make_batch(n: int = 8, seed: int = 1704, sides=(128, 256), ratio=(2.0, 8.0), blocks=(4, 32),
               compact: bool = False, side_range: tuple | None = None):
    """n independent problems of different sizes: side drawn from `sides`
    (uniformly), or, with side_range = (lo, hi), log-uniform in [lo, hi] and
    rounded to the nearest 16 * 2^a 3^b 5^c; M = r * L^2 with r log-uniform in
    `ratio`, block count uniform in `blocks`, strongly non-uniform coverage
    (std 0.1 pi)."""
    rng = np.random.default_rng(seed)
    grid = smooth_sides(*side_range) if side_range else None
    out = []
    for i in range(n):
        if grid:
            t = math.exp(rng.uniform(math.log(side_range[0]), math.log(side_range[1])))
            L = min(grid, key=lambda v: (abs(v - t), v))
        else:
            L = int(sides[int(rng.integers(0, len(sides)))])
        r = math.exp(rng.uniform(math.log(ratio[0]), math.log(ratio[1])))
        d = int(rng.integers(blocks[0], blocks[1] + 1))
        out.append(make_problem(f"batch_{i}", L=L, M=int(round(r * L * L)), n_blocks=d, uv_sigma=0.1,
                                seed=seed * 100 + i, compact=compact))
    return out


def make_batch32(seed: int = 1704):
    """32 independent problems, sides log-uniform in [256, 1024] rounded to the
    nearest 16 * 2^a 3^b 5^c, M = 2-8 x the pixel count, 4-32 blocks: the
    batched workload of independent problems."""
    return make_batch(32, seed=seed, ratio=(2.0, 8.0), blocks=(4, 32), compact=True, side_range=(256, 1024))


def make_problem(name: str = "c1_128", *, L: int | None = None, M: int | None = None,
                 n_blocks: int | None = None, uv_sigma: float | None = None,
                 seed: int | None = None, isnr_db: float = 30.0,
                 n_points: int = 20, n_blobs: int = 3, ggd_beta: float | None = None,
                 compact: bool | None = None, L1: int | None = None) -> Problem:
    """Build a seeded problem; keyword arguments override the named shape.
    compact: blobs kept well inside the image and their visibilities taken
    from the analytic Gaussian spectra (large problems; see sky_image).
    L1: number of image columns when it differs from L (rows)."""
    cfg = dict(CONFIGS.get(name, CONFIGS["c1_128"]))
    for k, v in dict(L=L, M=M, n_blocks=n_blocks, uv_sigma=uv_sigma, seed=seed, compact=compact).items():
        if v is not None:
            cfg[k] = v
    is_compact = bool(cfg.get("compact", False))
    rng = np.random.default_rng(cfg["seed"])
    Lv = int(cfg["L"])
    L1v = Lv if L1 is None else int(L1)
    params = []
    points, blob = sky_image(Lv, rng, n_points=n_points, n_blobs=n_blobs, compact=is_compact, params_out=params,
                             L1=L1v)
    x = blob.copy()
    for (p0, p1, f) in points:
        x[p0, p1] += f
    if ggd_beta is None:
        omega = sample_uv(int(cfg["M"]), float(cfg["uv_sigma"]), rng)
    else:
        omega = sample_uv_ggd(int(cfg["M"]), float(ggd_beta), float(cfg["uv_sigma"]), rng)
    block = radial_blocks(omega, int(cfg["n_blocks"]))
    if is_compact:
        y0 = point_visibilities(points, omega, Lv, L1=L1v) + gaussian_visibilities(params, omega, Lv, L1=L1v)
    else:
        y0 = exact_visibilities(points, blob, omega)
    Mv = omega.shape[0]
    sigma = math.sqrt(float(np.vdot(y0, y0).real) / Mv * 10.0 ** (-isnr_db / 10.0))
    noise = sigma * (rng.normal(size=Mv) + 1j * rng.normal(size=Mv)) / math.sqrt(2.0)
    return Problem(name=name, L=Lv, x_true=x, omega=omega, y=y0 + noise, sigma=sigma,
                   theta=np.full(Mv, 1.0 / sigma), block=block,
                   n_blocks=int(cfg["n_blocks"]), isnr_db=isnr_db, seed=int(cfg["seed"]), L1=L1v)


def active_sets(n_iters: int, n_blocks: int, p_data: float, p_prior: float, seed: int = 1706,
                n_bases: int = 9):
    """Seeded draws of the randomised active sets of Algorithm 3: every data
    block is in D with probability p_data and every basis (Dirac first) in P
    with probability p_prior, independently and identically along the
    iterations (Section 4.4 asks for nonzero probabilities and i.i.d. draws).
    Returns uint8 masks of shapes (n_iters, n_blocks) and (n_iters, n_bases)."""
    if not (0.0 < p_data <= 1.0 and 0.0 < p_prior <= 1.0):
        raise ValueError("activation probabilities must lie in (0, 1]")
    rng = np.random.default_rng(seed)
    blocks = (rng.random((n_iters, n_blocks)) < p_data).astype(np.uint8)
    bases = (rng.random((n_iters, n_bases)) < p_prior).astype(np.uint8)
    return blocks, bases


def splitmix64(counter: np.ndarray) -> np.ndarray:
    """SplitMix64 finaliser (Steele, Lea & Flood 2014) of uint64 counters:
    the generator's output for a state that has just been advanced to
    `counter`."""
    z = np.asarray(counter, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    return z ^ (z >> np.uint64(31))


def power_start(n0: int, n1: int, seed: int) -> np.ndarray:
    """Seeded start image of a power iteration (an input, like the data):
    all ones for seed 0, else x_i = 0.5 + 2^-53 (s_i >> 11) with s_i the
    SplitMix64 output for the counter seed + (i + 1) * 0x9E3779B97F4A7C15,
    i the row-major pixel index; normalised to unit l2 norm."""
    n = n0 * n1
    if seed == 0:
        x = np.ones(n)
    else:
        i = np.arange(1, n + 1, dtype=np.uint64)
        with np.errstate(over="ignore"):
            ctr = np.uint64(seed) + i * np.uint64(0x9E3779B97F4A7C15)
        x = 0.5 + (splitmix64(ctr) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
    x = x.reshape(n0, n1)
    return x / np.linalg.norm(x)
