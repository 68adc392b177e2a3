"""Benchmark of the PPD hot path on one GB300 (or N independent replicas).

Workload (default): 512 x 512 image, 524,288 visibilities drawn from a
strongly non-uniform Gaussian u-v density (std 0.1 pi), 16 uneven radial
blocks, 30 dB input SNR, seeded synthetic sky (point sources and Gaussian
blobs).  A step is one PPD iteration (Algorithm 3: forward FFT + degridding
with the data step, block norms, gridding with the dual update, inverse FFT,
SARA prior step, primal step) on inputs resident in HBM; L2 is flushed
(256 MiB write) between timed steps, outside the timed region.

Printed JSON line (rank 0): PPD iterations per second of the FP32-batched
path (FP32 arrays, FP64 norms, one CUDA graph per iteration), with the FP64
plain path, the SNR reached after 500 iterations (100 at 4096^2) by each, the iterations and
seconds the FP32 path needs to reach the FP64 path's SNR, an end-to-end
number through the host API, the roofline of the dominant kernel and the
FP64 oracle timed on the host cores.

--impl reference times the oracle itself (one oracle PPD iteration per step).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "PPD iters/s and time-to-target-SNR, FP32-batched vs FP64-plain on 1 GB300"
UNIT = "iters/s"
SNR_ITERS = 500
# iterations of the SNR comparison per workload (the FP64 plain path at 4096^2 runs a few iterations/s)
SNR_ITERS_BY_WORKLOAD = {"c5_4096": 100}
# workloads whose FP64 oracle iteration does not fit a bounded CPU sample (64M-visibility plans)
NO_ORACLE = {"c5_4096": "one oracle iteration at 4096^2 with 64M visibilities holds > 16 GB of FP64 tap tables "
                        "and runs for minutes on one core; the CPU baseline is reported on c2_512 and c3_1024"}
WORKLOAD = "c2_512"


_T0 = time.time()


def _log(msg: str):
    """Progress line on stderr (phase and elapsed seconds)."""
    print(f"[bench {time.time() - _T0:7.1f}s] {msg}", file=sys.stderr, flush=True)


def _env_rank():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


# ------------------------------------------------------------------ roofline model
def algorithmic_bytes_per_step(L: int, M: int, levels: int = 4, rsz: int = 4, xtrue: bool = True) -> dict:
    """Algorithmic HBM bytes per PPD iteration for each kernel name (all its launches).

    Complex = 2 * rsz bytes.  Every input read once and every output written
    once; halos, partial tiles and re-reads are implementation overhead and
    not counted.  N = L^2 pixels, K^2 = 4N grid cells, M visibilities.
    SARA analysis, level l (8 wavelet bases): the level input (xt once at
    level 0, the previous LL per basis after), the 3 detail quadrants of u
    read and written, the LL written (read and written in u at the last
    level).  Synthesis, level l >= 1: LL' and 3 detail quadrants read, the
    2h x 2h output written; level 0 (all bases summed): LL' and details read,
    ut written.  Primal: x, xt, g, ut, u_Dirac (and x_true for the SNR) read;
    x, xt, u_Dirac written; fused with the inverse and the next forward row
    pass (rows_primal), g never leaves the chip.
    """
    N, K2, c = L * L, 4 * L * L, 2 * rsz
    det = lambda l: 3 * N / 4 ** (l + 1)       # detail coefficients of level l, per basis
    ll = lambda l: N / 4 ** (l + 1)            # LL of level l, per basis
    ana = rsz * N                               # xt read once for all bases
    for l in range(levels):
        inp = 0 if l == 0 else ll(l - 1)
        last = l == levels - 1
        ana += 8 * rsz * (inp + 2 * det(l) + (2 * ll(l) if last else ll(l)))
    syn = 0.0
    for l in range(levels - 1, 0, -1):
        syn += 8 * rsz * (ll(l) + det(l) + 4 * ll(l))
    syn += 8 * rsz * (ll(0) + det(0)) + rsz * N
    return {
        "degrid_dual": (16 + 5 * c) * M + c * K2,     # record, v, y, p in; z, w out; grid once
        "grid_dual": (16 + 5 * c) * M,                # record, y, w, z in; v, p out (per-chunk partial tiles: overhead)
        "grid_combine": c * K2,                       # the combined grid written once (partial tiles in: overhead)
        "subiter": (16 + 4 * c) * M,
        "fft_fwd_rows": rsz * N + c * 2 * N,
        "fft_fwd_cols": c * 2 * N + c * K2,
        "fft_inv_cols": c * K2 + c * 2 * N,
        "fft_inv_rows": c * 2 * N + rsz * N,
        "sara_analysis": ana,
        "sara_synthesis": syn,
        "primal": rsz * N * (8 + (1 if xtrue else 0)),
        # inverse row pass (tmp_inv read), primal (x, xt, ut, u_Dirac [, x_true] read; x, xt,
        # u_Dirac written; g stays on chip) and the next forward row pass (tmp written)
        "rows_primal": c * 2 * N + rsz * N * (7 + (1 if xtrue else 0)) + c * 2 * N,
        "block_norms": 0.0,
    }


def source_digest() -> str:
    """sha256 over the library's CUDA sources (name and contents, sorted)."""
    import hashlib
    d = os.path.join(ROOT, "paper_1701_01748_gb300", "csrc")
    h = hashlib.sha256()
    for f in sorted(os.listdir(d)):
        h.update(f.encode())
        with open(os.path.join(d, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def dram_traffic(workload: str) -> tuple[dict, str]:
    """DRAM bytes per launch by kernel from the committed ncu summary of this
    workload (profiles/ncu_dram_<workload>.txt), if it was taken on the
    current sources; else ({}, why)."""
    path = os.path.join(ROOT, "profiles", f"ncu_dram_{workload}.txt")
    if not os.path.exists(path):
        return {}, "no ncu capture for this workload"
    out, digest = {}, None
    for line in open(path):
        line = line.strip()
        if line.startswith("sources sha256:"):
            digest = line.split(":", 1)[1].strip()
        elif line and not line.startswith("#") and ":" not in line:
            k, v = line.split()[:2]
            out[k] = float(v)
    if digest != source_digest():
        return {}, "kernels changed since the ncu capture"
    return out, "ncu dram__bytes_read.sum + dram__bytes_write.sum per launch, " + os.path.basename(path)


def read_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampling during the measured region."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        import tempfile
        self.path = os.path.join(tempfile.gettempdir(), f"ppd_bench_clocks_{os.getpid()}_{index}.csv")

    def __enter__(self):
        os.makedirs(os.path.dirname(self.path), exist_ok=True)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap,utilization.gpu")
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        try:
            rows = [r.split(",") for r in open(self.path).read().strip().splitlines() if r.strip()]
        except Exception:
            return out
        sm, smax, busy, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                s, mx, util = float(r[1]), float(r[2]), float(r[9])
            except Exception:
                continue
            sm.append(s)
            smax.append(mx)
            if util > 0:
                busy.append(s)
            for n, v in zip(names, r[5:9]):
                if v.strip() == "Active":
                    reasons.add(n)
        if sm:
            out["sm_mhz"] = statistics.median(busy if busy else sm)
            out["sm_max_mhz"] = max(smax)
            out["samples"] = len(sm)
            out["samples_busy"] = len(busy)
        out["reasons"] = sorted(reasons)
        return out


# ------------------------------------------------------------------ CPU oracle leg
GOLDEN_NORMS = os.path.join(ROOT, "tests", "golden", "op_norms.json")


def oracle_op_norm(p, P, U):
    """||U^{1/2} Phi||_S^2 of problem p for the oracle: the value stored by
    tests/golden/make_op_norms.py (the oracle's Lanczos routine, run offline)
    when it was made for this workload, seed and size, else the same routine
    now.  Returns (value, source)."""
    from oracle import ppd as oppd
    try:
        with open(GOLDEN_NORMS) as f:
            rec = json.load(f).get(p.name)
    except (OSError, ValueError):
        rec = None
    if rec and rec["seed"] == p.seed and rec["L"] == p.L and rec["M"] == p.M:
        return float(rec["op_norm_sq"]), "tests/golden/op_norms.json (oracle Lanczos, stored)"
    val, _ = oppd.op_norm_sq_lanczos(P, U, tol=1e-8)
    return val, "oracle Lanczos at set-up"


def oracle_setup(workload: str, seed: int):
    """The oracle's set-up of the workload (never timed): eta = 1/||U^{1/2} Phi||^2
    as Section 5.1 asks, so that the convergence condition holds."""
    from oracle import nufft, ppd as oppd
    from paper_1701_01748_gb300 import synth
    p = synth.make_problem(workload, seed=seed)
    P = nufft.Plan(p.omega, p.L, p.L, theta=p.theta)
    U = nufft.uniform_weights(p.omega, P.K0, P.K1)[0]
    norm, src = oracle_op_norm(p, P, U)
    S = oppd.make_setup(p.omega, p.y, p.theta, p.block, p.n_blocks, p.L, eta=1.0 / norm, U=U,
                        x_true=p.x_true)
    return p, S, {"op_norm_sq": norm, "eta_source": src, "convergence_lhs": oppd.convergence_lhs(S, 1.0, norm)}


def oracle_worker(args):
    """Run in a fresh single-threaded interpreter: time oracle PPD iterations,
    args.steps of them after args.warmup, or, with --oracle-seconds, as many
    as fit in that many seconds (at least 3)."""
    from oracle import ppd as oppd
    p, S, info = oracle_setup(args.workload, args.seed)
    st = oppd.init_state(S)
    times, snr = [], None
    budget = args.oracle_seconds
    i = 0
    while True:
        t0 = time.perf_counter()
        h = oppd.iterate(st, S)
        dt = time.perf_counter() - t0
        if not all(math.isfinite(r) for r in h["residual"]):
            raise RuntimeError(f"oracle iteration {i + 1} is not finite")
        snr = h.get("snr")
        if i >= args.warmup:
            times.append(dt)
        i += 1
        if budget > 0:
            if len(times) >= 3 and sum(times) >= budget:
                break
        elif len(times) >= args.steps:
            break
    print(json.dumps({"times": times, "snr_db": snr, **info}))


def run_oracle(workload: str, seed: int, steps: int, warmup: int, seconds: float = 0.0):
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    cmd = [sys.executable, os.path.abspath(__file__), "--oracle-worker", "--workload", workload,
           "--seed", str(seed), "--steps", str(steps), "--warmup", str(warmup),
           "--oracle-seconds", str(seconds)]
    r = subprocess.run(cmd, capture_output=True, text=True, env=env, timeout=1800)
    if r.returncode != 0:
        raise RuntimeError(r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


def workload_config(workload: str) -> dict:
    """The `config` block of a single-problem workload, from its generator settings."""
    from paper_1701_01748_gb300 import synth
    cfg = synth.CONFIGS[workload]
    return {"workload": workload, "image": f"{cfg['L']}x{cfg['L']}", "visibilities": cfg["M"],
            "blocks": cfg["n_blocks"], "uv_density": f"gaussian sigma={cfg['uv_sigma']}pi", "isnr_db": 30}


def cpu_info():
    model = ""
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part")) and not model:
                model = line.split(":", 1)[1].strip()
    except Exception:
        pass
    return model, os.cpu_count()


# ------------------------------------------------------------------ replicas
def max_over_ranks(seconds_per_step: float, dist=None, device=None) -> float:
    """Slowest rank's seconds per step (each rank runs its own replica)."""
    if dist is None:
        return float(seconds_per_step)
    import torch
    t = torch.tensor([seconds_per_step], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(seconds_per_step: float, world: int) -> float:
    """Whole-job iterations/s: every rank completes one iteration of its own
    problem per step, the step lasting as long as the slowest rank's."""
    return world / seconds_per_step


# ------------------------------------------------------------------ batched problems
def bench_batch(args, rank, world, local):
    """Independent problems of different sizes: each alone (one graph each,
    one after another) vs all in one group (one graph launch per iteration)."""
    import torch
    from paper_1701_01748_gb300 import ppd, synth
    n = int(args.workload[len("batch"):] or 8)
    # batch32: 32 problems of 256^2-1024^2, M = 2-8 x pixels, 4-32 blocks; other sizes: 128^2-256^2
    probs = synth.make_batch32(seed=1704 + 1000 * rank) if n == 32 else synth.make_batch(n, seed=1704 + 1000 * rank)
    dev = torch.device("cuda", local)
    solvers, tuned = [], []
    _log(f"{n} problems, {sum(p.M for p in probs)} visibilities in all")
    for p in probs:
        s = ppd.Solver(p.L, p.n_blocks, precision=ppd.PPD_FP32_FP64NORMS)
        s.set_problem(p.omega, p.y, p.block, theta=p.theta, x_true=p.x_true)
        if args.autotune:
            tuned.append(ppd.ppd_autotune(s.ctx, 5))
        solvers.append(s)
    _log("set-up done")
    for s in solvers:
        s.iterate(max(args.warmup, 3), stats=False)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for s in solvers:
        s.iterate(args.steps, stats=False)
    torch.cuda.synchronize(dev)
    t_seq = time.perf_counter() - t0
    g = ppd.ppd_group_create([s.ctx for s in solvers])
    ppd.ppd_group_iterate(g, max(args.warmup, 3))
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    ppd.ppd_group_iterate(g, args.steps)
    torch.cuda.synchronize(dev)
    t_grp = time.perf_counter() - t0
    ppd.ppd_group_destroy(g)
    total = n * args.steps
    if rank == 0:
        print(json.dumps({
            "metric": "PPD iterations/s summed over a batch of independent problems", "unit": "iters/s",
            "value": total / t_grp, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "higher_is_better": True, "dtype": "f32", "data": "synthetic",
            "config": {"workload": args.workload, "problems": [[p.L, p.M, p.n_blocks] for p in probs],
                       "visibilities": int(sum(p.M for p in probs)),
                       "gridding_tile_and_chunk": tuned if tuned else "library default (16, 1024)",
                       "timing": "wall clock between device synchronisations, one group graph launch per iteration"},
            "sequential_iters_per_s": total / t_seq, "batching_speedup": t_seq / t_grp}), flush=True)
    for s in solvers:
        s.close()


# ------------------------------------------------------------------ PD vs PPD study
def study_ggd(args, local):
    """Convergence speed of PPD (U = inverse sampling density) against PD
    (U = I) on generalised-Gaussian coverages of shape beta (Section 5.3): SNR
    every 10 iterations, and how many iterations PD needs to reach the SNR
    that PPD has at iteration 100."""
    import torch
    from paper_1701_01748_gb300 import ppd, synth
    torch.cuda.set_device(local)
    iters = max(args.steps, 200)
    out = {"metric": "iterations to reach PPD's SNR at iteration 100, PD vs PPD", "data": "synthetic",
           "config": {"workload": "ggd", "image": "256x256", "visibilities": 65536, "blocks": 4,
                      "uv_std": "0.15 pi", "isnr_db": args.isnr}, "results": []}
    for beta in (2.0, 0.5, 0.25):
        p = synth.make_problem("ggd", L=256, M=65536, n_blocks=4, uv_sigma=0.15, seed=1705,
                               ggd_beta=beta, isnr_db=args.isnr)
        curves = {}
        for name, precond in (("ppd", 1), ("pd", 0)):
            s = ppd.Solver(p.L, p.n_blocks, precision=ppd.PPD_FP32_FP64NORMS, precond=precond)
            s.set_problem(p.omega, p.y, p.block, theta=p.theta, x_true=p.x_true)
            curves[name] = [s.iterate(10)["snr_db"] for _ in range(iters // 10)]
            s.close()
        target = curves["ppd"][9]          # PPD at iteration 100
        reach = next((10 * (i + 1) for i, v in enumerate(curves["pd"]) if v >= target), None)
        out["results"].append({"beta": beta, "ppd_snr_at_100": target,
                               "pd_iters_to_ppd_snr_at_100": reach,
                               "speedup": (reach / 100.0) if reach else f">{iters / 100.0}",
                               "ppd_snr": curves["ppd"][::5], "pd_snr": curves["pd"][::5]})
    print(json.dumps(out), flush=True)


# ------------------------------------------------------------------ randomised active sets
def study_random(args, local):
    """Randomised active sets (Algorithm 3, sets P and D) on the bench
    workload: iterations/s of the FP32 path with every data block and basis
    active with probability p (seeded i.i.d. draws, Section 4.4), and the SNR
    after a fixed number of iterations, for p = 1 (plain), 0.75, 0.5."""
    import torch
    from paper_1701_01748_gb300 import ppd, synth
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    p = synth.make_problem(args.workload)
    stream = torch.cuda.Stream(dev)
    flush = torch.empty(256 * 2 ** 20 // 4, dtype=torch.float32, device=dev)
    s = ppd.Solver(p.L, p.n_blocks, precision=ppd.PPD_FP32_FP64NORMS, stream=stream.cuda_stream)
    s.set_problem(p.omega, p.y, p.block, theta=p.theta, x_true=p.x_true)
    zero = ppd.ppd_get_state(s.ctx)
    iters = args.snr_iters or SNR_ITERS
    out = {"metric": "PPD iterations/s and SNR with randomised active sets", "unit": "iters/s", "data": "synthetic",
           "dtype": "f32", "steps": args.steps, "warmup": args.warmup,
           "config": {"workload": args.workload, "image": f"{p.L}x{p.L}", "visibilities": p.M,
                      "blocks": p.n_blocks, "l2": "flushed (256 MiB write) between timed steps"},
           "results": []}
    for prob in (1.0, 0.75, 0.5):
        n_all = args.warmup + args.steps
        B, P = synth.active_sets(max(n_all, iters), p.n_blocks, prob, prob, seed=1706)

        def restart():
            ppd.ppd_set_state(s.ctx, zero)
            if prob < 1.0:
                ppd.ppd_set_active_sets(s.ctx, B, P)
            else:
                ppd.ppd_set_active_sets(s.ctx, n_iters=0)
        restart()
        for _ in range(args.warmup):
            ppd.ppd_iterate(s.ctx, 1, stats=False)
        torch.cuda.synchronize(dev)
        tot = 0.0
        for _ in range(args.steps):
            with torch.cuda.stream(stream):
                flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ppd.ppd_iterate(s.ctx, 1, stats=False)
            e1.record(stream)
            e1.synchronize()
            tot += e0.elapsed_time(e1)
        restart()             # SNR after `iters` iterations from zero with the same draws
        snr = [ppd.ppd_iterate(s.ctx, 10, p.n_blocks)["snr_db"] for _ in range(iters // 10)]
        out["results"].append({"p_active": prob, "iters_per_s": args.steps / (tot / 1e3),
                               "ms_per_iter": tot / args.steps, "snr_db_at_end": snr[-1],
                               "snr_db_every_50": snr[4::5]})
    print(json.dumps(out), flush=True)
    s.close()


# ------------------------------------------------------------------ main
def cufft_compare(K: int, dev, stream, flush, reps: int = 20) -> dict:
    """cuFFT (through torch.fft) on the full K x K complex64 grid, timed with CUDA
    events on the bench stream after 3 warm-ups, L2 flushed before each call:
    the comparison for the library's own forward and inverse 2-D FFT passes."""
    import torch
    a = torch.randn((K, K), dtype=torch.complex64, device=dev)
    out = {}
    with torch.cuda.stream(stream):
        for name, fn in (("cufft_fft2_us", lambda t: torch.fft.fft2(t)),
                         ("cufft_ifft2_us", lambda t: torch.fft.ifft2(t, norm="forward"))):
            for _ in range(3):
                fn(a)
            tot = 0.0
            for _ in range(reps):
                flush.zero_()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                fn(a)
                e1.record(stream)
                e1.synchronize()
                tot += e0.elapsed_time(e1)
            out[name] = 1e3 * tot / reps
    return out


def fft_pass_times(s, p, dev, stream, flush, reps: int = 20) -> dict:
    """The library's own 2-D transforms, every pass timed: the forward row and
    column passes of ppd_op_forward (Z fused, coverage pruning) and the
    inverse column and row passes of ppd_op_adjoint (crop, deapodisation and
    real part fused), per-kernel CUDA events on the bench stream, L2 flushed
    before each call; microseconds per pass, averaged over `reps` calls."""
    import torch
    from paper_1701_01748_gb300 import ppd
    real = torch.float32 if s.cfg.precision == ppd.PPD_FP32_FP64NORMS else torch.float64
    x = torch.rand((p.L, p.L), dtype=real, device=dev)
    y = torch.empty((p.M, 2), dtype=real, device=dev)
    sp = stream.cuda_stream
    for _ in range(3):
        ppd.ppd_op_forward(s.ctx, x.data_ptr(), y.data_ptr(), sp)
        ppd.ppd_op_adjoint(s.ctx, y.data_ptr(), x.data_ptr(), sp)
    torch.cuda.synchronize(dev)
    ppd.ppd_timing_enable(s.ctx, True)
    for _ in range(reps):
        with torch.cuda.stream(stream):
            flush.zero_()
        ppd.ppd_op_forward(s.ctx, x.data_ptr(), y.data_ptr(), sp)
        with torch.cuda.stream(stream):
            flush.zero_()
        ppd.ppd_op_adjoint(s.ctx, y.data_ptr(), x.data_ptr(), sp)
        ppd.ppd_timing_collect(s.ctx)
    kt = ppd.ppd_timing_read(s.ctx)
    ppd.ppd_timing_enable(s.ctx, False)
    return {k: 1e3 * kt[k][0] / kt[k][1] for k in ("fft_fwd_rows", "fft_fwd_cols", "fft_inv_cols", "fft_inv_rows")
            if k in kt}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--seed", type=int, default=None)
    ap.add_argument("--oracle-worker", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--oracle-seconds", type=float, default=20.0,
                    help="CPU baseline: oracle iterations until this many seconds (at least 3)")
    ap.add_argument("--snr-iters", type=int, default=0, help="iterations of the SNR comparison (0: per workload)")
    ap.add_argument("--tile", type=int, default=0, help="gridding tile side (0: library default)")
    ap.add_argument("--chunk", type=int, default=0, help="visibilities per work item (0: library default)")
    ap.add_argument("--study", default="", help="ggd: PD vs PPD convergence on generalised-Gaussian coverages; "
                                                "random: randomised active sets")
    ap.add_argument("--isnr", type=float, default=30.0, help="input SNR (dB) of the study problems")
    ap.add_argument("--autotune", action="store_true", help="batch workloads: autotune each problem's gridding")
    ap.add_argument("--no-autotune", action="store_true", help="main bench: keep the library's default gridding")
    ap.add_argument("--grid-warps", type=int, default=0, help="warps per gridding CTA (0: library default)")
    ap.add_argument("--degrid-threads", type=int, default=0,
                    help="threads per degridding CTA (0: library default)")
    ap.add_argument("--launch-overlap", action="store_true",
                    help="kernels start while their predecessor drains (programmatic dependent launch)")
    ap.add_argument("--quick", action="store_true",
                    help="only the timed FP32 steps (for profiler launch lists); eta from 20 power steps")
    args = ap.parse_args()
    if args.oracle_worker:
        oracle_worker(args)
        return
    rank, world, local = _env_rank()
    if args.study in ("ggd", "random"):
        from paper_1701_01748_gb300 import build
        build.build()
        if rank == 0:
            (study_ggd if args.study == "ggd" else study_random)(args, local)
        return
    from paper_1701_01748_gb300 import synth
    base_seed = synth.CONFIGS[args.workload]["seed"] if args.workload in synth.CONFIGS else 1704
    seed = (args.seed if args.seed is not None else base_seed) + 1000 * rank

    if args.impl == "reference":
        if rank != 0:
            return
        model, ncpu = cpu_info()
        if args.workload not in synth.CONFIGS or args.workload in NO_ORACLE:
            why = NO_ORACLE.get(args.workload, "the oracle runs single-problem workloads only")
            print(json.dumps({"impl": "reference", "unavailable": why}), flush=True)
            return
        r = run_oracle(args.workload, seed, args.steps, max(args.warmup, 0))
        times = r["times"]
        v = len(times) / sum(times)
        line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic", "config": workload_config(args.workload),
                "oracle": {"eta_source": r["eta_source"], "op_norm_sq": r["op_norm_sq"],
                           "convergence_lhs": r["convergence_lhs"], "snr_db_at_end": r["snr_db"]},
                "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                                 "sample": f"{len(times)} oracle PPD iterations of the workload after "
                                           f"{args.warmup} untimed (FP64 NumPy, 1 thread) on {model} "
                                           f"({ncpu} cores)"},
                "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return

    import torch
    from paper_1701_01748_gb300 import build, ppd
    build.build()
    torch.cuda.set_device(local)
    if args.workload.startswith("batch"):
        return bench_batch(args, rank, world, local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    dev = torch.device("cuda", local)
    _log(f"generating {args.workload}")
    p = synth.make_problem(args.workload, seed=seed)
    _log("problem ready")
    snr_iters = args.snr_iters or SNR_ITERS_BY_WORKLOAD.get(args.workload, SNR_ITERS)
    stream = torch.cuda.Stream(dev)
    sp = stream.cuda_stream

    def make(prec, **kw):
        shape = dict(grid_warps=args.grid_warps, degrid_threads=args.degrid_threads) \
            if prec == ppd.PPD_FP32_FP64NORMS else {}
        s = ppd.Solver(p.L, p.n_blocks, precision=prec, stream=sp, tile=args.tile, chunk=args.chunk,
                       launch_overlap=int(args.launch_overlap), **shape, **kw)
        s.set_problem(p.omega, p.y, p.block, theta=p.theta, x_true=p.x_true)
        return s

    flush = torch.empty(256 * 2 ** 20 // 4, dtype=torch.float32, device=dev)
    if args.quick:
        s32 = make(ppd.PPD_FP32_FP64NORMS, power_iters=20)
    else:
        _log("set-up FP32 (eta by power iteration)")
        s32 = make(ppd.PPD_FP32_FP64NORMS)
        if not args.no_autotune and args.tile == 0 and args.chunk == 0:
            _log("autotuning the gridding work decomposition")
            # enough iterations per candidate that the timing is stable (a 512^2
            # iteration is ~0.14 ms), fewer for the large workloads
            ppd.ppd_autotune(s32.ctx, 50 if p.M < 10_000_000 else 10)
        _log("set-up FP64 (eta by power iteration)")
        s64 = make(ppd.PPD_FP64_PLAIN)
    # the zero state of each solver, restored before every measured run (the
    # state blob resets x, xt, u, v and the warm start without a new eta)
    zero = {s.ctx: ppd.ppd_get_state(s.ctx) for s in ([s32] if args.quick else [s32, s64])}
    prm32 = s32.params()

    def timed_steps(s, steps, warmup, kernel_timing):
        ppd.ppd_timing_enable(s.ctx, kernel_timing)
        ppd.ppd_set_state(s.ctx, zero[s.ctx])             # reset to the zero state - untimed
        for _ in range(warmup):
            ppd.ppd_iterate(s.ctx, 1, stats=False)
        torch.cuda.synchronize(dev)
        ppd.ppd_timing_collect(s.ctx)
        ppd.ppd_timing_enable(s.ctx, kernel_timing)      # clears sums
        total = 0.0
        launches0 = ppd.ppd_launch_count(s.ctx)
        for _ in range(steps):
            with torch.cuda.stream(stream):
                flush.zero_()
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            ppd.ppd_iterate(s.ctx, 1, stats=False)
            ev1.record(stream)
            ev1.synchronize()
            total += ev0.elapsed_time(ev1)
            if kernel_timing:
                ppd.ppd_timing_collect(s.ctx)
        launches = ppd.ppd_launch_count(s.ctx) - launches0
        kt = ppd.ppd_timing_read(s.ctx) if kernel_timing else {}
        return total / 1e3, launches, kt

    def snr_run(s, iters):
        ppd.ppd_timing_enable(s.ctx, False)
        ppd.ppd_set_state(s.ctx, zero[s.ctx])
        snr = []
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for _ in range(iters // 10):
            st = ppd.ppd_iterate(s.ctx, 10, p.n_blocks)
            snr.append(st["snr_db"])
        dt = time.perf_counter() - t0
        return snr, dt

    if args.quick:
        ppd.ppd_timing_enable(s32.ctx, False)
        for _ in range(args.warmup):
            ppd.ppd_iterate(s32.ctx, 1, stats=False)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            ppd.ppd_iterate(s32.ctx, 1, stats=False)
        torch.cuda.synchronize(dev)
        print(json.dumps({"quick": True, "tile": args.tile, "chunk": args.chunk,
                          "ms_per_step": 1e3 * (time.perf_counter() - t0) / args.steps}))
        s32.close()
        return
    if dist is not None:
        dist.barrier()
    with Clocks(local) as clk:
        # timed region: FP32-batched, no per-kernel event nodes in the graph
        _log("timed FP32 steps")
        t32, launches, _ = timed_steps(s32, args.steps, max(args.warmup, 3), False)
        # same protocol again with an event pair around every kernel (roofline)
        _log("per-kernel timed FP32 steps")
        t32k, _, kt = timed_steps(s32, args.steps, max(args.warmup, 3), True)
        # FP64 plain, same protocol
        _log("timed FP64 steps")
        t64, _, _ = timed_steps(s64, max(3, args.steps // 4), 3, False)
        _log("SNR runs")
        snr32, wall32 = snr_run(s32, snr_iters)
        snr64, wall64 = snr_run(s64, snr_iters)
        # end to end through the host API: context, upload, set-up, snr_iters iterations with
        # per-10 stats, image back
        _log("end to end")
        e2e_t = []
        for _ in range(2):
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            se = ppd.Solver(p.L, p.n_blocks, precision=ppd.PPD_FP32_FP64NORMS, stream=sp,
                            tile=prm32["tile"], chunk=prm32["chunk"])
            ppd.ppd_set_visibilities(se.ctx, p.omega, p.y, p.block)
            ppd.ppd_set_weights(se.ctx, p.theta, None, None)
            ppd.ppd_set_ground_truth(se.ctx, p.x_true)
            for _ in range(snr_iters // 10):
                ppd.ppd_iterate(se.ctx, 10, p.n_blocks)
            img = ppd.ppd_get_image(se.ctx, p.L, p.L)
            se.close()
            e2e_t.append(time.perf_counter() - t0)
    clocks = clk.summary()
    _log("cuFFT comparison")
    cufft = cufft_compare(2 * p.L, dev, stream, flush) if rank == 0 else {}
    ours_fft = fft_pass_times(s32, p, dev, stream, flush) if rank == 0 else {}

    ips32 = args.steps / t32
    steps64 = max(3, args.steps // 4)
    ips64 = steps64 / t64
    per_step = max_over_ranks(t32 / args.steps, dist, dev)
    if dist is not None:
        dist.destroy_process_group()
    if rank != 0:
        return
    value = replica_throughput(per_step, world)
    target = snr64[-1]
    it_to_target = None
    for i, v in enumerate(snr32):
        if v >= target - 0.05:
            it_to_target = 10 * (i + 1)
            break
    # roofline of the dominant kernel: algorithmic bytes per iteration / its time per iteration
    peak, peak_kind = read_peaks()
    ab = algorithmic_bytes_per_step(p.L, p.M)
    ktot = sum(v[0] for v in kt.values()) if kt else 1.0
    kern = {}
    for k, (ms, n) in sorted(kt.items(), key=lambda kv: -kv[1][0]):
        per_step_s = ms / args.steps / 1e3
        bytes_step = ab.get(k, 0.0)
        kern[k] = {"avg_us": 1e3 * ms / n, "launches": n, "share": ms / ktot,
                   "gbs": (bytes_step / per_step_s / 1e9) if bytes_step else None}
    roof = None
    if kt:
        name, (ms, n) = max(kt.items(), key=lambda kv: kv[1][0])
        per_step_s = ms / args.steps / 1e3
        ach = ab.get(name, 0.0) / per_step_s / 1e9 if ab.get(name) else None
        traffic, why = dram_traffic(args.workload)
        roof = {"bound": "hbm", "kernel": name, "achieved": ach, "peak": peak, "unit": "GB/s",
                "frac": (ach / peak if ach else None), "traffic": traffic.get(name), "traffic_source": why,
                "peak_source": peak_kind,
                "algorithmic_bytes_per_launch": ab.get(name, 0.0) * args.steps / n,
                "avg_launch_us": 1e3 * ms / n, "share_of_kernel_time": ms / ktot,
                "ms_per_step_with_kernel_events": 1e3 * t32k / args.steps}
    fft_cmp = None
    if ours_fft and cufft:
        fwd = ours_fft.get("fft_fwd_rows", 0.0) + ours_fft.get("fft_fwd_cols", 0.0)
        inv = ours_fft.get("fft_inv_cols", 0.0) + ours_fft.get("fft_inv_rows", 0.0)
        fft_cmp = {"ours_forward_us": fwd, "ours_inverse_us": inv, "ours_passes_us": ours_fft, **cufft,
                   "forward_ratio": cufft["cufft_fft2_us"] / fwd if fwd else None,
                   "inverse_ratio": cufft["cufft_ifft2_us"] / inv if inv else None,
                   "note": "ours: both passes of each 2-D transform (row and column), each timed with "
                           "per-kernel events through ppd_op_forward / ppd_op_adjoint, L2 flushed; the "
                           "forward fuses zero-padding, deapodisation and coverage pruning, the inverse the "
                           "crop, deapodisation and real part; cuFFT: plain full-grid complex-to-complex "
                           "transform of the same 2L x 2L grid"}
    in_bytes = p.M * (16 + 16 + 4 + 8) + p.L * p.L * 8   # uv, y, block, theta; x_true
    out_bytes = p.L * p.L * 8
    stats_bytes = (snr_iters // 10) * (3 * 8 + p.n_blocks * 8 + 4)
    e2e_v = snr_iters / min(e2e_t)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {**workload_config(args.workload),
                   "l2": "flushed (256 MiB write) between timed steps", "graph": "one CUDA graph per iteration",
                   "replicas": world,
                   "launches": "overlapped (programmatic dependent launch)" if args.launch_overlap else "serial",
                   "gridding": {"tile": prm32["tile"], "chunk": prm32["chunk"], "work_items": prm32["n_chunks"],
                                "grid_warps": prm32["grid_warps"], "degrid_threads": prm32["degrid_threads"],
                                "autotuned": not args.no_autotune and args.tile == 0 and args.chunk == 0}},
        "snr_iters": snr_iters,
        "fp64_plain": {"iters_per_s": ips64, "snr_db_at_end": target, "seconds_all": wall64},
        "fp32_batched": {"iters_per_s": ips32, "snr_db_at_end": snr32[-1], "seconds_all": wall32,
                         "iters_to_target_snr": it_to_target,
                         "seconds_to_target_snr": (wall32 * it_to_target / snr_iters) if it_to_target else None},
        "speedup_iters_per_s": ips32 / ips64,
        "eta": {name: {k: prm[k] for k in ("op_norm_sq", "power_iters_done", "convergence_lhs")}
                for name, prm in (("fp32", prm32), ("fp64", s64.params()))},
        "e2e": {"value": e2e_v, "unit": UNIT, "h2d_bytes_per_step": in_bytes / snr_iters,
                "d2h_bytes_per_step": (out_bytes + stats_bytes) / snr_iters,
                "what": f"ppd_create + ppd_set_visibilities + ppd_set_weights (eta by power iteration) + "
                        f"{snr_iters} iterations "
                        "with stats every 10 + ppd_get_image, from host buffers"},
        "gpu_launches": launches,
        "fft_vs_cufft": fft_cmp,
        "roofline": roof,
        "kernels": kern,
        "clocks": clocks,
    }
    if args.workload in NO_ORACLE and world == 1:
        line["cpu_baseline"] = {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": "not run: " + NO_ORACLE[args.workload]}
    elif not args.no_cpu_baseline and world == 1:
        r = run_oracle(args.workload, seed, 0, 0, seconds=args.oracle_seconds)
        times = r["times"]
        model, ncpu = cpu_info()
        line["cpu_baseline"] = {"value": len(times) / sum(times), "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": f"{len(times)} oracle PPD iterations of the same workload from x = 0 "
                                          f"(about {args.oracle_seconds:.0f} s; FP64 NumPy, 1 thread) on "
                                          f"{model} ({ncpu} cores)",
                                "convergence_lhs": r["convergence_lhs"], "eta_source": r["eta_source"]}
    print(json.dumps(line), flush=True)
    s32.close()
    s64.close()


if __name__ == "__main__":
    main()
