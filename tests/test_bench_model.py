"""Host-side logic of the benchmark: the algorithmic byte model behind the
roofline figures and the rule that ties an ncu DRAM summary to the sources
it was captured on (traffic is reported only for unchanged kernels)."""
import os
import shutil

import pytest

import bench


def test_byte_model_counts_each_array_once():
    L, M = 512, 524288
    N, K2 = L * L, 4 * L * L
    b = bench.algorithmic_bytes_per_step(L, M)
    # degridding: 16-byte record, v, y, p read; z, w written (8 bytes each); the grid read once
    assert b["degrid_dual"] == 16 * M + 5 * 8 * M + 8 * K2
    # fused row kernel: inverse temporary read, forward temporary written (L x K complex each),
    # x, xt, ut, u_Dirac, x_true read and x, xt, u_Dirac written (4 bytes each)
    assert b["rows_primal"] == 2 * (8 * 2 * N) + 4 * N * 8
    # SARA analysis: xt once, then per level and basis the input LL, the three detail
    # quadrants read and written, the LL written (read and written in u at the last level)
    ana = 4 * N
    for lev in range(4):
        q = N / 4 ** (lev + 1)
        ana += 8 * 4 * ((0 if lev == 0 else 4 * q) + 2 * 3 * q + (2 * q if lev == 3 else q))
    assert b["sara_analysis"] == pytest.approx(ana)
    # gridding: record, y, w, z read; p, v written; its per-chunk partial tiles are
    # overhead, and the combined grid is counted once, in the combine pass
    assert b["grid_dual"] == 16 * M + 5 * 8 * M
    assert b["grid_combine"] == 8 * K2
    # the column passes: the L x K temporary and the K x K grid once each
    assert b["fft_fwd_cols"] == b["fft_inv_cols"] == 8 * 2 * N + 8 * K2
    # FP64 doubles every term
    b64 = bench.algorithmic_bytes_per_step(L, M, rsz=8)
    assert b64["fft_fwd_cols"] == 2 * b["fft_fwd_cols"]


def test_committed_dram_summaries_parse_and_name_their_sources():
    """Every profiles/ncu_dram_<workload>.txt names the sources digest it was
    captured on and holds one line per kernel timing name that the bench's
    byte model knows, with positive bytes per launch."""
    prof = os.path.join(bench.ROOT, "profiles")
    names = set(bench.algorithmic_bytes_per_step(64, 1000))
    files = [f for f in os.listdir(prof) if f.startswith("ncu_dram_") and f.endswith(".txt")]
    assert {"ncu_dram_c2_512.txt", "ncu_dram_c3_1024.txt", "ncu_dram_c5_4096.txt"} <= set(files)
    for f in files:
        lines = [ln.strip() for ln in open(os.path.join(prof, f)) if ln.strip()]
        digests = [ln for ln in lines if ln.startswith("sources sha256:")]
        assert len(digests) == 1 and len(digests[0].split(":", 1)[1].strip()) == 64, f
        rows = [ln.split() for ln in lines if not ln.startswith("#") and ":" not in ln]
        assert rows, f
        for k, v, n, t in rows:
            assert k in names and float(v) > 0 and int(n) >= 1 and float(t) > 0, (f, k)


def test_traffic_only_for_the_sources_it_was_captured_on(tmp_path, monkeypatch):
    root = tmp_path / "repo"
    shutil.copytree(os.path.join(bench.ROOT, "paper_1701_01748_gb300", "csrc"),
                    root / "paper_1701_01748_gb300" / "csrc")
    (root / "profiles").mkdir()
    monkeypatch.setattr(bench, "ROOT", str(root))
    assert bench.dram_traffic("w")[0] == {}                 # no capture
    digest = bench.source_digest()
    (root / "profiles" / "ncu_dram_w.txt").write_text(
        "# header\nsources sha256: " + digest + "\nsara_analysis 3075904 12 14.2\ngrid_dual 21047723 3 48.6\n")
    traffic, why = bench.dram_traffic("w")
    assert traffic == {"sara_analysis": 3075904.0, "grid_dual": 21047723.0} and "ncu" in why
    # any change to a kernel source voids the capture
    f = root / "paper_1701_01748_gb300" / "csrc" / "vis.cu"
    f.write_text(f.read_text() + "\n// changed\n")
    assert bench.dram_traffic("w") == ({}, "kernels changed since the ncu capture")


def test_reference_arm_prints_the_contract_line():
    """`bench.py --impl reference` times the oracle (one PPD iteration per step)
    and prints one JSON line with the contract's keys."""
    import json
    import subprocess
    import sys
    r = subprocess.run([sys.executable, os.path.join(bench.ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "0"], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["value"] > 0 and line["higher_is_better"] is True
    assert line["config"]["workload"] == bench.WORKLOAD
    assert line["config"] == bench.workload_config(bench.WORKLOAD)
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["cpu_baseline"]["kind"] == "oracle"
    # the oracle runs Algorithm 3 with the paper's eta (stored, not recomputed) and converges
    assert line["oracle"]["eta_source"].startswith("tests/golden/op_norms.json")
    assert line["oracle"]["convergence_lhs"] < 1.0


def test_oracle_setup_meets_the_convergence_condition_and_stays_finite():
    """The set-up the benchmark's oracle arm builds: eta = 1/||U^{1/2} Phi||^2 with
    the norm from the oracle's Lanczos routine, so tau eta ||U^{1/2} Phi||^2 +
    tau zeta ||Psi||^2 < 1 (Eq. "convergence-req-explicit-pd"), and the driver's
    steps + warm-up iterations (25) run without overflow."""
    import math
    from oracle import ppd as oppd
    p, S, info = bench.oracle_setup("c1_128", 1701)
    assert info["convergence_lhs"] < 1.0
    # the power iteration approaches the norm from below (a Rayleigh quotient)
    lo, _ = oppd.op_norm_sq(S.P, S.U, max_iter=30)
    assert lo <= info["op_norm_sq"] * (1 + 1e-9)
    st = oppd.init_state(S)
    for _ in range(25):
        h = oppd.iterate(st, S)
    assert all(math.isfinite(r) for r in h["residual"]) and math.isfinite(h["snr"]) and h["snr"] > 0


def test_stored_operator_norms_belong_to_the_benchmark_workloads():
    """tests/golden/op_norms.json was written for the workloads' current seeds and sizes."""
    import json
    from paper_1701_01748_gb300 import synth
    table = json.load(open(bench.GOLDEN_NORMS))
    for name in ("c2_512", "c3_1024"):
        cfg = synth.CONFIGS[name]
        rec = table[name]
        assert (rec["seed"], rec["L"], rec["M"], rec["n_blocks"]) == (cfg["seed"], cfg["L"], cfg["M"],
                                                                     cfg["n_blocks"])
        assert rec["op_norm_sq"] > 0
