"""Host-side helpers of bench.py that feed its JSON line (no GPU): the peak
denominators and the per-launch DRAM traffic read from the committed ncu summaries."""
import hashlib
import importlib.util
import os
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_host_module", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_measured_peaks_are_read_when_present():
    bench = _bench()
    p = bench.measured_peaks()
    if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")):
        assert p["source"] == "measured"
    else:
        assert p["source"] == "fallback" and p["hbm_gbs"] == 6800.0
    assert p["bf16_tflops_sustained"] > 0


def test_committed_8bit_traffic_matches_the_current_product_kernel():
    # the timed form's roofline.traffic comes from this capture; a change to the
    # product kernel makes it stale (bench.py then reports null) until it is re-taken
    bench = _bench()
    t = bench.gemm_traffic_per_launch(32768, "k_gemm_xyT_fp8_traffic.txt")
    assert t == pytest.approx(36.70e9, rel=1e-3), "k_gemm_xyT changed since profiles/k_gemm_xyT_fp8_traffic.txt was captured"


@pytest.mark.parametrize("name,gb", [("k_gemm_xyT_traffic.txt", 70.35), ("k_gemm_xyT_split_traffic.txt", 151.47),
                                     ("k_gemm_xyT_split8_traffic.txt", 96.87)])
def test_committed_traffic_of_every_timed_form_matches_the_current_product_kernel(name, gb):
    # each form's roofline.traffic: the mean of its two products' DRAM bytes at n = 32768
    bench = _bench()
    t = bench.gemm_traffic_per_launch(32768, name)
    assert t == pytest.approx(gb * 1e9, rel=1e-3), f"k_gemm_xyT changed since profiles/{name} was captured"


def test_traffic_is_dropped_when_the_kernel_source_changes(tmp_path):
    bench = _bench()
    root = tmp_path / "repo"
    (root / "profiles").mkdir(parents=True)
    (root / "paper_2111_05366_gb300" / "csrc").mkdir(parents=True)
    src = root / "paper_2111_05366_gb300" / "csrc" / "goat_gemm.cu"
    src.write_bytes(b"// kernel v1\n")
    digest = hashlib.sha256(b"// kernel v1\n").hexdigest()
    (root / "profiles" / "t.txt").write_text(f"# capture\nn: 1000\ndram_bytes_per_launch: 5e9\nsource_sha256: {digest}\n")
    bench.ROOT = str(root)
    assert bench.gemm_traffic_per_launch(1000, "t.txt") == 5e9
    # scaled to another size by the n^3 growth of the operand re-reads
    assert bench.gemm_traffic_per_launch(2000, "t.txt") == pytest.approx(40e9)
    src.write_bytes(b"// kernel v2\n")
    assert bench.gemm_traffic_per_launch(1000, "t.txt") is None
    assert bench.gemm_traffic_per_launch(1000, "missing.txt") is None
    shutil.rmtree(root)


def test_cpu_baseline_sample_runs_the_oracle_on_every_core_with_one_sinkhorn_count():
    # the cpu_baseline leg and the reference arm time the same oracle calls on all host
    # cores (a disjoint row block per thread) and charge the same Sinkhorn iterations
    # per FW iteration; here on a small pair so that the CPU suite stays fast
    bench = _bench()
    from paper_2111_05366_gb300 import synthetic
    gp = synthetic.large_sbm_pair(512, seed=5)
    r = bench.cpu_oracle_sample(gp, 2, cores=3)
    assert r["kind"] == "oracle" and r["cores"] == 3 and r["unit"] == bench.UNIT
    assert r["sinkhorn_iters_per_fw_iter"] == bench.SK_ITERS_PER_FW
    assert r["value"] > 0 and r["value"] == pytest.approx(1.0 / r["seconds_per_fw_iter"])
    assert "6 rows" in r["sample"] and "3 threads" in r["sample"]
    assert bench.host_cores() >= 1


def test_form_report_rates_from_the_library_timings():
    # the per-form figures come from the solves' own stats: FW iterations over the
    # timed ms, the products' mean launch time, and the Sinkhorn rate on 4 n^2 bytes
    # per iteration against the measured copy peak and the nominal 7.9 TB/s
    import numpy as np
    bench = _bench()
    n = 32768
    st = {"fw_iters": 5, "ms_gemm": 560.0, "gemm_launches": 10, "ms_fw": 760.0, "ms_sinkhorn": 170.0,
          "sk_iters_total": 254, "ms_project": 245.0, "objective": 1.0, "lap_gap": 0.0}
    truth = np.arange(8)
    outs = [(truth.copy(), 1.0, st), (truth.copy(), 1.0, st)]
    peaks = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "source": "fallback"}
    r = bench.form_report(outs, 2000.0, "bf16split8", n, peaks, 2.0e7, truth)
    assert r["value"] == pytest.approx(10 / 2.0) and r["ms_per_solve"] == pytest.approx(1000.0)
    assert r["gemm_ms_per_launch"] == pytest.approx(56.0) and r["accuracy"] == 1.0
    t_it = 340.0 / 508 / 1000.0
    assert r["sinkhorn_algorithmic_gbs"] == pytest.approx(4.0 * n * n / t_it / 1e9)
    assert r["sinkhorn_frac_of_hbm_peak"] == pytest.approx(r["sinkhorn_algorithmic_gbs"] / 6800.0)
    assert r["sinkhorn_frac_of_nominal_hbm"] == pytest.approx(r["sinkhorn_algorithmic_gbs"] / 7900.0)
    # split8: the second product is 1.5 BF16-equivalent passes
    assert r["roofline"]["executed_flop_per_launch"] == pytest.approx(2.0 * n ** 3 * 1.25)
