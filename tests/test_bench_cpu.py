"""Host logic of bench.py that needs no GPU: the oracle arm's JSON line, its
rank-0-only rule under a multi-rank launch, the loud failure of our arm
without a GPU (no CPU fallback), the clock-sample filter, the roofline of
the dominant kernel, and the traffic record's tie to the kernel source."""
import datetime
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _run(args, env_extra=None, timeout=600):
    env = dict(os.environ)
    env.update(env_extra or {})
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py")] + args, capture_output=True,
                          text=True, cwd=ROOT, env=env, timeout=timeout)


def test_reference_arm_prints_one_json_line():
    r = _run(["--impl", "reference", "--steps", "2", "--warmup", "3"])
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    out = json.loads(lines[0])
    assert out["impl"] == "reference"
    assert out["metric"] == bench.METRIC and out["unit"] == bench.UNIT
    assert out["higher_is_better"] is True and out["steps"] == 2 and out["warmup"] == 3
    assert out["value"] > 0 and out["ms_per_step"] > 0
    cb = out["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == out["value"] and cb["cores"] >= 1 and cb["sample"]
    assert out["e2e"] == {"value": out["value"], "unit": out["unit"], "h2d_bytes_per_step": 0,
                          "d2h_bytes_per_step": 0}
    assert out["config"]["n"] == 100000 and out["config"]["grid"] == [256, 256]


def test_reference_arm_runs_on_rank_zero_only():
    r = _run(["--impl", "reference", "--steps", "1", "--warmup", "3"],
             {"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"})
    assert r.returncode == 0 and r.stdout.strip() == ""


def test_our_arm_fails_loudly_without_a_gpu():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    r = _run(["--steps", "1", "--warmup", "3", "--no-cpu-baseline", "--no-batch-compare"])
    assert r.returncode != 0
    assert not any(l.lstrip().startswith("{") for l in r.stdout.splitlines())


def _row(ts, sm, reasons=()):
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    flags = ["Active" if n in reasons else "Not Active" for n in names]
    return ", ".join([ts.strftime("%Y/%m/%d %H:%M:%S.%f")[:-3], "0", str(sm), "2070", "900.5",
                      "0x0000000000000000"] + flags) + "\n"


def test_clock_samples_inside_the_region_only():
    t0 = datetime.datetime(2026, 1, 1, 12, 0, 0)
    ms = lambda k: t0 + datetime.timedelta(milliseconds=k)
    lines = [_row(ms(-100), 900, ("hw_slowdown",)),          # before the region: ignored
             _row(ms(10), 1950), _row(ms(60), 1965, ("sw_power_cap",)), _row(ms(110), 1980),
             "garbage line\n",
             _row(ms(400), 700, ("hw_thermal_slowdown",))]    # after the region: ignored
    c = bench.parse_clock_samples(lines, t0, ms(200))
    assert c["samples"] == 3 and c["sm_mhz"] == 1965 and c["sm_max_mhz"] == 2070
    assert c["reasons"] == ["sw_power_cap"]
    # a region shorter than the interval keeps the first sample after its start
    c = bench.parse_clock_samples(lines, ms(20), ms(30))
    assert c["samples"] == 1 and c["sm_mhz"] == 1965
    # a throttle reason inside the region is reported
    c = bench.parse_clock_samples(lines, ms(300), ms(500))
    assert c["reasons"] == ["hw_thermal_slowdown"] and c["sm_mhz"] == 700
    assert bench.parse_clock_samples(lines, ms(1000), ms(2000)) is None


def test_traffic_record_is_tied_to_the_kernel_source(tmp_path, monkeypatch):
    rec = {"kernel_source_hash": bench.kernel_hash(),
           "kernels": {"select2d_lag_f32": {"dram_bytes_per_algorithmic_byte": 0.25}}}
    p = tmp_path / "traffic.json"
    p.write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "PROFILE_FILE", str(p))
    assert bench.ncu_traffic("select2d_lag_f32", 1000.0) == pytest.approx(250.0)
    assert bench.ncu_traffic("another_kernel", 1000.0) is None
    rec["kernel_source_hash"] = "0" * 16      # the kernels changed since the capture
    p.write_text(json.dumps(rec))
    assert bench.ncu_traffic("select2d_lag_f32", 1000.0) is None


def test_host_cores_and_rank_seeds():
    assert 1 <= bench.host_cores() <= (os.cpu_count() or 1)
    seeds = {bench.rank_seed(2, r) for r in range(8)}
    assert len(seeds) == 8 and bench.rank_seed(2, 0) == 2


def test_all_core_oracle_baseline_runs_one_spawned_process_per_core():
    """The all-core baseline: `procs` spawned oracle processes each repeat the
    bounded sample; the job's rate sums their counts over the slowest wall
    time (here two processes on a small sample)."""
    from paper_1511_07482_gb300 import synthetic
    w = synthetic.small_case(n=300, d=2, M=[24, 20], seed=3, n_candidates=2)
    v1, n1, d1 = bench.oracle_throughput(w, 0.3, 1)
    v2, n2, d2 = bench.oracle_throughput(w, 0.3, 2)
    assert n1 >= 2 and n2 >= 4 and d1 >= 0.3 and d2 >= 0.3
    assert v1 == pytest.approx(n1 / d1) and v2 == pytest.approx(n2 / d2)


def test_search_parity_checker_sees_a_wrong_evaluation():
    """The check of the search kernel's records against the oracle: rows
    holding the oracle's own LSCV and SCV values and gradients give errors at
    rounding level, and one corrupted value is reported."""
    import numpy as np
    from oracle import binning, functionals as F, rules, selectors as S
    from paper_1511_07482_gb300 import synthetic
    w = synthetic.small_case(n=400, d=2, M=[30, 28], seed=5, n_candidates=2)
    c = binning.bin_linear(w.X, w.lo, w.hi, w.M)
    delta = rules.bin_width(w.lo, w.hi, w.M)
    a = F.autocorr_fft(c)
    rows = []
    for m, H in [(0, w.H[0]), (1, w.H[1]), (0, w.H[1])]:
        B = H if m == 0 else 2 * H + 2 * w.G
        L = rules.support_L(rules.lambda_max(B), delta, w.M)
        ev = lambda t: F.binned_direct(c, w.n, t, delta, L)
        f, g = S.lscv(ev, H, w.n, grad=True) if m == 0 else S.scv(ev, H, w.G, w.n, grad=True)
        rows.append([0, len(rows), m, H[0, 0], H[0, 1], H[1, 1], L[0], L[1], f, g[0, 0], g[0, 1], g[1, 1]])
    R = np.array(rows)
    out = bench.search_parity(w, R)
    assert out["lscv"]["evaluations"] == 2 and out["scv"]["evaluations"] == 1
    assert out["rel_err_max_search_lscv"] < 1e-10 and out["rel_err_max_search_scv"] < 1e-10
    R[2, 9] *= 1.001
    assert bench.search_parity(w, R)["rel_err_max_search_lscv"] > 1e-4


def test_roofline_of_the_dominant_kernel(monkeypatch, tmp_path):
    monkeypatch.setattr(bench, "PROFILE_FILE", str(tmp_path / "none.json"))   # no traffic record
    kstats = {
        "select2d_lag_f32": {"launches": 20, "ms": 7.3, "bytes": 282876800.0, "flops": 10326965600.0},
        "bin": {"launches": 20, "ms": 0.445, "bytes": 37242880.0, "flops": 16000000.0},
        "host:run": {"launches": 20, "ms": 99.0, "bytes": 0.0, "flops": 0.0},    # host phase: never the kernel
    }
    r = bench.roofline_of(kstats, 6800.7, 2070.0, "measured")
    assert r["kernel"] == "select2d_lag_f32" and r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    peak = 152 * 128 * 2 * 2070e6 / 1e12
    assert r["peak"] == pytest.approx(peak) and "derived" in r["peak_source"]
    assert r["avg_launch_us"] == pytest.approx(365.0)
    assert r["achieved"] == pytest.approx(10326965600.0 / 20 / 365e-6 / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / peak)
    assert r["share_of_kernel_time"] == pytest.approx(7.3 / 7.745)
    assert r["traffic"] is None
    # a kernel that moves many bytes per flop is reported against the HBM copy bandwidth
    r = bench.roofline_of({"copy": {"launches": 1, "ms": 1.0, "bytes": 5e9, "flops": 1e6}}, 6800.7, 2070.0,
                          "measured")
    assert r["bound"] == "hbm" and r["achieved"] == pytest.approx(5000.0) and r["frac"] == pytest.approx(5000 / 6800.7)
    assert bench.roofline_of({"host:run": kstats["host:run"]}, 6800.7, 2070.0, "measured") is None
