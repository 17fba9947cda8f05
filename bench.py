"""Throughput benchmark: candidate-bandwidth objective evaluations per second.

Workload (one "step" = the whole hot path on one dataset): the bivariate
3-component normal mixture with n = 100000 samples on a 256 x 256 grid
(synthetic.mixture_2d_large, seed 2): linear binning, count spectrum and
autocorrelation, then the full unconstrained LSCV minimisation and the full
SCV minimisation (pilot G = normal-scale matrix) over the 3 free entries of H,
each with exact gradients and `--n-starts` starts (both criteria in one
device-resident search launch), FP32 arithmetic with compensated sums.
metric = objective(+gradient) evaluations / step time.

value     : device-timed (CUDA events on the stream the library uses), sample
            already resident in HBM; L2 flushed (256 MiB write) before every
            step; the library's per-launch events off (launch sequences replay
            as CUDA graphs).
e2e       : the same step through the C ABI with the sample in pinned host
            memory (host->device copy inside the timed region) and host results.
roofline  : the kernel with the largest summed CUDA-event time over the same
            steps run again with the library's per-launch events on;
            algorithmic flops and bytes per launch, against the FP32 ALU peak
            and the measured HBM peak.
clocks    : nvidia-smi samples (50 ms) stamped inside the timed region.
cpu_baseline / --impl reference : the CPU FP64 oracle (test infrastructure)
            on a bounded sample of the same workload.

Multi-GPU (torchrun): every rank runs its own replica of the workload with its
own seed (independent datasets, no data-path collective); value = all ranks'
evaluations / max-over-ranks time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "candidate-H objective evals/sec (+grad) at stated rel err vs FP64; % HBM roofline"
UNIT = "evals/s"
SM_COUNT = 152
FP32_LANES_PER_SM = 128
PROFILE_FILE = os.path.join(ROOT, "profiles", "ncu_traffic.json")


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def rank_seed(base: int, rank: int, stride: int = 1000) -> int:
    """Seed of this rank's replica of the workload: independent datasets per
    rank, the same on every run."""
    return base + stride * rank


def combine_ranks(local, world: int, device=None):
    """[time_ms, evals, e2e_time_ms, e2e_evals] of this rank -> the whole
    job's: times are the maximum over ranks (the job ends with its slowest
    rank), evaluation counts the sum over ranks."""
    if world == 1:
        return [float(v) for v in local]
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v) for v in local], dtype=torch.float64, device=device)
    mx, sm = t.clone(), t.clone()
    dist.all_reduce(mx, op=dist.ReduceOp.MAX)
    dist.all_reduce(sm, op=dist.ReduceOp.SUM)
    return [mx[0].item(), sm[1].item(), mx[2].item(), sm[3].item()]


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d.get("hbm_gbs", 6800.0)), float(d.get("sm_max_mhz", 2070.0)), "measured"
    return 6800.0, 2070.0, "fallback"


class Clocks:
    """nvidia-smi sampling (every 50 ms) started before the warm-up; only the
    samples stamped inside the timed region count.  A region shorter than the
    sampling interval keeps the first sample after its start."""

    def __init__(self, index: int):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        q = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        self.t0 = self.t1 = None
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={index}", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                       "-lms", "50"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def start(self):
        import datetime
        self.t0 = datetime.datetime.now()

    def end(self):
        import datetime
        self.t1 = datetime.datetime.now()

    def stop(self):
        if self.p is None:
            return None
        time.sleep(0.12)   # let a sample land after the region
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        lines = self.f.readlines()
        os.unlink(self.f.name)
        return parse_clock_samples(lines, self.t0, self.t1)


def parse_clock_samples(lines, t0, t1, interval_ms=50):
    """nvidia-smi CSV rows (timestamp, index, clocks.sm, clocks.max.sm,
    power.draw, reasons.active, hw_slowdown, hw_thermal_slowdown,
    sw_thermal_slowdown, sw_power_cap) -> the clocks object of the bench
    line: median SM clock of the samples stamped inside [t0, t1] and every
    throttle reason active in any of them.  A region shorter than the
    sampling interval keeps the first sample after t0; no sample gives None."""
    import datetime
    rows = []
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in lines:
        parts = [x.strip() for x in line.split(",")]
        if len(parts) < 10:
            continue
        try:
            ts = datetime.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f")
            rows.append((ts, float(parts[2]), float(parts[3]),
                         [nm for nm, v in zip(names, parts[6:10]) if v.lower().startswith("active")]))
        except ValueError:
            continue
    inside = [r for r in rows if t0 and t1 and t0 <= r[0] <= t1]
    if not inside:
        inside = [r for r in rows if t0 and r[0] >= t0][:1]
    if not inside:
        return None
    reasons = sorted({nm for r in inside for nm in r[3]})
    return {"sm_mhz": statistics.median(r[1] for r in inside), "sm_max_mhz": inside[-1][2], "reasons": reasons,
            "samples": len(inside), "interval_ms": interval_ms}


def roofline_of(kstats, hbm, smmax, src):
    """The roofline object of the bench line for the kernel with the largest
    summed CUDA-event time: algorithmic flops and bytes per launch over the
    average launch time, against the FP32 ALU peak (152 SMs x 128 lanes x 2
    flop x the maximum SM clock) or the measured HBM copy bandwidth, whichever
    the kernel is closer to.  kstats: name -> {launches, ms, bytes, flops};
    names starting with "host:" are host phases, not kernels."""
    kernels = {k: v for k, v in kstats.items() if not k.startswith("host:")}
    if not kernels:
        return None
    kname = max(kernels, key=lambda k: kernels[k]["ms"])
    k = kernels[kname]
    avg_s = k["ms"] / 1000.0 / max(k["launches"], 1)
    fl = k["flops"] / max(k["launches"], 1)
    by = k["bytes"] / max(k["launches"], 1)
    alu_peak = SM_COUNT * FP32_LANES_PER_SM * 2 * smmax * 1e6 / 1e12        # TFLOP/s
    a_tf = fl / avg_s / 1e12
    a_gb = by / avg_s / 1e9
    if a_gb / hbm >= a_tf / alu_peak:
        roof = {"bound": "hbm", "achieved": a_gb, "peak": hbm, "unit": "GB/s", "frac": a_gb / hbm,
                "peak_source": f"{src} copy bandwidth"}
    else:
        roof = {"bound": "alu", "achieved": a_tf, "peak": alu_peak, "unit": "TFLOP/s", "frac": a_tf / alu_peak,
                "peak_source": f"derived: {SM_COUNT} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 flop x "
                               f"{smmax:.0f} MHz ({src} maximum SM clock)"}
    roof.update({"kernel": kname, "launches": k["launches"],
                 "avg_launch_us": avg_s * 1e6, "algorithmic_bytes_per_launch": by,
                 "algorithmic_flops_per_launch": fl, "traffic": ncu_traffic(kname, by),
                 "share_of_kernel_time": k["ms"] / sum(v["ms"] for v in kernels.values()),
                 "timing": "CUDA events around every launch on the library stream, over min(steps, 20) "
                           "identical steps run right after the timed region"})
    return roof


def kernel_hash():
    h = hashlib.sha256()
    for f in ("engine.cu", "engine.cuh", "lag.cu", "devutil.cuh"):
        h.update(open(os.path.join(ROOT, "paper_1511_07482_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def ncu_traffic(kname, alg_bytes_per_launch):
    """DRAM bytes per launch from the committed ncu capture (dram__bytes_read
    + write of one captured launch), scaled to this run's launches by their
    algorithmic bytes; None when the capture predates the current kernel
    source."""
    if not os.path.exists(PROFILE_FILE):
        return None
    try:
        d = json.load(open(PROFILE_FILE))
    except Exception:
        return None
    if d.get("kernel_source_hash") != kernel_hash():
        return None
    k = d.get("kernels", {}).get(kname)
    if k is None:
        return None
    return k["dram_bytes_per_algorithmic_byte"] * alg_bytes_per_launch


# ------------------------------------------------------------------ our arm

def run_ours(args):
    import torch
    import torch.distributed as dist
    from paper_1511_07482_gb300 import LSCV, SCV, Context, synthetic

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    ctx = Context(local)
    ctx.set_graphs(args.graphs == "on")
    from paper_1511_07482_gb300 import ENGINE_AUTO, ENGINE_FFT, ENGINE_MULTIPASS
    ctx.set_engine({"auto": ENGINE_AUTO, "fft": ENGINE_FFT, "multipass": ENGINE_MULTIPASS}[args.engine])
    stream = torch.cuda.current_stream(dev)
    if args.workload == "select2d":
        w = synthetic.mixture_2d_large(seed=rank_seed(2, rank))
        X_dev = torch.from_numpy(w.X).to(dev)
        X_pin = torch.from_numpy(w.X).pin_memory()

        def step(X):
            ds = ctx.bin(X, w.lo, w.hi, w.M)
            (H1, f1, e1), (H2, f2, e2) = ds.select_H_many([LSCV, SCV], G=w.G, n_starts=args.n_starts,
                                                          max_iter=args.max_iter)
            ds.close()
            return e1 + e2, (H1, f1, H2, f2)
        workload_desc = (w.name + ": bin + full LSCV and SCV minimisation (3 free entries of H, adjoint "
                         "gradients)")
    elif args.workload == "psi4_3d":
        w = synthetic.mixture_3d(seed=rank_seed(3, rank), **({"n_candidates": args.candidates} if args.candidates else {}))
        X_dev = torch.from_numpy(w.X).to(dev)
        X_pin = torch.from_numpy(w.X).pin_memory()

        def step(X):
            ds = ctx.bin(X, w.lo, w.hi, w.M)
            ds.psi(w.H, 4)
            ds.close()
            return len(w.H), None
        workload_desc = w.name + ": bin + psi_4 (15 unique partials) for 256 candidate H in one call"
    elif args.workload == "uneven512":
        ws = synthetic.batched_uneven(base_seed=rank_seed(4, rank, 100000))
        w = ws[0]
        X_dev = [torch.from_numpy(v.X).to(dev) for v in ws]
        X_pin = [torch.from_numpy(v.X).pin_memory() for v in ws]

        def step(Xs):
            dss = ctx.bin_many(Xs, [v.lo for v in ws], [v.hi for v in ws], [v.M for v in ws])
            ctx.batch_lscv(dss, [v.H for v in ws])
            for ds in dss:
                ds.close()
            return 16 * len(ws), None
        workload_desc = "512 bivariate datasets (n log-uniform 1e3..1e5, grids 64^2..256^2): batched binning + " \
                        "LSCV and gradient for 16 H each in one batched call"
    elif args.workload == "lscv_batch16":
        w = synthetic.mixture_2d_large(seed=rank_seed(2, rank))
        X_dev = torch.from_numpy(w.X).to(dev)
        X_pin = torch.from_numpy(w.X).pin_memory()

        def step(X):
            ds = ctx.bin(X, w.lo, w.hi, w.M)
            for _ in range(20):
                ds.lscv(w.H, grad=True)
            ds.close()
            return 20 * len(w.H), None
        workload_desc = w.name + ": bin + 20 batches of LSCV and gradient at 16 candidate H"
    elif args.workload == "qr_e8":
        # the V-statistics experiment's shape: a bivariate N(0, I) sample,
        # M = 100 per axis, Q_r for total derivative orders 0, 2, 4, 6, 8
        rng = np.random.default_rng(rank_seed(8, rank))
        Xq = rng.standard_normal((10000, 2))
        Sq = synthetic.normal_scale(Xq)
        loq, hiq = synthetic.grid_range(Xq, Sq)
        w = synthetic.Workload("normal-2d-n10000-M100", Xq, loq, hiq, [100, 100], [Sq], G=Sq)
        X_dev = torch.from_numpy(Xq).to(dev)
        X_pin = torch.from_numpy(Xq).pin_memory()

        def step(X):
            ds = ctx.bin(X, loq, hiq, [100, 100])
            for r in (0, 2, 4, 6, 8):
                ds.qr(Sq, r)
            ds.close()
            return 5, None
        workload_desc = "normal-2d-n10000-M100: bin + Q_r (Eq. 32) for total derivative orders 0, 2, 4, 6, 8"
    else:  # plugin4d
        w = synthetic.mixture_4d(seed=rank_seed(5, rank), n_candidates=args.candidates or 16)
        X_dev = torch.from_numpy(w.X).to(dev)
        X_pin = torch.from_numpy(w.X).pin_memory()
        from paper_1511_07482_gb300 import P_FIXED

        def step(X):
            ds = ctx.bin(X, w.lo, w.hi, w.M, P_rule=P_FIXED, P_fixed=w.P)
            ds.pi(w.H, w.G, grad=True)
            ds.eta02(w.H, w.G)
            ds.close()
            return 2 * len(w.H), None
        workload_desc = w.name + ": bin + psi_4(G) + PI(H) with gradient and eta_{0,2}(H, G) for 16 H"

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)

    clocks = Clocks(local)   # sampling starts before the warm-up
    for _ in range(args.warmup):
        step(X_dev)

    # ---- device-resident timed region (library profiling off, so that
    # repeated launch sequences replay as CUDA graphs, as in production use)
    times, evals = [], 0
    ctx.profile(0)   # clears the launch and copy counters
    clocks.start()
    for _ in range(args.steps):
        flush.fill_(1.0)
        barrier()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        e, res = step(X_dev)
        b.record(stream)
        torch.cuda.synchronize(dev)
        times.append(a.elapsed_time(b))
        evals += e
    clocks.end()
    _, launches, _, _ = ctx.profile_read()
    clk = clocks.stop()
    t_total = sum(times)

    # ---- end-to-end through the C ABI with host buffers
    e2e_times, e2e_evals = [], 0
    ctx.profile(0)
    for _ in range(args.steps):
        flush.fill_(1.0)
        barrier()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        e, _ = step(X_pin)
        b.record(stream)
        torch.cuda.synchronize(dev)
        e2e_times.append(a.elapsed_time(b))
        e2e_evals += e
    _, _, h2d, d2h = ctx.profile_read()

    # ---- per-kernel CUDA events (on the library's stream, bracketing every
    # launch) over the same number of identical steps, and host-side phase
    # times; kept out of the timed regions above because the per-launch
    # events bypass the graph replay
    prof_times = []
    prof_steps = min(args.steps, 20)
    ctx.profile(1)
    for _ in range(prof_steps):
        flush.fill_(1.0)
        barrier()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        step(X_dev)
        b.record(stream)
        torch.cuda.synchronize(dev)
        prof_times.append(a.elapsed_time(b))
    kstats, _, _, _ = ctx.profile_read()
    ctx.profile(0)

    # max over ranks
    tot = torch.tensor(combine_ranks([t_total, evals, sum(e2e_times), e2e_evals], world, dev), dtype=torch.float64)
    value = tot[1].item() / (tot[0].item() / 1000.0)
    e2e_value = tot[3].item() / (tot[2].item() / 1000.0)

    if rank != 0:
        if world > 1:
            dist.barrier()
            dist.destroy_process_group()
        return

    roof = roofline_of(kstats, *peaks())
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": tot[0].item() / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": workload_desc, "n": w.n, "d": w.d, "grid": w.M,
                   "n_starts": args.n_starts, "max_iter": args.max_iter, "precision": "fp32, fp64 reductions",
                   "l2": "flushed by a 256 MiB device write before every step",
                   "evals_per_step": evals / args.steps},
        "roofline": roof,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(h2d / args.steps),
                "d2h_bytes_per_step": int(d2h / args.steps)},
        "gpu_launches": int(launches),
        "kernel_times_ms": {k: round(v["ms"], 3) for k, v in kstats.items() if not k.startswith("host:")},
        "kernel_work": {k: {"launches": v["launches"], "alg_bytes": v["bytes"], "alg_flops": v["flops"]}
                        for k, v in kstats.items() if not k.startswith("host:")},
        "host_times_ms": {k[5:]: round(v["ms"], 3) for k, v in kstats.items() if k.startswith("host:")},
        "profiled_ms_per_step": sum(prof_times) / prof_steps,
        "clocks": clk,
    }
    if args.workload == "select2d":
        # one step is one LSCV and one SCV selection
        out["ms_per_selection"] = {"lscv_and_scv": out["ms_per_step"],
                                   "note": "one step selects H for both criteria (16 starts each)"}
    if world == 1 and args.workload == "select2d" and not args.no_fp64:
        out["fp64_path"], fp64_res = fp64_selection(ctx, w, dev, args)
    else:
        fp64_res = None
    if not args.no_cpu_baseline and world == 1 and args.workload == "select2d":
        rec = search_records(ctx, w, dev, args)
        out["cpu_baseline"] = cpu_baseline(w, args, res, fp64_res, rec)
        for k in ("rel_err_max_search_lscv", "rel_err_max_search_scv"):
            out[k] = out["cpu_baseline"]["search_parity"][k]
        if fp64_res is not None:
            out["fp64_path"].update(out["cpu_baseline"].pop("fp64_parity"))
    if world == 1 and args.workload == "select2d" and not args.no_batch_compare:
        out["batched_vs_single_h"] = batched_vs_single(ctx, w, dev)
    print(json.dumps(out))
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


def fp64_selection(ctx, w, dev, args, steps=3):
    """The same step (binning + LSCV and SCV selection, same starts) on an FP64
    dataset: FP64 arithmetic on the GPU, searched from the host with one
    batched evaluation per round.  Device-timed with CUDA events like the FP32
    line; returns (its line, the selected bandwidths and values)."""
    import torch
    from paper_1511_07482_gb300 import FP64, LSCV, SCV
    X = torch.from_numpy(w.X).to(dev)
    stream = torch.cuda.current_stream(dev)

    def step():
        ds = ctx.bin(X, w.lo, w.hi, w.M, precision=FP64)
        (H1, f1, e1), (H2, f2, e2) = ds.select_H_many([LSCV, SCV], G=w.G, n_starts=args.n_starts,
                                                      max_iter=args.max_iter)
        ds.close()
        return e1 + e2, (H1, f1, H2, f2)
    step()
    t, ev = 0.0, 0
    for _ in range(steps):
        torch.cuda.synchronize(dev)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        e, res = step()
        b.record(stream)
        torch.cuda.synchronize(dev)
        t += a.elapsed_time(b)
        ev += e
    line = {"value": ev / (t / 1000.0), "unit": UNIT, "ms_per_step": t / steps, "evals_per_step": ev / steps,
            "precision": "fp64 (every kernel value, transform and sum)", "search": "host-driven, one batched "
            "evaluation per round", "steps": steps}
    return line, res


def search_records(ctx, w, dev, args):
    """One more step of the FP32 selection with the search kernel recording
    every evaluation it makes (bandwidth, support, value, gradient): rows of
    12 values, outside every timed region."""
    import torch
    from paper_1511_07482_gb300 import LSCV, SCV
    cap = 400
    rec = torch.full((2 * args.n_starts * cap * 12,), float("nan"), dtype=torch.float64, device=dev)
    ds = ctx.bin(torch.from_numpy(w.X).to(dev), w.lo, w.hi, w.M)
    ctx.set_search_record(rec, cap)
    ds.select_H_many([LSCV, SCV], G=w.G, n_starts=args.n_starts, max_iter=args.max_iter)
    ctx.set_search_record(None)
    ds.close()
    R = rec.view(-1, 12).cpu().numpy()
    return R[np.isfinite(R[:, 0])]


def crossover(args):
    """Per-bandwidth device time of the lag-domain engine against the FFT
    route (the transforms of Eqs. 19-24) as the support L grows, on the
    benchmark datasets' shapes: LSCV with its gradient for 32 bandwidths per
    call, the bandwidth set to a multiple of the identity chosen so that Eq. 26
    gives the listed L on the first axis (the last rung is the untruncated
    support L = M - 1).  Times are the library's CUDA events around every
    kernel of a second, identical call (the count spectrum and
    autocorrelation are cached by the first); one JSON object per rung."""
    import torch
    from paper_1511_07482_gb300 import ENGINE_AUTO, ENGINE_FFT, L_FULL, P_FIXED, Context, synthetic
    torch.cuda.set_device(0)
    cases = [("mixture-2d-n100000-M256", synthetic.mixture_2d_large(), {}, [8, 16, 32, 64, 128, 255]),
             ("mixture-3d-n1000000-M128", synthetic.mixture_3d(n_candidates=4), {}, [4, 8, 16, 32, 64, 127]),
             ("mixture-4d-n1000000-M48", synthetic.mixture_4d(n_candidates=4), {"P_rule": P_FIXED}, [4, 8, 16, 24, 47])]
    per_dataset = ("acorr", "spec_df", "stage_a_f64", "mid_f64", "final_f64", "bin")
    rows = []
    for name, w, extra, Ls in cases:
        delta = (np.asarray(w.hi) - np.asarray(w.lo)) / (np.asarray(w.M) - 1)
        for L in Ls:
            full = L == w.M[0] - 1
            lam = (L * delta[0] / 3.7) ** 2 * (0.999 if not full else 1.0)
            Hs = np.stack([lam * np.eye(w.d)] * 32)
            row = {"workload": name, "d": w.d, "M": list(w.M), "L_target": L}
            for eng_name, eng in (("lag", ENGINE_AUTO), ("fft", ENGINE_FFT)):
                ctx = Context(0)
                ctx.set_engine(eng)
                opts = dict(extra)
                if "P_rule" in opts:
                    opts["P_fixed"] = w.P
                if full:
                    opts["L_basis"] = L_FULL
                ds = ctx.bin(w.X, w.lo, w.hi, w.M, **opts)
                try:
                    Lp, Pp = ds.plan(0, Hs[0])
                    if extra.get("P_rule") is not None and any(p < m + l for p, m, l in zip(Pp, w.M, Lp)):
                        row[eng_name] = None          # the fixed padding aliases at this support
                        continue
                    ds.lscv(Hs, grad=True)
                    torch.cuda.synchronize()
                    ctx.profile(1)
                    ds.lscv(Hs, grad=True)
                    torch.cuda.synchronize()
                    ks, _, _, _ = ctx.profile_read()
                    ctx.profile(0)
                except Exception as e:       # noqa: BLE001 - reported in the row
                    row[eng_name] = {"error": str(e)[:200]}
                    continue
                finally:
                    ds.close()
                    ctx.close()
                ker = {k: v for k, v in ks.items() if not k.startswith("host:") and k not in per_dataset}
                row.update({"L": Lp, "P": Pp})
                row[eng_name] = {"us_per_bandwidth": 1000.0 * sum(v["ms"] for v in ker.values()) / len(Hs),
                                 "kernels": sorted(ker)}
            rows.append(row)
            print(json.dumps(row), flush=True)
    return rows


def batched_vs_single(ctx, w, dev, reps=5):
    """LSCV + gradient at 256 candidate bandwidths around the normal-scale
    matrix of the bench dataset: all of them in one call against one call per
    bandwidth (the plain single-H path).  Both go through the synchronous
    public API, so each is timed on the host clock around the calls; the
    best of `reps` repetitions is kept."""
    import torch
    ds = ctx.bin(torch.from_numpy(w.X).to(dev), w.lo, w.hi, w.M)
    Hs = synthetic_candidates(w, 256)
    ds.lscv(Hs[:4], grad=True)   # autocorrelation and first-use set-up outside the timing
    tb = ts = float("inf")
    for _ in range(reps):
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        vb, _ = ds.lscv(Hs, grad=True)
        t1 = time.perf_counter()
        vs = [ds.lscv(h, grad=True)[0][0] for h in Hs]
        t2 = time.perf_counter()
        tb, ts = min(tb, t1 - t0), min(ts, t2 - t1)
    ds.close()
    return {"candidates": len(Hs), "batched_evals_per_s": len(Hs) / tb, "single_h_evals_per_s": len(Hs) / ts,
            "max_rel_diff": float(np.max(np.abs(np.asarray(vs) - vb) / np.abs(vb)))}


def synthetic_candidates(w, k):
    from paper_1511_07482_gb300 import synthetic
    H0 = synthetic.normal_scale(w.X)
    return synthetic.candidates_around(np.random.default_rng(11), H0, k)


# ------------------------------------------------------------------ oracle arm

def oracle_evals(w, Hs, G):
    """The oracle's LSCV+gradient and SCV+gradient at the given H (FP64,
    binned, the paper's FFT steps); returns (#evals, results)."""
    from oracle import binning, functionals as F, rules, selectors as S
    c = binning.bin_linear(w.X, w.lo, w.hi, w.M)
    delta = rules.bin_width(w.lo, w.hi, w.M)
    res = []
    for H in Hs:
        L = rules.support_L(rules.lambda_max(H), delta, w.M)
        P = rules.P_minimal(w.M, L)
        res.append(("lscv", S.lscv(lambda t: F.binned_fft(c, w.n, t, delta, L, P), H, w.n, grad=True)))
        L2 = rules.support_L(rules.lambda_max(2 * H + 2 * G), delta, w.M)
        P2 = rules.P_minimal(w.M, L2)
        res.append(("scv", S.scv(lambda t: F.binned_fft(c, w.n, t, delta, L2, P2), H, G, w.n, grad=True)))
    return 2 * len(Hs), res


def host_cores() -> int:
    """Host cores this process may run on."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def _oracle_worker(job):
    """One oracle process of the all-core baseline: repeats the bounded
    sample (binning of all n, then LSCV+gradient and SCV+gradient at one
    bandwidth) until `seconds` have passed; returns its evaluation count and
    wall time.  Started by spawn, it imports only the oracle and numpy."""
    import types
    X, lo, hi, M, Hs, G, name, seconds = job
    sys.path.insert(0, ROOT)
    wk = types.SimpleNamespace(X=X, lo=lo, hi=hi, M=M, n=X.shape[0], name=name)
    t0, n_ev, i = time.perf_counter(), 0, 0
    while time.perf_counter() - t0 < seconds:
        k, _ = oracle_evals(wk, [Hs[i % len(Hs)]], G)
        n_ev += k
        i += 1
    return n_ev, time.perf_counter() - t0


def oracle_throughput(w, seconds: float, procs: int):
    """Evaluations per second of `procs` concurrent oracle processes (spawned:
    no process inherits CUDA state), each running the bounded sample for
    `seconds`; the job's rate is the summed count over the slowest wall time."""
    import multiprocessing as mp
    job = (w.X, w.lo, w.hi, list(w.M), list(w.H), w.G, w.name, seconds)
    if procs == 1:
        n_ev, dt = _oracle_worker(job)
        return n_ev / dt, n_ev, dt
    with mp.get_context("spawn").Pool(procs) as pool:
        out = pool.map(_oracle_worker, [job] * procs)
    n_ev = sum(o[0] for o in out)
    dt = max(o[1] for o in out)
    return n_ev / dt, n_ev, dt


def search_parity(w, rec):
    """Max error of the search kernel's own evaluations (value and the three
    gradient entries of every recorded LSCV and SCV evaluation) against the
    FP64 oracle at the same FP32 bandwidth and support, each relative to
    max(|ref|, S/10), S the magnitude of the summed terms (the FP32
    tolerance's normalisation)."""
    from oracle import binning, functionals as F, rules, selectors as S
    c = binning.bin_linear(w.X, w.lo, w.hi, w.M)
    delta = rules.bin_width(w.lo, w.hi, w.M)
    a = F.autocorr_fft(c)
    err = {0: [0.0, 0.0, 0], 1: [0.0, 0.0, 0]}
    for r in rec:
        m = int(r[2])
        H = np.array([[r[3], r[4]], [r[4], r[5]]])
        L = [int(r[6]), int(r[7])]
        ev = lambda t: F.lag_sums(a, w.n, t, delta, L)[0]
        ea = lambda t: F.lag_sums(a, w.n, t, delta, L)[1]
        if m == 0:
            val, g = S.lscv(ev, H, w.n, grad=True)
            sv, sg = S.abs_scales(ea, "lscv", H, w.n)
        else:
            val, g = S.scv(ev, H, w.G, w.n, grad=True)
            sv, sg = S.abs_scales(ea, "scv", H, w.n, w.G)
        gg = np.array([[r[9], r[10]], [r[10], r[11]]])
        e = err[m]
        e[0] = max(e[0], abs(r[8] - val) / max(abs(val), 0.1 * sv))
        e[1] = max(e[1], float(np.max(np.abs(gg - g) / np.maximum(np.abs(g), 0.1 * sg))))
        e[2] += 1
    return {"rel_err_max_search_lscv": max(err[0][0], err[0][1]), "rel_err_max_search_scv": max(err[1][0], err[1][1]),
            "lscv": {"evaluations": err[0][2], "value": err[0][0], "gradient": err[0][1]},
            "scv": {"evaluations": err[1][2], "value": err[1][0], "gradient": err[1][1]},
            "normalisation": "|got - ref| / max(|ref|, S/10), S = magnitude of the summed terms; tolerance 1e-5"}


def cpu_baseline(w, args, gpu_res, fp64_res=None, rec=None):
    """The oracle, as it stands, on a bounded sample: binning of the full
    sample plus LSCV+grad and SCV+grad at one bandwidth per repetition, on one
    host core and on every host core (one oracle process per core); also the
    oracle's check of the GPU's results: the objective values at the selected
    bandwidths (FP32 and FP64 paths) and every evaluation the search kernel
    recorded."""
    H1, f1, H2, f2 = gpu_res
    _, res = oracle_evals(w, [H1], w.G)
    _, res2 = oracle_evals(w, [H2], w.G)
    rel_l = abs(f1 - res[0][1][0]) / abs(res[0][1][0])
    rel_s = abs(f2 - res2[1][1][0]) / abs(res2[1][1][0])
    ncore = host_cores()
    half = args.cpu_seconds / 2.0
    v1, n1, d1 = oracle_throughput(w, half, 1)
    vall, nall, dall = oracle_throughput(w, half, ncore)
    out = {"value": vall, "unit": UNIT, "cores": ncore, "kind": "oracle", "host_cores": ncore,
           "sample": f"{w.name}: repetitions of oracle binning of all n followed by LSCV+gradient and SCV+gradient "
                     f"in FP64 (numpy FFT) at one bandwidth; {ncore} processes x {half:.0f} s ({nall} evaluations) "
                     f"for the all-core value, one process x {half:.0f} s ({n1} evaluations) for one core",
           "one_core": {"value": v1, "unit": UNIT, "cores": 1, "evaluations": n1, "seconds": d1},
           "all_cores": {"value": vall, "unit": UNIT, "cores": ncore, "evaluations": nall, "seconds": dall},
           "rel_err_lscv_at_selected_H": rel_l, "rel_err_scv_at_selected_H": rel_s}
    if rec is not None:
        out["search_parity"] = search_parity(w, rec)
    if fp64_res is not None:
        G1, g1, G2, g2 = fp64_res
        _, r1 = oracle_evals(w, [G1], w.G)
        _, r2 = oracle_evals(w, [G2], w.G)
        out["fp64_parity"] = {"rel_err_lscv_at_selected_H": abs(g1 - r1[0][1][0]) / abs(r1[0][1][0]),
                              "rel_err_scv_at_selected_H": abs(g2 - r2[1][1][0]) / abs(r2[1][1][0])}
    return out


def run_reference(args):
    rank, world, local = dist_env()
    if world > 1 and rank != 0:
        return
    from paper_1511_07482_gb300 import synthetic
    w = synthetic.mixture_2d_large()
    Hs = list(w.H[:4])
    for _ in range(args.warmup):
        oracle_evals(w, Hs, w.G)
    t, ev = 0.0, 0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        n_ev, _ = oracle_evals(w, Hs, w.G)
        t += time.perf_counter() - t0
        ev += n_ev
    value = ev / t
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": 1000.0 * t / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": w.name + ": bin + LSCV and SCV objective+gradient evaluations (oracle)",
                      "n": w.n, "d": w.d, "grid": w.M},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "host_cores": host_cores(),
                            "sample": f"per step: oracle binning of all n plus {2 * len(Hs)} FP64 "
                                      f"objective+gradient evaluations, one process"},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--graphs", choices=["on", "off"], default="on",
                    help="CUDA-graph replay of repeated launch sequences (the timed regions run with the library's "
                         "per-launch events off, so they replay; the per-kernel profiled pass launches directly)")
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n-starts", type=int, default=16)
    ap.add_argument("--workload", default="select2d", choices=["select2d", "psi4_3d", "uneven512", "plugin4d", "lscv_batch16", "qr_e8"],
                    help="select2d (default): the n=1e5 bivariate selection workload; the others time the "
                         "batched 3-D psi_4, 512-dataset LSCV and 4-D plug-in configurations")
    ap.add_argument("--max-iter", type=int, default=60)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch-compare", action="store_true",
                    help="skip the batched-vs-single-H LSCV comparison of the select2d workload")
    ap.add_argument("--cpu-seconds", type=float, default=12.0,
                    help="oracle baseline budget: half on one core, half on every host core")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64-path line of the select2d workload")
    ap.add_argument("--engine", choices=["auto", "fft", "multipass"], default="auto",
                    help="evaluation engine of the library (auto: lag domain wherever the padding has no aliasing)")
    ap.add_argument("--candidates", type=int, default=0,
                    help="psi4_3d / plugin4d: number of candidate bandwidths (0: the configuration's)")
    ap.add_argument("--crossover", action="store_true",
                    help="print the lag-domain against FFT-route cost per bandwidth over the support L "
                         "(one JSON object per rung) instead of the benchmark line")
    args = ap.parse_args()
    if args.crossover:
        crossover(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
