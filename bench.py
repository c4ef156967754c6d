#!/usr/bin/env python
"""GOAT Frank-Wolfe throughput on GB300.

Workload: one rho-correlated 3-block SBM pair (blocks 40/35/25 %, p_in = 0.02,
p_out = 0.004, rho = 0.7, B vertex-permuted by a seeded sigma), n = 32768,
barycenter init, up to 30 Frank-Wolfe iterations, final GPU linear assignment.
A "step" is one whole solve (goat_match: gradient products, Sinkhorn, line
search, update for every FW iteration, then the projection and the exact
objective).  The metric is FW iterations per second of the chosen form
(tensor-core products with Q in BF16 and the intermediate Q B as a BF16 hi term
plus an E4M3 lo term -- the form whose matching accuracy equals the FP64
oracle's -- and FP32 log-domain Sinkhorn warm-started from the previous step's
duals), reported next to the other forms and the plain FP32-accurate GPU form
(two-term BF16 split products, cold- and warm-started Sinkhorn) on the same pair.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank solves its own pair (seed + rank): replicas, weak scaling.
The reference arm (--impl reference) times the FP64 CPU oracle on a bounded
row sample of the same workload on all host cores (one row a core per step).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "GOAT FW iters/s at n=32768, chosen vs plain FP32 on GB300 at equal match accuracy"
UNIT = "FW iters/s"
NOMINAL_HBM_GBS = 7900.0  # HBM3e of a GB300, nominal
T0 = time.time()


def log(msg: str):
    print(f"[bench {time.time() - T0:7.1f}s] {msg}", file=sys.stderr, flush=True)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n", type=int, default=32768)
    ap.add_argument("--max-iter", type=int, default=30)
    ap.add_argument("--fw-tol", type=float, default=1e-4)
    ap.add_argument("--sk-tol", type=float, default=1e-3)
    ap.add_argument("--sk-max-iter", type=int, default=500)
    ap.add_argument("--seed", type=int, default=3000)
    ap.add_argument("--plain-steps", type=int, default=1)
    ap.add_argument("--chosen", choices=["bf16split", "bf16split8", "fp8", "bf16"], default="bf16split8",
                    help="product form of the timed (chosen) solve; the other forms are reported beside it")
    ap.add_argument("--e2e-steps", type=int, default=1)
    ap.add_argument("--cpu-rows-per-core", type=int, default=4,
                    help="gradient rows a host core computes in the cpu_baseline sample")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-accuracy", action="store_true")
    ap.add_argument("--accuracy-seeds", type=int, default=20,
                    help="n = 1500 SBM pairs per rho in the accuracy comparison (the oracle's values are stored)")
    ap.add_argument("--pairs", type=int, default=512)
    ap.add_argument("--restarts", type=int, default=20)
    ap.add_argument("--train-pairs", type=int, default=32)
    ap.add_argument("--train-steps", type=int, default=2000)
    ap.add_argument("--no-learned", action="store_true", help="skip the learned warm-start leg")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched (C4) leg")
    ap.add_argument("--kernel-case", choices=["gemm", "sinkhorn", "lap", "batched", "warmstart", "lot", "faq"],
                    default=None,
                    help="run only one step kind a few times on the workload (the small cases profiled with ncu)")
    ap.add_argument("--repeat", type=int, default=3)
    ap.add_argument("--precision", choices=["bf16", "fp8", "fp32", "bf16split", "bf16split8"], default="bf16",
                    help="form of the products in --kernel-case gemm")
    return ap.parse_args()


def workload_config(args):
    return {"workload": f"rho-SBM pair, 3 blocks (40/35/25%), n={args.n}, p_in=0.02, p_out=0.004, rho=0.7, "
                        f"B vertex-permuted; barycenter init; <= {args.max_iter} FW iters; GPU LAP projection",
            "n": args.n, "max_fw_iters": args.max_iter, "fw_tol": args.fw_tol, "eps_rel": 0.03,
            "sinkhorn_tol": args.sk_tol, "sinkhorn_max_iter": args.sk_max_iter, "seed": args.seed,
            "l2": "inputs larger than L2 (FP32 G and P are 4.3 GB each at n=32768)"}


# ------------------------------------------------------------------ clocks

QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")


class ClockSampler:
    """Samples nvidia-smi every 200 ms while the timed region runs."""

    def __init__(self, gpu_index: int):
        self.proc = None
        self.path = f"/tmp/goat_clocks_{os.getpid()}.csv"
        self.gpu = gpu_index

    def start(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        load = [x for x in sm if x > 0.5 * max(sm)] or sm
        return {"sm_mhz": statistics.median(load), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------ peaks / profiles

def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return {"hbm_gbs": d.get("hbm_gbs"), "bf16_tflops": d.get("bf16_tflops"),
                "bf16_tflops_sustained": d.get("bf16_tflops_sustained"), "source": "measured"}
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "source": "fallback"}


def gemm_traffic_per_launch(n: int, name: str = "k_gemm_xyT_traffic.txt"):
    """DRAM bytes per GEMM launch from the committed ncu summary `name`, scaled to n, or None.

    The summary records the kernel source hash it was taken with; a changed
    kernel invalidates it."""
    path = os.path.join(ROOT, "profiles", name)
    if not os.path.exists(path):
        return None
    kv = {}
    for line in open(path):
        if ":" in line and not line.startswith("#"):
            k, v = line.split(":", 1)
            kv[k.strip()] = v.strip()
    src = open(os.path.join(ROOT, "paper_2111_05366_gb300", "csrc", "goat_gemm.cu"), "rb").read()
    if kv.get("source_sha256") != hashlib.sha256(src).hexdigest():
        return None
    try:
        bytes_ = float(kv["dram_bytes_per_launch"])
        n_cap = float(kv["n"])
    except (KeyError, ValueError):
        return None
    # the products are n x n x n: operand re-reads grow like n^3 / tile, outputs like n^2
    return bytes_ * (n / n_cap) ** 3 if n != n_cap else bytes_


# ------------------------------------------------------------------ per-form report

FORM_PRECISION = {"fp8": 2, "bf16": 0, "fp32": 1, "bf16split": 3, "bf16split8": 5}
# BF16 MMA passes of (product 1, product 2) relative to one n x n x n BF16 product:
# the FP32 form splits Q and Q B in two terms (K = 2n in both products), the split
# form only Q B (product 2); the 8-bit form runs its passes at twice the BF16 rate,
# the split8 form the lo pass of its second product (1.5 BF16-equivalent passes)
FORM_PASSES = {"fp8": (1.0, 1.0), "bf16": (1.0, 1.0), "fp32": (2.0, 2.0), "bf16split": (1.0, 2.0),
               "bf16split8": (1.0, 1.5)}


def gemm_roofline(precision: str, n: int, ms_per_launch: float, peaks: dict, nnz: float):
    """Roofline block of the tensor-core products of one precision form.  The FP32
    form runs each product as BF16 MMAs over K = 2n (two split terms): its executed
    work is 2 x 2 n^3 BF16 FLOP per launch, which is what the tensor pipe sees."""
    flop = 2.0 * n ** 3
    executed = flop * sum(FORM_PASSES[precision]) / 2.0  # mean over the two products
    if precision == "fp8":
        # no FP8 peak was measured on this machine: the measured BF16 sustained rate times
        # the nominal dense FP8 / BF16 ratio (4.5 / 2.25 PFLOP/s)
        peak = 2.0 * peaks["bf16_tflops_sustained"]
        kernel = "k_gemm_xyT (E4M3 kind::f8f6f4, one n x n x n product per launch)"
        peak_source = f"{peaks['source']} bf16_tflops_sustained x nominal fp8/bf16 ratio 2"
        traffic = gemm_traffic_per_launch(n, "k_gemm_xyT_fp8_traffic.txt")
    else:
        peak = peaks["bf16_tflops_sustained"]
        kernel = {"bf16": "k_gemm_xyT (BF16 kind::f16, one n x n x n product per launch)",
                  "bf16split": "k_gemm_xyT (BF16 kind::f16; product 2 over the two terms of Q B, K = 2n)",
                  "bf16split8": "k_gemm_xyT (BF16 kind::f16; product 2: the hi term of Q B in BF16, its lo "
                                "term in E4M3 kind::f8f6f4, one accumulator)",
                  "fp32": "k_gemm_xyT (BF16 kind::f16 over two split terms, K = 2n, in K chunks)"}[precision]
        peak_source = f"{peaks['source']} bf16_tflops_sustained"
        traffic = {"bf16": gemm_traffic_per_launch(n),
                   "bf16split": gemm_traffic_per_launch(n, "k_gemm_xyT_split_traffic.txt"),
                   "bf16split8": gemm_traffic_per_launch(n, "k_gemm_xyT_split8_traffic.txt")}.get(precision)
    sec = ms_per_launch / 1000.0
    achieved = executed / sec / 1e12
    # A and B are ~1 % dense: of the dense FLOP only 2 nnz(B) n (C1 = B Q^T) and
    # 2 nnz(A) n (A C1^T) multiply a nonzero
    return {"bound": "tensor", "kernel": kernel, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "traffic": traffic, "peak_source": peak_source,
            "algorithmic_flop_per_launch": flop, "executed_flop_per_launch": executed,
            "useful_flop_per_launch": nnz * n, "useful_tflops": nnz * n / sec / 1e12}


def form_report(outs, ms: float, precision: str, n: int, peaks: dict, nnz: float, truth) -> dict:
    """FW iterations per second, time to solution and per-phase figures of the solves
    `outs` (goat_match results) that took `ms` of device time."""
    solves = len(outs)
    it = sum(o[2]["fw_iters"] for o in outs)
    ms_gemm = sum(o[2]["ms_gemm"] for o in outs)
    n_gemm = max(sum(o[2]["gemm_launches"] for o in outs), 1)
    ms_fw = sum(o[2]["ms_fw"] for o in outs)
    ms_sk = sum(o[2]["ms_sinkhorn"] for o in outs)
    sk = sum(o[2]["sk_iters_total"] for o in outs)
    rep = {"precision": precision, "value": it / (ms / 1000.0), "unit": UNIT,
           "fw_loop_value": it / (ms_fw / 1000.0), "ms_per_solve": ms / solves,
           "fw_iters_per_solve": it / solves, "sinkhorn_iters_per_fw_iter": sk / max(it, 1),
           "gemm_ms_per_launch": ms_gemm / n_gemm, "ms_projection_per_solve": sum(o[2]["ms_project"] for o in outs) / solves,
           "accuracy": float((outs[-1][0] == truth).mean()), "objective": outs[-1][2]["objective"],
           "lap_gap": outs[-1][2]["lap_gap"],
           "roofline": gemm_roofline(precision, n, ms_gemm / n_gemm, peaks, nnz)}
    if sk:
        t_it = ms_sk / sk / 1000.0
        # algorithmic bytes of one Sinkhorn iteration: one read of FP32 G (4 n^2).  The
        # fused single-read iteration runs every iteration of a solve but its first
        # (which reads G twice); the figure averages over all of them, small kernels and
        # launch gaps included
        rep["sinkhorn_ms_per_iter"] = t_it * 1000.0
        rep["sinkhorn_algorithmic_gbs"] = 4.0 * n * n / t_it / 1e9
        rep["sinkhorn_frac_of_hbm_peak"] = rep["sinkhorn_algorithmic_gbs"] / peaks["hbm_gbs"]
        # and against the nominal HBM3e rate of a GB300 (7.9 TB/s)
        rep["sinkhorn_frac_of_nominal_hbm"] = rep["sinkhorn_algorithmic_gbs"] / NOMINAL_HBM_GBS
    return rep


# The paper's Sec. 4.3 rho-SBM at n = 1500 (3 equal blocks), where GOAT recovers a
# real fraction of the vertices: the forms' matching accuracy is compared there with
# the FP64 oracle's, stored in tests/golden/sbm1500_oracle.txt by the committed
# script beside it (bench.py itself never runs the oracle outside its CPU legs).
SBM1500_PB = [[0.2, 0.01, 0.01], [0.01, 0.1, 0.01], [0.01, 0.01, 0.2]]


def sbm1500_oracle_accuracy():
    path = os.path.join(ROOT, "tests", "golden", "sbm1500_oracle.txt")
    out = {}
    if not os.path.exists(path):
        return out
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        rho, seed, acc, obj, it = line.split()
        out[(float(rho), int(seed))] = float(acc)
    return out


def accuracy_comparison(goat, synthetic, torch, forms: dict, seeds: int) -> dict:
    """Each form's mean matching accuracy on the n = 1500 pairs (seeds 1..seeds) next
    to the oracle's stored accuracy on the same pairs, in percentage points."""
    ref = sbm1500_oracle_accuracy()
    res = {"workload": "rho-SBM n=1500, 3 equal blocks, B=[[.2,.01,.01],[.01,.1,.01],[.01,.01,.2]] (Sec. 4.3)",
           "seeds": seeds, "rho": {}}
    for rho in (0.9, 0.95):
        row = {}
        pairs = [synthetic.rho_sbm_pair([500, 500, 500], SBM1500_PB, rho, seed=s) for s in range(1, seeds + 1)]
        for name, prm in forms.items():
            accs = []
            for gp in pairs:
                perm, _, _ = goat.goat_match(torch.from_numpy(gp.A).cuda(), torch.from_numpy(gp.B).cuda(),
                                             eps_rel=0.03, max_iter=30, tol=1e-4, params=prm)
                accs.append(float((perm == gp.truth).mean()))
            row[name] = float(np.mean(accs))
        refs = [ref.get((rho, s)) for s in range(1, seeds + 1)]
        if all(r is not None for r in refs):
            row["oracle"] = float(np.mean(refs))
            row["max_abs_delta_points"] = max(abs(v - row["oracle"]) * 100 for k, v in row.items() if k != "oracle")
        res["rho"][str(rho)] = row
    return res


# ------------------------------------------------------------------ CPU oracle sample

# Sinkhorn iterations per FW iteration charged to the CPU oracle in both the
# cpu_baseline leg and the reference arm: the warm-started GPU form's count at this
# workload (about 25), i.e. the oracle is credited with the same Sinkhorn work as the
# form it is compared with (its own cold start takes more; the row-LSE share of its
# FW iteration is a few percent either way).
SK_ITERS_PER_FW = 25


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_oracle_sample(gp, rows_per_core: int, cores: int | None = None):
    """Times the FP64 oracle, as it stands, on a row sample of one FW iteration of the
    workload, on all host cores.

    Work timed: rows_per_core x cores rows of grad f(J) (oracle.gradient_rows, naive
    loops), then the Sinkhorn row scaling of those rows (oracle.lot_rows); each core
    takes a disjoint block of rows in its own thread (the oracle's C calls release the
    interpreter lock).  Scaled to one FW iteration as
    T = (n / rows) * (2 * T_grad + 2 * k_sk * T_rowlse): the oracle's step size forms
    the same naive products as the gradient (counted as a second gradient), and a
    Sinkhorn iteration is a row pass plus a column pass of equal work."""
    from concurrent.futures import ThreadPoolExecutor
    import oracle
    n = gp.n
    cores = cores or host_cores()
    rows = max(1, rows_per_core * cores)
    rng = np.random.default_rng(0)
    sel = np.sort(rng.choice(n, size=min(rows, n), replace=False)).astype(np.int32)
    blocks = [blk for blk in np.array_split(sel, cores) if blk.size]
    P = np.full((n, n), 1.0 / n, dtype=np.float32)
    with ThreadPoolExecutor(max_workers=len(blocks)) as pool:
        t0 = time.perf_counter()
        grads = list(pool.map(lambda blk: oracle.gradient_rows(gp.A, gp.B, P, blk), blocks))
        t_grad = time.perf_counter() - t0
        del P
        G_rows = [(-gr).astype(np.float32) for gr in grads]
        eps = 0.03 * max(float(np.abs(gr).max()) for gr in G_rows)
        g = np.zeros(n, dtype=np.float32)
        t0 = time.perf_counter()
        list(pool.map(lambda gr: oracle.lot_rows(gr, g, eps), G_rows))
        t_lse = time.perf_counter() - t0
    t_iter = (n / sel.size) * (2.0 * t_grad + 2.0 * SK_ITERS_PER_FW * t_lse)
    sample = (f"{sel.size} rows of grad f at the barycenter (naive FP64 loops) + their Sinkhorn row scaling, "
              f"n={n}, {len(blocks)} threads; one FW iteration = (n/rows) x (2 x gradient rows + "
              f"2 x {SK_ITERS_PER_FW} x row-LSE); measured {t_grad + t_lse:.1f} s")
    return {"value": 1.0 / t_iter, "unit": UNIT, "cores": len(blocks), "kind": "oracle", "sample": sample,
            "seconds_per_fw_iter": t_iter, "sinkhorn_iters_per_fw_iter": SK_ITERS_PER_FW}


# ------------------------------------------------------------------ reference arm

def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from paper_2111_05366_gb300 import synthetic
    gp = synthetic.large_sbm_pair(args.n, seed=args.seed)
    vals = []
    last = None
    for step in range(args.warmup + args.steps):
        # one row a core per step, so K + W steps end within a few minutes
        r = cpu_oracle_sample(gp, 1)
        if step >= args.warmup:
            vals.append(r["value"])
        last = r
    v = float(np.mean(vals))
    cb = dict(last)
    cb["value"] = v
    cb["sample"] = last["sample"] + f"; mean of {args.steps} timed samples after {args.warmup} warm-up"
    line = {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000.0 / v, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": workload_config(args),
            "impl": "reference", "cpu_baseline": cb,
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ single-kernel cases (for ncu)

def run_kernel_case(args):
    """Calls one step of the path `--repeat` times on the workload pair at size --n.

    gemm:     goat_gradient at a doubly stochastic P (two tensor-core products per call)
    sinkhorn: goat_sinkhorn on -grad f(J) for a fixed number of iterations (tol 0)
    lap:      goat_project on the entropic direction Q at the barycenter (a diffuse,
              degree-structured doubly stochastic matrix like the relaxed P of a hard pair)
    faq:      one goat_match solve with the LOT direction (GOAT, Alg. 3) and one with the
              exact assignment direction (FAQ, Alg. 1), --precision form, on the same pair"""
    import torch

    import paper_2111_05366_gb300 as goat
    from paper_2111_05366_gb300 import synthetic
    torch.cuda.set_device(0)
    goat.load()
    if args.kernel_case == "batched":
        return run_batched_case(args)
    if args.kernel_case == "warmstart":
        return run_warmstart_case(args)
    if args.kernel_case == "lot":
        return run_lot_case(args)
    n = args.n
    gp = synthetic.large_sbm_pair(n, seed=args.seed)
    A = torch.from_numpy(gp.A).cuda()
    B = torch.from_numpy(gp.B).cuda()
    P = torch.full((n, n), 1.0 / n, dtype=torch.float32, device="cuda")
    P[torch.arange(n, device="cuda"), torch.randperm(n, device="cuda")] += 1.0
    P /= 2.0
    out = {"case": args.kernel_case, "n": n}
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if args.kernel_case == "gemm":
        prec = FORM_PRECISION[args.precision]
        G = goat.goat_gradient(A, B, P, precision=prec)
        e0.record()
        for _ in range(args.repeat):
            goat.goat_gradient(A, B, P, precision=prec, out=G)
        e1.record()
        out["precision"] = args.precision
    elif args.kernel_case == "faq":
        prec = FORM_PRECISION[args.precision]
        del P
        out["precision"] = args.precision
        for name, direction in (("goat", goat.GOAT_DIR_LOT), ("faq", goat.GOAT_DIR_LAP)):
            prm = goat.default_params(precision=prec, sk_warm_start=1, sk_tol=args.sk_tol,
                                      sk_max_iter=args.sk_max_iter, profile=1, direction=direction)
            torch.cuda.synchronize()
            e0.record()
            perm, obj, st = goat.goat_match(A, B, eps_rel=0.03, max_iter=args.max_iter, tol=args.fw_tol, params=prm)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            out[name] = {"ms_solve": ms, "fw_iters": st["fw_iters"], "converged": st["converged"],
                         "fw_iters_per_s": st["fw_iters"] / (ms / 1000.0),
                         "ms_direction_steps": st["ms_sinkhorn"], "ms_products": st["ms_gemm"],
                         "ms_projection": st["ms_project"], "accuracy": float((perm == gp.truth).mean()),
                         "objective": obj}
            log(f"{name}: {st['fw_iters']} FW iterations in {ms:.0f} ms, accuracy {out[name]['accuracy']:.4f}")
    elif args.kernel_case == "sinkhorn":
        G = goat.goat_gradient(A, B, P)
        eps = 0.03 * float(G.abs().max())
        e0.record()
        for _ in range(args.repeat):
            goat.goat_sinkhorn(G, eps, 0.0, 10)
        e1.record()
    else:
        J = torch.full((n, n), 1.0 / n, dtype=torch.float32, device="cuda")
        G = goat.goat_gradient(A, B, J)
        del J
        eps = 0.03 * float(G.abs().max())
        _, _, Q, _, _ = goat.goat_sinkhorn(G, eps, args.sk_tol, args.sk_max_iter, want_Q=True)
        del G
        e0.record()
        for _ in range(args.repeat):
            _, cost, gap, info = goat.goat_project_ex(Q, allow_uncertified=True)
        e1.record()
        out["cost"], out["gap"], out["info"] = cost, gap, info
    torch.cuda.synchronize()
    if args.kernel_case != "faq":
        out["ms_per_call"] = e0.elapsed_time(e1) / args.repeat
    print(json.dumps(out), flush=True)
    return 0


def run_lot_case(args):
    """LOT against exact linear assignment on the paper's Fig. 1 workload (Sec. 3.3):
    i.i.d. Uniform(100, 150) costs, n = 250, 500, ..., 3000, lambda = 100 (eps = 0.01),
    --repeat matrices per n.  Per n: the device time of goat_sinkhorn to the marginal
    tolerance --sk-tol (Q written out) and of goat_project (certified optimum), and the
    relative objective gap (OFV_LAP - OFV_LOT) / OFV_LAP of the paper's Fig. 1."""
    import torch

    import paper_2111_05366_gb300 as goat
    from paper_2111_05366_gb300 import synthetic
    eps = 0.01
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn):
        torch.cuda.synchronize()
        e0.record()
        r = fn()
        e1.record()
        torch.cuda.synchronize()
        return r, e0.elapsed_time(e1)

    rows = []
    for n in range(250, 3001, 250):
        lot_ms, lap_ms, gaps, iters = [], [], [], []
        for k in range(args.repeat + 1):  # k = 0 warms up this size
            M = torch.from_numpy(synthetic.uniform_costs(n, 100, 150, 1000 * n + k, np.float32)).cuda()
            (_, _, Q, it, resid), t_lot = timed(lambda: goat.goat_sinkhorn(M, eps, args.sk_tol, 5000, want_Q=True))
            (_, cost, _), t_lap = timed(lambda: goat.goat_project(M, maximize=False))
            ofv = float((Q.double() * M.double()).sum())
            if k:
                lot_ms.append(t_lot)
                lap_ms.append(t_lap)
                gaps.append((cost - ofv) / cost)
                iters.append(it)
        rows.append({"n": n, "lot_ms": float(np.mean(lot_ms)), "lap_ms": float(np.mean(lap_ms)),
                     "lap_over_lot": float(np.mean(lap_ms) / np.mean(lot_ms)),
                     "max_abs_rel_gap": float(np.max(np.abs(gaps))), "mean_rel_gap": float(np.mean(gaps)),
                     "lot_iters": float(np.mean(iters))})
        log(f"n={n}: LOT {rows[-1]['lot_ms']:.2f} ms ({rows[-1]['lot_iters']:.0f} it), "
            f"LAP {rows[-1]['lap_ms']:.2f} ms, gap {rows[-1]['max_abs_rel_gap']:.2e}")
    print(json.dumps({"case": "lot_vs_lap", "costs": "Uniform(100, 150)", "eps": eps, "lambda": 1.0 / eps,
                      "sk_tol": args.sk_tol, "matrices_per_n": args.repeat, "rows": rows}), flush=True)
    return 0


def learned_warm_start_leg(args, n: int = 8192, fw_steps: int = 3) -> dict:
    """The learned Sinkhorn warm start, trained and measured.

    Training: converged duals of GOAT runs on --train-pairs correlated ER / SBM pairs
    (n in [500, 2000], half weighted; 3 FW steps each, Sinkhorn to 1e-5).
    Evaluation (the weighted workload: correlated ER, n = 8192, p = 0.05, rho = 0.8,
    lognormal(0, 1) weights; Sinkhorn to marginal tolerance 1e-4) at the barycenter
    gradient and the next FW steps: cold start (g = 0) against the network's duals,
    in iterations and in device ms with the features and the network included, and
    against the previous FW step's duals (free, the in-solve default) from step 1 on."""
    import torch

    import paper_2111_05366_gb300 as goat
    from paper_2111_05366_gb300 import synthetic, warmstart
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn):
        e0.record()
        out = fn()
        e1.record()
        torch.cuda.synchronize()
        return out, e0.elapsed_time(e1)

    t0 = time.time()
    X, T = warmstart.collect(warmstart.default_training_pairs(args.train_pairs, seed=args.seed), fw_steps=3)
    t_collect = time.time() - t0
    (master, adam, wb, losses), ms_train = timed(
        lambda: warmstart.train(X, T, steps=args.train_steps, batch=16384, lr=3e-3, seed=0))
    gp = synthetic.rho_er_pair(n, 0.05, 0.8, seed=args.seed + 5, weighted=True)
    A, B = torch.from_numpy(gp.A).cuda(), torch.from_numpy(gp.B).cuda()
    P = torch.full((n, n), 1.0 / n, dtype=torch.float32, device="cuda")
    G = goat.goat_gradient(A, B, P, precision=goat.GOAT_PREC_FP32)
    # one untimed pass of every call (first-use costs)
    eps = 0.03 * float(G.abs().max())
    goat.goat_sinkhorn(G, eps, 1e-4, 5000, g_init=goat.goat_mlp_warm_start(G, A, B, eps, wb))
    rows, g_prev = [], None
    for step in range(fw_steps):
        eps = 0.03 * float(G.abs().max())
        (f, g, Q, it_c, r_c), ms_c = timed(lambda: goat.goat_sinkhorn(G, eps, 1e-4, 5000, want_Q=True))
        (_, _, _, it_w, r_w), ms_w = timed(
            lambda: goat.goat_sinkhorn(G, eps, 1e-4, 5000, g_init=goat.goat_mlp_warm_start(G, A, B, eps, wb)))
        row = {"fw_step": step, "cold_iters": it_c, "learned_iters": it_w, "cold_ms": ms_c,
               "learned_ms_incl_features_and_mlp": ms_w, "cold_resid": r_c, "learned_resid": r_w}
        if g_prev is not None:
            (_, _, _, it_p, r_p), ms_p = timed(lambda: goat.goat_sinkhorn(G, eps, 1e-4, 5000, g_init=g_prev))
            row.update({"previous_step_iters": it_p, "previous_step_ms": ms_p, "previous_step_resid": r_p})
        rows.append(row)
        g_prev = g.clone()
        GQ = goat.goat_gradient(A, B, Q, precision=goat.GOAT_PREC_FP32)
        alpha, _, _ = goat.goat_line_search(G, GQ, P, Q)
        goat.goat_fw_update(P, G, Q, GQ, alpha)
        del Q, GQ
    del P, G
    torch.cuda.empty_cache()
    cold_ms = sum(r["cold_ms"] for r in rows)
    learned_ms = sum(r["learned_ms_incl_features_and_mlp"] for r in rows)
    return {"workload": f"weighted rho-ER n={n}, p=0.05, rho=0.8, lognormal(0,1) weights; Sinkhorn tol 1e-4",
            "train_pairs": args.train_pairs, "train_solves": args.train_pairs * 3, "train_samples": int(X.shape[0]),
            "collect_s": t_collect, "train_steps": args.train_steps, "train_ms": ms_train,
            "loss_first": losses[0], "loss_last": losses[-1], "eval": rows,
            "learned_over_cold_ms": learned_ms / cold_ms if cold_ms > 0 else None,
            "pays": learned_ms < cold_ms}


def run_warmstart_case(args):
    """The learned warm start alone (learned_warm_start_leg at n = --n)."""
    print(json.dumps({"case": "warmstart", **learned_warm_start_leg(args, n=args.n)}), flush=True)
    return 0


def batched_leg(args) -> dict:
    """The batched workload (configuration C4): --pairs correlated ER pairs with
    n ~ U{50..1000}, p ~ U[0.02, 0.2], rho ~ U[0.6, 1.0], each from --restarts starts
    (restart 0 the barycenter, the others (J + K)/2 random starts), one CUDA-graph
    replay per FW iteration.  Reports solved pairs per second, the mean matching
    accuracy of the best restarts, and the dense product work of the batch (4 n^3 per
    problem and FW iteration, the iterations each problem ran) over the batch time."""
    import torch

    import paper_2111_05366_gb300 as goat
    from paper_2111_05366_gb300 import synthetic
    rng = np.random.default_rng(args.seed)
    ns = rng.integers(50, 1001, size=args.pairs)
    ps = rng.uniform(0.02, 0.2, size=args.pairs)
    rhos = rng.uniform(0.6, 1.0, size=args.pairs)
    gps = [synthetic.rho_er_pair(int(n), float(p), float(r), seed=args.seed + 17 * k)
           for k, (n, p, r) in enumerate(zip(ns, ps, rhos))]
    nn = np.array([g.n for g in gps], dtype=np.int32)
    off = np.zeros(len(gps), dtype=np.int64)
    off[1:] = np.cumsum(nn.astype(np.int64) ** 2)[:-1]
    Ad = torch.from_numpy(np.concatenate([g.A.ravel() for g in gps])).cuda()
    Bd = torch.from_numpy(np.concatenate([g.B.ravel() for g in gps])).cuda()
    prm = goat.default_params(sk_tol=args.sk_tol, sk_max_iter=args.sk_max_iter)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    # the first call autotunes the Sinkhorn launch shape (cached per process)
    goat.goat_match_batched(None, None, restarts=args.restarts, seed=args.seed, max_iter=args.max_iter,
                            tol=args.fw_tol, params=prm, device_AB=(Ad, Bd, off, nn))
    torch.cuda.synchronize()
    e0.record()
    for _ in range(args.repeat):
        perms, obj, best, its = goat.goat_match_batched(None, None, restarts=args.restarts, seed=args.seed,
                                                        max_iter=args.max_iter, tol=args.fw_tol, params=prm,
                                                        device_AB=(Ad, Bd, off, nn))
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.repeat
    acc = float(np.mean([(perms[k] == gps[k].truth).mean() for k in range(len(gps))]))
    # dense product FLOP of the batch: every restart runs until its own stop test; the
    # per-pair count returned is the best restart's, so this is an estimate
    flop = float(np.sum(4.0 * nn.astype(np.float64) ** 3 * np.asarray(its, dtype=np.float64))) * args.restarts
    del Ad, Bd
    torch.cuda.empty_cache()
    return {"workload": f"{args.pairs} correlated ER pairs, n ~ U{{50..1000}}, p ~ U[0.02, 0.2], "
                        f"rho ~ U[0.6, 1.0], {args.restarts} starts each (barycenter + random (J + K)/2)",
            "pairs": args.pairs, "restarts": args.restarts, "problems": args.pairs * args.restarts,
            "ms_per_batch": ms, "pairs_per_s": args.pairs / (ms / 1000.0), "mean_accuracy_best_restart": acc,
            "mean_fw_iters_best_restart": float(np.mean(its)),
            "product_tflops_effective": flop / (ms / 1000.0) / 1e12,
            "note": "effective rate = dense product FLOP (4 n^3 per FW iteration, best restart's iteration count for "
                    "every restart) / whole batch time, Sinkhorn, steps and projections included"}


def run_batched_case(args):
    """The batched workload alone (batched_leg)."""
    print(json.dumps({"case": "batched", **batched_leg(args)}), flush=True)
    return 0


# ------------------------------------------------------------------ our arm

class Ranks:
    """Barrier and reductions over the ranks of a weak-scaling run (replicas: one
    independent pair per rank; the only communication is the timing reduction)."""

    def __init__(self, world: int, device: str):
        self.world = world
        self.device = device

    def barrier(self):
        if self.world > 1:
            import torch.distributed as dist
            dist.barrier()

    def _reduce(self, x: float, op) -> float:
        if self.world == 1:
            return x
        import torch
        import torch.distributed as dist
        t = torch.tensor([x], dtype=torch.float64, device=self.device)
        dist.all_reduce(t, op=op)
        return float(t.item())

    def max(self, x: float) -> float:
        import torch.distributed as dist
        return self._reduce(x, dist.ReduceOp.MAX)

    def sum(self, x: float) -> float:
        import torch.distributed as dist
        return self._reduce(x, dist.ReduceOp.SUM)


def whole_job_rate(ranks: Ranks, units: float, ms: float) -> float:
    """Units all ranks processed / the slowest rank's time (the timed region is
    bracketed by barriers, so the slowest rank spans the job)."""
    return ranks.sum(units) / (ranks.max(ms) / 1000.0)


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.kernel_case:
        return run_kernel_case(args)

    import torch
    import torch.distributed as dist

    import paper_2111_05366_gb300 as goat
    from paper_2111_05366_gb300 import synthetic

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")

    ranks = Ranks(world, "cuda")
    barrier, max_over_ranks, sum_over_ranks = ranks.barrier, ranks.max, ranks.sum

    goat.load()
    n = args.n
    log(f"generating the n={n} pair")
    gp = synthetic.large_sbm_pair(n, seed=args.seed + rank)
    nnz_A, nnz_B = int(gp.A.sum()), int(gp.B.sum())
    log(f"pair ready: {nnz_A} + {nnz_B} nonzeros")
    A = torch.from_numpy(gp.A).cuda()
    B = torch.from_numpy(gp.B).cuda()
    ws = torch.empty(max(goat.workspace_bytes(n, goat.GOAT_DTYPE_U8, pr) for pr in FORM_PRECISION.values()),
                     dtype=torch.uint8, device="cuda")
    chosen_prec = FORM_PRECISION[args.chosen]
    chosen = goat.default_params(precision=chosen_prec, sk_warm_start=1, sk_tol=args.sk_tol,
                                 sk_max_iter=args.sk_max_iter, profile=1)
    others = {f"{k}_warm": goat.default_params(precision=FORM_PRECISION[k], sk_warm_start=1, sk_tol=args.sk_tol,
                                               sk_max_iter=args.sk_max_iter, profile=1)
              for k in ("bf16split", "bf16split8", "bf16", "fp8") if k != args.chosen}
    plain = goat.default_params(precision=goat.GOAT_PREC_FP32, sk_warm_start=0, sk_tol=args.sk_tol,
                                sk_max_iter=args.sk_max_iter, profile=1)
    plain_warm = goat.default_params(precision=goat.GOAT_PREC_FP32, sk_warm_start=1, sk_tol=args.sk_tol,
                                     sk_max_iter=args.sk_max_iter, profile=1)

    def solve(params):
        return goat.goat_match(A, B, eps_rel=0.03, max_iter=args.max_iter, tol=args.fw_tol, params=params,
                               workspace=ws)

    def timed(params, warmup, steps, sampler=None):
        for _ in range(warmup):
            _, _, stw = solve(params)
            log(f"warmup solve: {stw['fw_iters']} FW iters, {stw['ms_total']:.0f} ms "
                f"(fw {stw['ms_fw']:.0f}, project {stw['ms_project']:.0f}, lap rounds {stw['lap_rounds']}, "
                f"tail bids {stw['lap_tail_bids']}, sap rows {stw['lap_sap_rows']} pops {stw['lap_sap_pops']}; "
                f"ms head {stw['lap_ms_head']:.0f} tail {stw['lap_ms_tail']:.0f} sap {stw['lap_ms_sap']:.0f})")
        barrier()
        torch.cuda.synchronize()
        if sampler:
            sampler.start()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        outs = [solve(params) for _ in range(steps)]
        e1.record()
        torch.cuda.synchronize()
        barrier()
        clocks = sampler.stop() if sampler else None
        ms = e0.elapsed_time(e1)
        return ms, outs, clocks

    sampler = ClockSampler(local)
    ms, outs, clocks = timed(chosen, args.warmup, args.steps, sampler)
    log(f"chosen form timed: {ms:.0f} ms for {args.steps} solves")
    fw_iters = sum(o[2]["fw_iters"] for o in outs)
    ms_max = max_over_ranks(ms)
    value = whole_job_rate(ranks, float(fw_iters), ms)
    st = outs[-1][2]
    acc = float((outs[-1][0] == gp.truth).mean())

    # per-phase breakdown and the roofline of the dominant kernel (the tensor-core products)
    peaks = measured_peaks()
    nnz = float(nnz_A + nnz_B)
    chosen_rep = form_report(outs, ms, args.chosen, n, peaks, nnz, gp.truth)
    roofline = chosen_rep["roofline"]
    ms_gemm = sum(o[2]["ms_gemm"] for o in outs)
    n_gemm = sum(o[2]["gemm_launches"] for o in outs)
    ms_sk = sum(o[2]["ms_sinkhorn"] for o in outs)
    ms_step = sum(o[2]["ms_step"] for o in outs)
    ms_proj = sum(o[2]["ms_project"] for o in outs)
    sk_total = sum(o[2]["sk_iters_total"] for o in outs)
    launches = sum(o[2]["launches"] for o in outs)
    ms_fw_loop = sum(o[2]["ms_fw"] for o in outs)
    breakdown = {"ms_per_fw_iter": ms / max(fw_iters, 1), "gemm_ms_per_launch": ms_gemm / max(n_gemm, 1),
                 "ms_fw_loop_per_solve": ms_fw_loop / args.steps, "ms_projection_per_solve": ms_proj / args.steps,
                 "gemm_share": ms_gemm / ms, "sinkhorn_share": ms_sk / ms, "step_share": ms_step / ms,
                 "projection_share": ms_proj / ms, "sinkhorn_iters_per_fw_iter": sk_total / max(fw_iters, 1),
                 "fw_iters_per_solve": fw_iters / args.steps, "accuracy": acc,
                 "objective": st["objective"], "disagreements": st["disagreements"], "lap_gap": st["lap_gap"],
                 "lap_rounds": st["lap_rounds"], "lap_tail_bids": st["lap_tail_bids"],
                 "lap_sap_rows": st["lap_sap_rows"], "lap_sap_pops": st["lap_sap_pops"],
                 "lap_ms_head": st["lap_ms_head"], "lap_ms_tail": st["lap_ms_tail"], "lap_ms_sap": st["lap_ms_sap"]}
    for k in ("sinkhorn_ms_per_iter", "sinkhorn_algorithmic_gbs", "sinkhorn_frac_of_hbm_peak",
              "sinkhorn_frac_of_nominal_hbm"):
        if k in chosen_rep:
            breakdown[k] = chosen_rep[k]

    fw_loop_value = sum_over_ranks(float(fw_iters)) / (max_over_ranks(ms_fw_loop) / 1000.0)
    result = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
              "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
              "scaling": "weak", "vs_baseline": None, "dtype": {"fp8": "e4m3", "bf16split8": "bf16+e4m3"}.get(args.chosen, "bf16"),
              "precision_form": {"bf16split": "BF16 products, Q B kept as two BF16 terms (GOAT_PREC_BF16_SPLIT)",
                                 "bf16split8": "BF16 products, Q B as a BF16 hi term and an E4M3 lo term "
                                               "(GOAT_PREC_BF16_SPLIT8)",
                                 "bf16": "BF16 products (GOAT_PREC_BF16)",
                                 "fp8": "E4M3 products (GOAT_PREC_FP8)"}[args.chosen],
              "data": "synthetic",
              "config": workload_config(args), "clocks": clocks, "gpu_launches": int(sum_over_ranks(launches)),
              "roofline": roofline, "breakdown": breakdown,
              # the Frank-Wolfe iterations alone (rows a1-a5): the projection runs once per
              # solve and is reported separately in breakdown.ms_projection_per_solve
              "fw_loop": {"value": fw_loop_value, "unit": UNIT},
              "warm_start": "each Sinkhorn solve starts from the previous Frank-Wolfe step's duals; the learned "
                            "(MLP) start is measured beside it (learned_warm_start) and not used in the timed "
                            "form"}

    # every form on the same pair, one timed solve each after one untimed one: the other
    # 16/8-bit form, and the plain FP32-accurate form cold- and warm-started, so that the
    # gain of the precision and the gain of warm-starting the duals show separately
    forms = {f"{args.chosen}_warm": chosen_rep}
    if not args.no_plain:
        legs = [(name, prm, name[:-5]) for name, prm in others.items()]
        legs += [("fp32_cold", plain, "fp32"), ("fp32_warm", plain_warm, "fp32")]
        for name, prm, prec in legs:
            ms_f, outs_f, _ = timed(prm, 1, args.plain_steps)
            forms[name] = form_report(outs_f, ms_f, prec, n, peaks, nnz, gp.truth)
            log(f"{name} form timed: {ms_f:.0f} ms ({forms[name]['fw_iters_per_solve']:.0f} FW iterations)")
        cold = forms["fp32_cold"]
        result["plain_fp32"] = {"value": cold["value"], "unit": UNIT, "accuracy": cold["accuracy"],
                                "fw_iters_per_solve": cold["fw_iters_per_solve"],
                                "sinkhorn_iters_per_fw_iter": cold["sinkhorn_iters_per_fw_iter"],
                                "gemm_ms_per_launch": cold["gemm_ms_per_launch"]}
        result["chosen_over_plain"] = value / cold["value"]
        result["fw_loop"]["plain_value"] = cold["fw_loop_value"]
        result["fw_loop"]["chosen_over_plain"] = fw_loop_value / cold["fw_loop_value"]
        # the same ratios by time to solution (the forms run different numbers of FW
        # iterations before the stop test ends them), against the cold and the warm plain form
        result["time_to_solution"] = {
            "ms": {k: v["ms_per_solve"] for k, v in forms.items()},
            "chosen_speedup_vs_plain_cold": cold["ms_per_solve"] / chosen_rep["ms_per_solve"],
            "chosen_speedup_vs_plain_warm": forms["fp32_warm"]["ms_per_solve"] / chosen_rep["ms_per_solve"],
            "iters_per_s_ratio_vs_plain_cold": value / cold["value"],
            "iters_per_s_ratio_vs_plain_warm": value / forms["fp32_warm"]["value"]}
    result["forms"] = forms
    if not args.no_accuracy and rank == 0:
        acc_forms = {f"{k}_{'warm' if w else 'cold'}": goat.default_params(
                         precision=FORM_PRECISION[k], sk_warm_start=w, sk_tol=args.sk_tol, sk_max_iter=args.sk_max_iter)
                     for k in ("bf16split", "bf16split8", "fp32", "bf16", "fp8") for w in (1, 0)}
        result["accuracy"] = accuracy_comparison(goat, synthetic, torch, acc_forms, args.accuracy_seeds)
        log(f"accuracy on the n=1500 SBM: {result['accuracy']['rho']}")
    if not args.no_batched and rank == 0:
        one = argparse.Namespace(**{**vars(args), "repeat": 1})  # one timed batch in the line
        result["batched_c4"] = batched_leg(one)
        bc = result["batched_c4"]
        log(f"batched C4: {bc['ms_per_batch']:.0f} ms per batch, {bc['pairs_per_s']:.1f} pairs/s, "
            f"accuracy {bc['mean_accuracy_best_restart']:.3f}")
    if not args.no_learned and rank == 0:
        result["learned_warm_start"] = learned_warm_start_leg(args)
        lw = result["learned_warm_start"]
        log(f"learned warm start: learned/cold ms {lw['learned_over_cold_ms']:.2f}; "
            f"{[(r['cold_iters'], r['learned_iters'], r.get('previous_step_iters')) for r in lw['eval']]}")

    # end to end through the host-buffer entry point: pinned host A, B in, permutation out
    if not args.no_e2e:
        Ah = torch.from_numpy(gp.A).pin_memory().numpy()
        Bh = torch.from_numpy(gp.B).pin_memory().numpy()
        ws_h = torch.empty(goat.workspace_bytes(n, goat.GOAT_DTYPE_U8, chosen_prec, host=True),
                           dtype=torch.uint8, device="cuda")
        del ws
        torch.cuda.empty_cache()
        goat.goat_match_host(Ah, Bh, eps_rel=0.03, max_iter=args.max_iter, tol=args.fw_tol, params=chosen,
                             workspace=ws_h)
        barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        it_e = 0
        for _ in range(args.e2e_steps):
            perm_h, obj_h, st_h = goat.goat_match_host(Ah, Bh, eps_rel=0.03, max_iter=args.max_iter,
                                                       tol=args.fw_tol, params=chosen, workspace=ws_h)
            it_e += st_h["fw_iters"]
        e1.record()
        torch.cuda.synchronize()
        barrier()
        ms_e = max_over_ranks(e0.elapsed_time(e1))
        result["e2e"] = {"value": sum_over_ranks(float(it_e)) / (ms_e / 1000.0), "unit": UNIT,
                         "h2d_bytes_per_step": int(2 * n * n), "d2h_bytes_per_step": int(4 * n),
                         "api": "goat_match_host (pinned host A, B; permutation read back)"}

    if not args.no_e2e:
        log("e2e done")
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        log("timing the CPU oracle sample")
        result["cpu_baseline"] = cpu_oracle_sample(gp, args.cpu_rows_per_core)

    if rank == 0:
        print(json.dumps(result), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
