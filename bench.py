#!/usr/bin/env python3
"""Throughput benchmark of the GB300 batched nested sampler.

Workload: the 10-D correlated Gaussian (covariance R diag(lambda) R^T, R a
seeded Haar-orthogonal matrix, lambda log-uniform in [0.01, 1], mean
uniform in [-2, 2]^10, prior [-10, 10]^10), N_live = 1000, m = 100 live
points replaced per iteration, 5 d = 50 slice steps, stop at a remaining-
evidence fraction of 1e-3.  Each GPU runs R independent runs (one seed and
one seeded covariance each), all in one persistent launch.  A step is the
whole job: every run from its initial live set to its stopping rule.

Reported (one JSON line from rank 0):
  value     likelihood evaluations per second over all GPUs, device time of
            ns_run with the problem already resident (L2 flushed between
            steps);
  e2e       the same metric through the C ABI from host buffers:
            ns_create (host->device) + ns_run + ns_result for every run
            (device->host of all samples) + ns_destroy;
  roofline  the run kernel against the FP32 ALU peak;
  cpu_baseline  the CPU oracle on the host cores, on a bounded sample;
  emulator_bf16_vs_fp32  the 27-D emulator-style MLP likelihood (N_live
            1500, m 150, 135 slice steps, one run per SM, first iterations):
            whole-run evals/s of the BF16 tensor-core path (FP32
            re-evaluation near the threshold) and of the FP32 path, and the
            tensor-core evaluator alone against the measured BF16 peak.

``--impl reference`` times the CPU oracle as the reference arm instead.
"""
import argparse
import json
import math
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "likelihood evals/s and wall-time to log Z at |ΔlogZ|<0.1; BF16 vs FP32 path"
UNIT = "evals/s"
D, N_LIVE, M, N_STEPS, STOP = 10, 1000, 100, 50, 1e-3
# algorithmic FP32 work of one correlated-Gaussian likelihood at d = 10:
# the triangular product z = L^T y with the Cholesky factor of the
# precision (d(d+1)/2 FMA = d(d+1) FLOP) plus y = theta - mean and |z|^2
# (2d FLOP): 130 FLOP; the slice arithmetic around the likelihood (the
# candidate x + t v, the unit-cube map) is not counted
FLOP_PER_EVAL = D * (D + 1) + 2 * D
# FP32 peak: SMs (from the device) x 128 FP32 lanes x 2 FLOP x 2070 MHz
# (the maximum SM clock)
FP32_LANES, SM_MAX_MHZ = 128, 2070.0


# the 27-D emulator-style likelihood (MLP 27 -> 512 x 4 -> 2000, SiLU),
# N_live = 1500, m = 150, 135 slice steps: BF16 tensor-core path with FP32
# re-evaluation near the threshold against the plain FP32 path, on the first
# EMU_ITERS iterations of one run per SM
EMU_N, EMU_M, EMU_STEPS, EMU_ITERS = 1500, 150, 135, 2
EMU_FLOP = 2 * (27 * 512 + 3 * 512 * 512 + 512 * 2000)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--runs", type=int, default=0,
                    help="independent runs per GPU (0: as many as the GPU holds resident, one wave)")
    ap.add_argument("--m", type=int, default=M)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--chunk", type=int, default=1000)
    ap.add_argument("--profile", action="store_true",
                    help="profiling case: short launches (--chunk), dead buffers of --dead-cap, run "
                         "status ignored; prints no bench line")
    ap.add_argument("--dead-cap", type=int, default=0)
    ap.add_argument("--no-emulator", action="store_true")
    ap.add_argument("--no-batch256", action="store_true",
                    help="skip the 256-run heterogeneous batch (one walker per thread vs autotuned)")
    ap.add_argument("--profile-mlp", type=int, default=0, metavar="N",
                    help="profiling case: the BF16 and FP32 MLP evaluators on N candidates of the 27-D emulator "
                         "network, three launches each; prints no bench line")
    ap.add_argument("--clustering-tests", type=int, default=0, metavar="SEEDS",
                    help="run the clustering tests of Table 1 with SEEDS runs per configuration (m = 1), print "
                         "the JSON table and exit")
    ap.add_argument("--emulator-convergence", type=int, default=0, metavar="SEEDS",
                    help="emulator runs to convergence: BF16 vs FP32 (widened data errors), and the emulator "
                         "configuration on BF16")
    ap.add_argument("--emulator-cases", default="target150,single150",
                    help="cases of --emulator-convergence (target150, target75, single150, single75, m1, paired)")
    ap.add_argument("--mapping-study", type=int, default=0, metavar="RUNS",
                    help="walker per thread vs per warp vs autotuned, RUNS runs per shape, and the 256-run batch")
    ap.add_argument("--comparison-shapes", type=int, default=0, metavar="SEEDS",
                    help="run the section-4 comparison shapes (Gaussian d = 2..32, Rosenbrock and the 49-Gaussian "
                         "array at N = 100..1000) with SEEDS runs each, print the JSON table and exit")
    ap.add_argument("--profile-mlp-runs", type=int, default=0, metavar="R",
                    help="profiling case: R runs of the 27-D emulator workload (BF16 path), one iteration per "
                         "launch, three launches, small dead buffers; prints no bench line")
    ap.add_argument("--depth-sweep", type=int, default=0, metavar="SEEDS",
                    help="the tree-depth study of section 2.3 (Test 2 truncated to d = 2..10, depth 0..6) and exit")
    ap.add_argument("--bracket", type=int, default=0, choices=[0, 1],
                    help="--depth-sweep and --clustering-tests: the slice bracket's unit (0 the cluster's Cholesky "
                         "factor, 1 that factor times the cluster's bounding radius)")
    ap.add_argument("--correction-sweep", type=int, default=0, metavar="SEEDS",
                    help="run the batching-error study (correction schemes x m/N) with SEEDS runs per point, "
                         "print its JSON table and exit")
    return ap.parse_args()


def workload_config(args, runs, note="as many as are resident at once"):
    return {"workload": f"10-D correlated Gaussian, prior [-10,10]^10, N_live={N_LIVE}, m={args.m}, "
                        f"{N_STEPS} slice steps, stop 1e-3; {runs} independent seeded runs per GPU "
                        f"({note})",
            "d": D, "n_live": N_LIVE, "m": args.m, "slice_steps": N_STEPS, "stop_frac": STOP,
            "runs_per_gpu": runs, "correction": "sorting + history (K=1)",
            "l2": "flushed between timed steps (256 MiB write)"}


# --------------------------------------------------------------------------
# CPU oracle (baseline and reference arm): one full run per process
# --------------------------------------------------------------------------
def _oracle_one(seed_m):
    seed, m = seed_m
    sys.path.insert(0, ROOT)
    from oracle import oracle as O
    from paper_2608_28514_gb300 import workloads as W
    t0 = time.perf_counter()
    r = O.run(W.corr_gauss10(seed), N_LIVE, m, N_STEPS, STOP, seed)
    return r["n_evals"], time.perf_counter() - t0, r["logz"]


def _oracle_mlp_one(seed_n):
    """FP64 oracle evaluations of the emulator likelihood at n seeded points."""
    seed, n = seed_n
    sys.path.insert(0, ROOT)
    import numpy as np
    from oracle import oracle as O
    from paper_2608_28514_gb300 import workloads as W
    p = W.mlp_emulator(1)
    lik = O.Lik(p)
    x = np.random.default_rng(seed).uniform(size=(n, p.d))
    t0 = time.perf_counter()
    O.loglike(lik, x)
    return n, time.perf_counter() - t0


def emulator_cpu_baseline(n_proc, per_proc=1000):
    """The emulator likelihood on the host cores: the FP64 oracle's MLP, one
    process per core, per_proc evaluations each (a sample of the likelihood
    work; whole oracle runs of this workload take hours)."""
    t0 = time.perf_counter()
    out = _spawn_map(_oracle_mlp_one, [(100 + k, per_proc) for k in range(n_proc)], n_proc)
    wall = time.perf_counter() - t0
    n = sum(o[0] for o in out)
    return {"value": n / wall, "unit": UNIT, "cores": n_proc, "kind": "oracle",
            "sample": f"{n} FP64 evaluations of the 27-512x4-2000 MLP likelihood at seeded points, {per_proc} per "
                      f"process, {wall:.1f} s wall (pool start-up included)"}


def _spawn_map(fn, items, n_proc):
    """fn over items in n_proc spawned processes (safe after CUDA has been
    initialised); a worker that dies raises BrokenProcessPool instead of
    leaving the caller waiting."""
    import concurrent.futures as cf
    with cf.ProcessPoolExecutor(max_workers=max(1, n_proc), mp_context=mp.get_context("spawn")) as ex:
        return list(ex.map(fn, items))


def oracle_sample(n_proc, seeds, m):
    t0 = time.perf_counter()
    out = _spawn_map(_oracle_one, [(s, m) for s in seeds], n_proc)
    wall = time.perf_counter() - t0
    evals = sum(o[0] for o in out)
    return evals, wall, out


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


# --------------------------------------------------------------------------
# clocks during the timed region
# --------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (FileNotFoundError, OSError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() in ("active", "1", "yes"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------------------
# the emulator likelihood: BF16 vs FP32 path
# --------------------------------------------------------------------------
def emulator_compare(nat, W, torch, n_sm, peaks, cpu_cores=0):
    p = W.mlp_emulator(1)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    runs = [(p, EMU_N, EMU_M, EMU_STEPS, 1e-3, s) for s in range(1, n_sm + 1)]
    out = {"workload": f"27-D emulator MLP 27-512x4-2000 (SiLU, BF16-exact weights), N_live={EMU_N}, m={EMU_M}, "
                       f"{EMU_STEPS} slice steps, {n_sm} runs (one per SM), first {EMU_ITERS} iterations of each "
                       "(early iterations: few candidates near the threshold; whole runs in whole_run_record)",
           "reeval": "16-bit stage when |logL - threshold| < 2 + 4e-3 |threshold|, FP32 when the 16-bit value is "
                     "within 0.05 + 1e-4 |threshold| (library defaults)"}
    for name, prec in (("bf16", 1), ("fp32_tc", 2), ("fp32", 0)):
        opt = nat.ns_default_options(precision=prec, max_iter=EMU_ITERS, chunk_iters=EMU_ITERS)
        h = nat.ns_create_batch(runs, opt)
        nat.ns_run(h, check=False)  # warm-up
        nat.ns_reset(h)
        flush.zero_()
        torch.cuda.synchronize()
        nat.ns_run(h, check=False)
        st = nat.ns_get_stats(h)
        res = [nat.ns_summary(h, r) for r in range(len(runs))]
        nat.ns_destroy(h)
        ev = sum(r["n_evals"] for r in res) - EMU_N * len(runs)  # slice-step evaluations (initial set excluded)
        re = sum(r["n_reeval"] for r in res)
        tf = ev * EMU_FLOP / (st["run_ms"] / 1e3) / 1e12
        # the useful MLP work of the runs against the peak of the pipe the path computes on: the
        # measured sustained BF16 tensor rate (launches of ~0.3 s), or the FP32 ALU rate
        if prec in (1, 2):
            pk = (peaks or {}).get("bf16_tflops_sustained") or (peaks or {}).get("bf16_tflops")
            basis = "measured bf16 (sustained)" if pk else None
        else:
            pk = n_sm * FP32_LANES * 2 * SM_MAX_MHZ * 1e6 / 1e12
            basis = f"FP32 FMA: {n_sm} SMs x 128 lanes x 2 FLOP x 2070 MHz"
        out[name] = {"evals_per_s": ev / (st["run_ms"] / 1e3), "ms": st["run_ms"], "evals": ev, "fp32_reevals": re,
                     "effective_tflops": tf, "peak_tflops": pk, "frac_of_peak": (tf / pk) if pk else None,
                     "peak_basis": basis}
    out["bf16_over_fp32"] = out["bf16"]["evals_per_s"] / out["fp32"]["evals_per_s"]
    out["bf16_over_fp32_tc"] = out["bf16"]["evals_per_s"] / out["fp32_tc"]["evals_per_s"]
    # whole runs to the stopping rule take minutes per path: their numbers come
    # from the study record (bench.py --emulator-convergence), while the kernel
    # sources still match the build that wrote it
    rec = os.path.join(ROOT, "profiles", "emulator_runs_N1500.json")
    out["whole_run_record"] = None
    if os.path.exists(rec):
        try:
            rj = json.load(open(rec))
            if rj.get("csrc_sha256_16") == csrc_hash():
                out["whole_run_record"] = rj.get("summary")
        except (ValueError, KeyError):
            pass
    out["cpu_baseline"] = emulator_cpu_baseline(cpu_cores) if cpu_cores > 0 else None
    # the tensor-core evaluator alone on a large batch (8 calls of 128 candidates per SM)
    nb = nat.ns_mlp_image_bytes(p)
    img = torch.empty(nb + 1024, dtype=torch.uint8, device="cuda")
    off = (-img.data_ptr()) % 1024
    img = img[off:off + nb]
    nat.ns_mlp_pack(p, img)
    n = n_sm * 128 * 8
    x = torch.rand(n, p.d, device="cuda", generator=torch.Generator(device="cuda").manual_seed(7))
    lo = torch.empty(n, device="cuda")
    for _ in range(3):
        nat.ns_mlp_loglike(p, img, x, lo, precision=1)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 5
    stream = torch.cuda.current_stream()
    e0.record(stream)
    for _ in range(reps):
        nat.ns_mlp_loglike(p, img, x, lo, precision=1, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    achieved = n * EMU_FLOP / (ms / 1e3) / 1e12
    peak = peaks.get("bf16_tflops") if peaks else None
    out["evaluator_roofline"] = {"bound": "tensor", "kernel": "k_mlp_bf16", "achieved": achieved,
                                 "peak": peak, "unit": "TFLOP/s", "frac": (achieved / peak) if peak else None,
                                 "peak_basis": "measured bf16 burst (cuBLAS 8192^3)" if peak else None,
                                 "candidates": n, "flop_per_eval": EMU_FLOP, "ms_per_launch": ms}
    return out


# --------------------------------------------------------------------------
# the batching-error study (section 3.2): correction schemes x m/N
# --------------------------------------------------------------------------
CORRECTION_SCHEMES = (("naive", 0, 1), ("sorting", 1, 1), ("history_K1", 2, 1), ("history_K2", 2, 2),
                      ("history_K10", 2, 10), ("best_of_worst", 3, 1))
# (m, N_live): m/N = 0.001 .. 0.2 at N = 1000, and m/N = 0.5 at N = 512
# (m = 256, the library's largest batch)
SWEEP_MN = tuple((m, 1000) for m in (1, 2, 5, 10, 20, 50, 100, 200)) + ((256, 512),)


def correction_sweep(n_seeds):
    """The 2-D unit Gaussian on [-7, 7]^2, 5 d = 10 slice steps: for every
    correction scheme and m/N in {0.001 .. 0.2} (N_live = 1000) and 0.5
    (N_live = 512, m = 256), the mean and standard deviation of
    log Z - log Z_true over n_seeds runs, all runs of a scheme in one batch.
    m/N = 1 lies outside the method as read here (m = N leaves no survivor
    to seed a walker)."""
    import numpy as np
    import torch

    from paper_2608_28514_gb300 import _native as nat
    from tests import analytic
    from paper_2608_28514_gb300 import workloads as W

    p = W.gauss2d_unit_box7()
    truth = analytic.logz(p)
    table = {}
    t_all = 0.0
    for name, corr, K in CORRECTION_SCHEMES:
        opt = nat.ns_default_options(correction=corr, history_iters=K)
        runs = [(p, n_live, m, 10, 1e-3, 1000 * m + s) for m, n_live in SWEEP_MN for s in range(1, n_seeds + 1)]
        h = nat.ns_create_batch(runs, opt)
        nat.ns_run(h)
        t_all += nat.ns_get_stats(h)["run_ms"]
        res = [nat.ns_summary(h, r) for r in range(len(runs))]
        nat.ns_destroy(h)
        rows = {}
        for i, (m, n_live) in enumerate(SWEEP_MN):
            z = np.array([r["log_z"] for r in res[i * n_seeds:(i + 1) * n_seeds]]) - truth
            rel = sum(r["n_relaxed"] for r in res[i * n_seeds:(i + 1) * n_seeds])
            rows[f"{m / n_live:g}"] = {"m": m, "n_live": n_live, "mean_dlogz": float(z.mean()),
                                       "std": float(z.std(ddof=1)), "sem": float(z.std(ddof=1) / np.sqrt(n_seeds)),
                                       "relaxed_points": int(rel)}
        table[name] = rows
    torch.cuda.synchronize()
    return {"study": "batching error vs m/N (section 3.2): 2-D unit Gaussian, prior [-7,7]^2, N_live=1000 "
                     "(512 at m/N=0.5), 10 slice steps, %d seeds per point" % n_seeds,
            "log_z_true": truth, "device_ms": t_all, "schemes": table}


# --------------------------------------------------------------------------
# the clustering tests of section 2.3 (Table 1)
# --------------------------------------------------------------------------
def clustering_tests(n_seeds, m=1, n_live=1000, bracket=0):
    """Table 1: Test 1 (49 Gaussians, tree depth 6), Test 2 (two separated
    10-D Gaussians, depth 1), Test 3 (Gaussian shell, depth 4), each with (+)
    and without (-) the cluster tree, re-clustering every 100 iterations,
    5 d slice steps; all seeds of one configuration in one batch.  bracket:
    the slice bracket's unit (0 the cluster's Cholesky factor, 1 that factor
    times the cluster's bounding radius)."""
    import numpy as np
    import torch

    from paper_2608_28514_gb300 import _native as nat
    from tests import analytic
    from paper_2608_28514_gb300 import workloads as W

    tests = (("test1_array49", W.array49(), 6), ("test2_bimodal10", W.bimodal(10), 1),
             ("test3_shell", W.shell2d(), 4))
    out = {}
    for name, p, depth in tests:
        row = {"log_z_true": analytic.logz(p)}
        for tag, dep in (("+", depth), ("-", 0)):
            h = nat.ns_create_batch([(p, n_live, m, 5 * p.d, 1e-3, 7000 + s) for s in range(n_seeds)],
                                    nat.ns_default_options(depth=dep, recluster_every=100, bracket=bracket))
            nat.ns_run(h)
            st = nat.ns_get_stats(h)
            res = [nat.ns_summary(h, r) for r in range(n_seeds)]
            nat.ns_destroy(h)
            z = np.array([r["log_z"] for r in res])
            row[tag] = {"depth": dep, "log_z_mean": float(z.mean()), "log_z_std": float(z.std(ddof=1)),
                        "evaluations_mean": float(np.mean([r["n_evals"] for r in res])),
                        "device_ms_all_runs": st["run_ms"], "runs_concurrent": n_seeds}
        out[name] = row
    torch.cuda.synchronize()
    return {"study": "clustering tests (section 2.3, Table 1): N_live=%d, m=%d, %d runs per configuration"
                     % (n_live, m, n_seeds), "bracket": bracket, "tests": out}


def depth_sweep(n_seeds, m=1, n_live=1000, dims=(2, 4, 6, 8, 10), depths=(0, 1, 2, 3, 4, 5, 6), bracket=0):
    """The depth study of section 2.3 (Fig. 1): Test 2 (two Gaussians of
    weights 1/10 and 1 at -10 and +10 in every coordinate, variances
    alternating 0.1 / 1, prior [-20, 20]^d) truncated to d = 2..10, with the
    cluster tree at depth 0..6, re-clustering every 100 iterations, 5 d
    slice steps, N_live = 1000, m = 1: mean likelihood evaluations per run
    and log Z over n_seeds runs; all dimensions of one depth in one batch."""
    import numpy as np
    import torch

    from paper_2608_28514_gb300 import _native as nat
    from tests import analytic
    from paper_2608_28514_gb300 import workloads as W

    probs = {d: W.bimodal(d) for d in dims}
    truth = {d: analytic.logz(p) for d, p in probs.items()}
    table = {str(d): {"log_z_true": truth[d]} for d in dims}
    t_all = 0.0
    for dep in depths:
        runs = [(probs[d], n_live, m, 5 * d, 1e-3, 9000 + s) for d in dims for s in range(n_seeds)]
        h = nat.ns_create_batch(runs, nat.ns_default_options(depth=dep, recluster_every=100, bracket=bracket,
                                                             walker_mapping=1 if m == 1 else 0))
        nat.ns_run(h)
        t_all += nat.ns_get_stats(h)["run_ms"]
        res = [nat.ns_summary(h, r) for r in range(len(runs))]
        nat.ns_destroy(h)
        for i, d in enumerate(dims):
            rr = res[i * n_seeds:(i + 1) * n_seeds]
            z = np.array([r["log_z"] for r in rr])
            ev = np.array([r["n_evals"] for r in rr], dtype=np.float64)
            table[str(d)][str(dep)] = {"evaluations_mean": float(ev.mean()), "evaluations_sem": float(
                ev.std(ddof=1) / np.sqrt(n_seeds)), "log_z_mean": float(z.mean()), "log_z_std": float(z.std(ddof=1))}
    for d in dims:
        e0 = table[str(d)]["0"]["evaluations_mean"]
        for dep in depths:
            row = table[str(d)][str(dep)]
            row["evaluations_vs_depth0"] = row["evaluations_mean"] / e0
    torch.cuda.synchronize()
    return {"study": "tree depth sweep (section 2.3, Fig. 1): Test 2 truncated to d, N_live=%d, m=%d, 5 d slice steps, "
                     "re-clustering every 100 iterations, %d runs per point" % (n_live, m, n_seeds),
            "bracket": bracket, "device_ms": t_all, "dims": table}


# --------------------------------------------------------------------------
# replicas over ranks: runs are independent, so ranks shard them by seed and
# exchange only the timing and the counts (no data-path collective)
# --------------------------------------------------------------------------
def rank_seeds(rank, runs_per_rank):
    """Seeds of this rank's runs: disjoint across ranks."""
    return [1 + rank * runs_per_rank + r for r in range(runs_per_rank)]


def combine_ranks(t_seconds, evals, dist, device):
    """Whole-job figures over the ranks of a process group (or one process
    when dist is None): the slowest rank's time and the total evaluations."""
    if dist is None:
        return float(t_seconds), float(evals)
    import torch
    tt = torch.tensor([float(t_seconds)], dtype=torch.float64, device=device)
    ee = torch.tensor([float(evals)], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    dist.all_reduce(ee, op=dist.ReduceOp.SUM)
    return float(tt.item()), float(ee.item())


def csrc_hash():
    """First 16 hex digits of the SHA-256 of the kernel sources (names and
    contents), identifying the build that a stored ncu figure belongs to."""
    import glob
    import hashlib
    h = hashlib.sha256()
    for f in sorted(glob.glob(os.path.join(ROOT, "paper_2608_28514_gb300", "csrc", "*"))):
        h.update(os.path.basename(f).encode())
        h.update(open(f, "rb").read())
    return h.hexdigest()[:16]


# --------------------------------------------------------------------------
# the comparison shapes of section 4 (the paper's own sampler settings)
# --------------------------------------------------------------------------
def comparison_shapes(n_seeds, m=1):
    """Section 4: the unit Gaussian on [-7, 7]^d for d in {2, 4, 8, 16, 32}
    (N = 1000); the 2-D Rosenbrock on [-10, 10]^2 and the array of 49
    Gaussians for N in {100, 200, 500, 1000}; sequential (m = 1), 5 d slice
    steps, stop 1e-3; all seeds of a configuration concurrently.  Reported:
    mean and spread of log Z - log Z_true, evaluations and device time."""
    import numpy as np
    import torch

    from paper_2608_28514_gb300 import _native as nat
    from tests import analytic
    from paper_2608_28514_gb300 import workloads as W

    cases = [(f"gauss_d{d}", W.gauss_unit_box7(d), 1000) for d in (2, 4, 8, 16, 32)]
    cases += [(f"rosenbrock_N{n}", W.rosenbrock2d_box10(), n) for n in (100, 200, 500, 1000)]
    cases += [(f"array49_N{n}", W.array49(), n) for n in (100, 200, 500, 1000)]
    out = {}
    for name, p, n_live in cases:
        truth = analytic.logz(p)
        h = nat.ns_create_batch([(p, n_live, m, 5 * p.d, 1e-3, 3000 + s) for s in range(n_seeds)])
        nat.ns_run(h)
        st = nat.ns_get_stats(h)
        res = [nat.ns_summary(h, r) for r in range(n_seeds)]
        nat.ns_destroy(h)
        dz = np.array([r["log_z"] for r in res]) - truth
        out[name] = {"log_z_true": truth, "mean_dlogz": float(dz.mean()), "std_dlogz": float(dz.std(ddof=1)),
                     "mean_reported_err": float(np.mean([r["log_z_err"] for r in res])),
                     "evaluations_mean": float(np.mean([r["n_evals"] for r in res])),
                     "device_ms_all_runs": st["run_ms"], "runs_concurrent": n_seeds, "n_live": n_live}
    torch.cuda.synchronize()
    return {"study": "comparison shapes (section 4): m=%d, %d runs per configuration" % (m, n_seeds),
            "cases": out}


def _run_mapping(nat, runs, mapping, warm=0, opt_kw=None):
    """One batch of runs with walker mapping `mapping` (0 per thread, 1 per
    warp, "auto" = ns_autotune's per-run choice after `warm` iterations).
    Returns evaluations per second over the wall time of the whole job
    (autotuner included, synchronised), the autotuner's share and choices."""
    import time

    import torch

    opt = nat.ns_default_options(walker_mapping=0 if mapping == "auto" else mapping, **(opt_kw or {}))
    h = nat.ns_create_batch(runs, opt)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    tune_s, choice, ratio = 0.0, None, None
    if mapping == "auto":
        choice, ratio = nat.ns_autotune(h, warm_iters=warm, probe_iters=3)
        tune_s = time.perf_counter() - t0
    nat.ns_run(h)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    res = [nat.ns_summary(h, r) for r in range(len(runs))]
    nat.ns_destroy(h)
    ev = sum(r["n_evals"] for r in res)
    return {"evals_per_s": ev / wall, "wall_s": wall, "evals": ev, "autotune_s": tune_s, "choice": choice,
            "ratio": ratio, "results": res}


def batch256(nat, W, analytic, n_runs=256, seed=1, mappings=(0, 1, "auto")):
    """The heterogeneous batch (d 2..30, N 100..2000, m = floor(0.05 N), four
    likelihood families) with one walker per thread, one per warp, and the
    autotuner's per-run choice: aggregate evaluations per second and each
    run's log Z error against its closed form (Gaussians, and Rosenbrock and
    mixture runs up to d = 10, where the closed forms are the pins)."""
    import numpy as np

    runs = W.batched_runs(n_runs, seed=seed)
    probs = [(p, N, m, 5 * p.d, 1e-3, s) for p, N, m, s in runs]
    out = {}
    for mapping in mappings:
        r = _run_mapping(nat, probs, mapping, warm=40)  # 2 N / m iterations: X = e^-2
        z = []
        for (p, N, m, s), res in zip(runs, r["results"]):
            if p.kind in (W.GAUSS_ISO, W.GAUSS_CORR) or p.d <= 10:
                z.append((res["log_z"] - analytic.logz(p)) / res["log_z_err"])
        z = np.array(z)
        key = {0: "per_thread", 1: "per_warp", "auto": "autotuned"}[mapping]
        out[key] = {"evals_per_s": r["evals_per_s"], "wall_s": r["wall_s"],
                    "mean_abs_dlogz_over_err": float(np.mean(np.abs(z))),
                    "frac_within_2sigma": float(np.mean(np.abs(z) < 2.0)), "runs_pinned": int(len(z))}
        if mapping == "auto":
            out[key]["autotune_s"] = r["autotune_s"]
            out[key]["runs_per_warp"] = int(sum(r["choice"]))
    return {"workload": "%d runs: d ~ U{2..30}, N ~ U{100..2000}, m = floor(0.05 N), 5 d slice steps, stop 1e-3, "
                        "families iso/corr Gaussian, chained Rosenbrock, 4-mode mixture" % n_runs, **out}


def mapping_study(n_runs):
    """Batching: one walker per thread vs one walker per warp vs the
    autotuner's per-run choice, from the sequential sampler (m = 1) to the
    headline batch (m = 100), n_runs seeded runs of each shape in one batch,
    each to its stopping rule; then the heterogeneous 256-run batch."""
    import numpy as np
    import torch

    from paper_2608_28514_gb300 import _native as nat
    from tests import analytic
    from paper_2608_28514_gb300 import workloads as W

    shapes = [("gauss2d_sigma05_N100_m1", W.gauss2d_sigma05(), 100, 1, 10),
              ("corr10_N1000_m1", W.corr_gauss10(1), 1000, 1, 50),
              ("gauss_unit_box7_d30_N300_m1", W.gauss_unit_box7(30), 300, 1, 150),
              ("corr10_N1000_m10", W.corr_gauss10(1), 1000, 10, 50),
              ("corr10_N1000_m100", W.corr_gauss10(1), 1000, 100, 50)]
    out = {}
    for name, p, N, m, ns in shapes:
        probs = [(p, N, m, ns, 1e-3, 9000 + s) for s in range(n_runs)]
        row = {}
        for mapping in (0, 1, "auto"):
            r = _run_mapping(nat, probs, mapping, warm=2 * N // m)
            key = {0: "per_thread", 1: "per_warp", "auto": "autotuned"}[mapping]
            row[key] = {"evals_per_s": r["evals_per_s"], "wall_s": r["wall_s"]}
            if mapping == "auto":
                row[key]["autotune_s"] = r["autotune_s"]
                row[key]["runs_per_warp"] = int(sum(r["choice"]))
                q = [x for x in r["ratio"] if x == x]
                row[key]["ratio_warp_over_thread"] = [float(min(q)), float(np.median(q)), float(max(q))]
        out[name] = row
    out["batch256"] = batch256(nat, W, analytic)
    # BF16 MLP runs: candidates per weight pass (the tensor-core N), which the
    # autotuner also picks; the first two iterations of 152 emulator runs
    p = W.mlp_emulator(1)
    probs = [(p, EMU_N, EMU_M, EMU_STEPS, 1e-3, s) for s in range(1, 153)]
    row = {}
    for cap in (128, 64, 0):
        opt = nat.ns_default_options(precision=1, mlp_batch_cap=cap, max_iter=EMU_ITERS, chunk_iters=EMU_ITERS,
                                     dead_cap=EMU_N + 4 * EMU_M)
        h = nat.ns_create_batch(probs, opt)
        nat.ns_run(h, check=False)
        st = nat.ns_get_stats(h)
        ev = sum(nat.ns_summary(h, r)["n_evals"] for r in range(len(probs)))
        nat.ns_destroy(h)
        row["cap_%d" % cap] = {"evals_per_s": ev / (st["run_ms"] * 1e-3), "device_ms": st["run_ms"]}
    opt = nat.ns_default_options(precision=1, max_iter=10, chunk_iters=10, dead_cap=EMU_N + 20 * EMU_M)
    h = nat.ns_create_batch(probs, opt)
    choice, ratio = nat.ns_autotune(h, warm_iters=1, probe_iters=1)
    nat.ns_destroy(h)
    row["autotuned_caps"] = {str(c): choice.count(c) for c in sorted(set(choice))}
    row["ratio_cap64_over_cap128_median"] = float(np.median([x for x in ratio if x == x]))
    out["emulator27_m150_candidates_per_pass"] = row
    torch.cuda.synchronize()
    return {"study": "walker mappings and the autotuner: %d runs per shape, evaluations/s over the wall time of the "
                     "job (autotuner included; warm-up 2 N / m iterations)" % n_runs, "cases": out}


def emulator_convergence(n_seeds, cases="target150,single150"):
    """Whole runs of the 27-D emulator likelihood (27-512x4-2000, sigma_k in
    [1e-3, 1e-1]) to their stopping rule, 135 slice steps, stop 1e-3, seeds
    500.., one network.  Cases (comma-separated; each prints one JSON line
    as soon as it ends):
      target150 / target75: the emulator configuration (N = 1500, m = 150 or
        75), n_seeds runs on the BF16 path (FP32 re-evaluation near the
        threshold) and the same n_seeds runs on the FP32 path of the tensor
        cores (precision 2), one SM per run, all runs of a path concurrently:
        log Z per seed on both paths, the paired difference BF16 - FP32 with
        its standard error, wall time to the stopping rule (device time of
        ns_run), evaluations/s, the FP32 re-evaluation share;
      cluster150 / cluster75: the same paired comparison with every run
        split over a 4-CTA cluster (n_seeds clusters side by side);
      single150 / single75: one run alone (seed 500) split over a 4-CTA
        cluster (4 SMs), BF16 and FP32 paths: its wall time to log Z;
      m1: m = 1 (the sequential sampler), one run on a 4-CTA cluster, the
        first 200 iterations on both paths: evaluations/s and iterations/s;
      paired: N = 200, m = 20, BF16 against the FP32 path of the CUDA cores
        (precision 0), n_seeds runs each."""
    import numpy as np
    import torch

    from paper_2608_28514_gb300 import _native as nat
    from paper_2608_28514_gb300 import workloads as W

    def runs_of(p, N, m, precision, seeds, cluster, max_iter=0):
        kw = dict(precision=precision, mlp_cluster=cluster)
        if max_iter:
            kw.update(max_iter=max_iter, chunk_iters=max_iter, dead_cap=N + 4 * m * max_iter)
        opt = nat.ns_default_options(**kw)
        h = nat.ns_create_batch([(p, N, m, 5 * p.d, 1e-3, s) for s in seeds], opt)
        nat.ns_run(h, check=False)
        st = nat.ns_get_stats(h)
        res = [nat.ns_summary(h, r) for r in range(len(seeds))]
        nat.ns_destroy(h)
        z = np.array([r["log_z"] for r in res])
        ev = np.array([r["n_evals"] for r in res], dtype=np.float64)
        cands = sum(r["n_cand_bf16"] for r in res)
        return {"device_s": st["run_ms"] * 1e-3, "runs": len(seeds), "cluster_ctas": cluster,
                "evals_per_run": float(ev.mean()), "evals_per_s": float(ev.sum() / (st["run_ms"] * 1e-3)),
                "iterations_per_run": float(np.mean([r["n_iter"] for r in res])),
                "fp32_evaluations_per_run": float(np.mean([r["n_cand_fp32"] for r in res])),
                "fp32_reeval_share": (float(sum(r["n_reeval"] for r in res) / max(1, cands)) if precision == 1
                                      else None),
                "x2_reeval_share": (float(sum(r["n_cand_x2"] for r in res) / max(1, cands)) if precision == 1
                                    else None),
                "rounds_per_run": float(np.mean([r["n_rounds"] for r in res])),
                "bf16_candidates_per_pass": (cands / max(1, sum(r["n_pass_bf16"] for r in res))) if cands else None,
                "log_z": z.tolist(), "log_z_mean": float(z.mean()), "log_z_std": float(z.std(ddof=1)) if len(z) > 1
                else 0.0, "log_z_err_mean": float(np.mean([r["log_z_err"] for r in res])),
                "info_h_mean": float(np.mean([r["info"] for r in res])),
                "status": sorted({int(r["status"]) for r in res})}

    def emit(name, obj):
        print(json.dumps({"case": name, **obj}), flush=True)
        return obj

    out = {}
    p = W.mlp_emulator(1)
    seeds = [500 + s for s in range(n_seeds)]
    for m in (150, 75):
        if f"target{m}" in cases:
            a = {"bf16": runs_of(p, 1500, m, 1, seeds, 1), "fp32_tc": runs_of(p, 1500, m, 2, seeds, 1)}
            dz = np.array(a["bf16"]["log_z"]) - np.array(a["fp32_tc"]["log_z"])
            se = float(dz.std(ddof=1) / np.sqrt(len(dz))) if len(dz) > 1 else float("nan")
            a["paired_dlogz"] = {"mean": float(dz.mean()), "std": float(dz.std(ddof=1)) if len(dz) > 1 else 0.0,
                                 "standard_error": se, "bound_abs_mean_plus_2se": float(abs(dz.mean()) + 2 * se),
                                 "max_abs": float(np.max(np.abs(dz))),
                                 "seeds_identical": int(np.sum(dz == 0.0)), "seeds": len(dz)}
            a["wall_time_ratio_fp32_over_bf16"] = a["fp32_tc"]["device_s"] / a["bf16"]["device_s"]
            out[f"target_N1500_m{m}"] = emit(f"target{m}", a)
        if f"cluster{m}" in cases:
            a = {"bf16": runs_of(p, 1500, m, 1, seeds, 4), "fp32_tc": runs_of(p, 1500, m, 2, seeds, 4)}
            dz = np.array(a["bf16"]["log_z"]) - np.array(a["fp32_tc"]["log_z"])
            se = float(dz.std(ddof=1) / np.sqrt(len(dz))) if len(dz) > 1 else float("nan")
            a["paired_dlogz"] = {"mean": float(dz.mean()), "std": float(dz.std(ddof=1)) if len(dz) > 1 else 0.0,
                                 "standard_error": se, "bound_abs_mean_plus_2se": float(abs(dz.mean()) + 2 * se),
                                 "max_abs": float(np.max(np.abs(dz))),
                                 "seeds_identical": int(np.sum(dz == 0.0)), "seeds": len(dz)}
            a["wall_time_ratio_fp32_over_bf16"] = a["fp32_tc"]["device_s"] / a["bf16"]["device_s"]
            out[f"cluster_N1500_m{m}_4cta"] = emit(f"cluster{m}", a)
        if f"single{m}" in cases:
            a = {"bf16": runs_of(p, 1500, m, 1, seeds[:1], 4), "fp32_tc": runs_of(p, 1500, m, 2, seeds[:1], 4)}
            a["wall_time_ratio_fp32_over_bf16"] = a["fp32_tc"]["device_s"] / a["bf16"]["device_s"]
            out[f"single_run_N1500_m{m}_4cta"] = emit(f"single{m}", a)
    if "m1" in cases:
        a = {"bf16": runs_of(p, 1500, 1, 1, seeds[:1], 4, max_iter=200),
             "fp32_tc": runs_of(p, 1500, 1, 2, seeds[:1], 4, max_iter=200)}
        for k in ("bf16", "fp32_tc"):
            a[k]["iterations_per_s"] = a[k]["iterations_per_run"] / a[k]["device_s"]
        out["m1_segment_200_iterations_4cta"] = emit("m1", a)
    if "paired" in cases:
        a = {"bf16": runs_of(p, 200, 20, 1, seeds, 1), "fp32_cuda_cores": runs_of(p, 200, 20, 0, seeds, 1)}
        a["dlogz_bf16_minus_fp32"] = a["bf16"]["log_z_mean"] - a["fp32_cuda_cores"]["log_z_mean"]
        a["dlogz_standard_error"] = float(np.sqrt((a["bf16"]["log_z_std"] ** 2 + a["fp32_cuda_cores"]["log_z_std"] ** 2)
                                                  / n_seeds))
        a["wall_time_ratio_fp32_over_bf16"] = a["fp32_cuda_cores"]["device_s"] / a["bf16"]["device_s"]
        out["paired_N200_m20"] = emit("paired", a)
    torch.cuda.synchronize()
    return {"study": "emulator runs to convergence: seeds 500.., 135 slice steps, stop 1e-3", "cases": out}


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return None


# --------------------------------------------------------------------------
# reference arm: the CPU oracle
# --------------------------------------------------------------------------
def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    cores = host_cores()
    n_proc = max(1, min(cores, 16))
    times, evals_all = [], 0
    seed = 1
    for step in range(args.warmup + args.steps):
        seeds = list(range(seed, seed + n_proc))
        seed += n_proc
        ev, wall, _ = oracle_sample(n_proc, seeds, args.m)
        if step >= args.warmup:
            times.append(wall)
            evals_all += ev
    total = sum(times)
    value = evals_all / total
    sample = (f"each step: {n_proc} full runs of the workload (one seeded run per process, "
              f"{n_proc} processes), FP64 oracle")
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(args, n_proc, "the reference arm: a bounded sample of the GPU arm's resident "
                                                    "wave, one run per host process"), "impl": "reference",
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": n_proc, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------
# the GB300 arm
# --------------------------------------------------------------------------
def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.profile_mlp > 0:
        import torch
        from paper_2608_28514_gb300 import _native as nat
        from paper_2608_28514_gb300 import workloads as W
        p = W.mlp_emulator(1)
        nb = nat.ns_mlp_image_bytes(p)
        img = torch.empty(nb + 1024, dtype=torch.uint8, device="cuda")
        img = img[(-img.data_ptr()) % 1024:][:nb]
        nat.ns_mlp_pack(p, img)
        x = torch.rand(args.profile_mlp, p.d, device="cuda", generator=torch.Generator(device="cuda").manual_seed(7))
        out = torch.empty(args.profile_mlp, device="cuda")
        for prec in (1, 0):
            for _ in range(3):
                nat.ns_mlp_loglike(p, img, x, out, precision=prec)
        torch.cuda.synchronize()
        print("profile case done", float(out[:8].sum()))
        return
    if args.profile_mlp_runs > 0:
        import torch
        from paper_2608_28514_gb300 import _native as nat
        from paper_2608_28514_gb300 import workloads as W
        p = W.mlp_emulator(1)
        opt = nat.ns_default_options(precision=1, max_iter=1, chunk_iters=1, dead_cap=EMU_N + 4 * EMU_M)
        h = nat.ns_create_batch([(p, EMU_N, EMU_M, EMU_STEPS, 1e-3, s)
                                 for s in range(1, args.profile_mlp_runs + 1)], opt)
        for _ in range(3):
            nat.ns_reset(h)
            nat.ns_run(h, check=False)
        torch.cuda.synchronize()
        print("profile case done", nat.ns_get_stats(h))
        nat.ns_destroy(h)
        return
    if args.emulator_convergence > 0:
        if int(os.environ.get("RANK", "0")) == 0:
            print(json.dumps(emulator_convergence(args.emulator_convergence, args.emulator_cases)), flush=True)
        return
    if args.mapping_study > 0:
        if int(os.environ.get("RANK", "0")) == 0:
            print(json.dumps(mapping_study(args.mapping_study)), flush=True)
        return
    if args.comparison_shapes > 0:
        if int(os.environ.get("RANK", "0")) == 0:
            print(json.dumps(comparison_shapes(args.comparison_shapes)), flush=True)
        return
    if args.clustering_tests > 0:
        if int(os.environ.get("RANK", "0")) == 0:
            print(json.dumps(clustering_tests(args.clustering_tests, bracket=args.bracket)), flush=True)
        return
    if args.depth_sweep > 0:
        if int(os.environ.get("RANK", "0")) == 0:
            print(json.dumps(depth_sweep(args.depth_sweep, bracket=args.bracket)), flush=True)
        return
    if args.correction_sweep > 0:
        if int(os.environ.get("RANK", "0")) == 0:
            print(json.dumps(correction_sweep(args.correction_sweep)), flush=True)
        return
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    # the CPU baseline pool starts before the first GPU call (spawned workers)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cores = host_cores()
        n_proc = max(1, min(cores, 16))
        ev, wall, _ = oracle_sample(n_proc, list(range(10001, 10001 + n_proc)), args.m)
        cpu = {"value": ev / wall, "unit": UNIT, "cores": n_proc, "kind": "oracle",
               "sample": f"{n_proc} full runs of the workload (seeds 10001..{10000 + n_proc}), one per process, "
                         f"{wall:.1f} s wall"}

    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2608_28514_gb300 import _native as nat
    from tests import analytic
    from paper_2608_28514_gb300 import workloads as W

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    R = args.runs
    if R <= 0:
        per_sm = nat.ns_resident_runs_per_sm(D, args.m, 0)
        R = max(1, per_sm) * torch.cuda.get_device_properties(local).multi_processor_count
    seeds = rank_seeds(rank, R)
    probs = [W.corr_gauss10(s) for s in seeds]
    truths = np.array([analytic.logz(p) for p in probs])
    runs = [(p, N_LIVE, args.m, N_STEPS, STOP, s) for p, s in zip(probs, seeds)]
    opt = nat.ns_default_options(chunk_iters=args.chunk, dead_cap=args.dead_cap)
    if args.profile:
        opt.max_iter = 3 * args.chunk
    h = nat.ns_create_batch(runs, opt)
    if args.profile:
        for _ in range(3):
            nat.ns_reset(h)
            nat.ns_run(h, check=False)
        torch.cuda.synchronize()
        print("profile case done", nat.ns_get_stats(h))
        nat.ns_destroy(h)
        return
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def one_step():
        nat.ns_reset(h, stream)
        flush.zero_()
        torch.cuda.synchronize()
        nat.ns_run(h, stream)
        st = nat.ns_get_stats(h)
        res = [nat.ns_summary(h, r) for r in range(R)]
        return st, res

    for _ in range(args.warmup):
        one_step()

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    sampler = ClockSampler(local)
    sampler.start()
    barrier()
    dev_ms, ker_ms, launches, evals, wall_first = 0.0, 0.0, 0, 0, None
    last_res = None
    for k in range(args.steps):
        st, res = one_step()
        dev_ms += st["run_ms"]
        ker_ms += st["kernel_ms"]
        launches += st["launches"]
        evals += sum(r["n_evals"] for r in res)
        last_res = res
    barrier()
    clocks = sampler.stop()

    t_dev, evals_all = combine_ranks(dev_ms / 1e3, evals, dist if world > 1 else None, "cuda")
    value = evals_all / t_dev

    phase = {k: 0 for k in nat.PHASES + nat.WALK_PHASES}
    for r in range(R):
        for k, v in nat.ns_phase_cycles(h, r, walk=True).items():
            phase[k] += v
    tot_c = max(1, sum(v for k, v in phase.items() if k in nat.PHASES))
    phase_frac = {k: round(v / tot_c, 4) for k, v in phase.items()}
    status = [r["status"] for r in last_res]
    logz = np.array([r["log_z"] for r in last_res])
    err = np.array([r["log_z_err"] for r in last_res])
    dz = logz - truths
    acc = {"mean_dlogz": float(np.mean(dz)), "mean_abs_dlogz": float(np.mean(np.abs(dz))),
           "frac_abs_dlogz_lt_0.1": float(np.mean(np.abs(dz) < 0.1)),
           "frac_within_2sigma": float(np.mean(np.abs(dz) < 2 * err)), "mean_logz_err": float(np.mean(err)),
           "all_status_ok": all(s == 0 for s in status)}

    # roofline of the run kernel (the only kernel of the timed region)
    avg_launch_s = (ker_ms / 1e3) / max(1, launches)
    flops_per_launch = FLOP_PER_EVAL * evals / max(1, launches)
    achieved = flops_per_launch / avg_launch_s / 1e12
    n_sm = torch.cuda.get_device_properties(local).multi_processor_count
    peak = n_sm * FP32_LANES * 2 * SM_MAX_MHZ * 1e6 / 1e12
    # DRAM bytes per launch from the ncu record of this kernel, scaled by the
    # run-iterations of a launch; null once the kernel sources have changed
    traffic = None
    tf = os.path.join(ROOT, "profiles", "traffic_k_run.json")
    if os.path.exists(tf):
        try:
            tj = json.load(open(tf))
            if tj.get("csrc_sha256_16") == csrc_hash():
                iters = sum(r["n_iter"] for r in last_res)
                traffic = tj["bytes_per_run_iteration"] * iters * args.steps / max(1, launches)
        except (ValueError, KeyError):
            traffic = None
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": traffic, "kernel": "nsd::k_run<10>",
                "peak_basis": f"FP32 FMA: {n_sm} SMs (device) x 128 lanes x 2 FLOP x 2070 MHz (max clock)",
                "flop_per_eval": FLOP_PER_EVAL}

    # end to end through the C ABI from host buffers
    e2e = None
    if not args.no_e2e:
        e2e_t, e2e_evals, h2d, d2h = 0.0, 0, 0, 0
        for k in range(args.steps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            h2 = nat.ns_create_batch(runs, opt)
            nat.ns_run(h2, stream)
            res = [nat.ns_result(h2, r) for r in range(R)]
            st2 = nat.ns_get_stats(h2)
            nat.ns_destroy(h2)
            torch.cuda.synchronize()
            e2e_t += time.perf_counter() - t0
            e2e_evals += sum(r["n_evals"] for r in res)
            h2d, d2h = st2["h2d_bytes"], st2["d2h_bytes"]
            del res
        e2e_t, e2e_evals = combine_ranks(e2e_t, e2e_evals, dist if world > 1 else None, "cuda")
        e2e = {"value": e2e_evals / e2e_t, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h), "includes": "ns_create + ns_run + ns_result(all runs) + ns_destroy"}

    nat.ns_destroy(h)
    emulator = None
    if not args.no_emulator:
        emulator = emulator_compare(nat, W, torch, torch.cuda.get_device_properties(local).multi_processor_count,
                                    measured_peaks(), cpu_cores=0 if args.no_cpu else min(16, host_cores()))
    hetero = None
    if not args.no_batch256 and world == 1:
        hetero = batch256(nat, W, analytic, mappings=(0, "auto"))
    # "wall time to log Z at |dlogZ| < 0.1": one run of this workload reports
    # an error of ~0.165, so an estimate with a standard error below 0.1 is the
    # mean of k = 4 independent runs of one problem; they run side by side, so
    # the time to it is the device time of one 4-run launch to the stopping rule
    k_pool = 4
    p0 = W.corr_gauss10(1)
    hp = nat.ns_create_batch([(p0, N_LIVE, args.m, N_STEPS, STOP, 9000 + j) for j in range(k_pool)],
                             nat.ns_default_options(chunk_iters=args.chunk))
    nat.ns_run(hp, stream)
    rp = [nat.ns_summary(hp, j) for j in range(k_pool)]
    pooled = {"runs": k_pool, "device_s": nat.ns_get_stats(hp)["run_ms"] * 1e-3,
              "log_z_mean": float(np.mean([r["log_z"] for r in rp])),
              "standard_error": float(np.sqrt(sum(r["log_z_err"] ** 2 for r in rp)) / k_pool),
              "log_z_true": float(analytic.logz(p0))}
    pooled["abs_dlogz"] = abs(pooled["log_z_mean"] - pooled["log_z_true"])
    nat.ns_destroy(hp)
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": 1e3 * t_dev / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": dict(workload_config(args, R), parallelism=f"replicas x{world} (runs sharded by seed)"),
                "wall_time_to_logz_s": t_dev / args.steps,
                "wall_time_to_logz_reading": "device time of one step: every run of the batch from its initial live "
                                             "set to its stopping rule (per-run error in accuracy.mean_logz_err)",
                "time_to_logz_se_below_0.1": pooled, "accuracy": acc, "clocks": clocks,
                "gpu_launches": launches, "roofline": roofline, "e2e": e2e, "cpu_baseline": cpu,
                "phase_cycle_share": phase_frac, "emulator_bf16_vs_fp32": emulator, "batch256": hetero}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
