"""Writes tests/golden/oracle_runs_50.json: whole FP64 oracle runs, 50
seeds per benchmark configuration, for the whole-run parity tests
(tests/test_gpu_whole_run_parity.py); with --batch256, writes
tests/golden/oracle_batch256_highd.json: one oracle run for each
Rosenbrock and mixture run above d = 10 of the 256-run heterogeneous batch
(workloads.batched_runs(256, seed=1)), for tests/test_gpu_batch.py.

Only the oracle (oracle/) and the seeded problem descriptions
(paper_2608_28514_gb300/workloads.py) are used.  Each configuration is run
with its own seeds (500000 + s), independent of the GPU runs' seeds (s),
on the same problem instance (problem seed s where the configuration draws
one per seed), so a GPU run and its oracle partner are two independent
draws of the same estimator.

Usage: python tests/golden/make_oracle_runs.py [--batch256] [workers]
"""
import hashlib
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

N_SEEDS = 50
ORACLE_SEED0 = 500000
OUT = os.path.join(HERE, "oracle_runs_50.json")
OUT_B256 = os.path.join(HERE, "oracle_batch256_highd.json")


def configs():
    """name -> (problem factory of the seed, N, m, slice steps, cluster depth)."""
    from paper_2608_28514_gb300 import workloads as W
    c = {"config1_gauss2d_m1": (lambda s: W.gauss2d_sigma05(), 100, 1, 10, 0)}
    for m in (1, 10, 50, 100):
        c[f"config2_corr10_m{m}"] = (lambda s: W.corr_gauss10(s), 1000, m, 50, 0)
    c["config3_rosenbrock2_m50"] = (lambda s: W.rosenbrock(2), 1000, 50, 10, 0)
    c["config3_rosenbrock10_m50"] = (lambda s: W.rosenbrock(10), 1000, 50, 50, 0)
    c["config3_mixture5_m200_depth3"] = (lambda s: W.mixture4_d5(s), 2000, 200, 25, 3)
    return c


def _one(job):
    name, s = job
    from oracle import oracle as O
    make, N, m, ns, depth = configs()[name]
    p = make(s)
    o = O.opts(p.d, m, depth=depth)
    t0 = time.perf_counter()
    r = O.run(p, N, m, ns, 1e-3, ORACLE_SEED0 + s, o=o)
    return {"config": name, "problem_seed": s, "oracle_seed": ORACLE_SEED0 + s, "logz": r["logz"],
            "logz_err": r["logz_err"], "n_evals": int(r["n_evals"]), "n_iter": int(r["n_iter"]),
            "status": int(r["status"]), "cpu_s": time.perf_counter() - t0}


def main(workers):
    import concurrent.futures as cf
    import multiprocessing as mp
    from oracle import build_oracle
    build_oracle.build()
    src = open(os.path.join(ROOT, "oracle", "ns_oracle.c"), "rb").read()
    jobs = [(name, s) for name in configs() for s in range(1, N_SEEDS + 1)]
    # longest configurations first keeps the pool busy to the end
    order = {"config3_rosenbrock10_m50": 0, "config3_mixture5_m200_depth3": 1, "config2_corr10_m1": 2}
    jobs.sort(key=lambda j: order.get(j[0], 9))
    t0 = time.perf_counter()
    with cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
        rows = list(ex.map(_one, jobs))
    out = {"about": "FP64 oracle whole runs (oracle/ns_oracle.c), 50 seeds per configuration; "
                    "written by tests/golden/make_oracle_runs.py",
           "oracle_c_sha256_16": hashlib.sha256(src).hexdigest()[:16], "stop_frac": 1e-3,
           "configs": {k: {"N": v[1], "m": v[2], "slice_steps": v[3], "depth": v[4]} for k, v in configs().items()},
           "runs": {}}
    for r in rows:
        out["runs"].setdefault(r["config"], []).append(r)
    for k in out["runs"]:
        out["runs"][k].sort(key=lambda r: r["problem_seed"])
    with open(OUT, "w") as f:
        json.dump(out, f, indent=0)
    print(f"{len(rows)} runs in {time.perf_counter() - t0:.0f} s -> {OUT}")


def batch256_highd():
    """(index in the batch, problem, N, m, run seed) of the batch's Rosenbrock
    and mixture runs above d = 10."""
    from paper_2608_28514_gb300 import workloads as W
    runs = W.batched_runs(256, seed=1)
    return [(i, p, N, m, s) for i, (p, N, m, s) in enumerate(runs)
            if p.d > 10 and p.kind in (W.ROSENBROCK, W.MIXTURE)]


def _one_b256(i):
    from oracle import oracle as O
    sel = {k: (p, N, m, s) for k, p, N, m, s in batch256_highd()}
    p, N, m, s = sel[i]
    t0 = time.perf_counter()
    r = O.run(p, N, m, 5 * p.d, 1e-3, ORACLE_SEED0 + s)
    return {"index": i, "name": p.name, "d": p.d, "N": N, "m": m, "run_seed": s, "oracle_seed": ORACLE_SEED0 + s,
            "logz": r["logz"], "logz_err": r["logz_err"], "n_evals": int(r["n_evals"]), "status": int(r["status"]),
            "cpu_s": time.perf_counter() - t0}


def main_b256(workers):
    import concurrent.futures as cf
    import multiprocessing as mp
    from oracle import build_oracle
    build_oracle.build()
    src = open(os.path.join(ROOT, "oracle", "ns_oracle.c"), "rb").read()
    sel = batch256_highd()
    # largest jobs first (d N is a rough cost)
    idx = [k for k, p, N, m, s in sorted(sel, key=lambda t: -t[1].d * t[2])]
    t0 = time.perf_counter()
    with cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
        rows = list(ex.map(_one_b256, idx))
    rows.sort(key=lambda r: r["index"])
    out = {"about": "FP64 oracle whole runs (oracle/ns_oracle.c) of the Rosenbrock and mixture runs above d = 10 "
                    "of workloads.batched_runs(256, seed=1), 5 d slice steps, stop 1e-3, oracle seed 500000 + the "
                    "run's seed; written by tests/golden/make_oracle_runs.py --batch256",
           "oracle_c_sha256_16": hashlib.sha256(src).hexdigest()[:16], "runs": rows}
    with open(OUT_B256, "w") as f:
        json.dump(out, f, indent=0)
    print(f"{len(rows)} runs in {time.perf_counter() - t0:.0f} s -> {OUT_B256}")


if __name__ == "__main__":
    args = [a for a in sys.argv[1:] if not a.startswith("--")]
    w = int(args[0]) if args else (os.cpu_count() or 1)
    if "--batch256" in sys.argv:
        main_b256(w)
    else:
        main(w)
