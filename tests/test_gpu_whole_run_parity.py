"""Whole runs of the benchmark configurations against the FP64 oracle, in
distribution, with the statistic the target names: over 50 seeds, the
fraction of runs whose |log Z_GPU - log Z_oracle| lies within twice the
combined reported error sqrt(err_GPU^2 + err_oracle^2).

Nested sampling is a random estimator, so a whole run can only be compared
in distribution: the GPU run of seed s and the oracle run of seed 500000 + s
(tests/golden/oracle_runs_50.json, written by make_oracle_runs.py from the
oracle alone) are two independent draws on the same problem.  If both are
unbiased and their errors sqrt(H / N) are right, each difference falls
within 2 combined errors with probability 0.9545; at least 44 of 50 must
(the 1 % point of Binomial(50, 0.9545)).  The mean difference must also lie
within 3 standard errors of zero.  Configurations: the 2-D Gaussian (m = 1),
the 10-D correlated Gaussian at m = 1, 10, 50, 100, Rosenbrock in 2 and 10
dimensions (m = 50) and the 4-mode mixture in 5-D (N = 2000, m = 200,
cluster tree of depth 3).

One exception is a property of the method, not of either implementation:
on the 10-D Rosenbrock valley at 5 d slice steps the reported error
sqrt(H / N) understates the run-to-run scatter about twofold (the oracle's
50 runs: scatter 0.40, mean reported error 0.19), so no sampler passes the
reported-error statistic there.  For that configuration the two samples of
50 runs are compared as distributions instead: the same statistic with each
side's measured scatter in place of its reported error, the means within 3
standard errors, the scatters within the 1 % bounds of their F ratio, and a
two-sample Kolmogorov-Smirnov test at the 1 % level.
"""
import json
import math
import os

import numpy as np
import pytest

from paper_2608_28514_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "oracle_runs_50.json")
MIN_WITHIN_2SIGMA = 44  # of 50: P(Binomial(50, 0.9545) < 44) = 0.007
# configurations whose reported errors understate the scatter (the method's, see above)
UNDERSTATED_ERRORS = {"config3_rosenbrock10_m50"}

PROBLEMS = {
    "config1_gauss2d_m1": lambda s: W.gauss2d_sigma05(),
    "config2_corr10_m1": W.corr_gauss10, "config2_corr10_m10": W.corr_gauss10,
    "config2_corr10_m50": W.corr_gauss10, "config2_corr10_m100": W.corr_gauss10,
    "config3_rosenbrock2_m50": lambda s: W.rosenbrock(2),
    "config3_rosenbrock10_m50": lambda s: W.rosenbrock(10),
    "config3_mixture5_m200_depth3": W.mixture4_d5,
}


@pytest.fixture(scope="module")
def nat():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2608_28514_gb300 import _native
    _native.lib()
    return _native


@pytest.fixture(scope="module")
def golden():
    with open(GOLDEN) as f:
        return json.load(f)


@pytest.mark.parametrize("name", list(PROBLEMS))
def test_fifty_seeds_within_two_combined_sigma(nat, golden, name):
    cfg = golden["configs"][name]
    orc = golden["runs"][name]
    assert len(orc) == 50 and all(r["status"] == 0 for r in orc)
    seeds = [r["problem_seed"] for r in orc]
    probs = [PROBLEMS[name](s) for s in seeds]
    opt = nat.ns_default_options(depth=cfg["depth"])
    h = nat.ns_create_batch([(p, cfg["N"], cfg["m"], cfg["slice_steps"], golden["stop_frac"], s)
                             for p, s in zip(probs, seeds)], opt)
    nat.ns_run(h)
    res = [nat.ns_summary(h, r) for r in range(len(seeds))]
    nat.ns_destroy(h)
    assert all(r["status"] == 0 for r in res)
    zg = np.array([r["log_z"] for r in res])
    eg = np.array([r["log_z_err"] for r in res])
    zo = np.array([r["logz"] for r in orc])
    eo = np.array([r["logz_err"] for r in orc])
    dz = zg - zo
    if name in UNDERSTATED_ERRORS:
        from scipy import stats
        comb = np.full(len(dz), math.hypot(zg.std(ddof=1), zo.std(ddof=1)))
        f = zg.var(ddof=1) / zo.var(ddof=1)
        n1 = len(zg) - 1
        assert stats.f.ppf(0.005, n1, n1) < f < stats.f.ppf(0.995, n1, n1), (name, f)
        assert stats.ks_2samp(zg, zo).pvalue > 0.01, name
    else:
        comb = np.sqrt(eg ** 2 + eo ** 2)
    within = int(np.sum(np.abs(dz) < 2 * comb))
    assert within >= MIN_WITHIN_2SIGMA, (name, within, dz.tolist(), comb.tolist())
    se = dz.std(ddof=1) / math.sqrt(len(dz))
    assert abs(dz.mean()) < 3 * se, (name, dz.mean(), se)
