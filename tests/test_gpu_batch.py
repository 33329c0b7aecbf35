"""Heterogeneous batches of independent runs in one call (the 256-run
workload: d uniform in 2..30, N uniform in 100..2000, m = floor(0.05 N), a
likelihood family uniform over isotropic / correlated Gaussian, chained
Rosenbrock and 4-mode mixture), through the C ABI.

Pins: the closed forms (Gaussians, mixture) and the transfer-operator
quadrature (Rosenbrock).  Gaussian runs of every dimension and the
Rosenbrock and mixture runs up to d = 10 agree with their pins; above that,
with 5 d slice steps and a fixed live-set size, the method itself drifts
(curved valleys, well separated narrow modes), so those 76 runs are checked
against independent FP64 oracle runs of the same problems instead.
"""
import math

import numpy as np
import pytest

from tests import analytic as A
from paper_2608_28514_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def nat():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2608_28514_gb300 import _native
    _native.lib()
    return _native


def _family(p):
    return {W.GAUSS_ISO: "gauss", W.GAUSS_CORR: "gauss", W.ROSENBROCK: "rosenbrock", W.MIXTURE: "mixture"}[p.kind]


@pytest.fixture(scope="module")
def batch256(nat):
    runs = W.batched_runs(256, seed=1)
    h = nat.ns_create_batch([(p, N, m, 5 * p.d, 1e-3, s) for p, N, m, s in runs])
    nat.ns_run(h)
    res = [nat.ns_result(h, r) for r in range(len(runs))]
    stats = nat.ns_get_stats(h)
    nat.ns_destroy(h)
    return runs, res, stats


def test_batch256_every_run_completes(batch256):
    runs, res, stats = batch256
    assert len({p.kind for p, *_ in runs}) == 4
    assert len({p.d for p, *_ in runs}) > 20
    for (p, N, m, s), r in zip(runs, res):
        assert r["status"] == 0 and r["d"] == p.d
        assert np.isfinite(r["log_z"]) and r["log_z_err"] > 0
        assert r["n_dead"] == r["n_iter"] * m + N
        nd = r["n_iter"] * m
        assert np.all(np.diff(r["dead_l"][:nd]) >= 0)
        w = r["dead_logw"]
        assert abs(np.log(np.sum(np.exp(w - w.max()))) + w.max() - r["log_z"]) < 1e-9
    assert stats["launches"] > 0


def test_batch256_against_pins(batch256):
    """The Gaussian runs of every dimension and the Rosenbrock and mixture
    runs up to d = 10 (180 runs) against their closed forms, with the
    target's statistic: the fraction of runs within twice their reported
    error at least the 1 % point of Binomial(n, 0.9545), per family group,
    and every run within 4 reported errors (the batch's runs are fixed by
    their seeds; the largest deviation is 3.6 errors, a 9-D Rosenbrock)."""
    from scipy.stats import binom
    runs, res, _ = batch256
    dz = {"gauss": [], "rosenbrock": [], "mixture": []}
    for (p, N, m, s), r in zip(runs, res):
        fam = _family(p)
        truth = A.logz(p)
        z = (r["log_z"] - truth) / r["log_z_err"]
        if fam == "gauss" or p.d <= 10:
            assert abs(z) < 4.0, (p.name, N, m, r["log_z"], truth, r["log_z_err"])
            dz[fam].append(z)
    g = np.array(dz["gauss"])
    low = np.array(dz["rosenbrock"] + dz["mixture"])
    assert len(g) > 100 and len(low) >= 20
    for zz in (g, low):
        n = len(zz)
        assert int(np.sum(np.abs(zz) < 2)) >= int(binom.ppf(0.01, n, 0.9545)), (n, int(np.sum(np.abs(zz) < 2)))
    assert abs(g.mean()) < 0.6 and 0.5 < g.std() < 1.6
    assert abs(low.mean()) < 1.5


def test_batch256_high_d_runs_match_the_oracle(batch256):
    """The batch's Rosenbrock and mixture runs above d = 10 (76 runs), whose
    closed forms the method at 5 d slice steps does not reach and whose
    reported errors understate the scatter (the method's drift, which the
    FP64 oracle shows as much as the GPU path), against one independent FP64
    oracle run each of the same problem (tests/golden/oracle_batch256_highd.json,
    written from the oracle alone), as distributions: the deviations from the
    pins in units of the reported error, (log Z - log Z_pin) / err, of the GPU
    runs and of the oracle runs pass a two-sample Kolmogorov-Smirnov test at
    the 1 % level and have equal means within 3 standard errors; and the
    paired differences log Z_GPU - log Z_oracle have mean zero within 3
    standard errors."""
    import json
    import os
    from scipy import stats
    runs, res, _ = batch256
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "oracle_batch256_highd.json")) as f:
        orc = json.load(f)["runs"]
    assert len(orc) >= 50 and all(o["status"] == 0 for o in orc)
    zg, zo, dz = [], [], []
    for o in orc:
        p, N, m, s = runs[o["index"]]
        assert (p.name, N, m, s) == (o["name"], o["N"], o["m"], o["run_seed"])
        r = res[o["index"]]
        truth = A.logz(p)
        zg.append((r["log_z"] - truth) / r["log_z_err"])
        zo.append((o["logz"] - truth) / o["logz_err"])
        dz.append(r["log_z"] - o["logz"])
    zg, zo, dz = np.array(zg), np.array(zo), np.array(dz)
    n = len(dz)
    assert stats.ks_2samp(zg, zo).pvalue > 0.01, (zg.mean(), zo.mean(), zg.std(), zo.std())
    assert abs(zg.mean() - zo.mean()) < 3 * math.sqrt((zg.var(ddof=1) + zo.var(ddof=1)) / n), (zg.mean(), zo.mean())
    assert abs(dz.mean()) < 3 * dz.std(ddof=1) / math.sqrt(n), (dz.mean(), dz.std(ddof=1))


def test_run_in_batch_equals_run_alone(nat, batch256):
    """A run's result does not depend on the other runs of its batch, nor on
    their register classes (the class groups run on their own streams)."""
    runs, res, _ = batch256
    picks = [0, 2, 3, 5]
    sel = [runs[i] for i in picks]
    h = nat.ns_create_batch([(p, N, m, 5 * p.d, 1e-3, s) for p, N, m, s in sel])
    nat.ns_run(h)
    for k, i in enumerate(picks):
        a = nat.ns_result(h, k)
        b = res[i]
        assert a["log_z"] == b["log_z"] and a["n_evals"] == b["n_evals"]
        np.testing.assert_array_equal(a["dead_l"], b["dead_l"])
        np.testing.assert_array_equal(a["dead_x"], b["dead_x"])
    nat.ns_destroy(h)


def test_high_d_rosenbrock_matches_oracle_in_distribution(nat, oracle):
    """14-D chained Rosenbrock, N = 200, m = 10, 70 slice steps: GPU and FP64
    oracle runs agree in distribution (means within 4 combined standard
    errors), and both sit below the quadrature value -- the drift is the
    method's at this slice budget, not the GPU path's."""
    p = W.rosenbrock(14)
    N, m, ns, n_seeds = 200, 10, 70, 8
    seeds = list(range(11, 11 + n_seeds))
    h = nat.ns_create_batch([(p, N, m, ns, 1e-3, s) for s in seeds])
    nat.ns_run(h)
    zg = np.array([nat.ns_result(h, r, samples=False)["log_z"] for r in range(n_seeds)])
    nat.ns_destroy(h)
    zo = np.array([oracle.run(p, N, m, ns, 1e-3, 1000 + s)["logz"] for s in seeds])
    se = math.sqrt(zg.var(ddof=1) / n_seeds + zo.var(ddof=1) / n_seeds)
    assert abs(zg.mean() - zo.mean()) < 4 * se + 0.05, (zg.mean(), zo.mean(), se)
    truth = A.logz(p)
    assert zg.mean() < truth and zo.mean() < truth, (zg.mean(), zo.mean(), truth)
