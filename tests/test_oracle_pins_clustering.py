"""Pins of the clustering-test likelihoods of section 2.3 (Tests 1-3) in the
CPU oracle: Table 1's printed true log-evidences (tests/golden), the
likelihoods against a library route (scipy's multivariate normal) and brute
force quadrature of the oracle's own likelihood on a grid, and short oracle
runs against the closed forms."""
import json
import math
import os

import numpy as np
import pytest
from scipy import special, stats

from tests import analytic as A
from paper_2608_28514_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
TABLE1 = json.load(open(os.path.join(GOLDEN, "table1_true_logz.json")))
MAKERS = {"array49_d2": W.array49, "bimodal_d10": lambda: W.bimodal(10), "shell_d2": W.shell2d}


@pytest.mark.parametrize("name", sorted(MAKERS))
def test_closed_forms_reproduce_table1(name):
    want = TABLE1[name]["log_z_true"]
    got = A.logz(MAKERS[name]())
    assert abs(got - want) <= 0.6 * 10.0 ** (-TABLE1[name]["printed_digits"]), (got, want)


def test_gmm_matches_scipy_multivariate_normal(oracle):
    """log sum_k w_k exp(-1/2 (x-mu_k)^T S_k^-1 (x-mu_k)) through scipy's
    normalised densities: logpdf + 1/2 log det(2 pi S_k) + log w_k."""
    rng = np.random.default_rng(31)
    for p in (W.array49(), W.bimodal(10), W.bimodal(3)):
        lik = oracle.Lik(p)
        x = rng.uniform(0.0, 1.0, size=(300, p.d))
        x[:5] = (p.centres[:5 if len(p.centres) >= 5 else len(p.centres)].mean(0) - p.lo) / (p.hi - p.lo)
        th = p.lo + (p.hi - p.lo) * x
        terms = []
        for c, v, lw in zip(p.centres, p.mode_var, p.mode_logw):
            S = np.diag(v)
            terms.append(lw + stats.multivariate_normal(c, S).logpdf(th)
                         + 0.5 * np.linalg.slogdet(2.0 * np.pi * S)[1])
        want = special.logsumexp(np.array(terms), axis=0)
        np.testing.assert_allclose(oracle.loglike(lik, x), want, rtol=1e-12, atol=1e-9)


@pytest.mark.parametrize("name", ["array49_d2", "shell_d2"])
def test_grid_quadrature_of_the_oracle_likelihood(oracle, name):
    """Midpoint rule of exp(oracle log L) on a 1600 x 1600 grid of the box
    against the closed form (Test 1: erf products, Test 3: radial quadrature)."""
    p = MAKERS[name]()
    lik = oracle.Lik(p)
    n = 1600
    g = (np.arange(n) + 0.5) / n
    X, Y = np.meshgrid(g, g, indexing="ij")
    ll = oracle.loglike(lik, np.stack([X.ravel(), Y.ravel()], 1))
    logz = math.log(np.exp(ll).mean())
    assert abs(logz - A.logz(p)) < 2e-5, (logz, A.logz(p))


def test_shell_values():
    """Special cases that fix the shell's formula: log L = 0 on the ridge
    |theta - c| = r0 and -1/2 k^2 at k widths from it."""
    from oracle import oracle as O
    p = W.shell2d()
    lik = O.Lik(p)
    span = p.hi - p.lo
    for k in (0.0, 1.0, 2.5):
        for ang in (0.3, 2.0, 4.4):
            r = p.a + k * p.sigma
            th = np.array([r * math.cos(ang), r * math.sin(ang)])
            x = (th - p.lo) / span
            assert abs(O.loglike(lik, x[None, :])[0] + 0.5 * k * k) < 1e-12


@pytest.mark.parametrize("name,depth,bracket", [("array49_d2", 3, 0), ("shell_d2", 3, 0), ("array49_d2", 3, 1),
                                                ("shell_d2", 3, 1)])
def test_oracle_runs_recover_table1(oracle, name, depth, bracket):
    """Sequential (m = 1) oracle runs of the 2-D tests with N = 300 live
    points and the cluster tree, under either bracket reading: the mean over
    6 seeds within 4 standard errors (of the runs' own error estimates) of
    the closed form."""
    p = MAKERS[name]()
    o = oracle.opts(p.d, 1, depth=depth, recluster_every=100, bracket=bracket)
    z, err = [], []
    for s in range(1, 7):
        r = oracle.run(p, 300, 1, 10, 1e-3, 500 + s, o=o)
        z.append(r["logz"])
        err.append(r["logz_err"])
    se = math.sqrt(np.mean(np.square(err)) / len(z))
    assert abs(np.mean(z) - A.logz(p)) < 4 * se + 0.01, (np.mean(z), A.logz(p), se)
