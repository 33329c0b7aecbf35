"""Closed-form and quadrature log-evidences of the synthetic workloads.

Z = (1 / V_prior) * integral over the prior box of L(theta), with the
unnormalised likelihoods of the paper (the Gaussian of section 3.2 has no
(2 pi sigma^2)^(-d/2) factor; Table 1's true values confirm this
convention).  These values are reference numbers for reporting, computed
from the mathematics alone; they use no code of the sampler.
"""
import math

import numpy as np
from scipy import integrate, special

from paper_2608_28514_gb300 import workloads as W

_SQ2 = math.sqrt(2.0)


def _log_box_volume(p):
    return float(np.sum(np.log(np.asarray(p.hi) - np.asarray(p.lo))))


def _log_gauss_1d(mu, sigma, lo, hi):
    """log integral_lo^hi exp(-(x-mu)^2 / (2 sigma^2)) dx."""
    return math.log(sigma * math.sqrt(math.pi / 2.0)
                    * (special.erf((hi - mu) / (sigma * _SQ2)) - special.erf((lo - mu) / (sigma * _SQ2))))


def logz_gauss_iso(p):
    s = sum(_log_gauss_1d(p.mean[i], p.sigma, p.lo[i], p.hi[i]) for i in range(p.d))
    return s - _log_box_volume(p)


def logz_gauss_corr(p):
    """Untruncated value 0.5 log det(2 pi Sigma) - log V.  The neglected box
    truncation is below sum_i 2 Phi(-dist_i / sigma_i) (union bound)."""
    sign, logdet = np.linalg.slogdet(2.0 * np.pi * p.cov)
    return 0.5 * logdet - _log_box_volume(p)


def truncation_bound_gauss_corr(p):
    sd = np.sqrt(np.diag(p.cov))
    dist = np.minimum(p.hi - p.mean, p.mean - p.lo)
    return float(np.sum(2.0 * special.ndtr(-dist / sd)))


def logz_mixture(p):
    terms = []
    for c in p.centres:
        terms.append(sum(_log_gauss_1d(c[i], p.sigma, p.lo[i], p.hi[i]) for i in range(p.d)))
    terms = np.array(terms)
    mx = terms.max()
    return mx + math.log(np.mean(np.exp(terms - mx))) - _log_box_volume(p)


def logz_gmm(p):
    """Weighted diagonal Gaussian mixture: each mode integrates to its weight
    times a product of truncated 1-D Gaussian integrals (erf)."""
    terms = []
    for c, v, lw in zip(p.centres, p.mode_var, p.mode_logw):
        terms.append(lw + sum(_log_gauss_1d(c[i], math.sqrt(v[i]), p.lo[i], p.hi[i]) for i in range(p.d)))
    terms = np.array(terms)
    mx = terms.max()
    return mx + math.log(np.sum(np.exp(terms - mx))) - _log_box_volume(p)


def logz_shell2d(p):
    """2-D Gaussian shell centred in a square box [lo, hi]^2: radial
    quadrature of 2 pi r exp(-(r - r0)^2 / (2 w^2)) over the inscribed disc,
    plus the corner annulus r in (h, h sqrt 2) weighted by the angle
    2 pi - 8 arccos(h / r) that stays in the box (h = half-width)."""
    assert p.d == 2
    c = np.asarray(p.mean)
    h = 0.5 * (p.hi[0] - p.lo[0])
    assert np.allclose(c, 0.5 * (p.hi + p.lo)) and np.isclose(p.hi[1] - p.lo[1], 2 * h)
    r0, w = p.a, p.sigma
    f = lambda r: math.exp(-0.5 * ((r - r0) / w) ** 2)
    inner = integrate.quad(lambda r: 2.0 * math.pi * r * f(r), 0.0, h, points=[r0], epsabs=0, epsrel=1e-12,
                           limit=400)[0]
    outer = integrate.quad(lambda r: (2.0 * math.pi - 8.0 * math.acos(h / r)) * r * f(r), h, h * _SQ2,
                           epsabs=0, epsrel=1e-12, limit=400)[0]
    return math.log(inner + outer) - _log_box_volume(p)


def logz_rosenbrock_2d(a, b, lo, hi):
    """log (1/V) int int exp(-(a-x)^2 - b (y-x^2)^2) dy dx over [lo,hi]^2,
    the inner integral in closed form (erf), the outer by adaptive
    quadrature."""
    sb = math.sqrt(b)

    def inner(x):
        return math.exp(-(a - x) ** 2) * (math.sqrt(math.pi) / (2 * sb)) * (
            special.erf(sb * (hi - x * x)) - special.erf(sb * (lo - x * x)))

    pts = [-1.0, 0.0, 1.0]
    val, err = integrate.quad(inner, lo, hi, points=pts, limit=500, epsabs=0, epsrel=1e-13)
    return math.log(val) - 2 * math.log(hi - lo)


def logz_rosenbrock_grid2d(a, b, lo, hi, n=4096):
    """Brute-force midpoint rule on an n x n grid (the paper-style check)."""
    h = (hi - lo) / n
    xs = lo + (np.arange(n) + 0.5) * h
    tot = 0.0
    for i0 in range(0, n, 256):
        x = xs[i0:i0 + 256][:, None]
        y = xs[None, :]
        tot += np.exp(-(a - x) ** 2 - b * (y - x * x) ** 2).sum()
    return math.log(tot * h * h) - 2 * math.log(hi - lo)


_CHAIN_CACHE = {}


def logz_rosenbrock_chain(d, a, b, lo, hi, h=0.002):
    """Chained Rosenbrock, L = prod_i exp(-(a-x_i)^2 - b (x_{i+1}-x_i^2)^2),
    by the transfer operator f_{i+1}(y) = int f_i(x) K(x, y) dx on a
    midpoint grid of spacing h.  One pass of the chain gives log Z for every
    dimension along the way; the pass is kept and extended on demand."""
    key = (float(a), float(b), float(lo), float(hi), float(h))
    st = _CHAIN_CACHE.get(key)
    if st is None:
        n = int(round((hi - lo) / h))
        hh = (hi - lo) / n
        xs = lo + (np.arange(n) + 0.5) * hh
        st = {"xs": xs, "h": hh, "f": np.ones(n), "logscale": 0.0, "ex": np.exp(-(a - xs) ** 2), "logz": {}}
        _CHAIN_CACHE[key] = st
    xs, hh, ex = st["xs"], st["h"], st["ex"]
    n = len(xs)
    while d not in st["logz"]:
        g = np.zeros(n)
        blk = 512
        f = st["f"]
        for j0 in range(0, n, blk):
            y = xs[j0:j0 + blk][None, :]
            K = np.exp(-b * (y - (xs * xs)[:, None]) ** 2)
            g[j0:j0 + blk] = (f * ex) @ K * hh
        s = g.max()
        st["logscale"] += math.log(s)
        st["f"] = g / s
        dim = len(st["logz"]) + 2  # the chain after k steps covers k + 1 variables
        st["logz"][dim] = math.log(st["f"].sum() * hh) + st["logscale"] - dim * math.log(hi - lo)
    return st["logz"][d]


def logz(p):
    """Closed-form (or quadrature) log Z of a Problem, where one exists."""
    if p.kind == W.GAUSS_ISO:
        return logz_gauss_iso(p)
    if p.kind == W.GAUSS_CORR:
        return logz_gauss_corr(p)
    if p.kind == W.MIXTURE:
        return logz_mixture(p)
    if p.kind == W.GMM:
        return logz_gmm(p)
    if p.kind == W.SHELL and p.d == 2:
        return logz_shell2d(p)
    if p.kind == W.ROSENBROCK:
        if p.d == 2:
            return logz_rosenbrock_2d(p.a, p.b, float(p.lo[0]), float(p.hi[0]))
        return logz_rosenbrock_chain(p.d, p.a, p.b, float(p.lo[0]), float(p.hi[0]))
    return None
