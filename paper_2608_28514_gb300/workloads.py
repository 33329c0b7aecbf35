"""Seeded synthetic problem descriptions (inputs only, no sampler arithmetic).

Each function returns a :class:`Problem`: the likelihood family, its
parameters and the prior box.  Both the CUDA path and the CPU oracle read
these; nothing of the nested-sampling method itself lives here.

Shapes follow the paper's workloads:
  - isotropic Gaussian (section 3.2, eq. for the Gaussian; section 4.1);
  - correlated Gaussian, covariance R diag(lambda) R^T with R a seeded
    Haar-orthogonal matrix and lambda log-uniform;
  - Rosenbrock, a = 1, b = 100 (section 4.2), chained for d > 2;
  - equal-weight mixture of isotropic Gaussians (the multimodal tests of
    sections 2.3 and 4.3);
  - the clustering tests of section 2.3: an array of 49 unit Gaussians
    (Test 1), two separated 10-D diagonal Gaussians of different heights
    (Test 2), a 2-D Gaussian shell (Test 3);
  - a 27-input SiLU MLP with a chi^2 likelihood standing in for the
    cosmological emulator of section 5 (whose weights and data are not
    available).
"""
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

GAUSS_ISO, GAUSS_CORR, ROSENBROCK, MIXTURE, MLP, GMM, SHELL = 0, 1, 2, 3, 4, 5, 6
KIND_NAMES = {GAUSS_ISO: "gauss_iso", GAUSS_CORR: "gauss_corr", ROSENBROCK: "rosenbrock",
              MIXTURE: "mixture", MLP: "mlp", GMM: "gmm", SHELL: "shell"}


@dataclass
class MLPSpec:
    widths: List[int]
    weights: List[np.ndarray]      # per layer [out, in], values exactly representable in bf16
    biases: List[np.ndarray]       # per layer [out]
    data: np.ndarray               # [widths[-1]]
    sigma_out: np.ndarray          # [widths[-1]]
    theta_star: Optional[np.ndarray] = None


@dataclass
class Problem:
    kind: int
    d: int
    lo: np.ndarray
    hi: np.ndarray
    mean: Optional[np.ndarray] = None
    prec_chol: Optional[np.ndarray] = None   # lower L, inverse covariance = L L^T
    cov: Optional[np.ndarray] = None         # kept for closed forms
    sigma: Optional[float] = None
    centres: Optional[np.ndarray] = None     # [n_modes, d]
    mode_var: Optional[np.ndarray] = None    # [n_modes, d] GMM diagonal variances
    mode_logw: Optional[np.ndarray] = None   # [n_modes] GMM log weights
    a: Optional[float] = None
    b: Optional[float] = None
    mlp: Optional[MLPSpec] = None
    name: str = ""
    extra: dict = field(default_factory=dict)


def _box(d, lo, hi):
    return np.full(d, float(lo)), np.full(d, float(hi))


def gauss_iso(d, sigma, lo, hi, mean=0.0, name=""):
    l, h = _box(d, lo, hi)
    return Problem(GAUSS_ISO, d, l, h, mean=np.full(d, float(mean)), sigma=float(sigma),
                   name=name or f"gauss_iso_d{d}")


def gauss_corr(d, seed, box=10.0, mean_range=2.0, lam_lo=0.01, lam_hi=1.0, name=""):
    """Correlated Gaussian: Sigma = R diag(lambda) R^T, R Haar-orthogonal
    (QR of a Gaussian matrix with the sign of diag(R) fixed), log lambda
    uniform, mean uniform in [-mean_range, mean_range]^d."""
    rng = np.random.default_rng([0x5EED, 2, int(seed)])
    A = rng.standard_normal((d, d))
    Q, Rq = np.linalg.qr(A)
    Q = Q * np.sign(np.diag(Rq))[None, :]
    lam = np.exp(rng.uniform(np.log(lam_lo), np.log(lam_hi), size=d))
    cov = (Q * lam[None, :]) @ Q.T
    cov = 0.5 * (cov + cov.T)
    prec = (Q * (1.0 / lam)[None, :]) @ Q.T
    prec = 0.5 * (prec + prec.T)
    Lp = np.linalg.cholesky(prec)
    mean = rng.uniform(-mean_range, mean_range, size=d)
    l, h = _box(d, -box, box)
    return Problem(GAUSS_CORR, d, l, h, mean=mean, prec_chol=Lp, cov=cov,
                   name=name or f"gauss_corr_d{d}_s{seed}", extra=dict(lam=lam))


def rosenbrock(d, box=5.0, a=1.0, b=100.0, name=""):
    l, h = _box(d, -box, box)
    return Problem(ROSENBROCK, d, l, h, a=float(a), b=float(b), name=name or f"rosenbrock_d{d}")


def mixture(d, seed, n_modes=4, sigma=0.1, centre_box=3.0, min_sep=1.0, box=5.0, name=""):
    """Equal-weight isotropic mixture; centres uniform in [-centre_box,
    centre_box]^d, redrawn until every pair is at least min_sep apart."""
    rng = np.random.default_rng([0x5EED, 3, int(seed)])
    centres = []
    while len(centres) < n_modes:
        c = rng.uniform(-centre_box, centre_box, size=d)
        if all(np.linalg.norm(c - q) >= min_sep for q in centres):
            centres.append(c)
    l, h = _box(d, -box, box)
    return Problem(MIXTURE, d, l, h, sigma=float(sigma), centres=np.array(centres),
                   name=name or f"mixture{n_modes}_d{d}_s{seed}")


def _bf16_round(a):
    """Round float64 values to the nearest bf16 (ties to even), returned as
    float32 arrays holding exactly those values."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    rounding = ((u >> 16) & 1) + 0x7FFF
    u = ((u + rounding) >> 16) << 16
    return u.astype(np.uint32).view(np.float32)


def mlp_emulator(seed, widths=(27, 512, 512, 512, 512, 2000), sig_lo=1e-3, sig_hi=1e-1, name=""):
    """Emulator-style likelihood: Xavier-uniform weights rounded to bf16
    (the fp32 masters are those same values), zero biases, data = MLP(theta*)
    + sigma_k * noise with theta* uniform in [0, 1]^27 and sigma_k
    log-uniform in [sig_lo, sig_hi]."""
    rng = np.random.default_rng([0x5EED, 4, int(seed)])
    widths = list(widths)
    Ws, Bs = [], []
    for nin, nout in zip(widths[:-1], widths[1:]):
        lim = np.sqrt(6.0 / (nin + nout))
        Ws.append(_bf16_round(rng.uniform(-lim, lim, size=(nout, nin))))
        Bs.append(np.zeros(nout, dtype=np.float32))
    d = widths[0]
    theta_star = rng.uniform(0.0, 1.0, size=d)
    sigma_out = np.exp(rng.uniform(np.log(sig_lo), np.log(sig_hi), size=widths[-1]))
    h = theta_star.astype(np.float64)
    for i, (W, B) in enumerate(zip(Ws, Bs)):
        h = W.astype(np.float64) @ h + B.astype(np.float64)
        if i + 1 < len(Ws):
            h = h / (1.0 + np.exp(-h))
    data = h + sigma_out * rng.standard_normal(widths[-1])
    spec = MLPSpec(widths, Ws, Bs, data, sigma_out, theta_star)
    l, hbox = _box(d, 0.0, 1.0)
    return Problem(MLP, d, l, hbox, mlp=spec, name=name or f"mlp{d}_s{seed}")


# --------------------------------------------------------------------------
# The workloads of the benchmark configurations, by what they are
# --------------------------------------------------------------------------
def gauss2d_sigma05():
    """2-D isotropic Gaussian, mean 0, sigma 0.5, prior [-5, 5]^2."""
    return gauss_iso(2, 0.5, -5.0, 5.0, name="gauss_iso_d2_sigma0.5_box5")


def gmm(d, centres, variances, log_weights, lo, hi, name=""):
    """Weighted Gaussian mixture with diagonal covariances:
    log L = log sum_k w_k exp(-1/2 sum_i (theta_i - mu_ki)^2 / s_ki^2)."""
    c = np.asarray(centres, dtype=np.float64).reshape(-1, d)
    v = np.asarray(variances, dtype=np.float64).reshape(c.shape)
    w = np.asarray(log_weights, dtype=np.float64).reshape(c.shape[0])
    l, h = _box(d, lo, hi)
    return Problem(GMM, d, l, h, centres=c, mode_var=v, mode_logw=w, name=name or f"gmm_d{d}_k{len(c)}")


def shell(d, radius, width, lo, hi, centre=0.0, name=""):
    """Gaussian shell: log L = -1/2 ((|theta - c| - r0) / w)^2."""
    l, h = _box(d, lo, hi)
    return Problem(SHELL, d, l, h, mean=np.full(d, float(centre)), a=float(radius), sigma=float(width),
                   name=name or f"shell_d{d}")


def array49():
    """Test 1 (section 2.3): 49 unit Gaussians at (4i, 4j), i, j = -3..3, each
    of weight 1, prior [-20, 20]^2."""
    c = np.array([[4.0 * i, 4.0 * j] for i in range(-3, 4) for j in range(-3, 4)])
    return gmm(2, c, np.ones_like(c), np.zeros(len(c)), -20.0, 20.0, name="array49_d2")


def bimodal(d=10):
    """Test 2 (section 2.3): weights 1/10 and 1, means -10 and +10 in every
    coordinate, diagonal variances alternating 0.1 / 1 (mode 1) and 1 / 0.1
    (mode 2), prior [-20, 20]^d.  d < 10 truncates the coordinates."""
    odd = np.arange(1, d + 1) % 2 == 1  # coordinate numbers 1, 3, 5, ... (1-based)
    v1 = np.where(odd, 0.1, 1.0)
    v2 = np.where(odd, 1.0, 0.1)
    c = np.array([np.full(d, -10.0), np.full(d, 10.0)])
    return gmm(d, c, np.array([v1, v2]), np.log([0.1, 1.0]), -20.0, 20.0, name=f"bimodal_d{d}")


def shell2d():
    """Test 3 (section 2.3): 2-D Gaussian shell of radius 5 and width 1 about
    the origin, prior [-10, 10]^2."""
    return shell(2, 5.0, 1.0, -10.0, 10.0, name="shell_d2")


def gauss_unit_box7(d):
    """The comparison Gaussian of section 4.1: log L = -|x|^2 / 2 on [-7, 7]^d."""
    return gauss_iso(d, 1.0, -7.0, 7.0, name=f"gauss_iso_d{d}_sigma1_box7")


def rosenbrock2d_box10():
    """The comparison Rosenbrock of section 4.2: a = 1, b = 100 on [-10, 10]^2."""
    return rosenbrock(2, box=10.0, name="rosenbrock_d2_box10")


def gauss2d_unit_box7():
    """2-D unit Gaussian, log L = -|x|^2 / 2, prior [-7, 7]^2 (the batching
    error study, section 3.2)."""
    return gauss_iso(2, 1.0, -7.0, 7.0, name="gauss_iso_d2_sigma1_box7")


def corr_gauss10(seed):
    """10-D correlated Gaussian on [-10, 10]^10."""
    return gauss_corr(10, seed)


def mixture4_d5(seed):
    """4-mode mixture in 5-D, sigma 0.1, centres in [-3, 3]^5, prior [-5, 5]^5."""
    return mixture(5, seed)


def batched_runs(n_runs, seed=0, d_lo=2, d_hi=30, n_lo=100, n_hi=2000, frac=0.05):
    """Heterogeneous batch of independent runs: d uniform in {d_lo..d_hi},
    N uniform in {n_lo..n_hi}, m = floor(frac N), likelihood family uniform
    over {isotropic, correlated, Rosenbrock, 4-mode mixture}.  Returns a
    list of (problem, N, m, seed) tuples."""
    rng = np.random.default_rng([0x5EED, 5, int(seed)])
    out = []
    for r in range(n_runs):
        d = int(rng.integers(d_lo, d_hi + 1))
        N = int(rng.integers(n_lo, n_hi + 1))
        m = max(1, int(np.floor(frac * N)))
        fam = int(rng.integers(0, 4))
        rs = int(seed) * 100003 + r + 1
        if fam == 0:
            p = gauss_iso(d, 1.0, -7.0, 7.0)
        elif fam == 1:
            p = gauss_corr(d, rs)
        elif fam == 2:
            p = rosenbrock(d)
        else:
            p = mixture(d, rs)
        out.append((p, N, m, rs))
    return out



def separated_blobs(n_blobs, d, per, seed, sd=0.005, min_sep=0.1, lo=0.2, hi=0.8):
    """Point sets for the cluster tree (section 2.1): n_blobs equally
    populated isotropic Gaussian blobs (spread sd) with centres uniform in
    [lo, hi]^d, redrawn until every pair is at least min_sep apart.  Returns
    x [n_blobs * per][d] in unit-cube coordinates (shuffled) and the blob
    label of each point."""
    rng = np.random.default_rng(seed)
    for _ in range(10000):
        c = rng.uniform(lo, hi, size=(n_blobs, d))
        dist = np.linalg.norm(c[:, None, :] - c[None, :, :], axis=-1)
        if np.all(dist[np.triu_indices(n_blobs, 1)] >= min_sep):
            break
    else:
        raise RuntimeError("separated_blobs: no layout found")
    labels = np.repeat(np.arange(n_blobs), per)
    x = c[labels] + sd * rng.standard_normal((n_blobs * per, d))
    perm = rng.permutation(len(x))
    return x[perm], labels[perm]
