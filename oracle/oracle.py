"""ctypes binding of the FP64 CPU oracle (``ns_oracle.c``).

TEST INFRASTRUCTURE ONLY.  Imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``; the product path never imports it.
The oracle shares no code with the CUDA path; the only thing both sides take
from a common module is the seeded problem description
(``paper_2608_28514_gb300.workloads.Problem``), which holds no arithmetic of
the method.
"""
import ctypes as C
import os

import numpy as np

from . import build_oracle

_lib = None

PURPOSE_SEED = 0x10000
PURPOSE_KMEANS = 0x20000
T_INIT = 0xFFFFFFFF

_dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_ip = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_up = np.ctypeslib.ndpointer(dtype=np.uint32, flags="C_CONTIGUOUS")


class OrcLik(C.Structure):
    _fields_ = [
        ("kind", C.c_int), ("d", C.c_int),
        ("lo", C.POINTER(C.c_double)), ("hi", C.POINTER(C.c_double)),
        ("mean", C.POINTER(C.c_double)), ("prec_chol", C.POINTER(C.c_double)),
        ("sigma", C.c_double), ("n_modes", C.c_int), ("centres", C.POINTER(C.c_double)),
        ("a", C.c_double), ("b", C.c_double),
        ("n_layers", C.c_int), ("widths", C.POINTER(C.c_int)),
        ("weights", C.POINTER(C.c_double)), ("biases", C.POINTER(C.c_double)),
        ("data", C.POINTER(C.c_double)), ("sigma_out", C.POINTER(C.c_double)),
        ("mode_var", C.POINTER(C.c_double)), ("mode_logw", C.POINTER(C.c_double)),
    ]


class OrcOpts(C.Structure):
    _fields_ = [
        ("depth", C.c_int), ("recluster_every", C.c_int), ("n_min", C.c_int),
        ("vol_frac", C.c_double), ("kmeans_iters", C.c_int), ("history_iters", C.c_int),
        ("t_max", C.c_int), ("e_max", C.c_int), ("s_max", C.c_int), ("width", C.c_double),
        ("max_iter", C.c_longlong), ("dead_cap", C.c_longlong), ("correction", C.c_int),
        ("bracket", C.c_int),
    ]


class OrcWalkerInfo(C.Structure):
    _fields_ = [("min_l_margin", C.c_double), ("min_box_margin", C.c_double),
                ("n_evals", C.c_longlong), ("flags", C.c_int)]


class OrcEvid(C.Structure):
    _fields_ = [("logz", C.c_double), ("info", C.c_double), ("k", C.c_longlong),
                ("n_live", C.c_int)]


class OrcResult(C.Structure):
    _fields_ = [("logz", C.c_double), ("logz_err", C.c_double), ("info", C.c_double),
                ("n_dead", C.c_longlong), ("n_evals", C.c_longlong), ("n_iter", C.c_longlong),
                ("n_relaxed", C.c_longlong), ("status", C.c_int)]


def lib():
    """Load (building first if needed) the oracle shared object."""
    global _lib
    if _lib is None:
        path = build_oracle.build()
        L = C.CDLL(path)
        L.orc_philox4x32_10.argtypes = [_up, _up, _up]
        L.orc_stream_draws.argtypes = [_up, C.c_uint32, C.c_uint32, C.c_uint32, C.c_uint32, C.c_int, _up]
        L.orc_loglike.argtypes = [C.POINTER(OrcLik), _dp]
        L.orc_loglike.restype = C.c_double
        L.orc_loglike_batch.argtypes = [C.POINTER(OrcLik), C.c_int, _dp, _dp]
        L.orc_loglike_batch.restype = None
        L.orc_default_opts.argtypes = [C.POINTER(OrcOpts), C.c_int, C.c_int]
        L.orc_select.argtypes = [C.c_int, C.c_int, _dp, _up, C.c_uint32, _ip, _ip]
        L.orc_slice_walker.argtypes = [C.POINTER(OrcLik), C.POINTER(OrcOpts), C.c_int, _up, C.c_uint32,
                                       C.c_int, _dp, C.c_double, _dp, C.c_double, C.c_double,
                                       _dp, C.POINTER(C.c_double), _dp, _dp, C.POINTER(C.c_int),
                                       C.POINTER(OrcWalkerInfo)]
        L.orc_batch_correct.argtypes = [C.c_int, C.c_int, C.c_int, _dp, _dp, _dp, _ip, C.c_int,
                                        _ip, _ip, _dp, _dp, _ip, _ip, _dp, _dp, C.POINTER(C.c_int)]
        L.orc_evid_init.argtypes = [C.POINTER(OrcEvid), C.c_int]
        L.orc_evid_add_dead.argtypes = [C.POINTER(OrcEvid), C.c_double]
        L.orc_evid_add_dead.restype = C.c_double
        L.orc_evid_add_live.argtypes = [C.POINTER(OrcEvid), C.c_double]
        L.orc_evid_add_live.restype = C.c_double
        L.orc_evid_should_stop.argtypes = [C.POINTER(OrcEvid), C.c_double, C.c_double]
        L.orc_evid_should_stop.restype = C.c_int
        L.orc_cluster.argtypes = [C.c_int, C.c_int, _dp, C.POINTER(OrcOpts), _up, C.c_uint32,
                                  _dp, _dp, _dp, _ip, _ip, _ip, _ip, _dp]
        L.orc_cluster.restype = C.c_int
        L.orc_nearest_leaf.argtypes = [C.c_int, C.c_int, _dp, _ip, _dp]
        L.orc_reg_cholesky.argtypes = [C.c_int, _dp, _dp]
        L.orc_reg_cholesky.restype = C.c_int
        L.orc_run.argtypes = [C.POINTER(OrcLik), C.c_int, C.c_int, C.c_int, C.c_double, C.c_uint64,
                              C.POINTER(OrcOpts), _dp, _dp, _dp, C.POINTER(OrcResult)]
        L.orc_run_sequential.argtypes = [C.POINTER(OrcLik), C.c_int, C.c_int, C.c_double, C.c_uint64,
                                         C.POINTER(OrcOpts), _dp, _dp, _dp, C.POINTER(OrcResult)]
        _lib = L
    return _lib


def _f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _key(seed):
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    return np.array([seed & 0xFFFFFFFF, seed >> 32], dtype=np.uint32)


class Lik:
    """Oracle-side likelihood: keeps the numpy buffers alive with the struct."""

    def __init__(self, problem):
        p = problem
        self._keep = []
        s = OrcLik()
        s.kind = int(p.kind)
        s.d = int(p.d)

        def ptr(a, ctype=C.c_double, dtype=np.float64):
            if a is None:
                return None
            arr = np.ascontiguousarray(np.asarray(a, dtype=dtype))
            self._keep.append(arr)
            return arr.ctypes.data_as(C.POINTER(ctype))

        s.lo = ptr(p.lo)
        s.hi = ptr(p.hi)
        s.mean = ptr(p.mean)
        s.prec_chol = ptr(p.prec_chol)
        s.sigma = float(p.sigma if p.sigma is not None else 0.0)
        s.n_modes = int(0 if p.centres is None else np.asarray(p.centres).shape[0])
        s.centres = ptr(p.centres)
        s.a = float(p.a if p.a is not None else 0.0)
        s.b = float(p.b if p.b is not None else 0.0)
        if p.mlp is not None:
            s.n_layers = len(p.mlp.widths) - 1
            s.widths = ptr(p.mlp.widths, C.c_int, np.int32)
            s.weights = ptr(np.concatenate([np.ravel(w) for w in p.mlp.weights]))
            s.biases = ptr(np.concatenate([np.ravel(b) for b in p.mlp.biases]))
            s.data = ptr(p.mlp.data)
            s.sigma_out = ptr(p.mlp.sigma_out)
        s.mode_var = ptr(p.mode_var)
        s.mode_logw = ptr(p.mode_logw)
        self.struct = s
        self.d = int(p.d)

    def ref(self):
        return C.byref(self.struct)


def opts(d, m, **kw):
    o = OrcOpts()
    lib().orc_default_opts(C.byref(o), int(d), int(m))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


def philox(ctr, key):
    ctr = np.ascontiguousarray(np.asarray(ctr, dtype=np.uint32).reshape(-1, 4))
    key = np.ascontiguousarray(np.asarray(key, dtype=np.uint32).reshape(2))
    out = np.empty_like(ctr)
    for i in range(ctr.shape[0]):
        o = np.empty(4, dtype=np.uint32)
        lib().orc_philox4x32_10(np.ascontiguousarray(ctr[i]), key, o)
        out[i] = o
    return out


def stream_draws(seed, t, walker, purpose, first, n):
    out = np.empty(n, dtype=np.uint32)
    lib().orc_stream_draws(_key(seed), t & 0xFFFFFFFF, walker & 0xFFFFFFFF, purpose, first, n, out)
    return out


def loglike(lik, X):
    X = np.ascontiguousarray(_f64(X).reshape(-1, lik.d))
    out = np.empty(len(X))
    lib().orc_loglike_batch(lik.ref(), len(X), X, out)
    return out


def select(logl, m, seed, t):
    logl = _f64(logl)
    worst = np.empty(m, dtype=np.int32)
    seeds = np.empty(m, dtype=np.int32)
    lib().orc_select(len(logl), m, logl, _key(seed), t, worst, seeds)
    return worst, seeds


def slice_walker(lik, o, n_steps, seed, t, walker, x_seed, l_seed, chol, thr_out, thr_in):
    d = lik.d
    x_out = np.empty(d)
    l_out = C.c_double()
    hist_l = np.full(o.t_max, np.nan)
    hist_x = np.full((o.t_max, d), np.nan)
    hlen = C.c_int()
    info = OrcWalkerInfo()
    lib().orc_slice_walker(lik.ref(), C.byref(o), n_steps, _key(seed), t, walker, _f64(x_seed),
                           float(l_seed), _f64(chol).reshape(-1), float(thr_out), float(thr_in),
                           x_out, C.byref(l_out), hist_l, hist_x.reshape(-1), C.byref(hlen),
                           C.byref(info))
    return dict(x=x_out, l=l_out.value, hist_l=hist_l[:hlen.value], hist_x=hist_x[:hlen.value],
                hist_len=hlen.value, n_evals=info.n_evals, flags=info.flags,
                min_l_margin=info.min_l_margin, min_box_margin=info.min_box_margin)


def batch_correct(W, newl, hist_l, hist_len, K=1, correction=2):
    m = len(W)
    hist_l = _f64(hist_l)
    t_max = hist_l.shape[1]
    out = {k: np.empty(m, dtype=np.int32) for k in ("acc_src", "acc_hpos", "rej_src", "rej_hpos")}
    out.update({k: np.empty(m) for k in ("acc_l", "acc_P", "rej_l", "rej_P")})
    nrel = C.c_int()
    lib().orc_batch_correct(m, K, correction, _f64(W), _f64(newl), hist_l.reshape(-1),
                            np.ascontiguousarray(np.asarray(hist_len, dtype=np.int32)), t_max,
                            out["acc_src"], out["acc_hpos"], out["acc_l"], out["acc_P"],
                            out["rej_src"], out["rej_hpos"], out["rej_l"], out["rej_P"], C.byref(nrel))
    out["n_relaxed"] = nrel.value
    return out


class Evidence:
    def __init__(self, n_live):
        self.s = OrcEvid()
        lib().orc_evid_init(C.byref(self.s), n_live)

    def add_dead(self, l):
        return lib().orc_evid_add_dead(C.byref(self.s), float(l))

    def add_live(self, l):
        return lib().orc_evid_add_live(C.byref(self.s), float(l))

    def should_stop(self, lmax, stop_frac):
        return bool(lib().orc_evid_should_stop(C.byref(self.s), float(lmax), float(stop_frac)))

    @property
    def logz(self):
        return self.s.logz

    @property
    def info(self):
        return self.s.info

    @property
    def k(self):
        return self.s.k


def reg_cholesky(cov):
    cov = _f64(cov)
    d = cov.shape[0]
    L = np.empty((d, d))
    flag = lib().orc_reg_cholesky(d, cov.reshape(-1), L.reshape(-1))
    return L, flag


def cluster(x, o, seed, t):
    """x: [N, d] unit-cube points.  Returns the node tables of the tree."""
    x = _f64(x)
    N, d = x.shape
    nn = (1 << (o.depth + 1)) - 1
    centres = np.zeros((nn, d))
    chol = np.zeros((nn, d, d))
    logvol = np.zeros(nn)
    count = np.zeros(nn, dtype=np.int32)
    split = np.zeros(nn, dtype=np.int32)
    mask = np.zeros(nn, dtype=np.int32)
    assign = np.zeros(N, dtype=np.int32)
    radius = np.zeros(nn)
    nl = lib().orc_cluster(N, d, x.reshape(-1), C.byref(o), _key(seed), t, centres.reshape(-1),
                           chol.reshape(-1), logvol, count, split, mask, assign, radius)
    return dict(centres=centres, chol=chol, logvol=logvol, count=count, split=split, mask=mask,
                assign=assign, n_leaves=nl, radius=radius)


def nearest_leaf(centres, mask, x):
    centres = _f64(centres)
    nn, d = centres.shape
    return lib().orc_nearest_leaf(d, nn, centres.reshape(-1),
                                  np.ascontiguousarray(np.asarray(mask, dtype=np.int32)), _f64(x))


def run(problem, N, m, n_steps, stop_frac, seed, o=None, sequential=False, dead_cap=None):
    """One whole nested-sampling run of the oracle."""
    lik = Lik(problem)
    d = lik.d
    if o is None:
        o = opts(d, m)
    cap = dead_cap if dead_cap is not None else N * 400 + 4 * m
    o.dead_cap = cap
    dx = np.empty((cap, d))
    dl = np.empty(cap)
    dw = np.empty(cap)
    res = OrcResult()
    if sequential:
        lib().orc_run_sequential(lik.ref(), N, n_steps, stop_frac, seed, C.byref(o), dx.reshape(-1),
                                 dl, dw, C.byref(res))
    else:
        lib().orc_run(lik.ref(), N, m, n_steps, stop_frac, seed, C.byref(o), dx.reshape(-1), dl, dw,
                      C.byref(res))
    n = res.n_dead
    return dict(logz=res.logz, logz_err=res.logz_err, info=res.info, n_dead=n,
                n_evals=res.n_evals, n_iter=res.n_iter, n_relaxed=res.n_relaxed,
                status=res.status, dead_x=dx[:n], dead_l=dl[:n], dead_logw=dw[:n])


def _run_summary(args):
    problem, N, m, n_steps, stop_frac, seed = args
    r = run(problem, N, m, n_steps, stop_frac, seed)
    return {k: r[k] for k in ("logz", "logz_err", "info", "n_evals", "n_iter", "status")}


def run_many(jobs, workers, fn=None):
    """Whole oracle runs (problem, N, m, n_steps, stop_frac, seed) in a pool
    of `workers` processes started with spawn (safe in a process that has
    already initialised CUDA).  Returns each run's summary, in order.  A
    worker that dies (a crash, a kill) is detected: the call raises
    RuntimeError naming the lost jobs instead of waiting for them."""
    import concurrent.futures as cf
    import multiprocessing as mp
    from concurrent.futures.process import BrokenProcessPool
    jobs = list(jobs)
    fn = fn or _run_summary
    with cf.ProcessPoolExecutor(max_workers=max(1, int(workers)), mp_context=mp.get_context("spawn")) as ex:
        futs = [ex.submit(fn, j) for j in jobs]
        out, lost = [], []
        for k, f in enumerate(futs):
            try:
                out.append(f.result())
            except BrokenProcessPool:
                lost.append(k)
                out.append(None)
    if lost:
        raise RuntimeError(f"oracle worker died: {len(lost)} of {len(jobs)} runs lost (jobs {lost[:8]})")
    return out


def _exit_worker(job):
    """A job that ends its worker process abruptly (for the failure-detection test)."""
    import os
    if job == "die":
        os._exit(3)
    return job
