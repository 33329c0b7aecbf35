"""ctypes binding of ``libns_gb300.so`` (argument marshalling only).

Every function here forwards to the C ABI declared in
``include/ns_gb300.h`` under the same name.  Device buffers are torch CUDA
tensors (torch is the device allocator and the source of streams); all
computation happens in the library's sm_103a kernels.  There is no CPU
fallback: if the library cannot be loaded, every call raises.
"""
import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libns_gb300.so")

NS_OK, NS_ERR_ARG, NS_ERR_CUDA, NS_ERR_OOM, NS_ERR_BUDGET, NS_ERR_STATE, NS_ERR_UNSUPPORTED = 0, -1, -2, -3, -4, -5, -6
STATUS_NAMES = {0: "NS_OK", -1: "NS_ERR_ARG", -2: "NS_ERR_CUDA", -3: "NS_ERR_OOM", -4: "NS_ERR_BUDGET",
                -5: "NS_ERR_STATE", -6: "NS_ERR_UNSUPPORTED"}
PURPOSE_SEED = 0x10000
PURPOSE_KMEANS = 0x20000
T_INIT = 0xFFFFFFFF


class NSError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class NsLikelihood(C.Structure):
    _fields_ = [
        ("kind", C.c_int), ("mean", C.POINTER(C.c_double)), ("prec_chol", C.POINTER(C.c_double)),
        ("sigma", C.c_double), ("n_modes", C.c_int), ("centres", C.POINTER(C.c_double)),
        ("a", C.c_double), ("b", C.c_double), ("n_layers", C.c_int), ("widths", C.POINTER(C.c_int)),
        ("weights", C.POINTER(C.c_float)), ("biases", C.POINTER(C.c_float)),
        ("data", C.POINTER(C.c_float)), ("sigma_out", C.POINTER(C.c_float)),
        ("mode_var", C.POINTER(C.c_double)), ("mode_logw", C.POINTER(C.c_double)),
    ]


class NsOptions(C.Structure):
    _fields_ = [
        ("depth", C.c_int), ("recluster_every", C.c_int), ("n_min", C.c_int), ("vol_frac", C.c_double),
        ("kmeans_iters", C.c_int), ("correction", C.c_int), ("history_iters", C.c_int), ("t_max", C.c_int),
        ("e_max", C.c_int), ("s_max", C.c_int), ("width", C.c_double), ("max_iter", C.c_longlong),
        ("dead_cap", C.c_longlong), ("chunk_iters", C.c_int), ("precision", C.c_int),
        ("reeval_margin", C.c_double), ("reeval_rel", C.c_double), ("reeval_defer", C.c_int),
        ("walker_mapping", C.c_int), ("mlp_batch_cap", C.c_int), ("mlp_cluster", C.c_int),
        ("two_plane", C.c_int), ("reeval2_margin", C.c_double), ("reeval2_rel", C.c_double),
        ("bracket", C.c_int),
    ]


class NsProblem(C.Structure):
    _fields_ = [
        ("lik", C.POINTER(NsLikelihood)), ("lo", C.POINTER(C.c_double)), ("hi", C.POINTER(C.c_double)),
        ("d", C.c_int), ("n_live", C.c_int), ("m", C.c_int), ("n_slice_steps", C.c_int),
        ("stop_frac", C.c_double), ("seed", C.c_uint64),
    ]


class NsStats(C.Structure):
    _fields_ = [("run_ms", C.c_double), ("kernel_ms", C.c_double), ("launches", C.c_longlong),
                ("h2d_bytes", C.c_longlong), ("d2h_bytes", C.c_longlong)]


class NsResult(C.Structure):
    _fields_ = [
        ("log_z", C.c_double), ("log_z_err", C.c_double), ("info_h", C.c_double),
        ("n_dead", C.c_longlong), ("n_evals", C.c_longlong), ("n_iter", C.c_longlong),
        ("n_relaxed", C.c_longlong), ("n_reeval", C.c_longlong), ("n_capped", C.c_longlong),
        ("status", C.c_int), ("d", C.c_int),
        ("dead_x", C.POINTER(C.c_float)), ("dead_logl", C.POINTER(C.c_float)),
        ("dead_logw", C.POINTER(C.c_double)),
        ("n_rounds", C.c_longlong), ("n_pass_bf16", C.c_longlong), ("n_cand_bf16", C.c_longlong),
        ("n_pass_fp32", C.c_longlong), ("n_cand_fp32", C.c_longlong),
        ("n_pass_x2", C.c_longlong), ("n_cand_x2", C.c_longlong),
    ]


_lib = None
_vp = C.c_void_p


def lib():
    """Load the shared library (it must have been built: __graft_entry__.build())."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it first (python -c 'import __graft_entry__ as g; g.build()')")
    L = C.CDLL(LIB_PATH)
    L.ns_default_options.argtypes = [C.POINTER(NsOptions)]
    L.ns_create.argtypes = [C.POINTER(NsLikelihood), C.POINTER(C.c_double), C.POINTER(C.c_double), C.c_int,
                            C.c_int, C.c_int, C.c_int, C.c_double, C.c_uint64, C.POINTER(NsOptions),
                            C.POINTER(_vp)]
    L.ns_create_batch.argtypes = [C.c_int, C.POINTER(NsProblem), C.POINTER(NsOptions), C.POINTER(_vp)]
    L.ns_run.argtypes = [_vp, _vp]
    L.ns_reset.argtypes = [_vp, _vp]
    L.ns_step.argtypes = [_vp, C.c_int, _vp]
    L.ns_autotune.argtypes = [_vp, C.c_int, C.c_int, _vp, _vp, _vp]
    L.ns_set_walker_mapping.argtypes = [_vp, C.c_int, C.c_int]
    L.ns_checkpoint_bytes.argtypes = [_vp]
    L.ns_checkpoint_bytes.restype = C.c_size_t
    L.ns_checkpoint.argtypes = [_vp, _vp, C.c_size_t, _vp]
    L.ns_restore.argtypes = [_vp, _vp, C.c_size_t, _vp]
    L.ns_result.argtypes = [_vp, C.c_int, C.POINTER(NsResult)]
    L.ns_summary.argtypes = [_vp, C.c_int, C.POINTER(NsResult)]
    L.ns_phase_cycles.argtypes = [_vp, C.c_int, C.POINTER(C.c_longlong)]
    L.ns_run_buffer_bytes.argtypes = [_vp, C.c_int, C.c_int]
    L.ns_run_buffer_bytes.restype = C.c_size_t
    L.ns_copy_run_buffer.argtypes = [_vp, C.c_int, C.c_int, _vp, C.c_size_t, _vp]
    L.ns_run_noalloc.argtypes = [C.POINTER(NsProblem), C.POINTER(NsOptions), _vp, _vp, _vp, C.c_longlong,
                                 C.POINTER(NsResult), _vp]
    L.ns_resident_runs_per_sm.argtypes = [C.c_int, C.c_int, C.c_int]
    L.ns_resident_runs_per_sm.restype = C.c_int
    L.ns_n_runs.argtypes = [_vp]
    L.ns_n_runs.restype = C.c_int
    L.ns_last_run_ms.argtypes = [_vp, C.POINTER(C.c_double)]
    L.ns_get_stats.argtypes = [_vp, C.POINTER(NsStats)]
    L.ns_last_error.argtypes = [_vp]
    L.ns_last_error.restype = C.c_char_p
    L.ns_destroy.argtypes = [_vp]
    L.ns_destroy.restype = None
    L.ns_philox4x32_10.argtypes = [_vp, C.c_uint32, C.c_uint32, C.c_int, _vp, _vp]
    L.ns_loglike.argtypes = [C.POINTER(NsLikelihood), C.POINTER(C.c_double), C.POINTER(C.c_double), C.c_int,
                             C.c_int, _vp, _vp, _vp]
    L.ns_select_worst.argtypes = [C.c_int, C.c_int, C.c_int, _vp, C.POINTER(C.c_uint64), C.c_uint32, _vp, _vp,
                                  _vp, _vp]
    L.ns_slice_replace.argtypes = [C.POINTER(NsLikelihood), C.POINTER(C.c_double), C.POINTER(C.c_double),
                                   C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.POINTER(NsOptions), C.c_uint64,
                                   C.c_uint32] + [_vp] * 15
    L.ns_slice_scratch_bytes.argtypes = [C.c_int, C.c_int, C.c_int]
    L.ns_slice_scratch_bytes.restype = C.c_size_t
    L.ns_batch_correct.argtypes = [C.c_int, C.c_int, C.c_int, _vp, _vp, _vp, _vp, C.c_int] + [_vp] * 10
    L.ns_evidence_update.argtypes = [C.c_int, C.c_int, _vp, _vp, _vp, C.c_int, _vp]
    L.ns_cluster.argtypes = [C.c_int, C.c_int, C.c_int, _vp, C.POINTER(NsOptions), C.c_uint64, C.c_uint32,
                             _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]
    L.ns_mlp_image_bytes.argtypes = [C.POINTER(NsLikelihood), C.c_int]
    L.ns_mlp_image_bytes.restype = C.c_size_t
    L.ns_mlp_pack.argtypes = [C.POINTER(NsLikelihood), C.c_int, _vp, _vp]
    L.ns_mlp_pack.restype = C.c_int
    L.ns_mlp_loglike.argtypes = [C.POINTER(NsLikelihood), C.POINTER(C.c_double), C.POINTER(C.c_double), C.c_int,
                                 _vp, C.c_int, _vp, _vp, C.c_int, _vp]
    L.ns_mlp_loglike.restype = C.c_int
    L.ns_mlp_loglike_cluster.argtypes = [C.POINTER(NsLikelihood), C.POINTER(C.c_double), C.POINTER(C.c_double),
                                         C.c_int, _vp, C.c_int, _vp, _vp, C.c_int, C.c_int, _vp]
    L.ns_mlp_loglike_cluster.restype = C.c_int
    L.ns_cluster_scratch_bytes.argtypes = [C.c_int, C.c_int, C.c_int]
    L.ns_cluster_scratch_bytes.restype = C.c_size_t
    for name in ("ns_default_options", "ns_create", "ns_create_batch", "ns_run", "ns_reset", "ns_result", "ns_summary",
                 "ns_phase_cycles", "ns_run_noalloc", "ns_step", "ns_autotune", "ns_set_walker_mapping", "ns_checkpoint", "ns_restore",
                 "ns_last_run_ms", "ns_get_stats", "ns_philox4x32_10", "ns_loglike", "ns_select_worst", "ns_slice_replace",
                 "ns_batch_correct", "ns_evidence_update", "ns_cluster", "ns_copy_run_buffer"):
        getattr(L, name).restype = C.c_int
    _lib = L
    return L


def _check(status, handle=None):
    if status != NS_OK:
        msg = lib().ns_last_error(handle)
        raise NSError(status, msg.decode() if msg else "")


# --------------------------------------------------------------------------
# marshalling helpers
# --------------------------------------------------------------------------
class _Keep:
    """Holds numpy buffers alive while a C struct points into them."""

    def __init__(self):
        self.bufs = []

    def dptr(self, a):
        if a is None:
            return None
        arr = np.ascontiguousarray(np.asarray(a, dtype=np.float64)).ravel()
        self.bufs.append(arr)
        return arr.ctypes.data_as(C.POINTER(C.c_double))

    def fptr(self, a):
        if a is None:
            return None
        arr = np.ascontiguousarray(np.asarray(a, dtype=np.float32)).ravel()
        self.bufs.append(arr)
        return arr.ctypes.data_as(C.POINTER(C.c_float))

    def iptr(self, a):
        if a is None:
            return None
        arr = np.ascontiguousarray(np.asarray(a, dtype=np.int32)).ravel()
        self.bufs.append(arr)
        return arr.ctypes.data_as(C.POINTER(C.c_int))


def likelihood_struct(problem, keep):
    p = problem
    s = NsLikelihood()
    s.kind = int(p.kind)
    s.mean = keep.dptr(p.mean)
    s.prec_chol = keep.dptr(p.prec_chol)
    s.sigma = float(p.sigma) if p.sigma is not None else 0.0
    s.n_modes = 0 if p.centres is None else int(np.asarray(p.centres).shape[0])
    s.centres = keep.dptr(p.centres)
    s.a = float(p.a) if p.a is not None else 0.0
    s.b = float(p.b) if p.b is not None else 0.0
    if p.mlp is not None:
        s.n_layers = len(p.mlp.widths) - 1
        s.widths = keep.iptr(p.mlp.widths)
        s.weights = keep.fptr(np.concatenate([np.ravel(w) for w in p.mlp.weights]))
        s.biases = keep.fptr(np.concatenate([np.ravel(b) for b in p.mlp.biases]))
        s.data = keep.fptr(p.mlp.data)
        s.sigma_out = keep.fptr(p.mlp.sigma_out)
    s.mode_var = keep.dptr(p.mode_var)
    s.mode_logw = keep.dptr(p.mode_logw)
    keep.bufs.append(s)
    return s


def ns_default_options(**kw):
    o = NsOptions()
    _check(lib().ns_default_options(C.byref(o)))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


def _stream_ptr(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _ptr(t):
    return None if t is None else t.data_ptr()


# --------------------------------------------------------------------------
# whole runs
# --------------------------------------------------------------------------
class Handle:
    def __init__(self, ptr, n_runs, keep):
        self.ptr = ptr
        self.n_runs = n_runs
        self._keep = keep

    def __del__(self):
        try:
            ns_destroy(self)
        except Exception:
            pass


def ns_create(problem, n_live, m, n_slice_steps, stop_frac, seed, opt=None):
    keep = _Keep()
    lik = likelihood_struct(problem, keep)
    h = _vp()
    _check(lib().ns_create(C.byref(lik), keep.dptr(problem.lo), keep.dptr(problem.hi), int(problem.d),
                           int(n_live), int(m), int(n_slice_steps), float(stop_frac), int(seed) & (2**64 - 1),
                           C.byref(opt) if opt is not None else None, C.byref(h)))
    return Handle(h, 1, keep)


def ns_create_batch(runs, opt=None):
    """runs: iterable of (problem, n_live, m, n_slice_steps, stop_frac, seed)."""
    keep = _Keep()
    runs = list(runs)
    arr = (NsProblem * len(runs))()
    liks = {}  # one struct per problem object: runs of one network share its arrays
    for i, (p, N, m, ns, sf, seed) in enumerate(runs):
        if id(p) not in liks:
            liks[id(p)] = likelihood_struct(p, keep)
        lik = liks[id(p)]
        arr[i].lik = C.pointer(lik)
        arr[i].lo = keep.dptr(p.lo)
        arr[i].hi = keep.dptr(p.hi)
        arr[i].d = int(p.d)
        arr[i].n_live = int(N)
        arr[i].m = int(m)
        arr[i].n_slice_steps = int(ns)
        arr[i].stop_frac = float(sf)
        arr[i].seed = int(seed) & (2**64 - 1)
    keep.bufs.append(arr)
    h = _vp()
    _check(lib().ns_create_batch(len(runs), arr, C.byref(opt) if opt is not None else None, C.byref(h)))
    return Handle(h, len(runs), keep)


def ns_run(h, stream=None, check=True):
    st = lib().ns_run(h.ptr, _stream_ptr(stream))
    if check:
        _check(st, h.ptr)
    return st


def ns_step(h, n_iters, stream=None, check=True):
    """Advance every unfinished run by at most n_iters iterations."""
    st = lib().ns_step(h.ptr, int(n_iters), _stream_ptr(stream))
    if check:
        _check(st, h.ptr)
    return st


def ns_checkpoint_bytes(h):
    """Size in bytes of the handle's checkpoint."""
    return int(lib().ns_checkpoint_bytes(h.ptr))


def ns_checkpoint(h, stream=None):
    """The handle's whole state as bytes (see ns_restore)."""
    n = int(lib().ns_checkpoint_bytes(h.ptr))
    buf = (C.c_char * n)()
    _check(lib().ns_checkpoint(h.ptr, buf, n, _stream_ptr(stream)), h.ptr)
    return bytes(buf)


def ns_restore(h, data, stream=None):
    """Load a checkpoint taken from a batch of the same runs and options."""
    buf = C.create_string_buffer(bytes(data), len(data))
    _check(lib().ns_restore(h.ptr, buf, len(data), _stream_ptr(stream)), h.ptr)


def ns_reset(h, stream=None):
    _check(lib().ns_reset(h.ptr, _stream_ptr(stream)), h.ptr)


def ns_autotune(h, warm_iters=0, probe_iters=3, stream=None):
    """Pick each run's configuration by measurement (ns_autotune); returns
    (choices, ratios): analytic runs 1 = one walker per warp; BF16 MLP runs
    the candidate cap per round; ratios of the second configuration's slice
    cycles per iteration over the default's (nan where not measured)."""
    n = int(lib().ns_n_runs(h.ptr))
    out = (C.c_int * max(1, n))()
    ratio = (C.c_double * max(1, n))()
    _check(lib().ns_autotune(h.ptr, int(warm_iters), int(probe_iters), C.cast(out, _vp), C.cast(ratio, _vp),
                             _stream_ptr(stream)), h.ptr)
    return [int(out[i]) for i in range(n)], [float(ratio[i]) for i in range(n)]


def ns_set_walker_mapping(h, run, warp):
    _check(lib().ns_set_walker_mapping(h.ptr, int(run), int(warp)), h.ptr)


def ns_resident_runs_per_sm(d, m, depth=0):
    return int(lib().ns_resident_runs_per_sm(int(d), int(m), int(depth)))


def ns_last_run_ms(h):
    ms = C.c_double()
    _check(lib().ns_last_run_ms(h.ptr, C.byref(ms)), h.ptr)
    return ms.value


def ns_get_stats(h):
    st = NsStats()
    _check(lib().ns_get_stats(h.ptr, C.byref(st)), h.ptr)
    return dict(run_ms=st.run_ms, kernel_ms=st.kernel_ms, launches=st.launches, h2d_bytes=st.h2d_bytes,
                d2h_bytes=st.d2h_bytes)


PHASES = ("cluster", "select", "slice", "correct", "update", "evidence")
MLP_PHASES = ("mlp_eval", "mlp_reeval")  # inside the slice phase of MLP runs
WALK_PHASES = ("draw", "walk")           # inside the slice phase of other runs (first warp)


# ns_buffer: name -> (enum value, numpy dtype)
RUN_BUFFERS = {"live_x": (0, np.float32), "live_l": (1, np.float32), "live_cid": (2, np.int32),
               "new_x": (3, np.float32), "new_l": (4, np.float32), "hist_l": (5, np.float32),
               "hist_x": (6, np.float32), "hist_len": (7, np.int32), "walker_evals": (8, np.int32),
               "walker_flags": (9, np.int32), "chol": (10, np.float32), "centres": (11, np.float32),
               "mask": (12, np.int32)}


def ns_run_buffer_bytes(h, run, name):
    """Size in bytes of one of a run's device buffers (0 for a bad run)."""
    return int(lib().ns_run_buffer_bytes(h.ptr, int(run), RUN_BUFFERS[name][0]))


def ns_copy_run_buffer(h, run, name, stream=None):
    """A host copy (flat numpy array) of one of a run's device buffers as the
    last iteration left it; see ns_copy_run_buffer in include/ns_gb300.h for
    the names, layouts and shapes."""
    which, dt = RUN_BUFFERS[name]
    nb = ns_run_buffer_bytes(h, run, name)
    out = np.empty(nb // np.dtype(dt).itemsize, dtype=dt)
    _check(lib().ns_copy_run_buffer(h.ptr, int(run), which, out.ctypes.data_as(_vp), nb, _stream_ptr(stream)), h.ptr)
    return out


def ns_phase_cycles(h, run=0, mlp=False, walk=False):
    """SM cycles per phase of one run; mlp=True adds the MLP evaluation and
    re-evaluation cycles, walk=True the direction-draw and walk cycles of the
    first warp (both parts of the slice phase)."""
    arr = (C.c_longlong * 8)()
    _check(lib().ns_phase_cycles(h.ptr, int(run), arr), h.ptr)
    out = {name: int(arr[i]) for i, name in enumerate(PHASES)}
    if mlp:
        out.update({name: int(arr[6 + i]) for i, name in enumerate(MLP_PHASES)})
    if walk:
        out.update({name: int(arr[6 + i]) for i, name in enumerate(WALK_PHASES)})
    return out


def ns_summary(h, run=0):
    return ns_result(h, run, samples=False)


def ns_result(h, run=0, samples=True):
    r = NsResult()
    fn = lib().ns_result if samples else lib().ns_summary
    _check(fn(h.ptr, int(run), C.byref(r)), h.ptr)
    out = dict(log_z=r.log_z, log_z_err=r.log_z_err, info=r.info_h, n_dead=r.n_dead, n_evals=r.n_evals,
               n_iter=r.n_iter, n_relaxed=r.n_relaxed, n_reeval=r.n_reeval, n_capped=r.n_capped,
               status=r.status, d=r.d, n_rounds=r.n_rounds, n_pass_bf16=r.n_pass_bf16, n_cand_bf16=r.n_cand_bf16,
               n_pass_fp32=r.n_pass_fp32, n_cand_fp32=r.n_cand_fp32, n_pass_x2=r.n_pass_x2,
               n_cand_x2=r.n_cand_x2)
    if samples and r.n_dead > 0:
        n, d = r.n_dead, r.d
        out["dead_x"] = np.ctypeslib.as_array(r.dead_x, shape=(n * d,)).reshape(n, d).copy()
        out["dead_l"] = np.ctypeslib.as_array(r.dead_logl, shape=(n,)).copy()
        out["dead_logw"] = np.ctypeslib.as_array(r.dead_logw, shape=(n,)).copy()
    return out


def ns_last_error(h=None):
    msg = lib().ns_last_error(h.ptr if h is not None else None)
    return msg.decode() if msg else ""


def ns_destroy(h):
    if h is not None and h.ptr is not None and h.ptr.value:
        lib().ns_destroy(h.ptr)
        h.ptr = _vp()


def noalloc_capacity(d, dead_x, dead_logl, dead_logw):
    """The dead-point capacity that ns_run_noalloc may write into the
    caller's tensors, after checking them: the C entry point gets bare
    device pointers and cannot see a buffer's size, so every tensor must be
    contiguous, of its dtype (float32, float32, float64), on one CUDA device,
    and dead_x must hold cap * d floats and dead_logw cap doubles, where cap
    = dead_logl.numel().  Raises NSError(NS_ERR_ARG) otherwise, before any
    device work."""
    import torch
    bufs = (("dead_x", dead_x, torch.float32), ("dead_logl", dead_logl, torch.float32),
            ("dead_logw", dead_logw, torch.float64))
    for name, t, dt in bufs:
        if not isinstance(t, torch.Tensor):
            raise NSError(NS_ERR_ARG, f"ns_run_noalloc: {name} must be a torch tensor")
        if t.dtype != dt:
            raise NSError(NS_ERR_ARG, f"ns_run_noalloc: {name} must be {dt}, got {t.dtype}")
        if not t.is_contiguous():
            raise NSError(NS_ERR_ARG, f"ns_run_noalloc: {name} must be contiguous")
    cap = int(dead_logl.numel())
    if int(dead_x.numel()) < cap * int(d):
        raise NSError(NS_ERR_ARG, f"ns_run_noalloc: dead_x holds {dead_x.numel()} floats, "
                                  f"fewer than cap * d = {cap} * {d}")
    if int(dead_logw.numel()) < cap:
        raise NSError(NS_ERR_ARG, f"ns_run_noalloc: dead_logw holds {dead_logw.numel()} values, "
                                  f"fewer than cap = {cap}")
    devs = {t.device for _, t, _ in bufs}
    if any(dv.type != "cuda" for dv in devs) or len(devs) != 1:
        raise NSError(NS_ERR_ARG, "ns_run_noalloc: dead_x, dead_logl and dead_logw must be on one CUDA "
                                  f"device, got {sorted(str(dv) for dv in devs)}")
    dev = next(iter(devs))
    if dev.index is not None and dev.index != torch.cuda.current_device():
        raise NSError(NS_ERR_ARG, f"ns_run_noalloc: the buffers are on {dev}, the current device is "
                                  f"cuda:{torch.cuda.current_device()}")
    return cap


def ns_run_noalloc(problem, n_live, m, n_slice_steps, stop_frac, seed, dead_x, dead_logl, dead_logw,
                   opt=None, stream=None, check=True):
    """One whole run that allocates no device memory: the library works in
    its fixed static device array and writes the samples into the caller's
    device tensors dead_x [cap, d], dead_logl [cap], dead_logw [cap]
    (float32, float32, float64).  For callers that cannot allocate device
    memory themselves (see ns_run_noalloc in include/ns_gb300.h).  Returns
    the scalar results; samples stay in the caller's tensors."""
    cap = noalloc_capacity(int(problem.d), dead_x, dead_logl, dead_logw)
    keep = _Keep()
    lik = likelihood_struct(problem, keep)
    pr = NsProblem()
    pr.lik = C.pointer(lik)
    pr.lo = keep.dptr(problem.lo)
    pr.hi = keep.dptr(problem.hi)
    pr.d = int(problem.d)
    pr.n_live = int(n_live)
    pr.m = int(m)
    pr.n_slice_steps = int(n_slice_steps)
    pr.stop_frac = float(stop_frac)
    pr.seed = int(seed) & (2**64 - 1)
    r = NsResult()
    st = lib().ns_run_noalloc(C.byref(pr), C.byref(opt) if opt is not None else None, _ptr(dead_x),
                              _ptr(dead_logl), _ptr(dead_logw), cap, C.byref(r), _stream_ptr(stream))
    if check:
        _check(st)
    return dict(log_z=r.log_z, log_z_err=r.log_z_err, info=r.info_h, n_dead=r.n_dead, n_evals=r.n_evals,
                n_iter=r.n_iter, n_relaxed=r.n_relaxed, n_reeval=r.n_reeval, n_capped=r.n_capped,
                status=r.status, d=r.d, ret=st)


# --------------------------------------------------------------------------
# step-level calls (torch CUDA tensors)
# --------------------------------------------------------------------------
def ns_philox4x32_10(ctr, key0, key1, out, stream=None):
    n = ctr.numel() // 4
    _check(lib().ns_philox4x32_10(_ptr(ctr), key0 & 0xFFFFFFFF, key1 & 0xFFFFFFFF, n, _ptr(out),
                                  _stream_ptr(stream)))


def ns_loglike(problem, x, out, stream=None):
    keep = _Keep()
    lik = likelihood_struct(problem, keep)
    n = x.shape[0]
    _check(lib().ns_loglike(C.byref(lik), keep.dptr(problem.lo), keep.dptr(problem.hi), int(problem.d), n,
                            _ptr(x), _ptr(out), _stream_ptr(stream)))


def ns_select_worst(logl, m, seeds, t, worst, W, seed_slot, stream=None):
    n_runs, N = logl.shape
    sd = (C.c_uint64 * n_runs)(*[int(s) & (2**64 - 1) for s in seeds])
    _check(lib().ns_select_worst(n_runs, N, int(m), _ptr(logl), sd, int(t) & 0xFFFFFFFF, _ptr(worst), _ptr(W),
                                 _ptr(seed_slot), _stream_ptr(stream)))


def ns_slice_scratch_bytes(d, m, n_steps):
    return int(lib().ns_slice_scratch_bytes(int(d), int(m), int(n_steps)))


def ns_slice_replace(problem, N, n_pad, m, n_steps, opt, seed, t, live_x, live_l, seed_slot, W, chol, cid,
                     new_x, new_l, hist_l, hist_x, hist_len, evals, flags, dir_scratch=None, stream=None):
    """dir_scratch: a device tensor of ns_slice_scratch_bytes(d, m, n_steps)
    bytes; allocated here with torch when not given."""
    if dir_scratch is None:
        import torch
        nb = ns_slice_scratch_bytes(problem.d, m, n_steps)
        dir_scratch = torch.empty((nb + 3) // 4, dtype=torch.float32, device=new_x.device)
    keep = _Keep()
    lik = likelihood_struct(problem, keep)
    _check(lib().ns_slice_replace(C.byref(lik), keep.dptr(problem.lo), keep.dptr(problem.hi), int(problem.d),
                                  int(N), int(n_pad), int(m), int(n_steps), C.byref(opt) if opt is not None else None,
                                  int(seed) & (2**64 - 1), int(t) & 0xFFFFFFFF, _ptr(live_x), _ptr(live_l),
                                  _ptr(seed_slot), _ptr(W), _ptr(chol), _ptr(cid), _ptr(new_x), _ptr(new_l),
                                  _ptr(hist_l), _ptr(hist_x), _ptr(hist_len), _ptr(evals), _ptr(flags),
                                  _ptr(dir_scratch), _stream_ptr(stream)))


def ns_batch_correct(m, K, correction, W, new_l, hist_l, hist_len, t_max, acc_src, acc_hpos, acc_l, acc_P,
                     rej_src, rej_hpos, rej_l, rej_P, n_relaxed, stream=None):
    _check(lib().ns_batch_correct(int(m), int(K), int(correction), _ptr(W), _ptr(new_l), _ptr(hist_l),
                                  _ptr(hist_len), int(t_max), _ptr(acc_src), _ptr(acc_hpos), _ptr(acc_l),
                                  _ptr(acc_P), _ptr(rej_src), _ptr(rej_hpos), _ptr(rej_l), _ptr(rej_P),
                                  _ptr(n_relaxed), _stream_ptr(stream)))


def ns_evidence_update(N, dead_l, state, logw, live=False, stream=None):
    _check(lib().ns_evidence_update(int(N), int(dead_l.numel()), _ptr(dead_l), _ptr(state), _ptr(logw),
                                    1 if live else 0, _stream_ptr(stream)))


def ns_mlp_image_bytes(problem):
    keep = _Keep()
    lik = likelihood_struct(problem, keep)
    return int(lib().ns_mlp_image_bytes(C.byref(lik), int(problem.d)))


def ns_mlp_pack(problem, image, stream=None):
    """image: a device uint8 tensor of ns_mlp_image_bytes(problem) bytes,
    1024-byte aligned."""
    keep = _Keep()
    lik = likelihood_struct(problem, keep)
    _check(lib().ns_mlp_pack(C.byref(lik), int(problem.d), _ptr(image), _stream_ptr(stream)))


_LIK_CACHE = {}


def _cached_likelihood(problem):
    """The marshalled likelihood of a problem object, kept while the object
    lives (batch evaluations are called many times on one network)."""
    key = id(problem)
    hit = _LIK_CACHE.get(key)
    if hit is not None and hit[0]() is problem:
        return hit[1], hit[2]
    import weakref
    keep = _Keep()
    lik = likelihood_struct(problem, keep)
    try:
        ref = weakref.ref(problem, lambda _r, k=key: _LIK_CACHE.pop(k, None))
    except TypeError:
        return lik, keep
    _LIK_CACHE[key] = (ref, lik, keep)
    return lik, keep


def ns_mlp_loglike(problem, image, x, logl, precision=1, stream=None):
    lik, _ = _cached_likelihood(problem)
    box = _Keep()
    _check(lib().ns_mlp_loglike(C.byref(lik), box.dptr(problem.lo), box.dptr(problem.hi), int(problem.d),
                                _ptr(image), int(x.shape[0]), _ptr(x), _ptr(logl), int(precision),
                                _stream_ptr(stream)))


def ns_mlp_loglike_cluster(problem, image, x, logl, precision=1, cluster=4, stream=None):
    """ns_mlp_loglike's tensor-core evaluators split over a cluster of
    `cluster` CTAs (see include/ns_gb300.h)."""
    lik, _ = _cached_likelihood(problem)
    box = _Keep()
    _check(lib().ns_mlp_loglike_cluster(C.byref(lik), box.dptr(problem.lo), box.dptr(problem.hi), int(problem.d),
                                        _ptr(image), int(x.shape[0]), _ptr(x), _ptr(logl), int(precision),
                                        int(cluster), _stream_ptr(stream)))


def ns_cluster_scratch_bytes(N, n_pad, d):
    return int(lib().ns_cluster_scratch_bytes(int(N), int(n_pad), int(d)))


def ns_cluster(N, n_pad, d, live_x, opt, seed, t, centres, chol, chol64, logvol, count, split, mask, cid,
               scratch=None, stream=None):
    """scratch: a device tensor of ns_cluster_scratch_bytes(N, n_pad, d)
    bytes (allocated here with torch when not given)."""
    if scratch is None:
        import torch
        nb = ns_cluster_scratch_bytes(N, n_pad, d)
        scratch = torch.empty(max(1, nb), dtype=torch.uint8, device=live_x.device)
    _check(lib().ns_cluster(int(N), int(n_pad), int(d), _ptr(live_x), C.byref(opt) if opt is not None else None,
                            int(seed) & (2**64 - 1), int(t) & 0xFFFFFFFF, _ptr(centres), _ptr(chol),
                            _ptr(chol64), _ptr(logvol), _ptr(count), _ptr(split), _ptr(mask), _ptr(cid),
                            _ptr(scratch), _stream_ptr(stream)))
