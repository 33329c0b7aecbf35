"""The C-ABI library loads and exports every symbol its header declares;
host-side argument validation rejects bad input before any CUDA call.
Runs without a GPU."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ns_gb300.h")


@pytest.fixture(scope="module")
def native():
    import __graft_entry__ as g
    from paper_2608_28514_gb300 import build as nb
    nb.build()
    from paper_2608_28514_gb300 import _native
    _native.lib()
    return _native


def _declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b(?:ns_status|void|int|size_t|const char\*)\s+(ns_\w+)\s*\(", text)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ("ns_create", "ns_create_batch", "ns_run", "ns_result", "ns_destroy", "ns_last_error",
                     "ns_select_worst", "ns_slice_replace", "ns_batch_correct", "ns_evidence_update",
                     "ns_cluster", "ns_loglike", "ns_philox4x32_10"):
        assert required in names


def test_library_exports_every_declared_symbol(native):
    lib = native.lib()
    missing = [n for n in _declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_names_match_header(native):
    for n in _declared_functions():
        if n in ("ns_n_runs",):
            continue
        assert hasattr(native, n), n


def test_validation_without_gpu(native):
    from paper_2608_28514_gb300 import workloads as W
    p = W.gauss2d_sigma05()
    bad = [
        dict(n_live=100, m=51),      # m > N/2
        dict(n_live=100, m=0),
        dict(n_live=1, m=1),
        dict(n_live=100, m=300),     # m > NS_MAX_BATCH
        dict(n_live=100, m=5, stop_frac=1.5),
        dict(n_live=100, m=5, n_slice_steps=0),
    ]
    for b in bad:
        args = dict(n_live=100, m=5, n_slice_steps=10, stop_frac=1e-3, seed=1)
        args.update(b)
        with pytest.raises(native.NSError) as ei:
            native.ns_create(p, **args)
        assert ei.value.status == native.NS_ERR_ARG
    # a bad box
    q = W.gauss2d_sigma05()
    q.hi = q.lo.copy()
    with pytest.raises(native.NSError) as ei:
        native.ns_create(q, 100, 5, 10, 1e-3, 1)
    assert ei.value.status == native.NS_ERR_ARG
    # non-finite likelihood parameters
    q = W.gauss2d_sigma05()
    q.mean = np.array([np.nan, 0.0])
    with pytest.raises(native.NSError):
        native.ns_create(q, 100, 5, 10, 1e-3, 1)
    q = W.gauss2d_sigma05()
    q.sigma = 0.0
    with pytest.raises(native.NSError):
        native.ns_create(q, 100, 5, 10, 1e-3, 1)
    # options out of range
    for k, v in [("depth", 9), ("t_max", 0), ("t_max", 65), ("correction", 7), ("width", -1.0),
                 ("precision", 2), ("reeval_margin", -1.0), ("reeval_rel", -1e-3), ("reeval_rel", float("inf")),
                 ("reeval_defer", -1), ("reeval_defer", 65), ("walker_mapping", 2), ("walker_mapping", -1),
                 ("mlp_batch_cap", -1), ("mlp_batch_cap", 129), ("mlp_cluster", 3), ("two_plane", 2),
                 ("reeval2_margin", -1.0), ("reeval2_rel", float("nan")), ("bracket", 2), ("bracket", -1)]:
        o = native.ns_default_options(**{k: v})
        with pytest.raises(native.NSError):
            native.ns_create(p, 100, 5, 10, 1e-3, 1, opt=o)
    assert native.ns_last_error() != ""


def test_step_level_validation_without_gpu(native):
    lib = native.lib()
    assert lib.ns_select_worst(1, 10, 6, None, None, 0, None, None, None, None) == native.NS_ERR_ARG
    assert lib.ns_batch_correct(0, 1, 2, *([None] * 4), 8, *([None] * 10)) == native.NS_ERR_ARG
    assert lib.ns_evidence_update(0, 1, None, None, None, 0, None) == native.NS_ERR_ARG
    assert lib.ns_philox4x32_10(None, 0, 0, -1, None, None) == native.NS_ERR_ARG


def test_default_options_match_header(native):
    o = native.ns_default_options()
    assert (o.depth, o.correction, o.history_iters, o.t_max, o.e_max, o.s_max) == (0, 2, 1, 64, 64, 128)
    assert o.width == 1.0 and o.vol_frac == 0.5 and o.kmeans_iters == 10
    assert o.precision == 0 and o.reeval_margin == 2.0 and o.reeval_rel == 4e-3 and o.reeval_defer == 4
    assert o.walker_mapping == 0 and o.mlp_batch_cap == 128
    assert o.mlp_cluster == 0 and o.two_plane == 1 and o.reeval2_margin == 0.05 and o.reeval2_rel == 1e-4
    assert o.bracket == 0


def test_autotune_and_mapping_arguments_without_gpu(native):
    lib = native.lib()
    assert lib.ns_autotune(None, 0, 3, None, None, None) == native.NS_ERR_ARG
    assert lib.ns_set_walker_mapping(None, 0, 1) == native.NS_ERR_ARG
    # a depth-6 tree's scratch: the points, then the deepest tree's FP64 node statistics
    assert native.ns_cluster_scratch_bytes(1000, 1024, 10) > 4 * 10 * 1024 + 4 * 1000 + 8 * 127 * 100
    assert native.ns_cluster_scratch_bytes(1, 32, 2) == 0


def test_noalloc_buffers_are_checked_before_any_launch():
    """ns_run_noalloc hands bare pointers to the library, which cannot see
    a buffer's size: the binding rejects a wrong dtype, a short or
    non-contiguous buffer, or host memory with NS_ERR_ARG before anything
    reaches the device (so this runs without a GPU)."""
    torch = pytest.importorskip("torch")
    from paper_2608_28514_gb300 import _native as nat
    cap, d = 100, 3
    ok = dict(dead_x=torch.empty(cap, d), dead_logl=torch.empty(cap), dead_logw=torch.empty(cap, dtype=torch.float64))
    bad = [
        (dict(ok, dead_logw=torch.empty(cap)), "float64"),
        (dict(ok, dead_x=torch.empty(cap, d, dtype=torch.float64)), "float32"),
        (dict(ok, dead_x=torch.empty(cap, d - 1)), "cap * d"),
        (dict(ok, dead_logw=torch.empty(cap - 1, dtype=torch.float64)), "cap ="),
        (dict(ok, dead_x=torch.empty(d, cap).t()), "contiguous"),
        (ok, "CUDA"),
    ]
    for kw, what in bad:
        with pytest.raises(nat.NSError) as ei:
            nat.noalloc_capacity(d, kw["dead_x"], kw["dead_logl"], kw["dead_logw"])
        assert ei.value.status == nat.NS_ERR_ARG and what in str(ei.value), (what, str(ei.value))
