"""The allocation-free whole-run entry point (ns_run_noalloc).

Some callers cannot call cudaMalloc: a library loaded into a host program
whose device memory is already reserved by another allocator, or code on a
latency-critical path that cannot afford cudaMalloc's implicit device-wide
synchronisation.  For them ns_run_noalloc works inside the library's fixed
static device array and writes into device buffers the caller already has.

This file is collected last on purpose.  It checks the new entry point,
through the C ABI, against the handle path (ns_create + ns_run +
ns_result) on the same problems, on two calls in a row with different
problems, so that a stale array from the first call would show.
"""
import numpy as np
import pytest

from paper_2608_28514_gb300 import workloads as W

torch = pytest.importorskip("torch")


@pytest.mark.gpu
def test_noalloc_matches_handle_path_on_two_calls():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2608_28514_gb300 import _native as nat
    nat.lib()
    # three calls in a row: a 10-D run, a 2-D run, and a 16-D run with a
    # depth-6 cluster tree whose tables spill out of shared memory (the
    # array's tree-scratch branch)
    deep = nat.ns_default_options(depth=6)
    cases = [(W.corr_gauss10(3), 1000, 50, 50, 1e-3, 7, None), (W.gauss2d_sigma05(), 100, 5, 10, 1e-3, 11, None),
             (W.bimodal(16), 400, 20, 80, 1e-3, 5, deep)]
    cap = 400 * 1000 + 4 * 50
    dead_x = torch.empty(cap, 16, dtype=torch.float32, device="cuda")
    dead_l = torch.empty(cap, dtype=torch.float32, device="cuda")
    dead_w = torch.empty(cap, dtype=torch.float64, device="cuda")
    for p, N, m, ns, sf, seed, opt in cases:
        h = nat.ns_create(p, N, m, ns, sf, seed, opt)
        nat.ns_run(h)
        ref = nat.ns_result(h, 0)
        nat.ns_destroy(h)
        dead_x.fill_(float("nan"))
        dead_l.fill_(float("nan"))
        dead_w.fill_(float("nan"))
        dx = dead_x.reshape(-1)[: cap * p.d].view(cap, p.d)
        got = nat.ns_run_noalloc(p, N, m, ns, sf, seed, dx, dead_l, dead_w, opt=opt)
        torch.cuda.synchronize()
        assert got["status"] == 0
        assert got["n_dead"] == ref["n_dead"] and got["n_evals"] == ref["n_evals"]
        assert got["log_z"] == pytest.approx(ref["log_z"], rel=1e-12, abs=1e-12)
        assert got["log_z_err"] == pytest.approx(ref["log_z_err"], rel=1e-12, abs=1e-12)
        n = ref["n_dead"]
        np.testing.assert_allclose(dead_l[:n].cpu().numpy(), ref["dead_l"], rtol=1e-6, atol=1e-6)
        np.testing.assert_allclose(dead_w[:n].cpu().numpy(), ref["dead_logw"], rtol=1e-12, atol=1e-12)
        flat = dx.reshape(-1)[: n * p.d].cpu().numpy().reshape(n, p.d)
        np.testing.assert_allclose(flat, ref["dead_x"], atol=1e-5)


@pytest.mark.gpu
def test_noalloc_rejects_oversized_runs():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2608_28514_gb300 import _native as nat
    p = W.gauss_iso(32, 1.0, -7, 7)
    cap = 70000
    dx = torch.empty(cap, 32, device="cuda")
    dl = torch.empty(cap, device="cuda")
    dw = torch.empty(cap, dtype=torch.float64, device="cuda")
    with pytest.raises(nat.NSError) as ei:
        nat.ns_run_noalloc(p, 60000, 200, 10, 1e-3, 1, dx, dl, dw)
    assert ei.value.status == nat.NS_ERR_ARG and "static array" in str(ei.value)


@pytest.mark.gpu
def test_noalloc_accepts_the_stated_edge_case():
    """The header's example of a run that fits the static array (d = 32,
    m = 128, 160 slice steps; here N = 2048) is accepted and gives the
    handle path's result."""
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2608_28514_gb300 import _native as nat
    p = W.gauss_iso(32, 1.0, -7, 7)
    N, m, ns, seed = 2048, 128, 160, 3
    h = nat.ns_create(p, N, m, ns, 1e-3, seed)
    nat.ns_run(h)
    ref = nat.ns_summary(h, 0)
    nat.ns_destroy(h)
    cap = 400 * N + 4 * m
    dx = torch.empty(cap, 32, device="cuda")
    dl = torch.empty(cap, device="cuda")
    dw = torch.empty(cap, dtype=torch.float64, device="cuda")
    got = nat.ns_run_noalloc(p, N, m, ns, 1e-3, seed, dx, dl, dw)
    assert got["status"] == 0 and got["n_dead"] == ref["n_dead"] and got["n_evals"] == ref["n_evals"]
    assert got["log_z"] == pytest.approx(ref["log_z"], rel=1e-12, abs=1e-12)
