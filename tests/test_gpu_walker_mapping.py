"""Walker-to-lane mappings and the autotuner (batching), through the C ABI.

One walker per warp (the lanes share the walker's coordinates) takes the
same decisions and draws as one walker per thread; the step-level parity
against the oracle is in test_gpu_parity.py.  Here: whole runs on the warp
mapping against their closed forms, and ns_autotune -- valid choices, the
probe's snapshot restored exactly, and each run afterwards identical to the
same run made alone with its chosen mapping.
"""
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


RUNS = [(W.corr_gauss10(3), 500, 10, 50, 1e-3, 21), (W.gauss2d_sigma05(), 100, 1, 10, 1e-3, 22),
        (W.mixture4_d5(2), 600, 30, 25, 1e-3, 23), (W.rosenbrock(2), 400, 1, 10, 1e-3, 24),
        (W.gauss_iso(30, 1.0, -7, 7), 300, 3, 150, 1e-3, 25), (W.shell2d(), 500, 5, 10, 1e-3, 26),
        (W.gauss_corr(32, 4), 400, 20, 160, 1e-3, 27)]


def test_warp_mapping_runs_match_closed_forms(nat):
    h = nat.ns_create_batch(RUNS, nat.ns_default_options(walker_mapping=1, depth=1))
    nat.ns_run(h)
    for r, (p, N, m, ns, sf, seed) in enumerate(RUNS):
        res = nat.ns_summary(h, r)
        assert res["status"] == 0
        truth = A.logz(p)
        assert abs(res["log_z"] - truth) < 4 * res["log_z_err"] + 0.05, (p.name, res["log_z"], truth)
    nat.ns_destroy(h)


def test_autotune_choices_and_exact_state(nat):
    """After a warm-up of 20 iterations the autotuner probes both mappings
    from one snapshot and restores it: every run then finishes bit for bit
    like the same run made alone -- 20 iterations one walker per thread, then
    the chosen mapping."""
    runs = RUNS + [(W.corr_gauss10(5), 1000, 100, 50, 1e-3, 31)]
    opt = nat.ns_default_options(depth=1)
    h = nat.ns_create_batch(runs, opt)
    choice, ratio = nat.ns_autotune(h, warm_iters=20, probe_iters=3)
    assert len(choice) == len(runs) and set(choice) <= {0, 1}
    assert all(np.isfinite(ratio))
    assert all((c == 1) == (q < 0.95) for c, q in zip(choice, ratio))
    # a walker per warp runs 100 walkers four at a time: the per-thread mapping wins there
    assert choice[-1] == 0 and ratio[-1] > 2.0
    assert all(nat.ns_summary(h, r)["n_iter"] == 20 for r in range(len(runs)))
    nat.ns_run(h)
    got = [nat.ns_result(h, r) for r in range(len(runs))]
    nat.ns_destroy(h)
    for r, run in enumerate(runs):
        h1 = nat.ns_create_batch([run], opt)
        nat.ns_step(h1, 20)
        nat.ns_set_walker_mapping(h1, 0, choice[r])
        nat.ns_run(h1)
        one = nat.ns_result(h1, 0)
        nat.ns_destroy(h1)
        assert one["log_z"] == got[r]["log_z"] and one["n_evals"] == got[r]["n_evals"], r
        np.testing.assert_array_equal(one["dead_l"], got[r]["dead_l"])
        np.testing.assert_array_equal(one["dead_x"], got[r]["dead_x"])


def test_autotune_arguments(nat):
    h = nat.ns_create_batch(RUNS[:2], nat.ns_default_options())
    for warm, probe in ((0, 0), (-1, 3), (0, 1001)):
        with pytest.raises(nat.NSError):
            nat.ns_autotune(h, warm, probe)
    choice, ratio = nat.ns_autotune(h, 0, 2)
    assert len(choice) == 2
    with pytest.raises(nat.NSError):
        nat.ns_set_walker_mapping(h, 2, 1)
    nat.ns_destroy(h)


def test_autotune_mlp_candidate_cap(nat):
    """BF16 MLP runs: the autotuner picks the candidates per weight pass
    (128, 64 or every candidate in equal calls); the runs are the same for
    every choice, so an autotuned run equals the run made without it."""
    p = W.mlp_emulator(2, widths=(4, 64, 64, 60), sig_lo=1e-2, sig_hi=1e-1)
    runs = [(p, 300, 150, 12, 1e-2, s) for s in (5, 6)] + [RUNS[0]]
    opt = nat.ns_default_options(precision=1, max_iter=60, chunk_iters=60)
    h = nat.ns_create_batch(runs, opt)
    choice, ratio = nat.ns_autotune(h, warm_iters=5, probe_iters=2)
    assert choice[0] in (128, 64, 0) and choice[1] in (128, 64, 0) and choice[2] in (0, 1)
    assert all(np.isfinite(ratio))
    nat.ns_run(h, check=False)
    got = [nat.ns_result(h, r) for r in range(2)]
    nat.ns_destroy(h)
    h = nat.ns_create_batch(runs, opt)
    nat.ns_step(h, 5, check=False)
    nat.ns_run(h, check=False)
    want = [nat.ns_result(h, r) for r in range(2)]
    nat.ns_destroy(h)
    for a, b in zip(got, want):
        assert a["n_iter"] == b["n_iter"] and a["n_iter"] > 5 and a["n_evals"] == b["n_evals"]
        np.testing.assert_array_equal(a["dead_l"], b["dead_l"])
        np.testing.assert_array_equal(a["dead_x"], b["dead_x"])
