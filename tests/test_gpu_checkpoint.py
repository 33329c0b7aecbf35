"""Checkpoint / resume through the C ABI: a run split into ns_step calls, or
checkpointed and restored into a fresh handle (another arena, so other
device pointers) through a file, finishes bit for bit like the run done in
one go; a checkpoint of another batch shape is refused."""
import numpy as np
import pytest

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


RUNS = [(W.corr_gauss10(3), 500, 25, 50, 1e-3, 11), (W.gauss2d_sigma05(), 300, 5, 10, 1e-3, 12),
        (W.mixture4_d5(2), 600, 30, 25, 1e-3, 13), (W.rosenbrock(3), 400, 20, 15, 1e-3, 14)]


def _results(nat, h):
    return [nat.ns_result(h, r) for r in range(len(RUNS))]


def _same(a, b):
    assert a["log_z"] == b["log_z"] and a["info"] == b["info"]
    assert a["n_iter"] == b["n_iter"] and a["n_evals"] == b["n_evals"] and a["n_dead"] == b["n_dead"]
    np.testing.assert_array_equal(a["dead_l"], b["dead_l"])
    np.testing.assert_array_equal(a["dead_x"], b["dead_x"])
    np.testing.assert_array_equal(a["dead_logw"], b["dead_logw"])


def test_steps_and_checkpoint_resume_are_bitwise(nat, tmp_path):
    opt = nat.ns_default_options(depth=1)
    h0 = nat.ns_create_batch(RUNS, opt)
    nat.ns_run(h0)
    ref = _results(nat, h0)
    nat.ns_destroy(h0)
    assert all(r["status"] == 0 and r["n_iter"] > 30 for r in ref)

    h1 = nat.ns_create_batch(RUNS, opt)
    nat.ns_step(h1, 13)
    nat.ns_step(h1, 7)
    mid = [nat.ns_summary(h1, r) for r in range(len(RUNS))]
    assert all(r["n_iter"] == 20 for r in mid)
    ck = nat.ns_checkpoint(h1)
    path = tmp_path / "runs.ckpt"
    path.write_bytes(ck)
    nat.ns_run(h1)
    for a, b in zip(_results(nat, h1), ref):
        _same(a, b)
    nat.ns_destroy(h1)

    h2 = nat.ns_create_batch(RUNS, opt)
    nat.ns_restore(h2, path.read_bytes())
    assert [nat.ns_summary(h2, r)["n_iter"] for r in range(len(RUNS))] == [20] * len(RUNS)
    nat.ns_run(h2)
    for a, b in zip(_results(nat, h2), ref):
        _same(a, b)
    nat.ns_destroy(h2)

    h3 = nat.ns_create_batch(RUNS[:3], opt)
    with pytest.raises(nat.NSError):
        nat.ns_restore(h3, ck)
    h4 = nat.ns_create_batch(RUNS, nat.ns_default_options(depth=2))
    with pytest.raises(nat.NSError):
        nat.ns_restore(h4, ck)
    with pytest.raises(nat.NSError):
        nat.ns_restore(h4, ck[:100])
    nat.ns_destroy(h3)
    nat.ns_destroy(h4)
