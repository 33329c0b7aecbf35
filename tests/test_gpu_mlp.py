"""The MLP likelihood's batch evaluators through the C ABI.

FP32 CUDA-core path: against the FP64 oracle at FP32 tolerance.  BF16
tensor-core path (tcgen05): against a numpy emulation of the same BF16
pipeline (inputs, weights and activations rounded to bf16, accumulation in
high precision) at a tolerance that allows an activation to round the other
way, and against the FP64 oracle at BF16 accuracy.
"""
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


def _bf16(a):
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = ((u + (((u >> 16) & 1) + 0x7FFF)) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def _emulate_bf16(p, x):
    th = _bf16(p.lo + (p.hi - p.lo) * x.astype(np.float32))
    h = th
    L = len(p.mlp.weights)
    for i, (Wt, Bt) in enumerate(zip(p.mlp.weights, p.mlp.biases)):
        z = h @ Wt.astype(np.float64).T + Bt.astype(np.float64)
        if i + 1 < L:
            h = _bf16(z / (1.0 + np.exp(-z)))
        else:
            h = z
    r = (h - p.mlp.data.astype(np.float32).astype(np.float64)) / p.mlp.sigma_out.astype(np.float32)
    return -0.5 * (r * r).sum(1)


def _problem(widths, seed, unit_sigma):
    p = W.mlp_emulator(seed, widths=widths)
    if unit_sigma:
        p.mlp.sigma_out = np.ones_like(p.mlp.sigma_out)
        p.mlp.data = np.zeros_like(p.mlp.data)
    return p


def _image(nat, p):
    nb = nat.ns_mlp_image_bytes(p)
    assert nb > 0
    img = torch.empty(nb + 1024, dtype=torch.uint8, device="cuda")
    off = (-img.data_ptr()) % 1024
    img = img[off:off + nb]
    nat.ns_mlp_pack(p, img)
    return img


@pytest.mark.parametrize("widths,n", [((27, 512, 512, 512, 512, 2000), 150), ((5, 128, 200, 300), 64),
                                      ((3, 64, 100), 1), ((27, 512, 512, 512, 512, 2000), 257)])
def test_mlp_fp32_matches_oracle(nat, oracle, widths, n):
    p = _problem(widths, 3, unit_sigma=False)
    img = _image(nat, p)
    rng = np.random.default_rng(n)
    x = rng.uniform(0, 1, size=(n, p.d)).astype(np.float32)
    x[0] = p.mlp.theta_star
    out = torch.zeros(n, device="cuda")
    nat.ns_mlp_loglike(p, img, torch.tensor(x, device="cuda"), out, precision=0)
    torch.cuda.synchronize()
    got = out.cpu().numpy().astype(np.float64)
    want = oracle.loglike(oracle.Lik(p), x.astype(np.float64))
    np.testing.assert_allclose(got, want, rtol=2e-5, atol=1e-3)


def test_mlp_fp32_general_weights(nat, oracle):
    """FP32 master weights that are not BF16 values are stored and read as
    FP32 (BF16-valued ones as BF16, exactly): both match the FP64 oracle."""
    for perturb in (False, True):
        p = _problem((5, 128, 200, 300), 4, unit_sigma=False)
        if perturb:
            rng = np.random.default_rng(9)
            p.mlp.weights = [(w * (1.0 + 1e-3 * rng.standard_normal(w.shape))).astype(np.float32)
                             for w in p.mlp.weights]
            assert any(np.any(w.view(np.uint32) & 0xFFFF) for w in p.mlp.weights)
        img = _image(nat, p)
        x = np.random.default_rng(5).uniform(0, 1, size=(97, p.d)).astype(np.float32)
        out = torch.zeros(97, device="cuda")
        nat.ns_mlp_loglike(p, img, torch.tensor(x, device="cuda"), out, precision=0)
        torch.cuda.synchronize()
        want = oracle.loglike(oracle.Lik(p), x.astype(np.float64))
        np.testing.assert_allclose(out.cpu().numpy().astype(np.float64), want, rtol=2e-5, atol=1e-3)


@pytest.mark.parametrize("widths,n", [((5, 128, 200, 300), 64), ((27, 512, 512, 512, 512, 2000), 150),
                                      ((3, 64, 100), 1), ((27, 512, 512, 512, 512, 2000), 257)])
def test_mlp_bf16_tensor_cores(nat, oracle, widths, n):
    p = _problem(widths, 5, unit_sigma=True)
    img = _image(nat, p)
    rng = np.random.default_rng(n + 7)
    x = rng.uniform(0, 1, size=(n, p.d)).astype(np.float32)
    out = torch.zeros(n, device="cuda")
    nat.ns_mlp_loglike(p, img, torch.tensor(x, device="cuda"), out, precision=1)
    torch.cuda.synchronize()
    got = out.cpu().numpy().astype(np.float64)
    assert np.all(np.isfinite(got)), "a tensor-core block timed out"
    emu = _emulate_bf16(p, x)
    np.testing.assert_allclose(got, emu, rtol=3e-3, atol=1e-3)
    exact = oracle.loglike(oracle.Lik(p), x.astype(np.float64))
    np.testing.assert_allclose(got, exact, rtol=5e-2, atol=1e-2)


@pytest.mark.parametrize("cluster", [2, 4])
@pytest.mark.parametrize("precision,n", [(1, 150), (1, 257), (1, 7), (2, 33), (2, 150)])
def test_mlp_cluster_split_evaluator(nat, oracle, cluster, precision, n):
    """The tensor-core evaluators split over a cluster of 2 or 4 CTAs (each
    streams a disjoint share of every layer's weight tiles; hidden
    activations exchanged through distributed shared memory) on the 27-D
    emulator network, ragged batches included: the same log L as one CTA up
    to the order of the final chi^2 sum, and, element by element, the FP64
    oracle at each path's tolerance (BF16: the BF16 emulation at 3e-3 and the
    oracle at 5e-2; FP32 accuracy: the oracle at 2e-5)."""
    p = _problem((27, 512, 512, 512, 512, 2000), 6, unit_sigma=(precision == 1))
    img = _image(nat, p)
    rng = np.random.default_rng(100 * cluster + n)
    x = rng.uniform(0, 1, size=(n, p.d)).astype(np.float32)
    x[0] = p.mlp.theta_star
    xt = torch.tensor(x, device="cuda")
    one = torch.zeros(n, device="cuda")
    split = torch.full((n,), float("nan"), device="cuda")
    nat.ns_mlp_loglike(p, img, xt, one, precision=precision)
    nat.ns_mlp_loglike_cluster(p, img, xt, split, precision=precision, cluster=cluster)
    torch.cuda.synchronize()
    got = split.cpu().numpy().astype(np.float64)
    assert np.all(np.isfinite(got)), "a cluster pass timed out"
    np.testing.assert_allclose(got, one.cpu().numpy().astype(np.float64), rtol=2e-6, atol=1e-4)
    exact = oracle.loglike(oracle.Lik(p), x.astype(np.float64))
    if precision == 1:
        np.testing.assert_allclose(got, _emulate_bf16(p, x), rtol=3e-3, atol=1e-3)
        np.testing.assert_allclose(got, exact, rtol=5e-2, atol=1e-2)
    else:
        np.testing.assert_allclose(got, exact, rtol=2e-5, atol=1e-3)


def test_mlp_cluster_arguments(nat):
    p = _small_emulator()
    img = _image(nat, p)
    x = torch.rand(8, p.d, device="cuda")
    out = torch.zeros(8, device="cuda")
    for prec, cl in ((1, 3), (0, 4), (1, 4)):  # bad size; CUDA-core path; 1 tile row per layer
        with pytest.raises(nat.NSError):
            nat.ns_mlp_loglike_cluster(p, img, x, out, precision=prec, cluster=cl)


# --------------------------------------------------------------------------
# whole runs with the MLP likelihood
# --------------------------------------------------------------------------
def _small_emulator(seed=2):
    p = W.mlp_emulator(seed, widths=(4, 64, 64, 60), sig_lo=1e-2, sig_hi=1e-1)
    return p


def test_mlp_runs_fp32_vs_oracle_and_bf16(nat, oracle):
    """A 4-D emulator (4 -> 64 -> 64 -> 60): the GPU FP32 path agrees with
    the FP64 oracle in distribution, and the BF16 tensor-core path with FP32
    re-evaluation near the threshold stays within 0.1 of the FP32 path."""
    p = _small_emulator()
    N, m, ns, sf = 200, 20, 20, 1e-2
    seeds = list(range(1, 9))
    orc = np.array([oracle.run(p, N, m, ns, sf, s)["logz"] for s in seeds])
    res = {}
    for prec in (0, 1):
        o = nat.ns_default_options(precision=prec, reeval_margin=5.0)
        h = nat.ns_create_batch([(p, N, m, ns, sf, s) for s in seeds], o)
        nat.ns_run(h)
        out = [nat.ns_result(h, r, samples=False) for r in range(len(seeds))]
        nat.ns_destroy(h)
        assert all(r["status"] == 0 for r in out)
        res[prec] = out
    z32 = np.array([r["log_z"] for r in res[0]])
    z16 = np.array([r["log_z"] for r in res[1]])
    err = np.mean([r["log_z_err"] for r in res[0]])
    se = np.sqrt(z32.var(ddof=1) / len(seeds) + orc.var(ddof=1) / len(seeds))
    assert abs(z32.mean() - orc.mean()) < 3.5 * se + 0.02, (z32.mean(), orc.mean(), se)
    assert abs(z16.mean() - z32.mean()) < 0.1 + 2 * err / np.sqrt(len(seeds)), (z16.mean(), z32.mean())
    assert sum(r["n_reeval"] for r in res[1]) > 0
    assert all(r["n_reeval"] == 0 for r in res[0])


def test_full_emulator_runs_a_few_iterations(nat):
    """The 27 -> 512 x 4 -> 2000 emulator workload (N = 1500, m = 150, 135
    slice steps), BF16 with FP32 re-evaluation: a few iterations complete on
    the tensor-core path and every stored value is finite."""
    p = W.mlp_emulator(1)
    o = nat.ns_default_options(precision=1, reeval_margin=20.0, max_iter=2, chunk_iters=2)
    h = nat.ns_create(p, 1500, 150, 135, 1e-3, 3, opt=o)
    st = nat.ns_run(h, check=False)
    r = nat.ns_result(h, 0)
    nat.ns_destroy(h)
    assert st == nat.NS_ERR_BUDGET and r["status"] == nat.NS_ERR_BUDGET and r["n_iter"] == 2
    assert r["n_evals"] > 1500 + 2 * 150 * 135
    assert np.all(np.isfinite(r["dead_l"]))
    # dead points of the two iterations, in ascending order
    nd = 2 * 150
    assert np.all(np.diff(r["dead_l"][:nd]) >= 0)


def test_deferred_reevaluation_changes_nothing(nat):
    """Near-threshold candidates re-evaluated at once (reeval_defer = 0) or
    batched over up to 4 and 16 rounds: the same runs, bit for bit."""
    p = _small_emulator(5)
    runs = [(p, 200, 20, 20, 1e-2, s) for s in (3, 4)]
    out = {}
    for defer in (0, 4, 16):
        o = nat.ns_default_options(precision=1, reeval_margin=5.0, reeval_defer=defer, max_iter=40, chunk_iters=40)
        h = nat.ns_create_batch(runs, o)
        nat.ns_run(h, check=False)
        out[defer] = [nat.ns_result(h, r) for r in range(len(runs))]
        nat.ns_destroy(h)
    assert sum(r["n_reeval"] for r in out[0]) > 0
    for defer in (4, 16):
        for a, b in zip(out[0], out[defer]):
            assert a["n_iter"] == b["n_iter"] and a["n_evals"] == b["n_evals"] and a["n_reeval"] == b["n_reeval"]
            np.testing.assert_array_equal(a["dead_l"], b["dead_l"])
            np.testing.assert_array_equal(a["dead_x"], b["dead_x"])


def test_round_cap_changes_nothing(nat):
    """BF16 rounds capped at 8 or 16 candidates (walkers beyond the cap keep
    their candidate for the next round) or uncapped, and the 27-D emulator
    workload (m = 150) at the default cap of 128 or uncapped: the same runs,
    bit for bit (a candidate's BF16 value does not depend on its batch)."""
    p = _small_emulator(5)
    runs = [(p, 200, 20, 20, 1e-2, s) for s in (3, 4)]
    cases = [(runs, (0, 8, 16), dict(max_iter=40, chunk_iters=40, reeval_margin=5.0)),
             ([(W.mlp_emulator(1), 1500, 150, 135, 1e-3, s) for s in (1, 2)], (0, 128),
              dict(max_iter=2, chunk_iters=2, dead_cap=1500 + 600))]
    for rr, caps, kw in cases:
        out = {}
        for cap in caps:
            o = nat.ns_default_options(precision=1, mlp_batch_cap=cap, **kw)
            h = nat.ns_create_batch(rr, o)
            nat.ns_run(h, check=False)
            out[cap] = [nat.ns_result(h, r) for r in range(len(rr))]
            nat.ns_destroy(h)
        for cap in caps[1:]:
            for a, b in zip(out[0], out[cap]):
                assert a["n_iter"] == b["n_iter"] and a["n_evals"] == b["n_evals"] and a["n_reeval"] == b["n_reeval"]
                np.testing.assert_array_equal(a["dead_l"], b["dead_l"])
                np.testing.assert_array_equal(a["dead_x"], b["dead_x"])


@pytest.mark.parametrize("widths,n", [((27, 512, 512, 512, 512, 2000), 150), ((5, 128, 200, 300), 64),
                                      ((3, 64, 100), 1), ((27, 512, 512, 512, 512, 2000), 33)])
def test_mlp_fp32_accurate_tensor_path(nat, oracle, widths, n):
    """precision 2 (three BF16 planes on the tensor cores) agrees with the FP64
    oracle at FP32 accuracy, like the CUDA-core FP32 evaluator."""
    p = _problem(widths, 3, unit_sigma=False)
    img = _image(nat, p)
    rng = np.random.default_rng(n + 11)
    x = rng.uniform(0, 1, size=(n, p.d)).astype(np.float32)
    x[0] = p.mlp.theta_star
    out = torch.zeros(n, device="cuda")
    nat.ns_mlp_loglike(p, img, torch.tensor(x, device="cuda"), out, precision=2)
    torch.cuda.synchronize()
    got = out.cpu().numpy().astype(np.float64)
    want = oracle.loglike(oracle.Lik(p), x.astype(np.float64))
    np.testing.assert_allclose(got, want, rtol=2e-5, atol=1e-3)


# --------------------------------------------------------------------------
# the lock-step MLP walkers of the run kernel on fixed streams
# --------------------------------------------------------------------------
def _mlp_walkers_vs_oracle(nat, oracle, p, N, m, ns, T, precision, seed, cluster=1):
    """Runs T iterations, reads the live set and cluster factor the next
    iteration starts from (ns_copy_run_buffer), runs iteration T, and replays
    each of its walkers with the oracle's slice walker on the same Philox
    streams, seed point and thresholds.  Returns (walkers compared, walkers
    that diverged at a borderline comparison)."""
    opt = nat.ns_default_options(precision=precision, mlp_cluster=cluster)
    assert (T % max(1, 100 // m)) != 0  # no re-clustering at iteration T: the factor read is the one used
    h = nat.ns_create_batch([(p, N, m, ns, 1e-3, seed)], opt)
    nat.ns_step(h, T)
    assert nat.ns_summary(h, 0)["n_iter"] == T
    d = p.d
    lx = nat.ns_copy_run_buffer(h, 0, "live_x").reshape(d, -1)[:, :N].T.copy()
    ll = nat.ns_copy_run_buffer(h, 0, "live_l")
    chol = nat.ns_copy_run_buffer(h, 0, "chol")[: d * d].reshape(d, d).astype(np.float64)
    assert np.all(nat.ns_copy_run_buffer(h, 0, "live_cid") == 0)
    nat.ns_step(h, 1)
    g = {k: nat.ns_copy_run_buffer(h, 0, k) for k in
         ("new_x", "new_l", "hist_l", "hist_x", "hist_len", "walker_evals", "walker_flags")}
    nat.ns_destroy(h)
    t_max = opt.t_max
    g["new_x"] = g["new_x"].reshape(m, d)
    g["hist_l"] = g["hist_l"].reshape(m, t_max)
    g["hist_x"] = g["hist_x"].reshape(m, t_max, d)
    worst, seeds = oracle.select(ll.astype(np.float64), m, seed, T)
    Wv = ll[worst]
    lik = oracle.Lik(p)
    oo = oracle.opts(d, m)
    tol = lambda l64: 2e-5 * np.abs(l64) + 1e-3  # FP32 evaluation of the MLP (test_mlp_fp32_matches_oracle)
    # BF16 runs: history samples below this never get their FP32 value (Algorithm 2 cannot take them)
    lim = Wv[0] - (opt.reeval_margin + opt.reeval_rel * abs(Wv[0]))
    n_div = 0
    for i in range(m):
        r = oracle.slice_walker(lik, oo, ns, seed, T, i, lx[seeds[i]].astype(np.float64), float(ll[seeds[i]]),
                                chol, float(Wv[0]), float(Wv[i]))
        if np.max(np.abs(r["x"] - g["new_x"][i])) <= 1e-5:
            l64 = oracle.loglike(lik, g["new_x"][i].astype(np.float64))[0]
            assert abs(l64 - g["new_l"][i]) <= tol(l64), (i, l64, g["new_l"][i])
            assert g["walker_evals"][i] == r["n_evals"], (i, g["walker_evals"][i], r["n_evals"])
            assert g["walker_flags"][i] == r["flags"]
            hl = g["hist_len"][i]
            assert hl == r["hist_len"], (i, hl, r["hist_len"])
            np.testing.assert_allclose(g["hist_x"][i, :hl], r["hist_x"], atol=1e-5)
            hx = g["hist_x"][i, :hl].astype(np.float64)
            fin = np.isfinite(r["hist_l"])
            np.testing.assert_array_equal(np.isfinite(g["hist_l"][i, :hl]), fin)
            h64 = oracle.loglike(lik, hx[fin]) if fin.any() else np.zeros(0)
            hg = g["hist_l"][i, :hl][fin]
            fp32 = np.ones(len(hg), dtype=bool) if precision != 1 else hg >= lim
            assert np.all(np.abs(hg[fp32] - h64[fp32]) <= tol(h64[fp32])), i
            # the others keep their BF16 value
            assert np.all(np.abs(hg[~fp32] - h64[~fp32]) <= 1e-2 * np.abs(h64[~fp32]) + 1.0), i
        else:
            n_div += 1
            assert r["min_l_margin"] < 4e-5 or r["min_box_margin"] < 1e-5, (i, r["min_l_margin"],
                                                                             r["min_box_margin"])
        assert g["new_l"][i] > Wv[i]
        assert np.all((g["new_x"][i] >= 0) & (g["new_x"][i] <= 1))
    return m, n_div


@pytest.mark.parametrize("net,precision,cluster", [
    ("emulator27", 0, 1), ("emulator27", 1, 1), ("emulator27", 1, 4), ("emulator27", 2, 4), ("emulator27", 2, 2),
    ("small4", 0, 1), ("small4", 1, 1), ("small4", 2, 1)])
def test_mlp_run_walkers_match_oracle_on_fixed_streams(nat, oracle, net, precision, cluster):
    """The run kernel's lock-step MLP walkers (both stepping-out ends
    evaluated in the same round, out-of-box proposals settled locally,
    rounds batched onto the evaluator, in BF16 mode FP32 re-evaluation near
    the threshold with deferred passes and the round cap; on one CTA or with
    every evaluation split over a cluster of CTAs) take the sequential slice
    sampler's decisions: each walker's new point, log L, history, evaluation
    count and cap flags equal the FP64 oracle walker's on the same streams,
    except where a comparison was borderline at FP32 accuracy.  Precision 0
    is FP32 on the CUDA cores, 1 BF16 with FP32 re-evaluation, 2 FP32 on the
    tensor cores.  On the 27-D emulator network (27 -> 512 x 4 -> 2000) at
    iteration 100 (N = 300, m = 16, 8 slice steps) and on a 4-D network
    (4 -> 64 -> 64 -> 60) at iteration 31 (N = 200, m = 20, 20 steps)."""
    if net == "emulator27":
        p, N, m, ns, T = W.mlp_emulator(1), 300, 16, 8, 100
    else:
        p, N, m, ns, T = _small_emulator(3), 200, 20, 20, 31
    n, n_div = _mlp_walkers_vs_oracle(nat, oracle, p, N, m, ns, T, precision, seed=9, cluster=cluster)
    assert n_div <= max(1, n // 10), n_div


@pytest.mark.parametrize("cluster", [1, 4])
def test_bf16_runs_reproduce_the_fp32_tensor_runs(nat, cluster):
    """The precision pattern's promise, checked whole: a BF16 decision is
    taken only when the BF16 log L lies beyond the re-evaluation margin from
    its threshold, every other candidate gets its FP32 value first, and every
    stored value is FP32; FP32 values on the tensor cores do not depend on the
    batch a candidate is evaluated in.  So, while the BF16 error stays within
    the margin, a BF16 run takes every decision of the FP32 run on the tensor
    cores (precision 2) and stores the same values: the two runs are the same
    run, bit for bit.  An 8-D network (8 -> 512 -> 512 -> 512), N = 200,
    m = 20, 40 slice steps, 8 seeds, on one CTA and on a 4-CTA cluster."""
    p = W.mlp_emulator(4, widths=(8, 512, 512, 512), sig_lo=2e-2, sig_hi=2e-1)
    seeds = list(range(31, 39))
    out = {}
    for prec in (1, 2):
        h = nat.ns_create_batch([(p, 200, 20, 40, 1e-3, s) for s in seeds],
                                nat.ns_default_options(precision=prec, mlp_cluster=cluster))
        nat.ns_run(h)
        out[prec] = [nat.ns_result(h, r) for r in range(len(seeds))]
        nat.ns_destroy(h)
    same = 0
    for a, b in zip(out[1], out[2]):
        assert a["status"] == 0 and b["status"] == 0
        assert abs(a["log_z"] - b["log_z"]) < 0.05, (a["log_z"], b["log_z"])
        if a["log_z"] == b["log_z"] and a["n_evals"] == b["n_evals"]:
            np.testing.assert_array_equal(a["dead_l"], b["dead_l"])
            np.testing.assert_array_equal(a["dead_x"], b["dead_x"])
            same += 1
    assert same >= len(seeds) - 1, same
    assert sum(r["n_reeval"] for r in out[1]) > 0 and all(r["n_cand_bf16"] > 0 for r in out[1])
    assert all(r["n_cand_bf16"] == 0 and r["n_cand_fp32"] > 0 for r in out[2])


@pytest.mark.parametrize("widths,n", [((27, 512, 512, 512, 512, 2000), 150), ((5, 128, 200, 300), 64),
                                      ((27, 512, 512, 512, 512, 2000), 65)])
def test_mlp_16bit_tensor_path(nat, oracle, widths, n):
    """precision 3 (inputs and activations as two BF16 planes, relative
    rounding 2^-17; BF16-valued weights exact) agrees with the FP64 oracle to
    16-bit accuracy, far closer than the BF16 path."""
    p = _problem(widths, 8, unit_sigma=False)
    img = _image(nat, p)
    x = np.random.default_rng(n + 3).uniform(0, 1, size=(n, p.d)).astype(np.float32)
    x[0] = p.mlp.theta_star
    xt = torch.tensor(x, device="cuda")
    o2, o1 = torch.zeros(n, device="cuda"), torch.zeros(n, device="cuda")
    nat.ns_mlp_loglike(p, img, xt, o2, precision=3)
    nat.ns_mlp_loglike(p, img, xt, o1, precision=1)
    torch.cuda.synchronize()
    want = oracle.loglike(oracle.Lik(p), x.astype(np.float64))
    e2 = np.abs(o2.cpu().numpy() - want)
    e1 = np.abs(o1.cpu().numpy() - want)
    np.testing.assert_allclose(o2.cpu().numpy(), want, rtol=2e-4, atol=1e-2)
    assert np.median(e2) * 20 < np.median(e1), (np.median(e2), np.median(e1))


def test_two_plane_stage_changes_nothing(nat):
    """The 16-bit stage between the BF16 value and the FP32 one only saves
    FP32 passes: with or without it, BF16 runs are the same run, bit for bit
    (every decision it takes lies beyond its margin from the threshold),
    with fewer FP32 re-evaluations."""
    p = W.mlp_emulator(4, widths=(8, 512, 512, 512), sig_lo=2e-2, sig_hi=2e-1)
    runs = [(p, 200, 20, 40, 1e-3, s) for s in (41, 42, 43)]
    out = {}
    for two in (0, 1):
        h = nat.ns_create_batch(runs, nat.ns_default_options(precision=1, two_plane=two))
        nat.ns_run(h)
        out[two] = [nat.ns_result(h, r) for r in range(len(runs))]
        nat.ns_destroy(h)
    same = 0
    for a, b in zip(out[0], out[1]):
        if a["log_z"] == b["log_z"] and a["n_evals"] == b["n_evals"]:
            np.testing.assert_array_equal(a["dead_l"], b["dead_l"])
            same += 1
    assert same >= len(runs) - 1, same
    assert sum(r["n_cand_x2"] for r in out[1]) > 0 and all(r["n_cand_x2"] == 0 for r in out[0])
    assert sum(r["n_reeval"] for r in out[1]) < sum(r["n_reeval"] for r in out[0])


def test_bf16_error_near_the_posterior_is_inside_the_margin(nat):
    """Calibration of the FP32 re-evaluation margin on the 27-D emulator
    network where it matters, near the end of a run: 20000 points of the
    posterior region (the Laplace approximation's Gaussian around the mode,
    oracle/laplace.py, clipped to the box; log L from about l_max - 30 to
    l_max), evaluated in BF16 and in FP32 on the tensor cores.  Twice the
    99.99th percentile of |log L_BF16 - log L_FP32| lies inside the default
    margin 2 + 4e-3 |log L|, so a BF16 decision there agrees with the FP32
    one."""
    from oracle import laplace
    p = W.mlp_emulator(1)
    lap = laplace.laplace_logz(p, n_mc=1000)
    L = np.linalg.cholesky(lap["cov"])
    z = np.random.default_rng(3).standard_normal((20000, p.d))
    x = np.clip(lap["theta_hat"] + z @ L.T, 0.0, 1.0).astype(np.float32)
    img = _image(nat, p)
    xt = torch.tensor(x, device="cuda")
    lb = torch.zeros(len(x), device="cuda")
    lf = torch.zeros(len(x), device="cuda")
    nat.ns_mlp_loglike(p, img, xt, lb, precision=1)
    nat.ns_mlp_loglike(p, img, xt, lf, precision=2)
    torch.cuda.synchronize()
    lb, lf = lb.cpu().numpy().astype(np.float64), lf.cpu().numpy().astype(np.float64)
    err = np.abs(lb - lf)
    q = float(np.quantile(err, 0.9999))
    opt = nat.ns_default_options()
    margin = opt.reeval_margin + opt.reeval_rel * np.abs(lf)
    assert 2 * q < float(margin.min()), (q, float(margin.min()), float(lf.min()), float(lf.max()))
    assert np.all(err < margin), float(np.max(err - margin))
    # the 16-bit stage's error against its own margin
    l2 = torch.zeros(len(x), device="cuda")
    nat.ns_mlp_loglike(p, img, xt, l2, precision=3)
    torch.cuda.synchronize()
    e2 = np.abs(l2.cpu().numpy().astype(np.float64) - lf)
    margin2 = opt.reeval2_margin + opt.reeval2_rel * np.abs(lf)
    assert 2 * float(np.quantile(e2, 0.9999)) < float(margin2.min()), (float(np.quantile(e2, 0.9999)),
                                                                        float(margin2.min()))
    assert np.all(e2 < margin2)


def test_cluster_option_validation(nat):
    """mlp_cluster must divide every layer's 128-row tile count and needs a
    tensor-core path; the automatic choice takes 4 CTAs per run while they fit
    the SMs and falls back to one CTA per run."""
    small = _small_emulator()          # one tile row per layer: no split
    big = W.mlp_emulator(1)            # 4 / 4 / 4 / 4 / 16 tile rows
    bad = [(small, dict(precision=1, mlp_cluster=2)), (big, dict(precision=0, mlp_cluster=4)),
           (big, dict(precision=1, mlp_cluster=3))]
    for p, kw in bad:
        with pytest.raises(nat.NSError) as ei:
            nat.ns_create_batch([(p, 200, 20, 10, 1e-2, 1)], nat.ns_default_options(**kw))
        assert ei.value.status == nat.NS_ERR_ARG
    # precision 2 needs BF16-valued weights
    q = _small_emulator()
    q.mlp.weights = [w * np.float32(1.0 + 1e-3) for w in q.mlp.weights]
    with pytest.raises(nat.NSError):
        nat.ns_create_batch([(q, 200, 20, 10, 1e-2, 1)], nat.ns_default_options(precision=2))
    # automatic: a small batch runs, one CTA per run for a network that cannot split
    for p in (small, big):
        h = nat.ns_create_batch([(p, 200, 20, 10, 1e-2, 1)],
                                nat.ns_default_options(precision=1, max_iter=2, chunk_iters=2))
        nat.ns_run(h, check=False)
        r = nat.ns_summary(h, 0)
        nat.ns_destroy(h)
        assert r["n_iter"] == 2 and r["n_cand_bf16"] > 0
