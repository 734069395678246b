"""The persistent batched engine (one launch over many problems, Alg. 2 with each step's
Alg. 1 loop as phases of a device work queue) against the FP64 oracle, against the
single-problem path, alone and in a mix (bit for bit), across column segmentations, and
at the edge cases of the stop test."""
import numpy as np
import pytest

from oracle import progot_oracle as O
from paper_2406_05061_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_MIXED = 1e-3


@pytest.fixture(scope="module")
def nat():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2406_05061_gb300 import native
    native.lib()
    yield native
    native.set_batch_engine("persistent")


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def host(t):
    return t.detach().cpu().numpy().astype(np.float64)


def schedule(p, K):
    """eps_k from 5 eps0 to sigma (closed-form end points of Alg. 4), constant-speed alpha."""
    x, y = p.x.astype(np.float64), p.y.astype(np.float64)
    mc = lambda u, v: np.mean(np.sum(u**2, 1)) + np.mean(np.sum(v**2, 1)) - 2 * u.mean(0) @ v.mean(0)
    al = O.alpha_schedule(K)
    t = O.progress_times(al)
    return al, (1 - t) * 5 * mc(x, y) / 20 + t * mc(y, y) / 20


def map_rms_rel(T, R, Y):
    Y = np.asarray(Y, dtype=np.float64)
    return float(np.sqrt(np.mean(np.sum((np.asarray(T) - R) ** 2, 1))) / np.sqrt(np.mean(np.sum((Y - Y.mean(0)) ** 2, 1))))


def marginal_l1(X, Y, f, g, eps, a=None, b=None):
    C = O.CostOperator(X, Y)
    n, m = C.n, C.m
    a = np.full(n, 1.0 / n) if a is None else a
    b = np.full(m, 1.0 / m) if b is None else b
    return float(np.abs(O.row_marginal(C, f, g, eps) - a).sum() + np.abs(O.col_marginal(C, f, g, eps) - b).sum())


def mixed_batch(count, seed, dims=(16, 64), lo=100, hi=1400):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n, m = (int(v) for v in np.exp(rng.uniform(np.log(lo), np.log(hi), 2)))
        d = int(rng.choice(dims))
        out.append(W.gmm_pair(n, m, d, seed=1000 * seed + i, k=3))
    return out


def specs_of(probs, K, tau=1e-4):
    specs = []
    for p in probs:
        al, eps = schedule(p, K)
        specs.append(dict(x=dev(p.x), y=dev(p.y), alpha=al, eps=eps, tau=[tau] * K))
    return specs


def test_batch_parity_with_oracle_every_step(nat):
    """Each problem of a mixed batch (ragged n, m; d in {1, 5, 16, 64}) against the oracle:
    the final map within the mixed bar of the oracle's own solve, and the last step's
    coupling (X^(K-1), Y, f, g_K) with both marginals recomputed in float64 by the oracle."""
    probs = [W.gmm_pair(300, 260, 16, seed=7, k=3), W.gmm_pair(129, 517, 64, seed=8, k=2),
             W.gmm_pair(257, 129, 5, seed=9, k=3), W.gmm_pair(77, 90, 1, seed=10, k=2),
             W.gmm_pair(640, 384, 64, seed=11, k=4)]
    K = 3
    specs = specs_of(probs, K)
    plan = nat.BatchPlan(specs, max_iter=5000, precision="bf16x3")
    plan.run()
    res = plan.collect()
    plan.close()
    # the GPU's own X^(K-1): the same batch with the schedules cut after K - 1 steps runs the
    # same arithmetic for those steps (a problem's results depend only on itself)
    cut = [dict(sp, alpha=sp["alpha"][:K - 1], eps=sp["eps"][:K - 1], tau=sp["tau"][:K - 1]) for sp in specs]
    plan = nat.BatchPlan(cut, max_iter=5000, precision="bf16x3")
    plan.run()
    res_cut = plan.collect()
    plan.close()
    for p, sp, r, rc in zip(probs, specs, res, res_cut):
        assert r["status"] == nat.PROGOT_OK
        assert torch.equal(r["g_all"][:K - 1], rc["g_all"])
        ref = O.progot(None, p.x, None, p.y, sp["eps"], sp["alpha"], [1e-6] * K)
        assert map_rms_rel(host(r["x_out"]), ref.x_out, p.y) <= TOL_MIXED
        # the last step's coupling (X^(K-1), Y, f, g_K), both marginals in float64
        assert marginal_l1(host(rc["x_out"]), p.y, host(r["f_last"]), host(r["g_all"])[K - 1],
                           sp["eps"][K - 1]) <= TOL_MIXED


def test_batch_matches_single_problem_path(nat):
    """The persistent engine and progot_solve on the same problems: maps within the mixed
    bar of each other, iteration counts within a few of each other."""
    probs = mixed_batch(8, seed=3)
    K = 4
    specs = specs_of(probs, K)
    res = nat.progot_solve_batched(specs, max_iter=5000, precision="bf16x3")
    for p, sp, r in zip(probs, specs, res):
        assert r["status"] == nat.PROGOT_OK
        solo = nat.progot_solve(sp["x"], sp["y"], sp["alpha"], sp["eps"], sp["tau"], max_iter=5000, precision="bf16x3")
        assert map_rms_rel(host(r["x_out"]), host(solo.x_out), p.y) <= TOL_MIXED
        assert all(abs(a - b) <= max(3, 0.1 * b) for a, b in zip(r["iters"], solo.iters))


def test_batch_results_same_alone_and_in_mix(nat):
    """A problem's results depend only on itself: alone in a batch of one and among 11
    others, bit for bit; two replays of the captured graph agree too."""
    probs = mixed_batch(12, seed=5)
    K = 3
    specs = specs_of(probs, K)
    plan = nat.BatchPlan(specs, max_iter=5000)
    plan.run()
    mix = plan.collect()
    plan.run()
    again = plan.collect()
    plan.close()
    for i in (0, 5, 11):
        solo_plan = nat.BatchPlan([specs[i]], max_iter=5000)
        solo_plan.run(graph=False)
        alone = solo_plan.collect()[0]
        solo_plan.close()
        assert torch.equal(alone["x_out"], mix[i]["x_out"])
        assert torch.equal(alone["g_all"], mix[i]["g_all"])
        assert alone["iters"] == mix[i]["iters"]
    for a, b in zip(mix, again):
        assert torch.equal(a["x_out"], b["x_out"]) and torch.equal(a["g_all"], b["g_all"])


@pytest.mark.parametrize("target", [1, 8, 256])
def test_batch_column_segments(nat, target):
    """Sweep tasks cut into 1 .. 8 column segments (combined in segment order) give maps
    within the mixed bar of the oracle; the wide problems get several segments."""
    probs = [W.gmm_pair(130, 1900, 64, seed=21, k=3), W.gmm_pair(1100, 140, 16, seed=22, k=3),
             W.gmm_pair(500, 700, 64, seed=23, k=3)]
    K = 2
    specs = specs_of(probs, K)
    plan = nat.BatchPlan(specs, max_iter=5000)
    plan.set_target(target)
    plan.run()
    res = plan.collect()
    plan.close()
    for p, sp, r in zip(probs, specs, res):
        ref = O.progot(None, p.x, None, p.y, sp["eps"], sp["alpha"], [1e-6] * K)
        assert map_rms_rel(host(r["x_out"]), ref.x_out, p.y) <= TOL_MIXED


def test_batch_weights_and_plain_entropic_map(nat):
    """Non-uniform weights a, b and K = 1, alpha = 1 (ProgOT reduces to the entropic map):
    the GPU potentials give marginals within the bar of (a, b), the map matches the
    oracle's entropic map from its own Sinkhorn potentials."""
    p = W.gmm_pair(400, 333, 16, seed=31, k=3)
    rng = np.random.default_rng(0)
    a = rng.uniform(0.5, 1.5, 400)
    a /= a.sum()
    b = rng.uniform(0.5, 1.5, 333)
    b /= b.sum()
    eps = 0.05 * O.mean_cost(p.x, p.y)
    spec = dict(x=dev(p.x), y=dev(p.y), alpha=[1.0], eps=[eps], tau=[1e-4], a=dev(a), b=dev(b))
    plan = nat.BatchPlan([spec], max_iter=5000)
    plan.run()
    r = plan.collect()[0]
    plan.close()
    assert r["status"] == nat.PROGOT_OK
    f, g = host(r["f_last"]), host(r["g_all"])[0]
    assert marginal_l1(p.x, p.y, f, g, eps, a, b) <= TOL_MIXED
    ref = O.sinkhorn(a, p.x, b, p.y, eps, 1e-7, max_iter=20000)
    assert map_rms_rel(host(r["x_out"]), O.entropic_map(p.x, p.y, ref.g, eps), p.y) <= TOL_MIXED


def test_batch_stop_test_edge_cases(nat):
    """max_iter = 0 ends every step after the first error measurement (NOT_CONVERGED,
    zero iterations, the map still applied); tau = 0 with a small max_iter runs exactly
    max_iter iterations; a NaN input stops its problem with NUMERIC while the others
    finish."""
    probs = mixed_batch(3, seed=9)
    K = 2
    specs = specs_of(probs, K)
    plan = nat.BatchPlan(specs, max_iter=0)
    plan.run()
    res = plan.collect(check=False)
    plan.close()
    assert all(r["status"] == nat.PROGOT_ERR_NOT_CONVERGED and r["iters"] == [0, 0] for r in res)
    specs0 = [dict(s, tau=[0.0] * K) for s in specs]
    plan = nat.BatchPlan(specs0, max_iter=7)
    plan.run()
    res = plan.collect(check=False)
    plan.close()
    assert all(r["iters"] == [7, 7] for r in res)
    xb = probs[1].x.copy()
    xb[3, 0] = np.nan
    bad = [specs[0], dict(specs[1], x=dev(xb)), specs[2]]
    plan = nat.BatchPlan(bad, max_iter=5000)
    plan.run()
    res = plan.collect(check=False)
    plan.close()
    assert res[1]["status"] == nat.PROGOT_ERR_NUMERIC
    assert res[0]["status"] == nat.PROGOT_OK and res[2]["status"] == nat.PROGOT_OK


def test_batch_autotune_picks_a_measured_target(nat):
    """The tuner times complete runs for each target and keeps the fastest; results after
    tuning stay within the bar of the oracle."""
    probs = mixed_batch(16, seed=13, lo=128, hi=2048)
    K = 2
    specs = specs_of(probs, K)
    plan = nat.BatchPlan(specs, max_iter=5000)
    target, ms = plan.autotune()
    assert target in (1, 4, 16, 64, 256) and ms > 0
    plan.run()
    res = plan.collect()
    plan.close()
    for i in (0, 7):
        p, sp = probs[i], specs[i]
        ref = O.progot(None, p.x, None, p.y, sp["eps"], sp["alpha"], [1e-6] * K)
        assert map_rms_rel(host(res[i]["x_out"]), ref.x_out, p.y) <= TOL_MIXED


def test_streams_engine_still_bit_identical_to_single(nat):
    """With the per-problem stream engine, batched results equal solving alone, bit for bit."""
    probs = mixed_batch(6, seed=17, dims=(2, 16, 64))
    K = 3
    specs = specs_of(probs, K)
    nat.set_batch_engine("streams")
    try:
        res = nat.progot_solve_batched(specs, max_iter=5000, precision="bf16x3", n_streams=3)
    finally:
        nat.set_batch_engine("persistent")
    for sp, r in zip(specs, res):
        solo = nat.progot_solve(sp["x"], sp["y"], sp["alpha"], sp["eps"], sp["tau"], max_iter=5000, precision="bf16x3")
        assert torch.equal(solo.x_out, r["x_out"]) and torch.equal(solo.g_all, r["g_all"])
