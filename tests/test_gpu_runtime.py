"""GPU tests of the batched solve and the continuous-batching server: results match
solving each problem alone (bit for bit) and the FP64 oracle (within the bars)."""
import numpy as np
import pytest

from oracle import progot_oracle as O
from paper_2406_05061_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nat():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2406_05061_gb300 import native
    native.lib()
    return native


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def schedule(p, K=4):
    """eps_k interpolating from 5 eps0 to sigma (Alg. 4's end points without the grid search),
    eps0 = mean cost(X, Y)/20 and sigma = mean cost(Y, Y)/20 in closed form."""
    x, y = p.x.astype(np.float64), p.y.astype(np.float64)
    mc = lambda u, v: np.mean(np.sum(u**2, 1)) + np.mean(np.sum(v**2, 1)) - 2 * u.mean(0) @ v.mean(0)
    al = O.alpha_schedule(K)
    t = O.progress_times(al)
    eps = (1 - t) * 5 * mc(x, y) / 20 + t * mc(y, y) / 20
    return al, eps


def batch(count=10, seed=5):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n, m = (int(v) for v in np.exp(rng.uniform(np.log(128), np.log(1500), 2)))
        d = int(rng.choice([2, 16, 64]))
        out.append(W.gmm_pair(n, m, d, seed=100 + i, k=3))
    return out


def map_rms_rel(T, R, Y):
    Y = np.asarray(Y, dtype=np.float64)
    return float(np.sqrt(np.mean(np.sum((np.asarray(T) - R) ** 2, 1))) / np.sqrt(np.mean(np.sum((Y - Y.mean(0)) ** 2, 1))))


@pytest.mark.parametrize("precision,tau", [("bf16x3", 1e-4), ("fp32", 1e-5)])
def test_batched_equals_single(nat, precision, tau):
    probs = batch()
    K = 4
    specs = []
    for p in probs:
        al, eps = schedule(p, K)
        specs.append(dict(x=dev(p.x), y=dev(p.y), alpha=al, eps=eps, tau=[tau] * K))
    nat.set_batch_engine("streams")  # the per-problem engine is the bit-identical one
    try:
        res = nat.progot_solve_batched(specs, max_iter=5000, precision=precision, n_streams=4)
    finally:
        nat.set_batch_engine("persistent")
    for sp, r in zip(specs, res):
        assert r["status"] == nat.PROGOT_OK
        solo = nat.progot_solve(sp["x"], sp["y"], sp["alpha"], sp["eps"], sp["tau"], max_iter=5000, precision=precision)
        assert torch.equal(solo.x_out, r["x_out"])
        assert torch.equal(solo.g_all, r["g_all"])
        assert list(solo.iters) == r["iters"]


def test_batched_parity_with_oracle(nat):
    probs = [W.gmm_pair(300, 260, 16, seed=7, k=3), W.gmm_pair(200, 333, 2, seed=8, k=2),
             W.gmm_pair(257, 129, 64, seed=9, k=3)]
    K = 3
    specs, refs = [], []
    for p in probs:
        al, eps = schedule(p, K)
        specs.append(dict(x=dev(p.x), y=dev(p.y), alpha=al, eps=eps, tau=[1e-4] * K))
        refs.append(O.progot(None, p.x, None, p.y, eps, al, [1e-6] * K))
    res = nat.progot_solve_batched(specs, max_iter=5000, precision="bf16x3", n_streams=3)
    for p, r, ref in zip(probs, res, refs):
        assert map_rms_rel(r["x_out"].cpu().numpy(), ref.x_out, p.y) <= 1e-3


def test_server_results_same_alone_and_in_mix(nat):
    probs = batch(12, seed=11)
    K = 4
    budget = 256 << 20
    srv = nat.Server(budget, n_workers=4, precision="bf16x3", max_iter=5000)
    try:
        ids = []
        for p in probs:
            al, eps = schedule(p, K)
            ids.append((p, al, eps, srv.submit(p.x, p.y, al, eps, [1e-4] * K)))
        outs = [(p, al, eps, srv.wait(i)) for p, al, eps, i in ids]
        st = srv.stats()
        assert st["completed"] == len(probs) and st["in_flight"] == 0 and st["bytes_in_use"] == 0
        assert 0 < st["peak_bytes"] <= budget
    finally:
        srv.close()
    for p, al, eps, o in outs:
        assert o["status"] == nat.PROGOT_OK and o["latency_ms"] > 0
        solo = nat.progot_solve(dev(p.x), dev(p.y), al, eps, [1e-4] * K, max_iter=5000, precision="bf16x3")
        np.testing.assert_array_equal(o["x_out"], solo.x_out.cpu().numpy())
        np.testing.assert_array_equal(o["g_all"], solo.g_all.cpu().numpy())


def test_server_memory_budget_serialises_large_requests(nat):
    """A budget that holds one request at a time still completes them all, in order."""
    probs = [W.gmm_pair(1024, 1024, 64, seed=20 + i, k=3) for i in range(3)]
    K = 2
    one = None
    srv = None
    try:
        al, eps = schedule(probs[0], K)
        # size the budget from the library's own workspace query: ~1.5 requests fit
        ws = nat.workspace_size(1024, 1024, 64, "bf16x3")
        one = ws + 4 * (2 * 1024 * 64 + 1024 * 64 + K * 1024 + 1024) + 8 * 256
        srv = nat.Server(int(one * 1.5), n_workers=3, precision="bf16x3", max_iter=5000)
        ids = [srv.submit(p.x, p.y, al, eps, [1e-4] * K) for p in probs]
        outs = [srv.wait(i) for i in ids]
        assert all(o["status"] == nat.PROGOT_OK for o in outs)
        assert srv.stats()["peak_bytes"] <= int(one * 1.5)
    finally:
        if srv is not None:
            srv.close()


def test_server_rejects_request_over_budget(nat):
    srv = nat.Server(1 << 20, n_workers=1)
    try:
        p = W.gmm_pair(4096, 4096, 64, seed=1, k=2)
        al, eps = schedule(p, 2)
        with pytest.raises(nat.ProgOTError) as ei:
            srv.submit(p.x, p.y, al, eps, [1e-4] * 2)
        assert ei.value.code == nat.PROGOT_ERR_OOM
    finally:
        srv.close()
