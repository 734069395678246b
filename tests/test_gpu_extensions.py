"""GPU parity of the widened entry points against the FP64 oracle: coupling metrics
(Sec. 5.2), the Sinkhorn divergence (eq. (8)), the theta-scaled eps rule (Sec. 5.2),
the linear tau schedule (Sec. 4) and the coupling diagonal of the blur benchmark
(Sec. 5.3, Prop. 3). Sizes span several 128-row tiles with ragged tails."""
import numpy as np
import pytest

from oracle import progot_oracle as O
from paper_2406_05061_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_FP32 = 1e-4
TOL_MIXED = 1e-3


@pytest.fixture(scope="module")
def nat():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2406_05061_gb300 import native
    native.lib()
    return native


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def host(t):
    return t.detach().cpu().numpy().astype(np.float64)


def map_rms_rel(T_gpu, T_ref, Y):
    Y = np.asarray(Y, dtype=np.float64)
    spread = np.sqrt(np.mean(np.sum((Y - Y.mean(0)) ** 2, 1)))
    return float(np.sqrt(np.mean(np.sum((np.asarray(T_gpu) - np.asarray(T_ref)) ** 2, 1))) / spread)


def _weights(rng, k):
    w = rng.uniform(0.5, 1.5, k)
    return (w / w.sum()).astype(np.float32)


# ------------------------------------------------------------ coupling metrics
@pytest.mark.parametrize("n,m,d,weighted", [(700, 530, 5, False), (300, 1000, 64, True), (129, 257, 2, True)])
def test_coupling_metrics_parity(nat, n, m, d, weighted):
    p = W.gmm_pair(n, m, d, seed=40 + d, k=3)
    rng = np.random.default_rng(41)
    a = _weights(rng, n) if weighted else None
    b = _weights(rng, m) if weighted else None
    eps = 0.05 * O.mean_cost(p.x, p.y)
    sk = O.sinkhorn(a, p.x, b, p.y, eps, 1e-7)
    # the GPU reads float32 potentials: give the oracle the very same values
    f32, g32 = sk.f.astype(np.float32), sk.g.astype(np.float32)
    f, g = f32.astype(np.float64), g32.astype(np.float64)
    met = nat.coupling_metrics(dev(p.x), dev(p.y), dev(f32), dev(g32), eps,
                               a=None if a is None else dev(a), b=None if b is None else dev(b))
    cost = O.coupling_cost(p.x, p.y, f, g, eps)
    ent = O.coupling_entropy(p.x, p.y, f, g, eps)
    dual = O.dual_objective(a, p.x, b, p.y, f, g, eps)
    C = O.CostOperator(p.x, p.y)
    r, c = O.row_marginal(C, f, g, eps), O.col_marginal(C, f, g, eps)
    aa = np.full(n, 1.0 / n) if a is None else a.astype(np.float64)
    bb = np.full(m, 1.0 / m) if b is None else b.astype(np.float64)
    assert met["transport_cost"] == pytest.approx(cost, rel=TOL_FP32)
    assert met["entropy"] == pytest.approx(ent, rel=TOL_FP32)
    assert met["dual"] == pytest.approx(dual, rel=TOL_FP32, abs=TOL_FP32 * cost)
    assert met["mass"] == pytest.approx(float(r.sum()), rel=TOL_FP32)
    assert met["err_row"] == pytest.approx(float(np.abs(r - aa).sum()), abs=TOL_FP32)
    assert met["err_col"] == pytest.approx(float(np.abs(c - bb).sum()), abs=TOL_FP32)


def test_coupling_metrics_at_scale(nat):
    # 4096 x 4096 d = 64 mixture (32 x 32 tiles) against the blocked float64 definitions
    p = W.gmm_pair(4096, 4096, 64, seed=42, k=8)
    eps = 0.05 * O.mean_cost(p.x, p.y)
    res = nat.sinkhorn_potentials(dev(p.x), dev(p.y), eps, 1e-5, max_iter=5000)
    f, g = host(res.f), host(res.g)
    met = nat.coupling_metrics(dev(p.x), dev(p.y), res.f, res.g, eps)
    assert met["transport_cost"] == pytest.approx(O.coupling_cost(p.x, p.y, f, g, eps), rel=TOL_FP32)
    assert met["entropy"] == pytest.approx(O.coupling_entropy(p.x, p.y, f, g, eps), rel=TOL_FP32)
    assert met["err_row"] + met["err_col"] <= 1e-5 + TOL_FP32


# ------------------------------------------------------- Sinkhorn divergence
@pytest.mark.parametrize("precision,tol", [("fp32", TOL_FP32), ("bf16x3", TOL_MIXED)])
def test_sinkhorn_divergence_parity(nat, precision, tol):
    p = W.gmm_pair(700, 450, 16, seed=43, k=3)
    eps = O.eps_divergence(p.y)
    tau = 1e-5
    D, parts, its, st = nat.sinkhorn_divergence(dev(p.x), dev(p.y), eps, tau, max_iter=20000, precision=precision)
    assert st == nat.PROGOT_OK, nat.last_error()
    Dr, pr, _ = O.sinkhorn_divergence(None, p.x, None, p.y, eps, 1e-9, max_iter=50000)
    scale = max(abs(v) for v in pr)
    for v, w in zip(parts, pr):
        assert abs(v - w) <= tol * scale
    assert abs(D - Dr) <= tol * scale
    assert D > 0
    # the self terms use the symmetric fixed point: tens of iterations, not thousands
    assert max(its[1:]) < 200


def test_sinkhorn_divergence_of_a_translate(nat):
    # D(X, X + v) = |v|^2 for every eps (the linear cost terms go into the potentials)
    rng = np.random.default_rng(44)
    x = rng.standard_normal((500, 8)).astype(np.float32)
    v = np.linspace(-0.5, 0.5, 8).astype(np.float32)
    D, parts, _, st = nat.sinkhorn_divergence(dev(x), dev(x + v), 2.0, 1e-5, max_iter=20000)
    assert st == nat.PROGOT_OK, nat.last_error()
    assert D == pytest.approx(float(v.astype(np.float64) @ v), rel=1e-3)


# ------------------------------------------------------------ theta rule
@pytest.mark.parametrize("precision,tol", [("fp32", TOL_FP32), ("bf16x3", TOL_MIXED)])
def test_progot_solve_theta_parity(nat, precision, tol):
    # theta = 1 puts eps_k at the usual mean-cost / 20 level, where a solve stopped at
    # tau = 1e-5 determines the map to the parity tolerance; smaller theta slows
    # Sinkhorn down (thousands of iterations) and the float32 and float64 runs then stop
    # at different points of a long, flat approach
    p = W.gmm_pair(600, 450, 16, seed=45, k=4)
    K, theta = 4, 1.0
    alpha = O.alpha_schedule(K)
    # both sides run the same linear tau schedule (equal accuracy); the mixed path ends
    # at 1e-4, the threshold its bf16 hi/lo products reach reliably
    tau = O.tau_schedule(K, 1e-4, 1e-5) if precision == "fp32" else O.tau_schedule(K, 1e-3, 1e-4)
    res, eps = nat.progot_solve_theta(dev(p.x), dev(p.y), alpha, theta, tau, max_iter=20000, precision=precision)
    assert res.status == nat.PROGOT_OK, nat.last_error()
    ref = O.progot(None, p.x, None, p.y, O.eps_theta_rule(theta, p.y), alpha, tau)
    # eps_1 comes from the input cloud itself: float64 closed form vs the definition
    assert eps[0] == pytest.approx(ref.eps_used[0], rel=1e-9)
    np.testing.assert_allclose(eps, ref.eps_used, rtol=10 * tol)
    assert map_rms_rel(host(res.x_out), ref.x_out, p.y) <= tol
    # teacher forcing: the rule on the GPU's own X^(K) gives the GPU's eps_K
    assert eps[-1] == pytest.approx(theta * O.mean_cost(host(res.x_last), p.y) / 20, rel=1e-6)


def test_progot_solve_theta_matches_progot_solve_with_its_eps(nat):
    # the theta path and the explicit-eps path run the same kernels: with the eps the
    # rule produced, progot_solve must give the same result bit for bit
    p = W.gmm_pair(500, 380, 24, seed=46, k=3)
    K = 3
    alpha = O.alpha_schedule(K, "accelerated")
    tau = [1e-5] * K
    r1, eps = nat.progot_solve_theta(dev(p.x), dev(p.y), alpha, 2.0 ** -4, tau, max_iter=20000)
    r2 = nat.progot_solve(dev(p.x), dev(p.y), alpha, eps, tau, max_iter=20000)
    assert torch.equal(r1.x_out, r2.x_out) and torch.equal(r1.g_all, r2.g_all)
    assert r1.iters == r2.iters


# ------------------------------------------------------------ coupling diagonal
def test_coupling_diagonal_parity_and_identity_recovery(nat):
    # Prop. 3: images and their blurs are optimally coupled by Id / n
    p = W.blur_pair(1500, side=8, sigma=2.0, seed=47)
    eps = 2.0 ** -6 * O.mean_cost(p.x, p.y) / 20
    res = nat.sinkhorn_potentials(dev(p.x), dev(p.y), eps, 1e-4, max_iter=30000)
    assert res.status in (nat.PROGOT_OK, nat.PROGOT_ERR_NOT_CONVERGED), nat.last_error()
    logd = torch.empty(p.n, dtype=torch.float32, device="cuda")
    tr, kl = nat.coupling_diagonal(dev(p.x), dev(p.y), res.f, res.g, eps, log_diag=logd)
    tr_r, kl_r = O.diagonal_metrics(p.x, p.y, host(res.f), host(res.g), eps)
    ld_r = O.coupling_diagonal(p.x, p.y, host(res.f), host(res.g), eps)
    np.testing.assert_allclose(host(logd), ld_r, rtol=1e-5, atol=1e-4)
    assert tr == pytest.approx(tr_r, rel=1e-6)
    assert kl == pytest.approx(kl_r, rel=1e-6, abs=1e-7)
    # a valid coupling: KL(Id/n || P) >= 0 (Gibbs) and Tr(P) <= 1, and at this small eps
    # the diagonal carries most of the mass (the independent coupling has Tr = 1/n)
    assert 0.5 < tr <= 1.0 + 1e-4 and 0 <= kl


# ------------------------------------------------- large d: A streamed with B
@pytest.mark.parametrize("n,m,d", [(300, 520, 320), (700, 900, 1024), (257, 130, 1000)])
def test_large_d_streamed_operand_parity_bf16x3(nat, n, m, d):
    # above d = 256 the bf16 hi/lo A operand of a row block no longer fits next to two B
    # stages, so the tensor-core sweep streams A one K block per stage
    p = W.gmm_pair(n, m, d, seed=n + m + d, k=4)
    eps = 0.05 * O.mean_cost(p.x, p.y)
    res = nat.sinkhorn_potentials(dev(p.x), dev(p.y), eps, 1e-4, max_iter=5000, precision="bf16x3")
    assert res.status == nat.PROGOT_OK, nat.last_error()
    ref = O.sinkhorn(None, p.x, None, p.y, eps, 1e-6, max_iter=5000)
    f, g = host(res.f), host(res.g)
    C = O.CostOperator(p.x, p.y)
    err = float(np.abs(O.row_marginal(C, f, g, eps) - 1.0 / n).sum() + np.abs(O.col_marginal(C, f, g, eps) - 1.0 / m).sum())
    assert err <= TOL_MIXED
    T_gpu = O.entropic_map(p.x, p.y, g, eps)
    T_ref = O.entropic_map(p.x, p.y, ref.g, eps)
    assert map_rms_rel(T_gpu, T_ref, p.y) <= TOL_MIXED


def test_large_d_map_step_parity_bf16x3(nat):
    # one ProgOT step at d = 1024: tensor-core LSE pass with streamed A, then the map
    p = W.blur_pair(600, side=32, sigma=2.0, seed=48)
    eps = 0.05 * O.mean_cost(p.x, p.y)
    alpha = [0.5, 1.0]
    res = nat.progot_solve(dev(p.x), dev(p.y), alpha, [eps, eps], [1e-4, 1e-4], max_iter=5000, precision="bf16x3")
    assert res.status == nat.PROGOT_OK, nat.last_error()
    ref = O.progot(None, p.x, None, p.y, [eps, eps], alpha, [1e-6, 1e-6])
    assert map_rms_rel(host(res.x_out), ref.x_out, p.y) <= TOL_MIXED


def test_overflowing_warm_start_keeps_iterating(nat):
    # potentials far above feasibility make the first row sums overflow float32; the loop
    # must treat that as "error above tau" and reach the zero-start coupling (oracle)
    p = W.gmm_pair(400, 300, 16, seed=49, k=3)
    eps = 0.05 * O.mean_cost(p.x, p.y)
    cmax = float(O.cost_matrix_rows(p.x, p.y).max())
    f0 = np.full(p.n, cmax, dtype=np.float32)
    g0 = np.full(p.m, cmax, dtype=np.float32)
    res = nat.sinkhorn_potentials(dev(p.x), dev(p.y), eps, 1e-5, max_iter=5000, f=dev(f0), g=dev(g0))
    assert res.status == nat.PROGOT_OK, nat.last_error()
    ref = O.sinkhorn(None, p.x, None, p.y, eps, 1e-7)
    T = O.entropic_map(p.x, p.y, host(res.g), eps)
    assert map_rms_rel(T, O.entropic_map(p.x, p.y, ref.g, eps), p.y) <= TOL_FP32


@pytest.mark.parametrize("d", [5, 64])
def test_coupling_cost_against_the_original_cloud(nat, d):
    # ProgOT's final coupling lives on X^(K) and is measured against the original X
    p = W.gmm_pair(600, 450, d, seed=50 + d, k=3)
    K = 3
    alpha = O.alpha_schedule(K)
    e0 = O.mean_cost(p.x, p.y) / 20
    res = nat.progot_solve(dev(p.x), dev(p.y), alpha, [3 * e0, 2 * e0, e0], [1e-5] * K, max_iter=5000)
    assert res.status == nat.PROGOT_OK, nat.last_error()
    xl, f, g = host(res.x_last), host(res.f_last), host(res.g_all[K - 1])
    met = nat.coupling_metrics(res.x_last, dev(p.y), res.f_last, res.g_all[K - 1], e0, x_cost=dev(p.x))
    want = O.coupling_cost(xl, p.y, f, g, e0, X_cost=p.x)
    assert met["transport_cost"] == pytest.approx(want, rel=TOL_FP32)
    assert met["entropy"] == pytest.approx(O.coupling_entropy(xl, p.y, f, g, e0), rel=TOL_FP32)
    # without x_cost the same call measures the cost on X^(K) itself
    met2 = nat.coupling_metrics(res.x_last, dev(p.y), res.f_last, res.g_all[K - 1], e0)
    assert met2["transport_cost"] == pytest.approx(O.coupling_cost(xl, p.y, f, g, e0), rel=TOL_FP32)


@pytest.mark.parametrize("nq,m,d", [(1000, 700, 64), (333, 517, 17), (129, 130, 2), (4096, 3000, 48)])
def test_map_step_on_tensor_cores(nat, nq, m, d):
    # Alg. 3 with the tcgen05 map kernel (S = X Y^T and P Y on the tensor cores, d <= 64)
    # against the oracle's Alg. 3 from the same g^(k), and against the float32 P Y path
    p = W.gmm_pair(nq, m, d, seed=nq + m + d, k=4)
    K = 2
    alpha = O.alpha_schedule(K)
    e0 = O.mean_cost(p.x, p.y) / 20
    eps = [2 * e0, e0]
    res = nat.progot_solve(dev(p.x), dev(p.y), alpha, eps, [1e-4] * K, max_iter=5000, precision="bf16x3")
    assert res.status == nat.PROGOT_OK, nat.last_error()
    g_all = host(res.g_all)
    xq = W.gmm_pair(nq, 10, d, seed=7 + d, k=4).x
    ref = O.progot_map(xq, p.y, g_all, eps, alpha)
    try:
        nat.set_map_tc(True)
        t_tc = host(nat.entropic_map_apply(dev(xq), dev(p.y), res.g_all, eps, alpha, precision="bf16x3"))
        nat.set_map_tc(False)
        t_f32 = host(nat.entropic_map_apply(dev(xq), dev(p.y), res.g_all, eps, alpha, precision="bf16x3"))
    finally:
        nat.set_map_tc(True)
    assert map_rms_rel(t_tc, ref, p.y) <= TOL_MIXED
    assert map_rms_rel(t_f32, ref, p.y) <= TOL_MIXED
    assert map_rms_rel(t_tc, t_f32, p.y) <= TOL_MIXED
    # in place (out aliasing the query points) gives the same result
    xq_dev = dev(xq)
    nat.entropic_map_apply(xq_dev, dev(p.y), res.g_all, eps, alpha, precision="bf16x3", out=xq_dev)
    assert map_rms_rel(host(xq_dev), t_tc, p.y) <= 1e-6


# ------------------------------------------- clouds far from the origin (centring)
@pytest.mark.parametrize("d,offset", [(32, 200.0), (300, 30.0)])
def test_tensor_core_path_far_from_the_origin(nat, d, offset):
    # the squared Euclidean cost and hence f, g are invariant under a common
    # translation; the tensor-core path centres its bf16 hi/lo operands, so a problem
    # moved far from the origin keeps the parity of the original (uncentred, the bf16x3
    # products of |x| |y| ~ d offset^2 would swamp the cost)
    p = W.gmm_pair(700, 600, d, seed=49 + d, k=4)
    v = np.full(d, offset, dtype=np.float64)
    x, y = p.x + v, p.y + v
    eps = 0.05 * O.mean_cost(p.x, p.y)
    res = nat.sinkhorn_potentials(dev(x), dev(y), eps, 1e-4, max_iter=5000, precision="bf16x3")
    assert res.status == nat.PROGOT_OK, nat.last_error()
    f, g = host(res.f), host(res.g)
    C = O.CostOperator(p.x, p.y)  # the same cost matrix
    err = float(np.abs(O.row_marginal(C, f, g, eps) - 1.0 / p.n).sum() +
                np.abs(O.col_marginal(C, f, g, eps) - 1.0 / p.m).sum())
    assert err <= TOL_MIXED
    ref = O.sinkhorn(None, p.x, None, p.y, eps, 1e-6, max_iter=5000)
    T_gpu = O.entropic_map(p.x, p.y, g, eps)
    assert map_rms_rel(T_gpu, O.entropic_map(p.x, p.y, ref.g, eps), p.y) <= TOL_MIXED


def test_progot_far_from_the_origin_matches_the_translate(nat):
    # Alg. 2 commutes with a common translation: X^(K)(X + v, Y + v) = X^(K)(X, Y) + v,
    # through the tensor-core map step (d <= 64)
    p = W.gmm_pair(900, 700, 16, seed=50, k=4)
    v = np.linspace(40.0, 80.0, 16)
    K = 3
    alpha = O.alpha_schedule(K)
    eps = [0.1 * O.mean_cost(p.x, p.y)] * K
    tau = [1e-4] * K
    res = nat.progot_solve(dev(p.x + v), dev(p.y + v), alpha, eps, tau, max_iter=5000, precision="bf16x3")
    assert res.status == nat.PROGOT_OK, nat.last_error()
    ref = O.progot(None, p.x, None, p.y, eps, alpha, [1e-6] * K)
    assert map_rms_rel(host(res.x_out) - v, ref.x_out, p.y) <= TOL_MIXED


# ------------------------------- more row blocks than SMs: whole row blocks in bands
@pytest.mark.parametrize("n,m,d", [(20000, 40000, 16), (39000, 20500, 320)])
def test_banded_work_split_sampled_parity(nat, n, m, d):
    # with at least G = 152 row blocks the tensor-core kernels hand whole row blocks to
    # the CTAs in bands (every CTA walks the column tiles together) and split only the
    # remaining row blocks; checked on rows and columns sampled and computed one by one
    # by the oracle from the GPU's potentials, and against the float32 path
    p = W.gmm_pair(n, m, d, seed=51 + d, k=4)
    x, y = dev(p.x), dev(p.y)
    eps = 0.1 * O.mean_cost(p.x[:2000], p.y[:2000])
    res = nat.sinkhorn_potentials(x, y, eps, 1e-4, max_iter=3000, precision="bf16x3")
    assert res.status == nat.PROGOT_OK, nat.last_error()
    f, g = host(res.f), host(res.g)
    rng = np.random.default_rng(52)
    X64, Y64 = p.x.astype(np.float64), p.y.astype(np.float64)
    rows, cols = rng.choice(n, 48, replace=False), rng.choice(m, 48, replace=False)
    r = np.exp((f[rows, None] + g[None, :] - O.cost_matrix_rows(X64[rows], Y64)) / eps).sum(1)
    c = np.exp((g[cols, None] + f[None, :] - O.cost_matrix_rows(Y64[cols], X64)) / eps).sum(1)
    # the last update was a g-update: column sums are exact up to rounding, row sums
    # carry the (converged) row error
    np.testing.assert_allclose(c * m, 1.0, rtol=2e-3)
    assert float(np.abs(r * n - 1.0).max()) <= 2e-2
    ref = nat.sinkhorn_potentials(x, y, eps, 1e-5, max_iter=3000, precision="fp32")
    T_tc = O.entropic_map(X64[rows], Y64, g, eps)
    T_32 = O.entropic_map(X64[rows], Y64, host(ref.g), eps)
    assert map_rms_rel(T_tc, T_32, p.y) <= TOL_MIXED
    # one map step (Alg. 3) on the tensor cores with the same split (d <= 64) or the
    # float32 P Y sweep after a banded log-sum-exp pass (d > 64)
    out = nat.entropic_map_apply(x, y, res.g.reshape(1, -1), [eps], [1.0], precision="bf16x3")
    assert map_rms_rel(host(out)[rows], T_tc, p.y) <= TOL_MIXED


# ------------------------------------------------ map Jacobian (conditional covariance)
@pytest.mark.parametrize("precision,h,tol", [("fp32", 3e-3, 2e-3), ("bf16x3", 3e-2, 2e-2)])
def test_map_jacobian_is_conditional_covariance(nat, precision, h, tol):
    # grad T_eps(x) = (2 / eps) Cov_p(x)(Y) for c = |x - y|^2 (the Lipschitz lemma of the
    # appendix, with the factor 2 of this cost): central differences of the GPU map on
    # query points against the covariance the oracle forms from the GPU's own g
    p = W.gmm_pair(600, 500, 3, seed=53, k=3)
    eps = 0.2 * O.mean_cost(p.x, p.y)
    res = nat.sinkhorn_potentials(dev(p.x), dev(p.y), eps, 1e-5, max_iter=5000, precision=precision)
    assert res.status == nat.PROGOT_OK, nat.last_error()
    g = host(res.g)
    d = 3
    xq = np.random.default_rng(54).normal(size=(6, d)) * 1.5
    pts = np.concatenate([xq[:, None, :] + s * h * np.eye(d)[None] for s in (1.0, -1.0)], axis=1).reshape(-1, d)
    T = host(nat.entropic_map_apply(dev(pts), dev(p.y), res.g.reshape(1, -1), [eps], [1.0],
                                    precision=precision)).reshape(6, 2, d, d)
    J = (T[:, 0] - T[:, 1]) / (2 * h)  # J[q, k, :] = dT / dx_k at point q
    Y64 = p.y.astype(np.float64)
    for q in range(6):
        logits = (g - np.sum((xq[q] - Y64) ** 2, 1)) / eps
        w = np.exp(logits - logits.max())
        w /= w.sum()
        mu = w @ Y64
        cov = (Y64 - mu).T @ ((Y64 - mu) * w[:, None])
        want = 2.0 / eps * cov
        assert np.abs(J[q].T - want).max() <= tol * np.abs(want).max() + 1e-6


# ---------------------------------------------------------------- one dimension
@pytest.mark.parametrize("precision,tol", [("fp32", TOL_FP32), ("bf16x3", TOL_MIXED)])
def test_one_dimensional_clouds(nat, precision, tol):
    # d = 1 (K padded to 64 on the tensor cores): Sinkhorn and a two-step ProgOT against
    # the oracle; in 1-D the entropic map is monotone, checked on the sorted queries
    p = W.gmm_pair(700, 530, 1, seed=55, k=3)
    eps = 0.05 * O.mean_cost(p.x, p.y)
    res = nat.sinkhorn_potentials(dev(p.x), dev(p.y), eps, 1e-5, max_iter=5000, precision=precision)
    assert res.status == nat.PROGOT_OK, nat.last_error()
    ref = O.sinkhorn(None, p.x, None, p.y, eps, 1e-7, max_iter=5000)
    T_gpu = O.entropic_map(p.x, p.y, host(res.g), eps)
    assert map_rms_rel(T_gpu, O.entropic_map(p.x, p.y, ref.g, eps), p.y) <= tol
    xs = np.sort(p.x[:, 0])[:, None]
    Ts = host(nat.entropic_map_apply(dev(xs), dev(p.y), res.g.reshape(1, -1), [eps], [1.0], precision=precision))
    assert np.all(np.diff(Ts[:, 0]) >= -tol * np.ptp(p.y))
    K = 2
    alpha = O.alpha_schedule(K)
    r2 = nat.progot_solve(dev(p.x), dev(p.y), alpha, [eps, eps / 2], [1e-5, 1e-5], max_iter=5000, precision=precision)
    assert r2.status == nat.PROGOT_OK, nat.last_error()
    o2 = O.progot(None, p.x, None, p.y, [eps, eps / 2], alpha, [1e-7, 1e-7])
    assert map_rms_rel(host(r2.x_out), o2.x_out, p.y) <= tol
