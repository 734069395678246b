"""Pins of the oracle's widened pieces (theta rule, tau schedule, Sinkhorn divergence,
coupling diagonal) against facts that do not come from the oracle: brute-force loops
on tiny inputs, exact invariances, limits and Gibbs' inequality. CPU only."""
import itertools
import math

import numpy as np
import pytest

from oracle import progot_oracle as O


def _rng(seed):
    return np.random.default_rng(seed)


# ------------------------------------------------------------ tau schedule (Sec. 4)
def test_tau_schedule_is_linear_between_its_ends():
    t = O.tau_schedule(6, 0.1, 1e-3)
    assert t[0] == pytest.approx(0.1, rel=1e-15) and t[-1] == pytest.approx(1e-3, rel=1e-12)
    steps = np.diff(t)
    np.testing.assert_allclose(steps, np.full(5, (1e-3 - 0.1) / 5), rtol=1e-12)
    assert np.all(steps < 0)
    assert O.tau_schedule(1, 0.1, 1e-3).tolist() == [1e-3]


# ------------------------------------------------ theta rule (Sec. 5.2, App. details)
def _brute_mean_cost(X, Y):
    tot = 0.0
    for x in X:
        for y in Y:
            tot += sum((float(u) - float(v)) ** 2 for u, v in zip(x, y))
    return tot / (len(X) * len(Y))


def test_theta_rule_uses_the_cloud_of_each_step():
    # eps_k = theta * sum_ij ||x^(k)_i - y_j||^2 / (20 n m) on the cloud solve k sees,
    # checked by a plain double loop on every step's input cloud
    rng = _rng(10)
    X, Y = rng.normal(size=(5, 2)), rng.normal(size=(4, 2)) * 1.5 + 2.0
    theta, K = 0.5, 3
    res = O.progot(None, X, None, Y, O.eps_theta_rule(theta, Y), O.alpha_schedule(K), [1e-10] * K)
    assert len(res.eps_used) == K
    for k in range(K):
        want = theta * _brute_mean_cost(res.x_steps[k], Y) / 20.0
        assert res.eps_used[k] == pytest.approx(want, rel=1e-12)
    # the cloud moves towards Y, so the regularisation shrinks along the path
    assert res.eps_used[0] > res.eps_used[1] > res.eps_used[2]


def test_theta_rule_single_step_is_plain_entropic_map():
    rng = _rng(11)
    X, Y = rng.normal(size=(9, 3)), rng.normal(size=(7, 3)) + 1.0
    theta = 2.0 ** -4
    eps = theta * _brute_mean_cost(X, Y) / 20.0
    res = O.progot(None, X, None, Y, O.eps_theta_rule(theta, Y), [1.0], [1e-12])
    sk = O.sinkhorn(None, X, None, Y, eps, 1e-12)
    np.testing.assert_allclose(res.x_out, O.entropic_map(X, Y, sk.g, eps), rtol=1e-9, atol=1e-9)


def test_theta_rule_translation_and_scale():
    rng = _rng(12)
    X, Y = rng.normal(size=(8, 2)), rng.normal(size=(6, 2)) + 1.0
    K, theta = 3, 0.25
    al, ta = O.alpha_schedule(K), [1e-11] * K
    base = O.progot(None, X, None, Y, O.eps_theta_rule(theta, Y), al, ta)
    v = np.array([3.0, -2.0])
    sh = O.progot(None, X + v, None, Y + v, O.eps_theta_rule(theta, Y + v), al, ta)
    np.testing.assert_allclose(sh.eps_used, base.eps_used, rtol=1e-10)
    np.testing.assert_allclose(sh.x_out, base.x_out + v, rtol=1e-8, atol=1e-8)
    s = 3.0
    sc = O.progot(None, s * X, None, s * Y, O.eps_theta_rule(theta, s * Y), al, ta)
    np.testing.assert_allclose(sc.eps_used, np.asarray(base.eps_used) * s * s, rtol=1e-10)
    np.testing.assert_allclose(sc.x_out, s * base.x_out, rtol=1e-8, atol=1e-8)


# ------------------------------------------------------- Sinkhorn divergence, eq. (8)
def test_divergence_of_a_translate_is_squared_shift():
    # cost |x_i - x_j - v|^2 = C_ij - 2 v.x_i + 2 v.x_j + |v|^2: the linear terms are
    # absorbed by the potentials, so OT(X, X + v) = OT(X, X) + |v|^2 for every eps and
    # the divergence is exactly |v|^2
    rng = _rng(20)
    X = rng.normal(size=(12, 3))
    v = np.array([0.7, -0.2, 0.4])
    for eps in (1.0, 5.0):
        D, parts, _ = O.sinkhorn_divergence(None, X, None, X + v, eps, 1e-12)
        assert D == pytest.approx(float(v @ v), rel=1e-9)
        assert parts[0] == pytest.approx(parts[1] + float(v @ v), rel=1e-9)


def test_divergence_of_a_cloud_with_itself_is_zero_and_symmetric():
    rng = _rng(21)
    X, Y = rng.normal(size=(10, 2)), rng.normal(size=(8, 2)) * 0.7 + 0.3
    D0, _, _ = O.sinkhorn_divergence(None, X, None, X, 0.2, 1e-12)
    assert abs(D0) < 1e-10
    Dxy, _, _ = O.sinkhorn_divergence(None, X, None, Y, 0.2, 1e-12)
    Dyx, _, _ = O.sinkhorn_divergence(None, Y, None, X, 0.2, 1e-12)
    assert Dxy > 0 and Dxy == pytest.approx(Dyx, rel=1e-9)


def test_divergence_large_eps_is_squared_mean_difference():
    # eps -> inf: P -> a b^T and OT_eps -> sum a_i b_j C_ij, so the divergence tends to
    # E|x - y|^2 - E|x - x'|^2 / 2 - E|y - y'|^2 / 2 = |xbar - ybar|^2
    rng = _rng(22)
    X, Y = rng.normal(size=(15, 3)), rng.normal(size=(11, 3)) + np.array([1.0, 0.0, -0.5])
    want = float(np.sum((X.mean(0) - Y.mean(0)) ** 2))
    D, _, _ = O.sinkhorn_divergence(None, X, None, Y, 1e5, 1e-13)
    assert D == pytest.approx(want, rel=1e-3)


def test_divergence_small_eps_is_exact_ot_cost():
    # eps -> 0: OT_eps(X, Y) -> min over permutations (n = m, uniform) and the entropic
    # terms of the three problems cancel, so D -> W2^2 of the brute-force assignment
    rng = _rng(23)
    n = 6
    X, Y = rng.normal(size=(n, 2)), rng.normal(size=(n, 2)) + 0.5
    C = np.array([[np.sum((x - y) ** 2) for y in Y] for x in X])
    best = min(sum(C[i, p[i]] for i in range(n)) / n for p in itertools.permutations(range(n)))
    D, _, _ = O.sinkhorn_divergence(None, X, None, Y, 2e-3, 1e-9, max_iter=200000)
    assert D == pytest.approx(best, rel=2e-3)


def test_eps_divergence_is_five_percent_of_intra_cost():
    rng = _rng(24)
    Y = rng.normal(size=(7, 2))
    assert O.eps_divergence(Y) == pytest.approx(0.05 * _brute_mean_cost(Y, Y), rel=1e-12)


# --------------------------------------------------- coupling diagonal (Prop. 3)
def test_diagonal_metrics_at_identity_coupling():
    # potentials that make P = Id / n on the diagonal: Tr = 1 and KL = 0 exactly
    rng = _rng(30)
    n = 9
    X, Y = rng.normal(size=(n, 4)), rng.normal(size=(n, 4))
    eps = 0.3
    cdiag = np.sum((X - Y) ** 2, axis=1)
    f = cdiag - eps * math.log(n) - 0.25
    g = np.full(n, 0.25)
    tr, kl = O.diagonal_metrics(X, Y, f, g, eps)
    assert tr == pytest.approx(1.0, rel=1e-13) and abs(kl) < 1e-13


def test_diagonal_kl_is_nonnegative_and_vanishes_as_eps_shrinks():
    # Gibbs' inequality on the n^2 grid: KL(Id/n || P) >= 0 for every coupling of mass 1;
    # for Y = X G with G SPD the optimal coupling is Id / n (Prop. 3), so KL -> 0, Tr -> 1
    rng = _rng(31)
    n, d = 12, 3
    X = rng.normal(size=(n, d))
    A = rng.normal(size=(d, d))
    G = A @ A.T + 0.5 * np.eye(d)
    Y = X @ G
    kls, trs = [], []
    for eps in (5.0, 0.5, 0.01):
        r = O.sinkhorn(None, X, None, Y, eps, 1e-11, max_iter=100000)
        tr, kl = O.diagonal_metrics(X, Y, r.f, r.g, eps)
        assert kl > -1e-9 and tr <= 1.0 + 1e-9
        kls.append(kl)
        trs.append(tr)
    assert kls[0] > kls[1] > kls[2] and kls[2] < 1e-3
    assert trs[2] > 0.999


def test_coupling_diagonal_matches_rows_of_p():
    rng = _rng(32)
    n = 6
    X, Y = rng.normal(size=(n, 2)), rng.normal(size=(n, 2))
    f, g, eps = rng.normal(size=n), rng.normal(size=n), 0.7
    logd = O.coupling_diagonal(X, Y, f, g, eps)
    for i in range(n):
        c = sum((X[i, k] - Y[i, k]) ** 2 for k in range(2))
        assert logd[i] == pytest.approx((f[i] + g[i] - c) / eps, rel=1e-13)


def test_symmetric_self_transport_matches_alternating_sinkhorn():
    # the symmetric fixed point and plain Alg. 1 reach the same maximiser of eq. (5):
    # equal OT values, symmetric potentials satisfying the f-update, marginals = a
    rng = _rng(25)
    X = rng.normal(size=(14, 3))
    a = rng.uniform(0.5, 1.5, 14)
    a /= a.sum()
    eps = 0.8
    sym = O.sinkhorn_symmetric(a, X, eps, 1e-12)
    alt = O.sinkhorn(a, X, a, X, eps, 1e-12, max_iter=200000)
    assert sym.converged and alt.converged and sym.iters < alt.iters
    v_sym = O.dual_objective(a, X, a, X, sym.f, sym.g, eps)
    v_alt = O.dual_objective(a, X, a, X, alt.f, alt.g, eps)
    assert v_sym == pytest.approx(v_alt, rel=1e-10)
    C = O.CostOperator(X, X)
    np.testing.assert_allclose(O.row_marginal(C, sym.f, sym.f, eps), a, atol=1e-12)
    np.testing.assert_allclose(O.col_marginal(C, sym.f, sym.f, eps), a, atol=1e-12)
    # potentials are unique up to (f + k, g - k); the symmetric one has k = 0
    kappa = np.mean(alt.f - sym.f)
    np.testing.assert_allclose(alt.f - kappa, sym.f, atol=1e-9)
    np.testing.assert_allclose(alt.g + kappa, sym.f, atol=1e-9)


def test_coupling_cost_against_another_cloud_by_loops():
    # P from (X, f, g), cost from X_cost: a plain double loop over the definition
    rng = _rng(33)
    X, Xc, Y = rng.normal(size=(5, 2)), rng.normal(size=(5, 2)), rng.normal(size=(4, 2))
    f, g, eps = rng.normal(size=5), rng.normal(size=4), 0.8
    for cost in (None, O.PNorm(1.5)):
        h = (lambda z: float(np.sum(z * z))) if cost is None else (lambda z: float(np.sum(np.abs(z) ** 1.5) / 1.5))
        want = 0.0
        for i in range(5):
            for j in range(4):
                want += math.exp((f[i] + g[j] - h(X[i] - Y[j])) / eps) * h(Xc[i] - Y[j])
        assert O.coupling_cost(X, Y, f, g, eps, cost, X_cost=Xc) == pytest.approx(want, rel=1e-12)
        same = O.coupling_cost(X, Y, f, g, eps, cost)
        assert O.coupling_cost(X, Y, f, g, eps, cost, X_cost=X) == pytest.approx(same, rel=1e-14)
