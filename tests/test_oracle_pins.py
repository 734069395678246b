"""Pins of the FP64 oracle against facts that do not come from the oracle itself:
closed forms, brute-force optima, library routines, invariants and the paper's
printed Table 7. CPU only."""
import itertools
import math
import os

import numpy as np
import pytest
from scipy import optimize, special
from scipy.linalg import sqrtm

import closed_forms as CF
from oracle import progot_oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rng(seed):
    return np.random.default_rng(seed)


# ---------------------------------------------------------------- primitives
def test_softmin_matches_library_logsumexp():
    rng = _rng(0)
    S = rng.normal(size=(7, 11)) * 30.0
    for eps in (0.01, 0.3, 5.0):
        ref = -eps * special.logsumexp(-S / eps, axis=1)
        np.testing.assert_allclose(O.softmin(S, eps), ref, rtol=1e-13, atol=1e-12)


def test_cost_is_squared_euclidean_distance():
    rng = _rng(1)
    X, Y = rng.normal(size=(5, 3)), rng.normal(size=(4, 3))
    C = O.cost_matrix_rows(X, Y)
    for i in range(5):
        for j in range(4):
            assert abs(C[i, j] - np.linalg.norm(X[i] - Y[j]) ** 2) < 1e-12


def test_mean_cost_matches_closed_form():
    # mean_ij ||x_i - y_j||^2 = mean ||x||^2 + mean ||y||^2 - 2 xbar . ybar
    rng = _rng(2)
    X, Y = rng.normal(size=(37, 5)) + 1.0, rng.normal(size=(23, 5)) * 2.0
    closed = np.mean(np.sum(X**2, 1)) + np.mean(np.sum(Y**2, 1)) - 2 * X.mean(0) @ Y.mean(0)
    assert abs(O.mean_cost(X, Y) - closed) < 1e-10 * closed


# ------------------------------------------------------ Sinkhorn (Alg. 1)
def _small_problem(seed=3, n=13, m=9, d=3, weights=True):
    rng = _rng(seed)
    X, Y = rng.normal(size=(n, d)), rng.normal(size=(m, d)) + 0.5
    if weights:
        a = rng.uniform(0.5, 1.5, n)
        b = rng.uniform(0.5, 1.5, m)
        return a / a.sum(), X, b / b.sum(), Y
    return None, X, None, Y


def test_sinkhorn_fixed_point_marginals():
    a, X, b, Y = _small_problem()
    eps, tau = 0.2, 1e-10
    r = O.sinkhorn(a, X, b, Y, eps, tau)
    assert r.converged
    C = O.CostOperator(X, Y)
    # after the g-update the column marginal is exact; the row one within tau
    np.testing.assert_allclose(O.col_marginal(C, r.f, r.g, eps), b, atol=1e-14)
    assert np.sum(np.abs(O.row_marginal(C, r.f, r.g, eps) - a)) <= tau


def test_sinkhorn_matches_independent_dual_ascent():
    """Maximise the eq. (5) dual with L-BFGS (its gradient is a - P1, b - P^T 1, written
    here from the Lagrangian, not from the Sinkhorn updates) and compare the
    gauge-invariant sums f_i + g_j."""
    a, X, b, Y = _small_problem(seed=4)
    eps = 0.3
    C = np.array([[np.sum((x - y) ** 2) for y in Y] for x in X])
    n, m = C.shape

    def neg_dual(z):
        f, g = z[:n], z[n:]
        P = np.exp((f[:, None] + g[None, :] - C) / eps)
        val = f @ a + g @ b - eps * P.sum()
        grad = np.concatenate([a - P.sum(1), b - P.sum(0)])
        return -val, -grad

    sol = optimize.minimize(neg_dual, np.zeros(n + m), jac=True, method="L-BFGS-B",
                            options=dict(maxiter=20000, gtol=1e-13, ftol=1e-15))
    fd, gd = sol.x[:n], sol.x[n:]
    r = O.sinkhorn(a, X, b, Y, eps, 1e-12)
    np.testing.assert_allclose(r.f[:, None] + r.g[None, :], fd[:, None] + gd[None, :], atol=5e-6)


def test_two_point_closed_form_plan():
    """n = m = 2, uniform weights: P = [[p, 1/2 - p], [1/2 - p, p]] with
    (p / (1/2 - p))^2 = exp((C12 + C21 - C11 - C22)/eps)."""
    X = np.array([[0.0, 0.0], [1.0, 0.5]])
    Y = np.array([[0.2, -0.1], [1.3, 0.9]])
    eps = 0.4
    C = np.array([[np.sum((x - y) ** 2) for y in Y] for x in X])
    q = math.sqrt(math.exp((C[0, 1] + C[1, 0] - C[0, 0] - C[1, 1]) / eps))
    p = q / (2 * (1 + q))
    r = O.sinkhorn(None, X, None, Y, eps, 1e-14)
    P = np.exp((r.f[:, None] + r.g[None, :] - C) / eps)
    np.testing.assert_allclose(P, [[p, 0.5 - p], [0.5 - p, p]], atol=1e-12)


def test_strong_duality_primal_equals_dual():
    """At the eq. (5) optimum: dual = <P, C> - eps E(P), E(P) = -sum P (log P - 1)."""
    a, X, b, Y = _small_problem(seed=5, weights=False)
    eps = 0.25
    r = O.sinkhorn(a, X, b, Y, eps, 1e-12)
    dual = O.dual_objective(a, X, b, Y, r.f, r.g, eps)
    primal = O.coupling_cost(X, Y, r.f, r.g, eps) - eps * O.coupling_entropy(X, Y, r.f, r.g, eps)
    assert abs(dual - primal) < 1e-9 * max(1.0, abs(dual))


def test_sinkhorn_warm_start_meeting_tau_does_no_work():
    a, X, b, Y = _small_problem(seed=6)
    r = O.sinkhorn(a, X, b, Y, 0.3, 1e-9)
    r2 = O.sinkhorn(a, X, b, Y, 0.3, 1e-9, r.f, r.g)
    assert r2.iters == 0 and r2.converged


def test_sinkhorn_max_iter_reports_not_converged():
    a, X, b, Y = _small_problem(seed=7)
    r = O.sinkhorn(a, X, b, Y, 0.01, 1e-14, max_iter=3)
    assert r.iters == 3 and not r.converged


# ----------------------------------------------- entropic potential / map
def test_entropic_map_is_gradient_of_potential():
    """eq. (7): T(x) = x - grad h*(grad f_hat(x)) = x - grad f_hat(x) / 2, checked with
    central differences of the eq. (6) potential."""
    rng = _rng(8)
    Y = rng.normal(size=(15, 3))
    g = rng.normal(size=15)
    eps = 0.7
    x = rng.normal(size=3)
    hstep = 1e-5
    grad = np.array([(O.entropic_potential(x + hstep * e, Y, g, eps)[0]
                      - O.entropic_potential(x - hstep * e, Y, g, eps)[0]) / (2 * hstep)
                     for e in np.eye(3)])
    np.testing.assert_allclose(O.entropic_map(x, Y, g, eps)[0], x - grad / 2, atol=1e-7)


def test_entropic_potential_on_training_points_gives_f():
    """At a Sinkhorn fixed point, f_hat(x_i) + eps log a_i = f_i (eq. (6) vs Alg. 1)."""
    a, X, b, Y = _small_problem(seed=9)
    eps = 0.3
    r = O.sinkhorn(a, X, b, Y, eps, 1e-13)
    np.testing.assert_allclose(O.entropic_potential(X, Y, r.g, eps) + eps * np.log(a), r.f, atol=1e-10)


def test_jacobian_is_conditional_covariance():
    """grad T_eps(x) = (2/eps) Cov_p(Y) for c = ||x - y||^2 (the Lipschitz lemma of the
    appendix states Cov/eps for h = ||.||^2 / 2)."""
    rng = _rng(10)
    Y = rng.normal(size=(25, 2))
    g = rng.normal(size=25) * 0.3
    eps = 0.9
    x = np.array([0.3, -0.2])
    hstep = 1e-5
    J = np.stack([(O.entropic_map(x + hstep * e, Y, g, eps)[0] - O.entropic_map(x - hstep * e, Y, g, eps)[0])
                  / (2 * hstep) for e in np.eye(2)], axis=1)
    logits = (g - np.sum((x - Y) ** 2, 1)) / eps
    p = np.exp(logits - logits.max())
    p /= p.sum()
    mu = p @ Y
    cov = (Y - mu).T @ ((Y - mu) * p[:, None])
    np.testing.assert_allclose(J, 2.0 / eps * cov, atol=1e-6)


def test_large_eps_map_is_target_mean():
    rng = _rng(11)
    X, Y = rng.normal(size=(10, 2)), rng.normal(size=(12, 2)) + 3.0
    eps = 1e6
    r = O.sinkhorn(None, X, None, Y, eps, 1e-12)
    T = O.entropic_map(X, Y, r.g, eps)
    np.testing.assert_allclose(T, np.broadcast_to(Y.mean(0), T.shape), atol=1e-4)


# ---------------------------------------------------- exact OT special cases
def test_brute_force_assignment_small_eps():
    """n = m = 6: the optimal permutation by enumeration; as eps -> 0 the entropic map
    sends x_i to y_sigma(i), and ProgOT (K = 3) recovers the same assignment."""
    rng = _rng(12)
    n = 6
    X, Y = rng.normal(size=(n, 2)), rng.normal(size=(n, 2)) * 1.5 + 0.3
    C = np.array([[np.sum((x - y) ** 2) for y in Y] for x in X])
    best, gap = _assignment_gap(C)
    eps = gap / 30.0
    r = O.sinkhorn(None, X, None, Y, eps, 1e-7, max_iter=50000)
    T = O.entropic_map(X, Y, r.g, eps)
    np.testing.assert_allclose(T, Y[list(best)], atol=1e-4)
    al = O.alpha_schedule(3)
    pr = O.progot(None, X, None, Y, [eps] * 3, al, [1e-7] * 3, max_iter=50000)
    np.testing.assert_allclose(pr.x_out, Y[list(best)], atol=1e-4)


def _assignment_gap(C):
    n = C.shape[0]
    costs = {perm: sum(C[i, perm[i]] for i in range(n)) for perm in itertools.permutations(range(n))}
    ranked = sorted(costs.values())
    return min(costs, key=costs.get), ranked[1] - ranked[0]


def test_one_dimensional_monotone_rearrangement():
    """d = 1: the optimal matching pairs the sorted x with the sorted y; as eps -> 0 the
    entropic map sends the k-th smallest x to the k-th smallest y."""
    rng = _rng(13)
    n = 7
    # well-separated points in shuffled order
    X = (np.cumsum(rng.uniform(0.3, 1.0, n)) - 2.0)[rng.permutation(n)][:, None]
    Y = np.cumsum(rng.exponential(0.5, n) + 0.1)[rng.permutation(n)][:, None]
    C = (X - Y.T) ** 2
    _, gap = _assignment_gap(C)
    eps = gap / 30.0
    r = O.sinkhorn(None, X, None, Y, eps, 1e-7, max_iter=50000)
    T = O.entropic_map(X, Y, r.g, eps)
    order = np.argsort(X[:, 0])
    np.testing.assert_allclose(T[order, 0], np.sort(Y[:, 0]), atol=1e-4)


def test_linear_spd_coupling_is_identity():
    """Prop. 3: for Y = G X with G symmetric positive definite the optimal coupling is
    Id/n, so at small eps n Tr(P) -> 1 and T(x_i) -> y_i."""
    rng = _rng(14)
    n, d = 30, 4
    X = rng.normal(size=(n, d))
    Q, _ = np.linalg.qr(rng.normal(size=(d, d)))
    G = Q @ np.diag([0.5, 0.8, 1.3, 2.0]) @ Q.T
    Y = X @ G.T
    eps = 2e-3
    r = O.sinkhorn(None, X, None, Y, eps, 1e-8, max_iter=100000)
    C = O.cost_matrix_rows(X, Y)
    P = np.exp((r.f[:, None] + r.g[None, :] - C) / eps)
    assert n * np.trace(P) > 0.999
    np.testing.assert_allclose(O.entropic_map(X, Y, r.g, eps), Y, atol=1e-3)


def test_gaussian_entropic_map_closed_form():
    """Population entropic OT between N(m1, A) and N(m2, B) for c = ||x - y||^2: the plan
    is Gaussian and E[Y | X = x] = m2 + A^-1/2 N A^-1/2 (x - m1) with
    N = (-eps I + (eps^2 I + 16 A^1/2 B A^1/2)^1/2) / 4 (derived from the Schroedinger
    system of eq. (13)). The empirical map's least-squares linear part must match it
    (statistical tolerance); eps and 2 eps give clearly different answers."""
    rng = _rng(15)
    n = 1500
    A = np.array([[1.0, 0.3], [0.3, 0.6]])
    B = np.array([[2.0, -0.4], [-0.4, 1.0]])
    m1, m2 = np.array([0.5, -1.0]), np.array([-1.0, 2.0])
    X = rng.multivariate_normal(m1, A, size=n)
    Y = rng.multivariate_normal(m2, B, size=n)
    eps = 1.5

    def slope(e):
        Ah = np.real(sqrtm(A))
        Aih = np.linalg.inv(Ah)
        N = (-e * np.eye(2) + np.real(sqrtm(e * e * np.eye(2) + 16 * Ah @ B @ Ah))) / 4
        return Aih @ N @ Aih

    r = O.sinkhorn(None, X, None, Y, eps, 1e-8)
    T = O.entropic_map(X, Y, r.g, eps)
    Xc = np.hstack([X - X.mean(0), np.ones((n, 1))])
    coef, *_ = np.linalg.lstsq(Xc, T, rcond=None)
    M_hat = coef[:2].T
    M_eps, M_2eps = slope(eps), slope(2 * eps)
    err = np.linalg.norm(M_hat - M_eps) / np.linalg.norm(M_eps)
    assert err < 0.08, err
    assert np.linalg.norm(M_2eps - M_eps) / np.linalg.norm(M_eps) > 3 * err


# ------------------------------------------------------- ProgOT (Alg. 2, 3)
def test_progot_single_full_step_is_entropic_map():
    a, X, b, Y = _small_problem(seed=16, weights=False)
    eps = 0.4
    pr = O.progot(a, X, b, Y, [eps], [1.0], [1e-12])
    r = O.sinkhorn(a, X, b, Y, eps, 1e-12)
    np.testing.assert_allclose(pr.x_out, O.entropic_map(X, Y, r.g, eps), atol=1e-10)


def test_alg3_on_training_points_reproduces_alg2():
    a, X, b, Y = _small_problem(seed=17, weights=False, n=20, m=15)
    K = 4
    al = O.alpha_schedule(K)
    eps = [1.2, 0.8, 0.5, 0.3]
    pr = O.progot(a, X, b, Y, eps, al, [1e-12] * K)
    Tq = O.progot_map(X, Y, pr.g_all, eps, al)
    np.testing.assert_allclose(Tq, pr.x_out, atol=1e-8)


def test_progot_equivariances():
    rng = _rng(18)
    X, Y = rng.normal(size=(14, 3)), rng.normal(size=(11, 3)) + 1.0
    K = 3
    al = O.alpha_schedule(K)
    eps = [0.9, 0.6, 0.4]
    tau = [1e-12] * K
    base = O.progot(None, X, None, Y, eps, al, tau).x_out
    v = np.array([0.3, -2.0, 1.0])
    np.testing.assert_allclose(O.progot(None, X + v, None, Y + v, eps, al, tau).x_out, base + v, atol=1e-8)
    Q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    np.testing.assert_allclose(O.progot(None, X @ Q.T, None, Y @ Q.T, eps, al, tau).x_out, base @ Q.T, atol=1e-8)
    perm = rng.permutation(11)
    np.testing.assert_allclose(O.progot(None, X, None, Y[perm], eps, al, tau).x_out, base, atol=1e-8)
    s = 1.7
    np.testing.assert_allclose(O.progot(None, s * X, None, s * Y, [e * s * s for e in eps], al, tau).x_out,
                               s * base, atol=1e-8)


def test_progot_target_to_itself_small_eps_is_identity():
    """Alg. 4's premise: the map from the target to itself is the identity."""
    rng = _rng(19)
    Y = rng.normal(size=(12, 2)) * 2
    eps = 1e-3
    r = O.sinkhorn(None, Y, None, Y, eps, 1e-10, max_iter=100000)
    np.testing.assert_allclose(O.entropic_map(Y, Y, r.g, eps), Y, atol=1e-4)


# -------------------------------------------------------------- schedules
def test_table7_progress_times_golden():
    with open(os.path.join(GOLDEN, "table7_progress_times.txt")) as fh:
        rows = [ln.split() for ln in fh if ln.strip() and not ln.startswith("#")]
    assert rows
    for kind, K, *ts in rows:
        t = O.progress_times(O.alpha_schedule(int(K), kind))
        np.testing.assert_allclose(t, [float(v) for v in ts], atol=1e-15)


def test_alpha_schedules_end_with_full_step():
    for K in (1, 2, 4, 8, 16):
        for kind in ("constant", "accelerated", "decelerated"):
            al = O.alpha_schedule(K, kind)
            assert al[-1] == 1.0 and np.all(al > 0) and np.all(al <= 1)
            assert O.progress_times(al)[-1] == 1.0
        np.testing.assert_allclose(O.alpha_schedule(K), [1.0 / (K - k + 1) for k in range(1, K + 1)])


def test_eps_schedule_alg4_structure():
    rng = _rng(20)
    X, Y = rng.normal(size=(40, 2)), rng.normal(size=(35, 2)) + 1
    Yt = rng.normal(size=(16, 2)) + 1
    al = O.alpha_schedule(4)
    sched, info = O.eps_schedule(X, None, Y, Yt, al, tau=1e-8)
    assert abs(info["eps0"] - O.mean_cost(X, Y) / 20) < 1e-14
    assert abs(info["sigma"] - O.mean_cost(Y, Y) / 20) < 1e-14
    assert info["p_star"] == int(np.argmin(info["errors"]))
    assert abs(sched[-1] - info["eps_K"]) < 1e-14
    t = O.progress_times(al)
    np.testing.assert_allclose(sched, (1 - t) * 5 * info["eps0"] + t * info["eps_K"], rtol=1e-14)


# Two-point targets (closed form in tests/closed_forms.py). Case A: uniform b, the default
# grid s_p = 2^-3..2^3; case B: b = (0.7, 0.3) on a grid that keeps the Gibbs kernel's
# off-diagonal entry away from zero, so the score depends on the potential g.
ALG4_Y = (np.array([0.0, 0.0]), np.array([2.0, 0.0]))
ALG4_CASES = {
    "A": dict(b=(0.5, 0.5), Z=np.array([[0.6, 0.0], [1.4, 0.3], [1.0, -0.2]]),
              s_grid=[2.0 ** e for e in range(-3, 4)]),
    "B": dict(b=(0.7, 0.3), Z=np.array([[0.7, 0.0], [1.3, 0.1]]), s_grid=[10.0, 14.0, 20.0, 28.0, 40.0]),
}


def _alg4_case(name):
    c = ALG4_CASES[name]
    X = _rng(5).normal(size=(5, 2))
    Y = np.stack(ALG4_Y)
    b = None if c["b"] == (0.5, 0.5) else np.array(c["b"])
    return X, Y, b, c


@pytest.mark.parametrize("name", ["A", "B"])
def test_eps_schedule_two_point_closed_form(name):
    """Alg. 4 against its closed form on a two-point target: eps0, sigma, every s_p's
    score (the eq. (7) map of the held-out points from the two-point Sinkhorn plan), p*
    and the interpolated schedule."""
    X, Y, b, c = _alg4_case(name)
    K = 4
    al = O.alpha_schedule(K)
    sched, info = O.eps_schedule(X, b, Y, c["Z"], al, s_grid=c["s_grid"], tau=1e-13)
    want, scores, p, eps0, sigma = CF.two_point_alg4(X, *ALG4_Y, c["Z"], K, c["s_grid"], b=c["b"])
    assert abs(info["eps0"] - eps0) <= 1e-13 * eps0 and abs(info["sigma"] - sigma) <= 1e-13 * sigma
    np.testing.assert_allclose(info["errors"], scores, rtol=1e-9, atol=1e-12)
    srt = np.sort(scores)
    assert srt[1] - srt[0] > 0.05 * srt[0]  # the minimiser is clear
    assert info["p_star"] == p
    np.testing.assert_allclose(sched, want, rtol=1e-12)
    if name == "B":
        assert 0 < p < len(c["s_grid"]) - 1  # an interior choice: the scores are not monotone


# ------------------------------------------------ planted mistakes are caught
@pytest.mark.filterwarnings("ignore::RuntimeWarning")
def test_planted_mistakes_are_caught(monkeypatch):
    """Plant plausible mistakes in the oracle and check that a pin above fails."""
    # (1) dropping the 1/2 of grad h* breaks the closed-form Gaussian map pin
    monkeypatch.setattr(O, "grad_h_star", lambda w: w)
    with pytest.raises(AssertionError):
        test_entropic_map_is_gradient_of_potential()
    monkeypatch.undo()
    # (2) the printed sign of the f-update ("- min_eps") breaks the fixed-point pin
    def bad_update_f(C, f, g, eps, a):
        out = np.empty_like(f)
        for i0, Cb in C.row_blocks():
            i1 = i0 + Cb.shape[0]
            S = Cb - O.tensor_sum(f[i0:i1], g)
            out[i0:i1] = eps * np.log(a[i0:i1]) - O.softmin(S, eps) + f[i0:i1]
        return out
    monkeypatch.setattr(O, "_update_f", bad_update_f)
    with pytest.raises(AssertionError):
        test_two_point_closed_form_plan()
    monkeypatch.undo()
    # (3) a transposed cost (C^T used for the f-update) breaks the dual-ascent pin
    orig = O.CostOperator.row_blocks
    monkeypatch.setattr(O.CostOperator, "row_blocks", O.CostOperator.col_blocks)
    with pytest.raises(Exception):
        test_sinkhorn_matches_independent_dual_ascent()
    monkeypatch.setattr(O.CostOperator, "row_blocks", orig)
    # (4) a b_j factor put back into Alg. 3 breaks the Alg. 3 == Alg. 2 pin (non-uniform b)
    a, X, b, Y = _small_problem(seed=21, n=10, m=8)
    K = 2
    al = O.alpha_schedule(K)
    pr = O.progot(a, X, b, Y, [0.8, 0.5], al, [1e-12] * K)
    good = O.progot_map(X, Y, pr.g_all, [0.8, 0.5], al)
    np.testing.assert_allclose(good, pr.x_out, atol=1e-8)
    bad = O.progot_map(X, Y, [gk + e * np.log(b) for gk, e in zip(pr.g_all, [0.8, 0.5])], [0.8, 0.5], al)
    assert np.max(np.abs(bad - pr.x_out)) > 1e-4
    # (5) Alg. 4 scoring the held-out points with a zero potential (the Sinkhorn solve
    # ignored) picks another s_p on the two-point target with non-uniform b
    orig_map = O.progot_map
    monkeypatch.setattr(O, "progot_map", lambda Xq, Yy, g_all, eps, al: orig_map(Xq, Yy, [np.zeros_like(g) for g in g_all], eps, al))
    with pytest.raises(AssertionError):
        test_eps_schedule_two_point_closed_form("B")
    monkeypatch.undo()
    # (6) sigma taken from the source-target cost instead of C_YY moves the eps grid
    orig_mc = O.mean_cost
    monkeypatch.setattr(O, "mean_cost", lambda U, V, *a, **k: orig_mc(U, V, *a, **k) if U is not V else orig_mc(_rng(5).normal(size=(5, 2)), V, *a, **k))
    with pytest.raises(AssertionError):
        test_eps_schedule_two_point_closed_form("A")
    monkeypatch.undo()


def test_sinkhorn_continues_through_an_overflowing_error():
    # a warm start far from feasible makes P overflow (error = inf > tau); Alg. 1 keeps
    # iterating and reaches the same coupling as the zero start (f (+) g is unique)
    a, X, b, Y = _small_problem(seed=9)
    eps = 0.05
    ref = O.sinkhorn(a, X, b, Y, eps, 1e-10, max_iter=100000)
    with np.errstate(over="ignore"):
        hot = O.sinkhorn(a, X, b, Y, eps, 1e-10, f_init=np.full(X.shape[0], 50.0),
                         g_init=np.full(Y.shape[0], 50.0), max_iter=100000)
    assert math.isinf(hot.errs[0]) and hot.converged
    np.testing.assert_allclose(hot.f[:, None] + hot.g[None, :], ref.f[:, None] + ref.g[None, :], atol=1e-8)
