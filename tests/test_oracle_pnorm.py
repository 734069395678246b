"""Pins of the oracle's non-quadratic cost h(z) = (1/p) sum_k |z_k|^p (Sec. 5.2, p = 1.5)
against facts that do not come from the oracle: convex duality, brute-force optima,
the 1-D monotone rearrangement, finite differences and the exact reduction of p = 2 to
the squared Euclidean cost. CPU only."""
import itertools

import numpy as np
import pytest

from oracle import progot_oracle as O

P15 = O.PNorm(1.5)


def _rng(seed):
    return np.random.default_rng(seed)


def test_pnorm_gradients_are_conjugate():
    # grad h* inverts grad h, and Fenchel-Young holds with equality at w = grad h(z):
    # h(z) + h*(w) = z . w with h*(w) = (1/q) sum |w|^q, 1/p + 1/q = 1
    rng = _rng(0)
    z = rng.normal(size=(50, 7)) * 3.0
    for p in (1.2, 1.5, 2.0, 3.0):
        c = O.PNorm(p)
        q = p / (p - 1.0)
        w = c.grad_h(z)
        np.testing.assert_allclose(c.grad_h_star(w), z, rtol=1e-10, atol=1e-12)
        hstar = np.sum(np.abs(w) ** q, axis=-1) / q
        np.testing.assert_allclose(c.h(z) + hstar, np.sum(z * w, axis=-1), rtol=1e-11)
    # p = 2 is half the squared Euclidean cost
    np.testing.assert_allclose(O.PNorm(2.0).h(z), 0.5 * np.sum(z * z, axis=-1), rtol=1e-14)


def test_pnorm_cost_matrix_by_loops():
    rng = _rng(1)
    X, Y = rng.normal(size=(4, 3)), rng.normal(size=(5, 3))
    C = O.cost_matrix_rows(X, Y, P15)
    for i in range(4):
        for j in range(5):
            want = sum(abs(float(X[i, k]) - float(Y[j, k])) ** 1.5 for k in range(3)) / 1.5
            assert C[i, j] == pytest.approx(want, rel=1e-13)
    Cop = O.CostOperator(X, Y, cost=P15, cache_limit=0)
    for j0, CbT in Cop.col_blocks():
        np.testing.assert_allclose(CbT, C.T[j0:j0 + CbT.shape[0]], rtol=1e-14)


def test_pnorm_sinkhorn_fixed_point():
    rng = _rng(2)
    X, Y = rng.normal(size=(11, 3)), rng.normal(size=(8, 3)) + 0.4
    eps = 0.3
    r = O.sinkhorn(None, X, None, Y, eps, 1e-12, cost=P15)
    C = O.CostOperator(X, Y, cost=P15)
    np.testing.assert_allclose(O.row_marginal(C, r.f, r.g, eps), np.full(11, 1 / 11), atol=1e-12)
    np.testing.assert_allclose(O.col_marginal(C, r.f, r.g, eps), np.full(8, 1 / 8), atol=1e-14)


def test_pnorm_map_is_gradient_of_potential():
    # eq. (7) with a general h: T(x) = x - grad h*(grad f_hat(x)), grad f_hat by central
    # differences of the eq. (6) potential
    rng = _rng(3)
    X, Y = rng.normal(size=(9, 2)), rng.normal(size=(7, 2)) + 1.0
    eps = 0.4
    r = O.sinkhorn(None, X, None, Y, eps, 1e-12, cost=P15)
    xq = rng.normal(size=(5, 2))
    hstep = 1e-6
    grad = np.zeros_like(xq)
    for k in range(2):
        e = np.zeros(2)
        e[k] = hstep
        grad[:, k] = (O.entropic_potential(xq + e, Y, r.g, eps, P15) -
                      O.entropic_potential(xq - e, Y, r.g, eps, P15)) / (2 * hstep)
    want = xq - P15.grad_h_star(grad)
    np.testing.assert_allclose(O.entropic_map(xq, Y, r.g, eps, P15), want, rtol=1e-6, atol=1e-6)


def test_pnorm_brute_force_assignment_small_eps():
    # a shuffled, noisy, shifted copy of X; the h_1.5-optimal permutation (brute force
    # over all 720) is not the shuffle itself for this draw
    rng = _rng(22)
    n = 6
    X = rng.uniform(-6, 6, (n, 2))
    Y = X[rng.permutation(n)] + rng.normal(size=(n, 2)) * 0.8 + np.array([1.0, -0.5])
    C = O.cost_matrix_rows(X, Y, P15)
    perms = list(itertools.permutations(range(n)))
    costs = sorted((sum(C[i, q[i]] for i in range(n)), q) for q in perms)
    (best, sigma), gap = costs[0], costs[1][0] - costs[0][0]
    eps = gap / 30.0
    r = O.sinkhorn(None, X, None, Y, eps, 1e-5, max_iter=50000, cost=P15)
    assert r.converged
    T = O.entropic_map(X, Y, r.g, eps, P15)
    np.testing.assert_allclose(T, Y[list(sigma)], atol=1e-4)


def test_pnorm_one_dimensional_monotone_rearrangement():
    # for a strictly convex h of x - y in 1-D the optimal matching pairs the sorted x with
    # the sorted y (checked by brute force here); at small eps every row of the entropic
    # plan puts its largest mass on that partner and the map lands next to it
    rng = _rng(13)
    n = 7
    X = np.cumsum(rng.uniform(0.5, 1.5, n))[rng.permutation(n)][:, None]
    Y = (np.cumsum(rng.uniform(0.5, 1.5, n)) * 2.0 - 1.0)[rng.permutation(n)][:, None]
    C = O.cost_matrix_rows(X, Y, P15)
    costs = sorted((sum(C[i, q[i]] for i in range(n)), q) for q in itertools.permutations(range(n)))
    sigma = np.array(costs[0][1])
    rank_x, rank_y = np.argsort(np.argsort(X[:, 0])), np.argsort(np.argsort(Y[:, 0]))
    assert np.all(rank_y[sigma] == rank_x)  # brute force agrees with the sorted matching
    eps = (costs[1][0] - costs[0][0]) / 10.0
    r = O.sinkhorn(None, X, None, Y, eps, 1e-4, max_iter=100000, cost=P15)
    assert r.converged
    P = np.exp((r.f[:, None] + r.g[None, :] - C) / eps)
    assert np.all(np.argmax(P, axis=1) == sigma)
    T = O.entropic_map(X, Y, r.g, eps, P15)[:, 0]
    np.testing.assert_allclose(T, Y[sigma, 0], atol=5e-2)


def test_pnorm_two_is_half_the_squared_euclidean_problem():
    # h_2 = |z|^2 / 2: at eps / 2 the potentials are half those of |.|^2 at eps and the
    # maps, couplings and ProgOT trajectories coincide
    rng = _rng(6)
    X, Y = rng.normal(size=(10, 3)), rng.normal(size=(9, 3)) + 0.7
    eps = 0.5
    sq = O.sinkhorn(None, X, None, Y, eps, 1e-12)
    p2 = O.sinkhorn(None, X, None, Y, eps / 2, 1e-12, cost=O.PNorm(2.0))
    np.testing.assert_allclose(p2.f[:, None] + p2.g[None, :], 0.5 * (sq.f[:, None] + sq.g[None, :]), atol=1e-10)
    np.testing.assert_allclose(O.entropic_map(X, Y, p2.g, eps / 2, O.PNorm(2.0)),
                               O.entropic_map(X, Y, sq.g, eps), atol=1e-9)
    al = O.alpha_schedule(3)
    a = O.progot(None, X, None, Y, [eps, eps / 2, eps / 4], al, [1e-11] * 3)
    b = O.progot(None, X, None, Y, [eps / 2, eps / 4, eps / 8], al, [1e-11] * 3, cost=O.PNorm(2.0))
    np.testing.assert_allclose(b.x_out, a.x_out, atol=1e-8)


def test_pnorm_coordinate_permutation_and_sign_equivariance():
    # h is a sum over coordinates of an even function: permuting coordinates or flipping
    # the sign of one coordinate in both clouds permutes / flips the map (rotations do not)
    rng = _rng(7)
    X, Y = rng.normal(size=(12, 3)), rng.normal(size=(10, 3)) * 1.3 + 0.2
    eps, al, ta = 0.3, O.alpha_schedule(2), [1e-11] * 2
    base = O.progot(None, X, None, Y, [eps, eps / 2], al, ta, cost=P15)
    perm = [2, 0, 1]
    pp = O.progot(None, X[:, perm], None, Y[:, perm], [eps, eps / 2], al, ta, cost=P15)
    np.testing.assert_allclose(pp.x_out, base.x_out[:, perm], atol=1e-8)
    s = np.array([1.0, -1.0, 1.0])
    fl = O.progot(None, X * s, None, Y * s, [eps, eps / 2], al, ta, cost=P15)
    np.testing.assert_allclose(fl.x_out, base.x_out * s, atol=1e-8)
    v = np.array([0.5, -1.0, 2.0])
    tr = O.progot(None, X + v, None, Y + v, [eps, eps / 2], al, ta, cost=P15)
    np.testing.assert_allclose(tr.x_out, base.x_out + v, atol=1e-8)


def test_pnorm_progot_reductions():
    rng = _rng(8)
    X, Y = rng.normal(size=(9, 2)), rng.normal(size=(8, 2)) + 1.0
    eps = 0.4
    one = O.progot(None, X, None, Y, [eps], [1.0], [1e-12], cost=P15)
    sk = O.sinkhorn(None, X, None, Y, eps, 1e-12, cost=P15)
    np.testing.assert_allclose(one.x_out, O.entropic_map(X, Y, sk.g, eps, P15), atol=1e-9)
    K = 3
    res = O.progot(None, X, None, Y, [eps, eps / 2, eps / 3], O.alpha_schedule(K), [1e-12] * K, cost=P15)
    T3 = O.progot_map(X, Y, res.g_all, [eps, eps / 2, eps / 3], O.alpha_schedule(K), P15)
    np.testing.assert_allclose(T3, res.x_out, atol=1e-8)
