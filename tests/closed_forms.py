"""Closed forms the tests pin the oracle (and the GPU) against; nothing here calls the
oracle or the library.

Alg. 4 on a two-point target. With Y = {y1, y2}, D = ||y1 - y2||^2 and weights
b = (b1, b2), the self-transport problem Sink(b, Y, b, Y) has the Gibbs kernel
K = [[1, k], [k, 1]], k = exp(-D / eps), and a symmetric plan P = diag(v) K diag(v)
(the cost is symmetric and both marginals are b). Its row sums give
    v1 (v1 + k v2) = b1,   v2 (k v1 + v2) = b2,
so the ratio r = v2 / v1 solves b1 r^2 + k (b1 - b2) r - b2 = 0 (positive root).
exp(g_j / eps) is proportional to v_j (the scaling of the Y side; any gauge gives the
same map), so the eq. (7) map of a test point z is
    T(z) = sum_j w_j y_j,   w_j proportional to v_j exp(-||z - y_j||^2 / eps),
and Alg. 4's score for s_p is sum_z ||z - T(z)||^2 at eps = s_p sigma.
sigma is the unweighted mean of C_YY over its four entries (two zeros, two D) over 20,
i.e. D / 40; eps0 the unweighted mean of C_XY over 20.

Only the regime where Sinkhorn reaches this plan is usable: when k underflows the plan
degenerates to diag(b), v is no longer determined by the marginals and an iteration
from zero stops at a different (equally feasible) split. With b uniform, v1 = v2 at
every iterate and at the solution, so any s_p works; with b non-uniform the grid must
keep k well above zero."""
from __future__ import annotations

import numpy as np


def two_point_scaling_ratio(k: float, b1: float, b2: float) -> float:
    """v2 / v1 of the symmetric scaling of K = [[1, k], [k, 1]] with marginals (b1, b2)."""
    return (-k * (b1 - b2) + np.sqrt(k * k * (b1 - b2) ** 2 + 4.0 * b1 * b2)) / (2.0 * b1)


def two_point_map(Z, y1, y2, eps: float, b=(0.5, 0.5)):
    """eq. (7) map of the rows of Z for the two-point self-transport solution at eps."""
    Z = np.asarray(Z, dtype=np.float64)
    Y = np.stack([np.asarray(y1, np.float64), np.asarray(y2, np.float64)])
    D = float(np.sum((Y[0] - Y[1]) ** 2))
    k = np.exp(-D / eps)
    v = np.array([1.0, two_point_scaling_ratio(k, b[0], b[1])])
    out = np.empty_like(Z)
    for i, z in enumerate(Z):
        w = v * np.exp(-np.sum((z - Y) ** 2, axis=1) / eps)
        out[i] = (w / w.sum()) @ Y
    return out


def two_point_alg4(X, y1, y2, Z, K: int, s_grid, b=(0.5, 0.5), beta0: float = 5.0):
    """Alg. 4 with the constant-speed t_k = k / K for a two-point target: returns
    (eps_1..eps_K, scores per s_p, p*, eps0, sigma), p* the first minimiser."""
    X = np.asarray(X, dtype=np.float64)
    Y = np.stack([np.asarray(y1, np.float64), np.asarray(y2, np.float64)])
    D = float(np.sum((Y[0] - Y[1]) ** 2))
    eps0 = float(np.mean([[np.sum((x - y) ** 2) for y in Y] for x in X])) / 20.0
    sigma = D / 40.0
    Z = np.asarray(Z, dtype=np.float64)
    scores = []
    for s in s_grid:
        T = two_point_map(Z, y1, y2, s * sigma, b)
        scores.append(float(np.sum((Z - T) ** 2)))
    scores = np.array(scores)
    p = int(np.argmin(scores))
    t = np.arange(1, K + 1) / K
    return (1.0 - t) * beta0 * eps0 + t * s_grid[p] * sigma, scores, p, eps0, sigma
