"""FP64 CPU oracle for the ProgOT hot path (arXiv 2406.05061).

TEST INFRASTRUCTURE. Only the tests, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
module. The CUDA path never calls it and shares no code with it.

What it computes, in float64, step by step in the paper's order and notation:

* Sec. 2 "Entropic OT": the cost c(x, y) = h(x - y) with h = ||.||^2, the soft-min
  min_eps(S)_i = -eps log sum_j exp(-S_ij / eps), the tensor sum f (+) g.
* Alg. 1 (Sinkhorn, log domain) with the dual convention of eq. (5):
  P_ij = exp((f_i + g_j - C_ij) / eps).
* eq. (6) / eq. (7): entropic potential and entropic map.
* Alg. 2 (ProgOT): warm-started Sinkhorn solves, row renormalisation
  Q = diag(1 / P 1) P and the displacement X <- X - alpha_k Z.
* Alg. 3: the progressive map applied to new points from the stored g^(k).
* Sec. 4 "Setting step lengths" and Table 7: alpha schedules and t_k.
* Alg. 4: the epsilon scheduler.
* Sec. 5.2: coupling cost <P, C>, entropy E(P), marginal L1 error; the
  iterate-dependent rule eps_k = theta cbar_k of the coupling experiments and the
  linear threshold schedule tau_k of Sec. 4.
* eq. (8): the Sinkhorn divergence D_eps(X, Y) built from the eq. (5) objective.
* Sec. 5.3 / Prop. 3: trace and KL of the coupling diagonal against Id / n.

Readings where the paper's printed formulas are garbled or silent:

* Alg. 1 loop condition: iterate WHILE ||P 1 - a||_1 > tau (the printed "<" would
  never start the loop).
* Alg. 1 updates: f <- eps log a + min_eps(C - f (+) g) + f and likewise for g
  (the printed "- min_eps" doubles f; with "+" the row sums become exactly a).
* Alg. 1 coupling / eq. (5) kernel: P_ij = exp((f_i + g_j - C_ij)/eps),
  K_ij = exp(-h(x_i - y_j)/eps) (the printed exp((C - f (+) g)/eps) has the sign
  flipped and K drops h).
* eq. (6): f_hat(x) = min_eps([h(x - y_j) - g_j]_j) (the printed argument has the
  sign of the bracket flipped).
* Alg. 3 weights: p_j proportional to exp((g_j - h(y - y_j))/eps) WITHOUT a b_j
  factor, because under the Alg. 1 convention g already absorbs eps log b. This
  makes Alg. 3 on a training point equal to Alg. 2's displaced point.
* Step indexing: K solves indexed k = 1..K (Def. 1 says K steps; Alg. 2's
  "k = 0..K" would give K + 1). Constant speed: alpha_k = 1 / (K - k + 1),
  so t_k = k / K and alpha_K = 1 (Table 7's printed 1/(K - k + 2) contradicts
  both t_k = k/K and alpha_K = 1).
* Warm start (Alg. 2): f_init, g_init = (1 - alpha_k) f, (1 - alpha_k) g^(k-1)
  with the CURRENT step's alpha_k, zero at the first step.
* Alg. 4: the value returned as "eps_1" is eps_K; eps_k = (1 - t_k) beta0 eps0 +
  t_k eps_K. Grid s_p = 2^-3 .. 2^3, beta0 = 5, ties broken by the smallest p.
* eps0 and sigma: unweighted means of the cost matrices over all pairs.
* theta rule: cbar_k is the unweighted mean of h(x_i^(k) - y_j) over all pairs,
  divided by 20, on the cloud X^(k) that solve k transports (the input of its
  Sinkhorn call); eps_k = theta cbar_k.
* tau schedule: tau_k falls linearly in k from tau_1 to tau_K.
* eq. (8) objective: OT_eps is the eq. (5) dual value at the Sinkhorn potentials;
  eps_D = 5% of the unweighted mean of the target's intra cost C_YY. The self terms
  OT(X, X), OT(Y, Y) are solved by the symmetric (averaged) fixed point, whose
  maximiser is the same and which converges much faster than alternating updates.
* Costs: the squared Euclidean h = ||.||^2 everywhere by default; the coupling
  experiments' h = (1/p) ||.||_p^p (p = 1.5) through the ``cost`` argument, with its
  gradient and the gradient of its conjugate written coordinate by coordinate.
* Blur benchmark KL: KL(P* || P) = -log n - (1/n) sum_i log P_ii (the printed
  "n sum_i" would not vanish at P = P* = Id / n).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "h", "grad_h", "grad_h_star", "cost_matrix_rows", "softmin", "tensor_sum",
    "CostOperator", "row_marginal", "col_marginal", "marginal_error",
    "sinkhorn", "SinkhornResult", "entropic_potential", "entropic_map",
    "barycentric_displacement", "progot", "ProgOTResult", "progot_map",
    "alpha_schedule", "progress_times", "mean_cost", "eps_schedule",
    "coupling_cost", "coupling_entropy", "dual_objective",
    "eps_theta_rule", "tau_schedule", "eps_divergence", "ot_value", "sinkhorn_symmetric",
    "sinkhorn_divergence", "coupling_diagonal", "diagonal_metrics",
    "SqEuclidean", "PNorm", "SQEUCLIDEAN",
]

# Rows per block: the oracle never holds more than BLOCK_ELEMS doubles of an
# (n x m x d) difference tensor at a time.
BLOCK_ELEMS = 1 << 22


# --------------------------------------------------------------------------
# Sec. 2: cost h, its gradient and the gradient of its convex conjugate.
# --------------------------------------------------------------------------
def h(z: np.ndarray) -> np.ndarray:
    """Translation-invariant cost h(z) = ||z||_2^2 (squared Euclidean, Sec. 2)."""
    return np.sum(z * z, axis=-1)


def grad_h(z: np.ndarray) -> np.ndarray:
    """Gradient of h = ||.||^2: 2 z."""
    return 2.0 * z


def grad_h_star(w: np.ndarray) -> np.ndarray:
    """Gradient of the convex conjugate h*(w) = ||w||^2 / 4 (Brenier's theorem,
    Sec. 2): w / 2."""
    return 0.5 * w


class SqEuclidean:
    """The workload cost h = ||.||^2 with grad h = 2z and grad h* = w/2."""

    name = "sqeuclidean"

    @staticmethod
    def h(z):
        return h(z)

    @staticmethod
    def grad_h(z):
        return grad_h(z)

    @staticmethod
    def grad_h_star(w):
        return grad_h_star(w)


class PNorm:
    """The non-quadratic cost of the coupling experiments (Sec. 5.2),
    h(z) = (1/p) sum_k |z_k|^p with p > 1, coordinate by coordinate:
    grad h(z)_k = sign(z_k) |z_k|^(p-1); its convex conjugate is
    h*(w) = (1/q) sum_k |w_k|^q with 1/p + 1/q = 1, so
    grad h*(w)_k = sign(w_k) |w_k|^(q-1) = sign(w_k) |w_k|^(1/(p-1))."""

    def __init__(self, p: float):
        if not p > 1.0:
            raise ValueError("p > 1")
        self.p = float(p)
        self.name = f"pnorm{self.p:g}"

    def h(self, z):
        return np.sum(np.abs(z) ** self.p, axis=-1) / self.p

    def grad_h(self, z):
        return np.sign(z) * np.abs(z) ** (self.p - 1.0)

    def grad_h_star(self, w):
        return np.sign(w) * np.abs(w) ** (1.0 / (self.p - 1.0))


SQEUCLIDEAN = SqEuclidean()


def _cost(cost):
    return SQEUCLIDEAN if cost is None else cost


def _rows_per_block(m: int, d: int) -> int:
    return max(1, BLOCK_ELEMS // max(1, m * d))


def cost_matrix_rows(X: np.ndarray, Y: np.ndarray, cost=None) -> np.ndarray:
    """C_ij = h(x_i - y_j) for all rows of X against all rows of Y, computed from the
    differences x_i - y_j themselves (the definition, no norm expansion); h is the
    squared Euclidean cost unless another cost is given."""
    diff = X[:, None, :] - Y[None, :, :]
    return _cost(cost).h(diff)


def softmin(S: np.ndarray, eps: float) -> np.ndarray:
    """Row-wise soft-min of Sec. 2: min_eps(S)_i = -eps log sum_j exp(-S_ij / eps).

    Evaluated with the row minimum factored out so that no exponent is positive."""
    s0 = np.min(S, axis=1)
    return s0 - eps * np.log(np.sum(np.exp(-(S - s0[:, None]) / eps), axis=1))


def tensor_sum(f: np.ndarray, g: np.ndarray) -> np.ndarray:
    """f (+) g := [f_i + g_j]_ij (Sec. 2)."""
    return f[:, None] + g[None, :]


class CostOperator:
    """Blocks of the cost matrix C = [h(x_i - y_j)]_ij of Alg. 1.

    Small problems keep C (computed once from the definition); larger ones
    recompute row blocks on demand, never holding more than one block."""

    def __init__(self, X: np.ndarray, Y: np.ndarray, cache_limit: int = 1 << 24, cost=None):
        self.X = np.asarray(X, dtype=np.float64)
        self.Y = np.asarray(Y, dtype=np.float64)
        self.cost = _cost(cost)
        self.n, self.m = self.X.shape[0], self.Y.shape[0]
        self._full = None
        if self.n * self.m <= cache_limit:
            self._full = np.concatenate(list(self._compute_row_blocks()), axis=0) if self.n else np.zeros((0, self.m))

    def _compute_row_blocks(self):
        step = _rows_per_block(self.m, self.X.shape[1])
        for i0 in range(0, self.n, step):
            yield cost_matrix_rows(self.X[i0:i0 + step], self.Y, self.cost)

    def row_blocks(self):
        """Yield (i0, C[i0:i1, :])."""
        if self._full is not None:
            yield 0, self._full
            return
        step = _rows_per_block(self.m, self.X.shape[1])
        for i0 in range(0, self.n, step):
            yield i0, cost_matrix_rows(self.X[i0:i0 + step], self.Y, self.cost)

    def col_blocks(self):
        """Yield (j0, C[:, j0:j1]^T), i.e. blocks of C^T."""
        if self._full is not None:
            yield 0, self._full.T
            return
        step = _rows_per_block(self.n, self.X.shape[1])
        for j0 in range(0, self.m, step):
            # both costs are even (h(-z) = h(z)), so C^T rows are costs from y_j to X
            yield j0, cost_matrix_rows(self.Y[j0:j0 + step], self.X, self.cost)


def _uniform(k: int) -> np.ndarray:
    return np.full(k, 1.0 / k)


def _weights(w, k: int) -> np.ndarray:
    return _uniform(k) if w is None else np.asarray(w, dtype=np.float64)


# --------------------------------------------------------------------------
# Alg. 1: log-domain Sinkhorn.
# --------------------------------------------------------------------------
def row_marginal(C: CostOperator, f: np.ndarray, g: np.ndarray, eps: float) -> np.ndarray:
    """r = P 1_m with P_ij = exp((f_i + g_j - C_ij)/eps) (Alg. 1 coupling)."""
    r = np.empty(C.n)
    for i0, Cb in C.row_blocks():
        P = np.exp((tensor_sum(f[i0:i0 + Cb.shape[0]], g) - Cb) / eps)
        r[i0:i0 + Cb.shape[0]] = P.sum(axis=1)
    return r


def col_marginal(C: CostOperator, f: np.ndarray, g: np.ndarray, eps: float) -> np.ndarray:
    """c = P^T 1_n."""
    c = np.empty(C.m)
    for j0, Cb in C.col_blocks():
        P_T = np.exp((tensor_sum(g[j0:j0 + Cb.shape[0]], f) - Cb) / eps)
        c[j0:j0 + Cb.shape[0]] = P_T.sum(axis=1)
    return c


def marginal_error(C: CostOperator, f, g, eps, a=None) -> float:
    """||exp((f (+) g - C)/eps) 1_m - a||_1: the stopping statistic of Alg. 1."""
    a = _weights(a, C.n)
    return float(np.sum(np.abs(row_marginal(C, f, g, eps) - a)))


def _update_f(C: CostOperator, f, g, eps, a):
    """f <- eps log a + min_eps(C - f (+) g) + f   (Alg. 1, sign as read)."""
    out = np.empty_like(f)
    for i0, Cb in C.row_blocks():
        i1 = i0 + Cb.shape[0]
        S = Cb - tensor_sum(f[i0:i1], g)
        out[i0:i1] = eps * np.log(a[i0:i1]) + softmin(S, eps) + f[i0:i1]
    return out


def _update_g(C: CostOperator, f, g, eps, b):
    """g <- eps log b + min_eps(C^T - g (+) f) + g   (Alg. 1, sign as read)."""
    out = np.empty_like(g)
    for j0, Cb in C.col_blocks():
        j1 = j0 + Cb.shape[0]
        S = Cb - tensor_sum(g[j0:j1], f)
        out[j0:j1] = eps * np.log(b[j0:j1]) + softmin(S, eps) + g[j0:j1]
    return out


@dataclass
class SinkhornResult:
    f: np.ndarray
    g: np.ndarray
    iters: int
    err: float
    converged: bool
    errs: list = field(default_factory=list)


def sinkhorn(a, X, b, Y, eps: float, tau: float, f_init=None, g_init=None,
             max_iter: int = 10000, C: CostOperator | None = None, cost=None) -> SinkhornResult:
    """Sink(a, X, b, Y, eps, tau, f_init, g_init) of Alg. 1.

    Potentials start at f_init, g_init (zero by default). While the row-marginal
    L1 error of P = exp((f (+) g - C)/eps) exceeds tau, update f then g. The
    error is checked before every iteration (so a warm start that already meets
    tau does no work). ``iters`` counts completed (f, g) update pairs; after
    ``max_iter`` of them the result is returned with converged = False. An error that
    overflows (a warm start far from feasible at small eps) is still above tau, so the
    loop goes on; only a NaN error stops it."""
    X = np.asarray(X, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    n, m = X.shape[0], Y.shape[0]
    a = _weights(a, n)
    b = _weights(b, m)
    C = C if C is not None else CostOperator(X, Y, cost=cost)
    f = np.zeros(n) if f_init is None else np.array(f_init, dtype=np.float64)
    g = np.zeros(m) if g_init is None else np.array(g_init, dtype=np.float64)
    it = 0
    errs = []
    while True:
        err = marginal_error(C, f, g, eps, a)
        errs.append(err)
        if math.isnan(err):
            return SinkhornResult(f, g, it, err, False, errs)
        if err <= tau:
            return SinkhornResult(f, g, it, err, True, errs)
        if it >= max_iter:
            return SinkhornResult(f, g, it, err, False, errs)
        f = _update_f(C, f, g, eps, a)
        g = _update_g(C, f, g, eps, b)
        it += 1


# --------------------------------------------------------------------------
# eq. (6), eq. (7): entropic potential and entropic map.
# --------------------------------------------------------------------------
def _softmax_rows(L: np.ndarray) -> np.ndarray:
    L0 = np.max(L, axis=1, keepdims=True)
    E = np.exp(L - L0)
    return E / np.sum(E, axis=1, keepdims=True)


def entropic_potential(xq, Y, g, eps: float, cost=None) -> np.ndarray:
    """f_hat(x) = min_eps([h(x - y_j) - g_j]_j)   (eq. (6), bracket sign as read)."""
    xq = np.atleast_2d(np.asarray(xq, dtype=np.float64))
    Y = np.asarray(Y, dtype=np.float64)
    g = np.asarray(g, dtype=np.float64)
    out = np.empty(xq.shape[0])
    step = _rows_per_block(Y.shape[0], Y.shape[1])
    for i0 in range(0, xq.shape[0], step):
        S = cost_matrix_rows(xq[i0:i0 + step], Y, cost) - g[None, :]
        out[i0:i0 + step] = softmin(S, eps)
    return out


def entropic_map(xq, Y, g, eps: float, cost=None) -> np.ndarray:
    """T_hat(x) = x - grad h*(grad f_hat(x))   (eq. (7)).

    grad f_hat(x) = sum_j p_j grad h(x - y_j) with p = softmax_j((g_j - h(x - y_j))/eps),
    the gradient of the soft-min in eq. (6)."""
    xq = np.atleast_2d(np.asarray(xq, dtype=np.float64))
    Y = np.asarray(Y, dtype=np.float64)
    g = np.asarray(g, dtype=np.float64)
    c = _cost(cost)
    out = np.empty_like(xq)
    step = _rows_per_block(Y.shape[0], Y.shape[1])
    for i0 in range(0, xq.shape[0], step):
        xb = xq[i0:i0 + step]
        diff = xb[:, None, :] - Y[None, :, :]
        p = _softmax_rows((g[None, :] - c.h(diff)) / eps)
        grad_f = np.einsum("ij,ijk->ik", p, c.grad_h(diff))
        out[i0:i0 + step] = xb - c.grad_h_star(grad_f)
    return out


# --------------------------------------------------------------------------
# Alg. 2: ProgOT.
# --------------------------------------------------------------------------
def barycentric_displacement(X, Y, f, g, eps: float, alpha: float, cost=None) -> np.ndarray:
    """Q <- diag(1/P 1) P; Z_i = grad h*(sum_j Q_ij grad h(x_i - y_j)); X <- X - alpha Z.

    P_ij = exp((f_i + g_j - C_ij)/eps). Row i of Q is P's row i divided by its sum;
    the common factor exp(f_i/eps) cancels, so each row is formed as a softmax of
    (f_i + g_j - C_ij)/eps with its maximum factored out (same value, no overflow)."""
    X = np.asarray(X, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    c = _cost(cost)
    out = np.empty_like(X)
    step = _rows_per_block(Y.shape[0], Y.shape[1])
    for i0 in range(0, X.shape[0], step):
        xb = X[i0:i0 + step]
        diff = xb[:, None, :] - Y[None, :, :]
        Q = _softmax_rows((tensor_sum(f[i0:i0 + step], g) - c.h(diff)) / eps)
        Z = c.grad_h_star(np.einsum("ij,ijk->ik", Q, c.grad_h(diff)))
        out[i0:i0 + step] = xb - alpha * Z
    return out


@dataclass
class ProgOTResult:
    x_out: np.ndarray          # X after the last displacement = T_Prog(x_i)
    g_all: np.ndarray          # (K, m) stored g^(k)
    f_last: np.ndarray         # f of the last solve
    x_last: np.ndarray         # X^(K): the cloud the last coupling P is defined on
    iters: list
    errs: list
    converged: list
    x_steps: list              # X^(1) .. X^(K) (inputs of each solve)
    eps_used: list = field(default_factory=list)  # eps_k of each solve


def progot(a, X, b, Y, eps_sched, alpha_sched, tau_sched, max_iter: int = 10000, cost=None) -> ProgOTResult:
    """ProgOT(a, X, b, Y, (eps_k, alpha_k, tau_k)_k) of Alg. 2, K = len(alpha_sched) solves.

    f = 0, g^(0) = 0; for k = 1..K: warm start (1 - alpha_k) f, (1 - alpha_k) g^(k-1);
    Sinkhorn at (eps_k, tau_k); displace X <- X - alpha_k Z. Returns the coupling
    potentials of the last solve and the map-estimator state (g^(k), eps_k, alpha_k).

    eps_sched is a sequence of K values, or a function (k, X^(k)) -> eps_k (k = 0..K-1)
    evaluated on the cloud that solve k transports (the theta rule of Sec. 5.2)."""
    X = np.array(X, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    K = len(alpha_sched)
    n, m = X.shape[0], Y.shape[0]
    f = np.zeros(n)
    g_prev = np.zeros(m)
    g_all = np.zeros((K, m))
    iters, errs, conv, steps, used = [], [], [], [], []
    x_last = X.copy()
    for k in range(K):
        alpha = float(alpha_sched[k])
        eps = float(eps_sched(k, X) if callable(eps_sched) else eps_sched[k])
        f_init, g_init = (1.0 - alpha) * f, (1.0 - alpha) * g_prev
        steps.append(X.copy())
        used.append(eps)
        x_last = X.copy()
        res = sinkhorn(a, X, b, Y, eps, float(tau_sched[k]), f_init, g_init, max_iter, cost=cost)
        f, g_prev = res.f, res.g
        g_all[k] = res.g
        iters.append(res.iters)
        errs.append(res.err)
        conv.append(res.converged)
        X = barycentric_displacement(X, Y, f, g_prev, eps, alpha, cost)
    return ProgOTResult(X, g_all, f, x_last, iters, errs, conv, steps, used)


# --------------------------------------------------------------------------
# Alg. 3: the progressive map on new points.
# --------------------------------------------------------------------------
def progot_map(xq, Y, g_all, eps_sched, alpha_sched, cost=None) -> np.ndarray:
    """T_Prog[b, Y, (g^(k), eps_k, alpha_k)_k](x) of Alg. 3 with alpha_K reset to 1.

    For each step: p = softmax_j((g^(k)_j - h(y - y_j))/eps_k) (no b_j factor, see the
    module notes), Delta = [grad h(y - y_j)]_j, z = grad h*(p^T Delta), y <- y - alpha_k z."""
    Yt = np.asarray(Y, dtype=np.float64)
    yq = np.array(np.atleast_2d(xq), dtype=np.float64)
    c = _cost(cost)
    K = len(eps_sched)
    alphas = [float(a) for a in alpha_sched]
    alphas[K - 1] = 1.0
    step = _rows_per_block(Yt.shape[0], Yt.shape[1])
    for k in range(K):
        g = np.asarray(g_all[k], dtype=np.float64)
        for i0 in range(0, yq.shape[0], step):
            yb = yq[i0:i0 + step]
            diff = yb[:, None, :] - Yt[None, :, :]
            p = _softmax_rows((g[None, :] - c.h(diff)) / float(eps_sched[k]))
            z = c.grad_h_star(np.einsum("ij,ijk->ik", p, c.grad_h(diff)))
            yq[i0:i0 + step] = yb - alphas[k] * z
    return yq


# --------------------------------------------------------------------------
# Sec. 4 "Setting step lengths" / Table 7.
# --------------------------------------------------------------------------
def alpha_schedule(K: int, kind: str = "constant") -> np.ndarray:
    """alpha_1..alpha_K for the three schedules, with alpha_K = 1 (Sec. 4).

    Each alpha_k is the fraction of the remaining path that step k covers, so for a
    target progress t_k: alpha_k = (t_k - t_{k-1}) / (1 - t_{k-1}), t_0 = 0.
    constant: t_k = k/K; accelerated: t_k = (k/K)^2; decelerated: alpha_k = 1/e."""
    if K < 1:
        raise ValueError("K >= 1")
    if kind == "decelerated":
        al = np.full(K, 1.0 / math.e)
        al[-1] = 1.0
        return al
    if kind == "constant":
        t = np.arange(0, K + 1) / K
    elif kind == "accelerated":
        t = (np.arange(0, K + 1) / K) ** 2
    else:
        raise ValueError(kind)
    al = (t[1:] - t[:-1]) / (1.0 - t[:-1])
    al[-1] = 1.0
    return al


def progress_times(alphas) -> np.ndarray:
    """t_k = 1 - prod_{l <= k} (1 - alpha_l), k = 1..K (Sec. 4)."""
    return 1.0 - np.cumprod(1.0 - np.asarray(alphas, dtype=np.float64))


# --------------------------------------------------------------------------
# Alg. 4: epsilon scheduler.
# --------------------------------------------------------------------------
def mean_cost(X, Y, cost=None) -> float:
    """(1/(n m)) sum_ij h(x_i - y_j), summed block by block from the definition."""
    C = CostOperator(X, Y, cache_limit=0, cost=cost)
    tot = 0.0
    for _, Cb in C.row_blocks():
        tot += float(np.sum(Cb))
    return tot / (C.n * C.m)


def eps_schedule(X, b, Y, Y_test, alphas, s_grid=None, beta0: float = 5.0, tau: float = 1e-6,
                 max_iter: int = 10000):
    """Alg. 4: eps0 = mean(C_XY)/20, sigma = mean(C_YY)/20; for each s_p solve
    Sink(b, Y, b, Y, s_p sigma, tau), map Y_test with (g, eps, alpha = 1) and score
    ||Y_test - T(Y_test)||^2; eps_K = s_{p*} sigma; eps_k = (1 - t_k) beta0 eps0 + t_k eps_K.

    Returns (eps_sched, info) with info = dict(eps0, sigma, errors, p_star, eps_K)."""
    if s_grid is None:
        s_grid = [2.0 ** e for e in range(-3, 4)]
    eps0 = mean_cost(X, Y) / 20.0
    sigma = mean_cost(Y, Y) / 20.0
    Yd = np.asarray(Y, dtype=np.float64)
    CYY = CostOperator(Yd, Yd)
    errors = []
    for s in s_grid:
        eps = s * sigma
        res = sinkhorn(b, Yd, b, Yd, eps, tau, max_iter=max_iter, C=CYY)
        T = progot_map(Y_test, Yd, [res.g], [eps], [1.0])
        errors.append(float(np.sum((np.asarray(Y_test, dtype=np.float64) - T) ** 2)))
    p_star = int(np.argmin(errors))  # first minimiser on ties
    eps_K = s_grid[p_star] * sigma
    t = progress_times(alphas)
    sched = (1.0 - t) * beta0 * eps0 + t * eps_K
    return sched, dict(eps0=eps0, sigma=sigma, errors=errors, p_star=p_star, eps_K=eps_K)


# --------------------------------------------------------------------------
# Sec. 5.2 coupling metrics and the eq. (5) dual objective.
# --------------------------------------------------------------------------
def coupling_cost(X, Y, f, g, eps: float, cost=None, X_cost=None) -> float:
    """<P, C> for P = exp((f (+) g - C)/eps).

    X_cost (optional, same number of rows as X): integrate the cost from X_cost instead,
    sum_ij P_ij h(xc_i - y_j) with P still defined on X. ProgOT's coupling is computed on
    the displaced cloud X^(K) but couples the original points (row i is point i), so
    Sec. 5.2 measures its transport cost against the original X."""
    C = CostOperator(X, Y, cache_limit=0, cost=cost)
    Cc = C if X_cost is None else CostOperator(X_cost, Y, cache_limit=0, cost=cost)
    tot = 0.0
    for (i0, Cb), (_, Ccb) in zip(C.row_blocks(), Cc.row_blocks()):
        P = np.exp((tensor_sum(f[i0:i0 + Cb.shape[0]], g) - Cb) / eps)
        tot += float(np.sum(P * Ccb))
    return tot


def coupling_entropy(X, Y, f, g, eps: float, cost=None) -> float:
    """E(P) = -sum_ij P_ij (log P_ij - 1)."""
    C = CostOperator(X, Y, cache_limit=0, cost=cost)
    tot = 0.0
    for i0, Cb in C.row_blocks():
        logP = (tensor_sum(f[i0:i0 + Cb.shape[0]], g) - Cb) / eps
        tot += float(-np.sum(np.exp(logP) * (logP - 1.0)))
    return tot


def dual_objective(a, X, b, Y, f, g, eps: float, cost=None) -> float:
    """<f, a> + <g, b> - eps <e^{f/eps}, K e^{g/eps}>, K_ij = exp(-C_ij/eps)   (eq. (5))."""
    X = np.asarray(X, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    a = _weights(a, X.shape[0])
    b = _weights(b, Y.shape[0])
    C = CostOperator(X, Y, cache_limit=0, cost=cost)
    mass = 0.0
    for i0, Cb in C.row_blocks():
        mass += float(np.sum(np.exp((tensor_sum(f[i0:i0 + Cb.shape[0]], g) - Cb) / eps)))
    return float(f @ a + g @ b - eps * mass)


# --------------------------------------------------------------------------
# Sec. 5.2 (coupling experiments): eps_k = theta cbar_k; Sec. 4: tau_k schedule.
# --------------------------------------------------------------------------
def eps_theta_rule(theta: float, Y, cost=None):
    """The rule (k, X^(k)) -> theta cbar_k, cbar_k = sum_ij h(x^(k)_i - y_j) / (20 n m),
    for ``progot``'s eps_sched."""
    Yd = np.asarray(Y, dtype=np.float64)

    def rule(k, Xk):
        return float(theta) * mean_cost(Xk, Yd, cost) / 20.0
    return rule


def tau_schedule(K: int, tau_first: float, tau_last: float) -> np.ndarray:
    """tau_1..tau_K decreasing linearly in k from tau_first to tau_last (Sec. 4)."""
    if K < 1:
        raise ValueError("K >= 1")
    if K == 1:
        return np.array([float(tau_last)])
    k = np.arange(K, dtype=np.float64)
    return tau_first + (tau_last - tau_first) * k / (K - 1)


# --------------------------------------------------------------------------
# eq. (8): Sinkhorn divergence.
# --------------------------------------------------------------------------
def eps_divergence(Y) -> float:
    """eps_D: 5% of the unweighted mean intra cost of the target cloud."""
    return 0.05 * mean_cost(Y, Y)


def sinkhorn_symmetric(a, X, eps: float, tau: float, max_iter: int = 10000) -> SinkhornResult:
    """Self-transport Sink(a, X, a, X, eps, tau) by the symmetric fixed point: with
    f_new = eps log a + min_eps(C - f (+) f) + f (the Alg. 1 f-update with g = f), stop
    when ||P 1 - a||_1 <= tau for P = exp((f (+) f - C)/eps), else f <- (f + f_new) / 2.
    The maximiser of eq. (5) for (a, X, a, X) is symmetric (f = g), so this reaches the
    same OT value as alternating updates, in far fewer iterations. Returns g = f."""
    X = np.asarray(X, dtype=np.float64)
    n = X.shape[0]
    a = _weights(a, n)
    C = CostOperator(X, X)
    f = np.zeros(n)
    it = 0
    errs = []
    while True:
        f_new = _update_f(C, f, f, eps, a)
        # row sums of P at the current f: a_i exp((f_i - f_new_i) / eps)
        err = float(np.sum(np.abs(a * np.expm1((f - f_new) / eps))))
        errs.append(err)
        if math.isnan(err):
            return SinkhornResult(f, f.copy(), it, err, False, errs)
        if err <= tau:
            return SinkhornResult(f, f.copy(), it, err, True, errs)
        if it >= max_iter:
            return SinkhornResult(f, f.copy(), it, err, False, errs)
        f = 0.5 * (f + f_new)
        it += 1


def ot_value(a, X, b, Y, eps: float, tau: float, max_iter: int = 10000, symmetric: bool = False):
    """OT_eps(X, Y): the eq. (5) objective at the potentials Alg. 1 returns (or the
    symmetric fixed point for a self term, Y = X, b = a). Returns (value, result)."""
    if symmetric:
        res = sinkhorn_symmetric(a, X, eps, tau, max_iter=max_iter)
    else:
        res = sinkhorn(a, X, b, Y, eps, tau, max_iter=max_iter)
    return dual_objective(a, X, b, Y, res.f, res.g, eps), res


def sinkhorn_divergence(a, X, b, Y, eps: float, tau: float, max_iter: int = 10000):
    """D_eps(X, Y) = OT_eps(X, Y) - (OT_eps(X, X) + OT_eps(Y, Y)) / 2   (eq. (8)), the
    self terms by the symmetric fixed point.
    Returns (D, (OT_xy, OT_xx, OT_yy), (iters_xy, iters_xx, iters_yy))."""
    oxy, rxy = ot_value(a, X, b, Y, eps, tau, max_iter)
    oxx, rxx = ot_value(a, X, a, X, eps, tau, max_iter, symmetric=True)
    oyy, ryy = ot_value(b, Y, b, Y, eps, tau, max_iter, symmetric=True)
    return oxy - 0.5 * (oxx + oyy), (oxy, oxx, oyy), (rxy.iters, rxx.iters, ryy.iters)


# --------------------------------------------------------------------------
# Sec. 5.3 / Prop. 3: the coupling diagonal against the identity coupling.
# --------------------------------------------------------------------------
def coupling_diagonal(X, Y, f, g, eps: float) -> np.ndarray:
    """log P_ii = (f_i + g_i - h(x_i - y_i)) / eps for n = m."""
    X = np.asarray(X, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    if X.shape != Y.shape:
        raise ValueError("the diagonal needs n = m")
    return (np.asarray(f, dtype=np.float64) + np.asarray(g, dtype=np.float64) - h(X - Y)) / eps


def diagonal_metrics(X, Y, f, g, eps: float):
    """(Tr(P), KL(Id/n || P)) with KL = -log n - (1/n) sum_i log P_ii."""
    logd = coupling_diagonal(X, Y, f, g, eps)
    n = logd.shape[0]
    return float(np.sum(np.exp(logd))), float(-math.log(n) - np.mean(logd))
