"""GPU parity of the p-norm cost h(z) = (1/p) sum_k |z_k|^p (Sec. 5.2, p = 1.5; float32
CUDA cores) against the FP64 oracle with the same cost: Sinkhorn, ProgOT with a fixed
schedule and with the theta rule, Alg. 3, coupling metrics and the pairwise mean cost.
Sizes span several 128-row tiles with ragged tails."""
import numpy as np
import pytest

from oracle import progot_oracle as O
from paper_2406_05061_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_FP32 = 1e-4
P15 = O.PNorm(1.5)


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


def marginal_l1(X, Y, f, g, eps, cost):
    C = O.CostOperator(X, Y, cost=cost)
    return float(np.abs(O.row_marginal(C, f, g, eps) - 1.0 / C.n).sum() +
                 np.abs(O.col_marginal(C, f, g, eps) - 1.0 / C.m).sum())


@pytest.mark.parametrize("n,m,d,p", [(300, 260, 16, 1.5), (129, 517, 3, 1.5), (640, 384, 47, 1.5),
                                     (257, 129, 2, 1.5), (300, 400, 8, 1.25), (200, 300, 12, 3.0)])
def test_sinkhorn_pnorm_parity(nat, n, m, d, p):
    cost = O.PNorm(p)
    pr = W.gmm_pair(n, m, d, seed=n + m + d, k=4)
    eps = 0.05 * O.mean_cost(pr.x, pr.y, cost)
    tau = 1e-5
    res = nat.sinkhorn_potentials_pnorm(dev(pr.x), dev(pr.y), p, eps, tau, max_iter=10000)
    assert res.status == nat.PROGOT_OK, nat.last_error()
    ref = O.sinkhorn(None, pr.x, None, pr.y, eps, 1e-7, max_iter=20000, cost=cost)
    f, g = host(res.f), host(res.g)
    assert marginal_l1(pr.x, pr.y, f, g, eps, cost) <= TOL_FP32 + tau
    T_gpu_g = O.entropic_map(pr.x, pr.y, g, eps, cost)
    T_ref = O.entropic_map(pr.x, pr.y, ref.g, eps, cost)
    assert map_rms_rel(T_gpu_g, T_ref, pr.y) <= TOL_FP32


def test_pnorm_two_matches_squared_euclidean_path(nat):
    # h_2 = |z|^2 / 2 at eps / 2 is the squared Euclidean problem at eps: the p-norm
    # kernels (general p) and the dot-product kernels give the same map
    pr = W.gmm_pair(500, 420, 24, seed=60, k=3)
    eps = 0.05 * O.mean_cost(pr.x, pr.y)
    a = nat.sinkhorn_potentials(dev(pr.x), dev(pr.y), eps, 1e-5)
    b = nat.sinkhorn_potentials_pnorm(dev(pr.x), dev(pr.y), 2.0, eps / 2, 1e-5)
    Ta = O.entropic_map(pr.x, pr.y, host(a.g), eps)
    Tb = O.entropic_map(pr.x, pr.y, host(b.g), eps / 2, O.PNorm(2.0))
    assert map_rms_rel(Ta, Tb, pr.y) <= 2 * TOL_FP32


def test_progot_pnorm_parity_and_alg3(nat):
    pr = W.gmm_pair(600, 500, 16, seed=61, k=4)
    K = 4
    alpha = O.alpha_schedule(K)
    e0 = O.mean_cost(pr.x, pr.y, P15) / 20
    eps = [4 * e0, 3 * e0, 2 * e0, e0]
    tau = [1e-5] * K
    res, _ = nat.progot_solve_pnorm(dev(pr.x), dev(pr.y), 1.5, alpha, tau, eps=eps, max_iter=10000)
    assert res.status == nat.PROGOT_OK, nat.last_error()
    ref = O.progot(None, pr.x, None, pr.y, eps, alpha, tau, cost=P15)
    assert map_rms_rel(host(res.x_out), ref.x_out, pr.y) <= TOL_FP32
    assert map_rms_rel(host(res.x_last), ref.x_last, pr.y) <= TOL_FP32
    assert marginal_l1(host(res.x_last), pr.y, host(res.f_last), host(res.g_all[K - 1]), eps[-1], P15) <= TOL_FP32
    # Alg. 3 with the stored g^(k) on the training points reproduces x_out
    Tq = nat.entropic_map_apply_pnorm(dev(pr.x), dev(pr.y), 1.5, res.g_all, eps, alpha)
    assert map_rms_rel(host(Tq), host(res.x_out), pr.y) <= TOL_FP32
    # ... and so does the oracle's Alg. 3 on fresh points, against the GPU's Alg. 3
    xq = W.gmm_pair(300, 10, 16, seed=62, k=4).x
    Tg = nat.entropic_map_apply_pnorm(dev(xq), dev(pr.y), 1.5, res.g_all, eps, alpha)
    To = O.progot_map(xq, pr.y, host(res.g_all), eps, alpha, P15)
    assert map_rms_rel(host(Tg), To, pr.y) <= TOL_FP32


def test_progot_pnorm_theta_rule(nat):
    pr = W.gmm_pair(400, 350, 12, seed=63, k=3)
    K, theta = 3, 1.0
    alpha = O.alpha_schedule(K)
    tau = O.tau_schedule(K, 1e-4, 1e-5)
    res, eps = nat.progot_solve_pnorm(dev(pr.x), dev(pr.y), 1.5, alpha, tau, theta=theta, max_iter=10000)
    assert res.status == nat.PROGOT_OK, nat.last_error()
    ref = O.progot(None, pr.x, None, pr.y, O.eps_theta_rule(theta, pr.y, P15), alpha, tau, cost=P15)
    assert eps[0] == pytest.approx(ref.eps_used[0], rel=1e-5)
    np.testing.assert_allclose(eps, ref.eps_used, rtol=1e-3)
    assert map_rms_rel(host(res.x_out), ref.x_out, pr.y) <= TOL_FP32


def test_coupling_metrics_and_mean_cost_pnorm(nat):
    pr = W.gmm_pair(700, 530, 9, seed=64, k=3)
    eps = 0.05 * O.mean_cost(pr.x, pr.y, P15)
    sk = O.sinkhorn(None, pr.x, None, pr.y, eps, 1e-8, cost=P15)
    f32, g32 = sk.f.astype(np.float32), sk.g.astype(np.float32)
    f, g = f32.astype(np.float64), g32.astype(np.float64)
    met = nat.coupling_metrics_pnorm(dev(pr.x), dev(pr.y), 1.5, dev(f32), dev(g32), eps)
    assert met["transport_cost"] == pytest.approx(O.coupling_cost(pr.x, pr.y, f, g, eps, P15), rel=TOL_FP32)
    assert met["entropy"] == pytest.approx(O.coupling_entropy(pr.x, pr.y, f, g, eps, P15), rel=TOL_FP32)
    dual = O.dual_objective(None, pr.x, None, pr.y, f, g, eps, P15)
    assert met["dual"] == pytest.approx(dual, rel=TOL_FP32, abs=TOL_FP32 * met["transport_cost"])
    mc = nat.progot_mean_cost_pnorm(dev(pr.x), dev(pr.y), 1.5)
    assert mc == pytest.approx(O.mean_cost(pr.x, pr.y, P15), rel=1e-5)


def test_coupling_metrics_pnorm_against_the_original_cloud(nat):
    pr = W.gmm_pair(500, 400, 10, seed=65, k=3)
    K = 2
    alpha = O.alpha_schedule(K)
    e0 = O.mean_cost(pr.x, pr.y, P15) / 20
    res, _ = nat.progot_solve_pnorm(dev(pr.x), dev(pr.y), 1.5, alpha, [1e-5] * K, eps=[2 * e0, e0], max_iter=10000)
    assert res.status == nat.PROGOT_OK, nat.last_error()
    xl, f, g = host(res.x_last), host(res.f_last), host(res.g_all[K - 1])
    met = nat.coupling_metrics_pnorm(res.x_last, dev(pr.y), 1.5, res.f_last, res.g_all[K - 1], e0, x_cost=dev(pr.x))
    assert met["transport_cost"] == pytest.approx(O.coupling_cost(xl, pr.y, f, g, e0, P15, X_cost=pr.x), rel=TOL_FP32)
