"""GPU parity of the C-ABI entry points against the FP64 oracle, on the same seeded
inputs. Sizes span several 128-row / 128-column tiles with ragged tails.

Tolerances (float32 path): map RMS error relative to the target spread <= 1e-4 and
marginal L1 error (recomputed by the oracle in float64 from the GPU's potentials)
<= 1e-4 plus the solve's own tau."""
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

import closed_forms as CF
from oracle import progot_oracle as O
from paper_2406_05061_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
TOL_FP32 = 1e-4


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


def marginal_l1(X, Y, f, g, eps, a=None, b=None):
    C = O.CostOperator(X, Y)
    n, m = C.n, C.m
    a = np.full(n, 1.0 / n) if a is None else a
    b = np.full(m, 1.0 / m) if b is None else b
    return float(np.abs(O.row_marginal(C, f, g, eps) - a).sum() + np.abs(O.col_marginal(C, f, g, eps) - b).sum())


def fp64_marginals(X, Y, f, g, eps, rows_per_block=8):
    """Row and column sums of P = exp((f (+) g - C)/eps) over ALL pairs in float64, C
    from the oracle's cost (differences, no norm expansion) in blocks of rows; the blocks
    run on host threads and are summed in block order."""
    X, Y = np.asarray(X, np.float64), np.asarray(Y, np.float64)
    f, g = np.asarray(f, np.float64), np.asarray(g, np.float64)
    n = X.shape[0]

    def block(i0):
        i1 = min(n, i0 + rows_per_block)
        P = np.exp((f[i0:i1, None] + g[None, :] - O.cost_matrix_rows(X[i0:i1], Y)) / eps)
        return i0, P.sum(1), P.sum(0)

    row, col = np.empty(n), np.zeros(Y.shape[0])
    with ThreadPoolExecutor(max(1, min(32, os.cpu_count() or 1))) as ex:
        for i0, r, c in ex.map(block, range(0, n, rows_per_block)):
            row[i0:i0 + r.shape[0]] = r
            col += c
    return row, col


def eps_for(p, frac=0.05):
    return frac * O.mean_cost(p.x, p.y)


SHAPES = [(300, 260, 16), (129, 517, 3), (1000, 700, 64), (257, 129, 17), (640, 384, 2), (200, 333, 96)]


@pytest.mark.parametrize("n,m,d", SHAPES)
def test_sinkhorn_potentials_parity(nat, n, m, d):
    p = W.gmm_pair(n, m, d, seed=n + m + d, k=4)
    eps = eps_for(p)
    tau = 1e-5
    res = nat.sinkhorn_potentials(dev(p.x), dev(p.y), eps, tau, max_iter=5000)
    ref = O.sinkhorn(None, p.x, None, p.y, eps, tau, max_iter=5000)
    assert ref.converged
    assert res.status == nat.PROGOT_OK, nat.last_error()
    f, g = host(res.f), host(res.g)
    assert abs(res.iters - ref.iters) <= max(2, ref.iters // 20)
    assert marginal_l1(p.x, p.y, f, g, eps) <= TOL_FP32 + tau
    T_gpu_g = O.entropic_map(p.x, p.y, g, eps)
    T_ref = O.entropic_map(p.x, p.y, ref.g, eps)
    assert map_rms_rel(T_gpu_g, T_ref, p.y) <= TOL_FP32
    # same initialisation and iteration -> same gauge: potentials agree directly
    scale = max(1.0, np.abs(ref.f).max())
    assert np.max(np.abs(f - ref.f)) <= 1e-3 * scale


def test_sinkhorn_weighted_marginals(nat):
    rng = np.random.default_rng(7)
    p = W.gmm_pair(300, 200, 8, seed=11, k=3)
    a = rng.uniform(0.5, 1.5, 300)
    b = rng.uniform(0.5, 1.5, 200)
    a, b = a / a.sum(), b / b.sum()
    eps = eps_for(p)
    res = nat.sinkhorn_potentials(dev(p.x), dev(p.y), eps, 1e-6, a=dev(a), b=dev(b))
    assert res.status == nat.PROGOT_OK, nat.last_error()
    ref = O.sinkhorn(a, p.x, b, p.y, eps, 1e-6)
    af, bf = a.astype(np.float32).astype(np.float64), b.astype(np.float32).astype(np.float64)
    assert marginal_l1(p.x, p.y, host(res.f), host(res.g), eps, af, bf) <= TOL_FP32
    assert map_rms_rel(O.entropic_map(p.x, p.y, host(res.g), eps), O.entropic_map(p.x, p.y, ref.g, eps),
                       p.y) <= TOL_FP32


@pytest.mark.parametrize("nq,m,d,K", [(333, 517, 17, 1), (1000, 700, 64, 3), (130, 129, 2, 2), (77, 1000, 256, 2)])
def test_entropic_map_apply_parity(nat, nq, m, d, K):
    p = W.gmm_pair(nq, m, d, seed=3 * nq + d, k=4)
    rng = np.random.default_rng(nq)
    base = eps_for(p)
    eps = [base * (1.0 - 0.3 * k) for k in range(K)]
    g_all = rng.normal(size=(K, m)) * base
    alpha = O.alpha_schedule(K)
    out = nat.entropic_map_apply(dev(p.x), dev(p.y), dev(g_all), eps, alpha)
    g32 = g_all.astype(np.float32).astype(np.float64)
    ref = O.progot_map(p.x, p.y, g32, eps, alpha)
    assert map_rms_rel(host(out), ref, p.y) <= TOL_FP32


def test_entropic_map_in_place_alias(nat):
    p = W.gmm_pair(200, 150, 16, seed=2, k=2)
    eps = [eps_for(p)]
    g = np.zeros((1, 150))
    xq = dev(p.x)
    out = nat.entropic_map_apply(xq, dev(p.y), dev(g), eps, [1.0], out=xq)
    assert out.data_ptr() == xq.data_ptr()
    assert map_rms_rel(host(out), O.progot_map(p.x, p.y, g, eps, [1.0]), p.y) <= TOL_FP32


@pytest.mark.parametrize("n,m,d", [(300, 260, 16), (1000, 700, 64), (129, 517, 3)])
def test_coupling_marginals_parity(nat, n, m, d):
    p = W.gmm_pair(n, m, d, seed=5 + n, k=3)
    eps = eps_for(p)
    ref = O.sinkhorn(None, p.x, None, p.y, eps, 1e-4)
    f32, g32 = ref.f.astype(np.float32), ref.g.astype(np.float32)
    row, col, err = nat.coupling_marginals(dev(p.x), dev(p.y), dev(f32), dev(g32), eps)
    C = O.CostOperator(p.x, p.y)
    r_ref = O.row_marginal(C, f32.astype(np.float64), g32.astype(np.float64), eps)
    c_ref = O.col_marginal(C, f32.astype(np.float64), g32.astype(np.float64), eps)
    np.testing.assert_allclose(host(row), r_ref, rtol=2e-4, atol=1e-9)
    np.testing.assert_allclose(host(col), c_ref, rtol=2e-4, atol=1e-9)
    err_ref = np.abs(r_ref - 1.0 / n).sum() + np.abs(c_ref - 1.0 / m).sum()
    assert abs(err - err_ref) <= 1e-4 * max(err_ref, 1e-3) + 2e-6


def test_mean_cost_closed_form_matches_definition(nat):
    p = W.gmm_pair(700, 333, 64, seed=9, k=3)
    assert abs(nat.progot_mean_cost(dev(p.x), dev(p.y)) - O.mean_cost(p.x, p.y)) <= 1e-9 * O.mean_cost(p.x, p.y)


def test_progot_solve_small_parity(nat):
    p = W.gmm_pair(600, 500, 16, seed=21, k=4)
    K = 4
    alpha = O.alpha_schedule(K)
    e0 = O.mean_cost(p.x, p.y) / 20
    eps = [5 * e0, 3 * e0, 2 * e0, e0]
    tau = [1e-5] * K
    res = nat.progot_solve(dev(p.x), dev(p.y), alpha, eps, tau, max_iter=5000)
    assert res.status == nat.PROGOT_OK, nat.last_error()
    ref = O.progot(None, p.x, None, p.y, eps, alpha, tau)
    assert map_rms_rel(host(res.x_out), ref.x_out, p.y) <= TOL_FP32
    assert map_rms_rel(host(res.x_last), ref.x_last, p.y) <= TOL_FP32
    for k in range(K):
        assert abs(res.iters[k] - ref.iters[k]) <= max(2, ref.iters[k] // 10)
    # final coupling (x_last, y, f_last, g_K): marginals recomputed in float64
    assert marginal_l1(host(res.x_last), p.y, host(res.f_last), host(res.g_all[K - 1]), eps[-1]) <= TOL_FP32 + tau[-1]
    # Alg. 3 with the returned state on the training points reproduces x_out
    Tq = nat.entropic_map_apply(dev(p.x), dev(p.y), res.g_all, eps, alpha)
    assert map_rms_rel(host(Tq), host(res.x_out), p.y) <= TOL_FP32


def test_progot_solve_config1_golden(nat):
    """The 2-D Gaussian workload (n = m = 512, K = 4, tau = 1e-6) against the stored
    oracle solve (tests/golden/make_golden.py)."""
    gold = np.load(os.path.join(HERE, "golden", "c1_progot.npz"))
    p = W.gaussian_affine(512, 512, 0)
    res = nat.progot_solve(dev(p.x), dev(p.y), gold["alpha"], gold["eps"], gold["tau"], max_iter=10000)
    assert res.status in (nat.PROGOT_OK, nat.PROGOT_ERR_NOT_CONVERGED)
    assert map_rms_rel(host(res.x_out), gold["x_out"], p.y) <= TOL_FP32
    assert map_rms_rel(host(res.x_last), gold["x_last"], p.y) <= TOL_FP32
    eK = float(gold["eps"][-1])
    assert marginal_l1(host(res.x_last), p.y, host(res.f_last), host(res.g_all[-1]), eK) <= TOL_FP32


def test_schedule_eps_alg4_parity(nat):
    p = W.gmm_pair(400, 300, 4, seed=31, k=3)
    yt = W.heldout_target(p, 100)
    al = O.alpha_schedule(4)
    eps_gpu, scores, pstar = nat.progot_schedule_eps(dev(p.x), dev(p.y), dev(yt), al, tau=1e-5)
    eps_ref, info = O.eps_schedule(p.x, None, p.y, yt, al, tau=1e-5)
    np.testing.assert_allclose(scores, info["errors"], rtol=1e-3)
    srt = np.sort(info["errors"])
    if srt[1] - srt[0] > 1e-2 * srt[0]:
        assert pstar == info["p_star"]
        np.testing.assert_allclose(eps_gpu, eps_ref, rtol=1e-9)


@pytest.mark.parametrize("precision", ["fp32", "bf16x3"])
def test_schedule_eps_two_point_closed_form(nat, precision):
    """Alg. 4 on the GPU against its closed form on a two-point target with weights
    b = (0.7, 0.3) (tests/closed_forms.py): every s_p's score, p* and the schedule."""
    y1, y2 = np.array([0.0, 0.0]), np.array([2.0, 0.0])
    Z = np.array([[0.7, 0.0], [1.3, 0.1]])
    X = np.random.default_rng(5).normal(size=(5, 2)).astype(np.float32).astype(np.float64)
    s_grid = [10.0, 14.0, 20.0, 28.0, 40.0]
    b = np.array([0.7, 0.3])
    al = O.alpha_schedule(4)
    eps_gpu, scores, pstar = nat.progot_schedule_eps(dev(X), dev(np.stack([y1, y2])), dev(Z), al, s_grid=s_grid,
                                                     tau=1e-6, b=dev(b), precision=precision)
    want, cf_scores, p, eps0, sigma = CF.two_point_alg4(X, y1, y2, Z, 4, s_grid, b=(0.7, 0.3))
    tol = 1e-4 if precision == "fp32" else 1e-3
    np.testing.assert_allclose(scores, cf_scores, rtol=tol)
    assert pstar == p
    np.testing.assert_allclose(eps_gpu, want, rtol=1e-6)


# ------------------------------------------------------------ edge cases
def test_max_iter_zero_reports_initial_error(nat):
    p = W.gmm_pair(200, 150, 4, seed=1, k=2)
    eps = eps_for(p)
    res = nat.sinkhorn_potentials(dev(p.x), dev(p.y), eps, 1e-9, max_iter=0)
    assert res.status == nat.PROGOT_ERR_NOT_CONVERGED and res.iters == 0
    err0 = O.marginal_error(O.CostOperator(p.x, p.y), np.zeros(200), np.zeros(150), eps)
    assert abs(res.err - err0) <= 1e-5 * err0


def test_warm_start_at_fixed_point_does_no_work(nat):
    p = W.gmm_pair(300, 200, 8, seed=4, k=2)
    eps = eps_for(p)
    r1 = nat.sinkhorn_potentials(dev(p.x), dev(p.y), eps, 1e-5)
    r2 = nat.sinkhorn_potentials(dev(p.x), dev(p.y), eps, 1e-5, f=r1.f.clone(), g=r1.g.clone())
    assert r2.iters == 0 and r2.status == nat.PROGOT_OK


def test_single_point_target(nat):
    """m = 1: every x maps to the single target point; g-sweeps see one column."""
    rng = np.random.default_rng(3)
    x = rng.normal(size=(257, 5))
    y = rng.normal(size=(1, 5))
    res = nat.sinkhorn_potentials(dev(x), dev(y), 1.0, 1e-6)
    out = nat.entropic_map_apply(dev(x), dev(y), res.g.reshape(1, 1), [1.0], [1.0])
    np.testing.assert_allclose(host(out), np.repeat(y, 257, 0).astype(np.float32), atol=1e-6)


def test_huge_eps_maps_to_target_mean(nat):
    p = W.gmm_pair(300, 400, 16, seed=8, k=2)
    res = nat.sinkhorn_potentials(dev(p.x), dev(p.y), 1e7, 1e-6)
    out = nat.entropic_map_apply(dev(p.x), dev(p.y), res.g.reshape(1, -1), [1e7], [1.0])
    np.testing.assert_allclose(host(out), np.broadcast_to(p.y.astype(np.float64).mean(0), (300, 16)), atol=1e-4)


def test_non_finite_input_reports_numeric(nat):
    p = W.gmm_pair(200, 150, 4, seed=1, k=2)
    x = p.x.copy()
    x[17, 2] = np.nan
    with pytest.raises(nat.ProgOTError) as ei:
        nat.sinkhorn_potentials(dev(x), dev(p.y), eps_for(p), 1e-6, max_iter=50)
    assert ei.value.code == nat.PROGOT_ERR_NUMERIC


def test_invalid_eps_on_device_call(nat):
    p = W.gmm_pair(64, 64, 4, seed=1, k=2)
    with pytest.raises(nat.ProgOTError) as ei:
        nat.sinkhorn_potentials(dev(p.x), dev(p.y), -1.0, 1e-6)
    assert ei.value.code == nat.PROGOT_ERR_INVALID_ARG


# ---------------------------------------------------- full-size sampled parity
def test_full_size_gmm64_sampled_parity(nat):
    """n = m = 8192, d = 64 (the benchmark workload), in the benchmark's launch
    configuration: one Sinkhorn solve at the first scheduled eps, then the coupling
    marginals and the entropic map checked on 48 sampled rows computed one by one by
    the oracle from the same potentials."""
    p = W.gmm_pair(8192, 8192, 64, seed=1)
    eps = 5 * O.mean_cost(p.x[:2048], p.y[:2048]) / 20
    x, y = dev(p.x), dev(p.y)
    res = nat.sinkhorn_potentials(x, y, eps, 1e-5, max_iter=2000)
    assert res.status == nat.PROGOT_OK, nat.last_error()
    f, g = host(res.f), host(res.g)
    row, col, err = nat.coupling_marginals(x, y, res.f, res.g, eps)
    out = nat.entropic_map_apply(x, y, res.g.reshape(1, -1), [eps], [1.0])
    rows = np.random.default_rng(0).choice(8192, 48, replace=False)
    X64, Y64 = p.x.astype(np.float64), p.y.astype(np.float64)
    Cs = O.cost_matrix_rows(X64[rows], Y64)
    r_ref = np.exp((f[rows, None] + g[None, :] - Cs) / eps).sum(1)
    np.testing.assert_allclose(host(row)[rows], r_ref, rtol=2e-4)
    T_ref = O.entropic_map(X64[rows], Y64, g, eps)
    assert map_rms_rel(host(out)[rows], T_ref, p.y) <= TOL_FP32
    assert err <= 1e-5 + TOL_FP32


# ---------------------------------------------------- tensor-core (bf16 split) path
TOL_MIXED = 1e-3
TC_SHAPES = [(300, 260, 16), (1000, 700, 64), (257, 129, 17), (129, 517, 3), (640, 384, 128), (333, 200, 256)]


@pytest.mark.parametrize("n,m,d", TC_SHAPES)
def test_sinkhorn_potentials_parity_bf16x3(nat, n, m, d):
    p = W.gmm_pair(n, m, d, seed=n + m + d, k=4)
    eps = eps_for(p)
    tau = 1e-4
    res = nat.sinkhorn_potentials(dev(p.x), dev(p.y), eps, tau, max_iter=5000, precision="bf16x3")
    assert res.status == nat.PROGOT_OK, nat.last_error()
    ref = O.sinkhorn(None, p.x, None, p.y, eps, 1e-6, max_iter=5000)
    f, g = host(res.f), host(res.g)
    assert marginal_l1(p.x, p.y, f, g, eps) <= TOL_MIXED
    assert map_rms_rel(O.entropic_map(p.x, p.y, g, eps), O.entropic_map(p.x, p.y, ref.g, eps), p.y) <= TOL_MIXED


def test_bf16_single_product_runs_and_is_coarser(nat):
    """The hi-only product is a speed option without the mixed-precision accuracy
    claim: it must run and stay within 1e-2 here, and bf16x3 must be at least as
    accurate."""
    p = W.gmm_pair(600, 500, 64, seed=77, k=4)
    eps = eps_for(p)
    ref = O.sinkhorn(None, p.x, None, p.y, eps, 1e-6)
    T_ref = O.entropic_map(p.x, p.y, ref.g, eps)
    errs = {}
    for prec in ("bf16", "bf16x3"):
        res = nat.sinkhorn_potentials(dev(p.x), dev(p.y), eps, 1e-4, precision=prec)
        errs[prec] = map_rms_rel(O.entropic_map(p.x, p.y, host(res.g), eps), T_ref, p.y)
    assert errs["bf16"] <= 1e-2
    assert errs["bf16x3"] <= errs["bf16"] + 1e-6


def test_progot_solve_parity_bf16x3(nat):
    p = W.gmm_pair(700, 600, 64, seed=23, k=4)
    K = 4
    alpha = O.alpha_schedule(K)
    e0 = O.mean_cost(p.x, p.y) / 20
    eps = [5 * e0, 3 * e0, 2 * e0, e0]
    res = nat.progot_solve(dev(p.x), dev(p.y), alpha, eps, [1e-4] * K, max_iter=5000, precision="bf16x3")
    assert res.status == nat.PROGOT_OK, nat.last_error()
    ref = O.progot(None, p.x, None, p.y, eps, alpha, [1e-6] * K)
    assert map_rms_rel(host(res.x_out), ref.x_out, p.y) <= TOL_MIXED
    assert marginal_l1(host(res.x_last), p.y, host(res.f_last), host(res.g_all[K - 1]), eps[-1]) <= TOL_MIXED


def test_full_size_gmm64_parity_bf16x3(nat):
    """n = m = 8192, d = 64 in the benchmark's launch configuration, bf16x3 sweeps at
    eps = 5 eps0 (the first scheduled step): both marginals of the GPU's (f, g)
    recomputed over all 8192^2 pairs in float64 (L1 <= 1e-3), and the GPU's map on 48
    sampled rows against the oracle's eq. (7) map from the same g."""
    p = W.gmm_pair(8192, 8192, 64, seed=1)
    eps = 5 * O.mean_cost(p.x[:2048], p.y[:2048]) / 20
    x, y = dev(p.x), dev(p.y)
    res = nat.sinkhorn_potentials(x, y, eps, 1e-4, max_iter=2000, precision="bf16x3")
    assert res.status == nat.PROGOT_OK, nat.last_error()
    f, g = host(res.f), host(res.g)
    row, col = fp64_marginals(p.x, p.y, f, g, eps)
    l1 = np.abs(row - 1.0 / 8192).sum() + np.abs(col - 1.0 / 8192).sum()
    assert l1 <= TOL_MIXED, l1
    rows = np.random.default_rng(1).choice(8192, 48, replace=False)
    X64, Y64 = p.x.astype(np.float64), p.y.astype(np.float64)
    out = nat.entropic_map_apply(x, y, res.g.reshape(1, -1), [eps], [1.0], precision="bf16x3")
    T_ref = O.entropic_map(X64[rows], Y64, g, eps)
    assert map_rms_rel(host(out)[rows], T_ref, p.y) <= TOL_MIXED


def test_full_size_sphere_65536_d256_sampled_parity(nat):
    """n = m = 65536 points on the sphere in d = 256 (the large coupling workload; the
    cost matrix would be 17 GB): one bf16x3 Sinkhorn solve, then row marginals and the
    map on 32 sampled rows computed one by one by the oracle from the GPU's potentials."""
    p = W.sphere_mixture_pair(65536, 65536, 256, seed=2)
    X64, Y64 = p.x.astype(np.float64), p.y.astype(np.float64)
    sub = np.random.default_rng(0).choice(65536, 1024, replace=False)
    eps = O.mean_cost(X64[sub], Y64[sub]) / 20
    x, y = dev(p.x), dev(p.y)
    res = nat.sinkhorn_potentials(x, y, eps, 1e-4, max_iter=3000, precision="bf16x3")
    assert res.status == nat.PROGOT_OK, nat.last_error()
    f, g = host(res.f), host(res.g)
    rows = np.random.default_rng(3).choice(65536, 32, replace=False)
    Cs = O.cost_matrix_rows(X64[rows], Y64)
    r_ref = np.exp((f[rows, None] + g[None, :] - Cs) / eps).sum(1)
    assert np.abs(r_ref - 1.0 / 65536).sum() * 65536 / 32 <= 2 * TOL_MIXED
    out = nat.entropic_map_apply(x, y, res.g.reshape(1, -1), [eps], [1.0], precision="bf16x3")
    T_ref = O.entropic_map(X64[rows], Y64, g, eps)
    assert map_rms_rel(host(out)[rows], T_ref, p.y) <= TOL_MIXED


def test_benchmark_workload_every_step_teacher_forced_bf16x3(nat):
    """The benchmark workload exactly as bench.py runs it: n = m = 8192, d = 64, K = 8
    constant-speed steps, bf16x3, tau = 1e-4, eps_k from the GPU's Alg. 4 scheduler on
    the held-out target draw. Every step k is teacher-forced on 48 sampled rows: the
    oracle applies eq. (7) with the GPU's g^(k) to the GPU's X^(k-1), and the GPU's
    displacement (X^(k) - (1 - alpha_k) X^(k-1)) / alpha_k must match it within map RMS
    1e-3; the sampled rows' float64 row sums of (f^(k), g^(k)), scaled to all rows, stay
    within 1e-3. X^(k) and f^(k) come from solves truncated after step k, which repeat
    the full solve's launches: their g's must equal the full solve's bit for bit. At the
    last step both marginals of (X^(K-1), Y, f_K, g_K) are recomputed over all 8192^2
    pairs in float64: L1 <= 1e-3."""
    p = W.gmm_pair(8192, 8192, 64, seed=1, k=8)
    yt = W.heldout_target(p)
    K = 8
    alpha = nat.progot_schedule_alpha(K, "constant")
    tau = [1e-4] * K
    x, y = dev(p.x), dev(p.y)
    eps, _, _ = nat.progot_schedule_eps(x, y, dev(yt), alpha, tau=tau[-1], precision="bf16x3")
    eps = [float(e) for e in eps]
    full = nat.progot_solve(x, y, alpha, eps, tau, max_iter=10000, precision="bf16x3")
    assert full.status == nat.PROGOT_OK, nat.last_error()
    rows = np.random.default_rng(56).choice(8192, 48, replace=False)
    Y64 = p.y.astype(np.float64)
    X_prev = p.x.astype(np.float64)
    for k in range(K):
        if k < K - 1:
            part = nat.progot_solve(x, y, alpha[:k + 1], eps[:k + 1], tau[:k + 1], max_iter=10000,
                                    precision="bf16x3")
            assert part.status == nat.PROGOT_OK, nat.last_error()
            assert torch.equal(part.g_all, full.g_all[:k + 1])
            X_k, f_k = host(part.x_out), host(part.f_last)
        else:
            assert np.array_equal(host(full.x_last), X_prev)
            X_k, f_k = host(full.x_out), host(full.f_last)
        g_k = host(full.g_all[k])
        T_ref = O.entropic_map(X_prev[rows], Y64, g_k, eps[k])
        T_gpu = (X_k[rows] - (1.0 - alpha[k]) * X_prev[rows]) / alpha[k]
        assert map_rms_rel(T_gpu, T_ref, p.y) <= TOL_MIXED, (k, map_rms_rel(T_gpu, T_ref, p.y))
        C = O.cost_matrix_rows(X_prev[rows], Y64)
        r = np.exp((f_k[rows, None] + g_k[None, :] - C) / eps[k]).sum(1)
        assert np.abs(r - 1.0 / 8192).sum() * 8192 / 48 <= TOL_MIXED, k
        X_prev = X_k
    row, col = fp64_marginals(host(full.x_last), p.y, host(full.f_last), host(full.g_all[K - 1]), eps[-1])
    l1 = np.abs(row - 1.0 / 8192).sum() + np.abs(col - 1.0 / 8192).sum()
    assert l1 <= TOL_MIXED, l1


def test_large_coupling_progot_sampled_steps_bf16x3(nat):
    """The large coupling configuration as the bench runs it: two 32-component mixtures on
    the unit sphere, n = m = 65536, d = 256, K = 16 constant-speed steps, bf16x3, tau = 1e-4,
    eps_k from the GPU's Alg. 4 on the held-out draw. Steps 1, 8 and 16 are teacher-forced
    on 32 sampled rows: the oracle applies eq. (7) with the GPU's g^(k) to the GPU's
    X^(k-1) (from solves truncated after step k - 1, whose g's equal the full solve's bit
    for bit), and the GPU's displacement must match it within map RMS 1e-3; the sampled
    rows' float64 row sums of (f^(k), g^(k)), scaled to all rows, stay within 1e-3."""
    p = W.sphere_mixture_pair(65536, 65536, 256, seed=2)
    yt = W.heldout_target(p)
    K = 16
    alpha = nat.progot_schedule_alpha(K, "constant")
    tau = [1e-4] * K
    x, y = dev(p.x), dev(p.y)
    eps, _, _ = nat.progot_schedule_eps(x, y, dev(yt), alpha, tau=tau[-1], precision="bf16x3")
    eps = [float(e) for e in eps]
    full = nat.progot_solve(x, y, alpha, eps, tau, max_iter=10000, precision="bf16x3")
    assert full.status == nat.PROGOT_OK, nat.last_error()
    rows = np.random.default_rng(57).choice(65536, 32, replace=False)
    Y64 = p.y.astype(np.float64)

    def upto(k):  # X^(k) and f^(k) from the solve cut after step k (k = 0: the input cloud)
        if k == 0:
            return p.x.astype(np.float64), None
        part = nat.progot_solve(x, y, alpha[:k], eps[:k], tau[:k], max_iter=10000, precision="bf16x3")
        assert part.status == nat.PROGOT_OK, nat.last_error()
        assert torch.equal(part.g_all, full.g_all[:k])
        return host(part.x_out), host(part.f_last)

    for k in (0, 7, K - 1):  # steps 1, 8, 16
        X_prev, _ = upto(k)
        if k < K - 1:
            X_k, f_k = upto(k + 1)
        else:
            assert np.array_equal(host(full.x_last), X_prev)
            X_k, f_k = host(full.x_out), host(full.f_last)
        g_k = host(full.g_all[k])
        T_ref = O.entropic_map(X_prev[rows], Y64, g_k, eps[k])
        T_gpu = (X_k[rows] - (1.0 - alpha[k]) * X_prev[rows]) / alpha[k]
        assert map_rms_rel(T_gpu, T_ref, p.y) <= TOL_MIXED, (k, map_rms_rel(T_gpu, T_ref, p.y))
        r = np.array([np.exp((f_k[i] + g_k - O.cost_matrix_rows(X_prev[i:i + 1], Y64)[0]) / eps[k]).sum()
                      for i in rows])
        assert np.abs(r - 1.0 / 65536).sum() * 65536 / len(rows) <= TOL_MIXED, k
