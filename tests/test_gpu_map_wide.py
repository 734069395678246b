"""The tensor-core map step for 64 < d <= 256 (Alg. 2's displacement and Alg. 3) against
the FP64 oracle: the progressive map on query clouds with ragged sizes, a full ProgOT
solve, in-place use, the 65536-point, d = 256 configuration on sampled rows, and the
hi-only precision on the tensor-core maps of every width."""
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
    native.set_map_tc(True)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def host(t):
    return t.detach().cpu().numpy().astype(np.float64)


def map_rms_rel(T_gpu, T_ref, Y):
    Y = np.asarray(Y, dtype=np.float64)
    spread = np.sqrt(np.mean(np.sum((Y - Y.mean(0)) ** 2, 1)))
    return float(np.sqrt(np.mean(np.sum((np.asarray(T_gpu) - np.asarray(T_ref)) ** 2, 1))) / spread)


@pytest.mark.parametrize("nq,m,d,K", [(333, 517, 96, 1), (1000, 700, 128, 3), (129, 130, 200, 2), (700, 1100, 256, 2),
                                      (257, 65, 130, 1), (1, 31, 65, 1), (130, 33, 256, 2)])
def test_wide_map_apply_parity_bf16x3(nat, nq, m, d, K):
    """Alg. 3 with given g^(k) on the bf16x3 path (tensor-core map, S once per 32-column
    tile and every 64-coordinate chunk of O in TMEM) against the oracle's progressive map
    from the same g (float32 round trip), map RMS relative to the target spread <= 1e-3;
    ragged m below one tile and a single query row included."""
    p = W.gmm_pair(nq, m, d, seed=5 * nq + d, k=4)
    rng = np.random.default_rng(d + nq)
    base = 0.05 * O.mean_cost(p.x, p.y)
    eps = [base * (1.0 - 0.25 * k) for k in range(K)]
    g_all = rng.normal(size=(K, m)) * base
    alpha = O.alpha_schedule(K)
    out = nat.entropic_map_apply(dev(p.x), dev(p.y), dev(g_all), eps, alpha, precision="bf16x3")
    ref = O.progot_map(p.x, p.y, g_all.astype(np.float32).astype(np.float64), eps, alpha)
    assert map_rms_rel(host(out), ref, p.y) <= TOL_MIXED


def test_wide_map_matches_cuda_core_map_and_aliases(nat):
    """The tensor-core map and the float32 CUDA-core map of the same step agree within the
    mixed bar, and the in-place call (out = xq) gives the same result."""
    p = W.gmm_pair(900, 800, 192, seed=17, k=5)
    eps = [0.04 * O.mean_cost(p.x, p.y)]
    g = np.random.default_rng(3).normal(size=(1, 800)) * eps[0]
    gd = dev(g)
    outs = {}
    for tc in (True, False):
        nat.set_map_tc(tc)
        outs[tc] = host(nat.entropic_map_apply(dev(p.x), dev(p.y), gd, eps, [1.0], precision="bf16x3"))
    nat.set_map_tc(True)
    assert map_rms_rel(outs[True], outs[False], p.y) <= TOL_MIXED
    xq = dev(p.x)
    o2 = nat.entropic_map_apply(xq, dev(p.y), gd, eps, [1.0], out=xq, precision="bf16x3")
    assert o2.data_ptr() == xq.data_ptr()
    np.testing.assert_array_equal(host(o2), outs[True])


@pytest.mark.parametrize("d", [128, 256])
def test_progot_solve_parity_bf16x3_wide(nat, d):
    """A K = 3 ProgOT solve with the tensor-core map for d > 64 against the oracle's solve."""
    p = W.gmm_pair(600, 500, d, seed=29 + d, k=4)
    K = 3
    alpha = O.alpha_schedule(K)
    e0 = O.mean_cost(p.x, p.y) / 20
    eps = [4 * e0, 2 * e0, e0]
    res = nat.progot_solve(dev(p.x), dev(p.y), alpha, eps, [1e-4] * K, max_iter=5000, precision="bf16x3")
    assert res.status == nat.PROGOT_OK, nat.last_error()
    ref = O.progot(None, p.x, None, p.y, eps, alpha, [1e-6] * K)
    assert map_rms_rel(host(res.x_out), ref.x_out, p.y) <= TOL_MIXED


@pytest.mark.parametrize("n", [4096, 65536])
def test_wide_map_full_size_sphere_d256_sampled(nat, n):
    """n x n points on the sphere in d = 256 (65536: the large coupling configuration;
    4096: every CTA runs tens of tiles over several row blocks, so the operand stages,
    TMEM buffers and the P hand-off all wrap): one bf16x3 map step with a given g,
    checked on 32 sampled rows computed one by one by the oracle."""
    p = W.sphere_mixture_pair(n, n, 256, seed=2)
    X64, Y64 = p.x.astype(np.float64), p.y.astype(np.float64)
    sub = np.random.default_rng(0).choice(n, 1024, replace=False)
    eps = O.mean_cost(X64[sub], Y64[sub]) / 20
    g = np.random.default_rng(4).normal(size=n) * 0.1 * eps
    out = nat.entropic_map_apply(dev(p.x), dev(p.y), dev(g.reshape(1, -1)), [eps], [1.0], precision="bf16x3")
    rows = np.random.default_rng(5).choice(n, 32, replace=False)
    T_ref = O.entropic_map(X64[rows], Y64, g.astype(np.float32).astype(np.float64), eps)
    assert map_rms_rel(host(out)[rows], T_ref, p.y) <= TOL_MIXED


@pytest.mark.parametrize("d", [64, 128, 256])
def test_hi_only_precision_map_and_solve(nat, d):
    """precision = bf16 (hi parts only, one product per term) on the tensor-core maps for
    d <= 64 and d > 64: the map step within 1e-2 of the oracle's, a K = 2 solve within
    1e-2 of the oracle's solve, and bf16x3 at least as accurate on the same step."""
    p = W.gmm_pair(500, 450, d, seed=41 + d, k=4)
    eps = [0.05 * O.mean_cost(p.x, p.y)]
    g = np.random.default_rng(d).normal(size=(1, 450)) * eps[0]
    ref = O.progot_map(p.x, p.y, g.astype(np.float32).astype(np.float64), eps, [1.0])
    errs = {}
    for prec in ("bf16", "bf16x3"):
        out = nat.entropic_map_apply(dev(p.x), dev(p.y), dev(g), eps, [1.0], precision=prec)
        errs[prec] = map_rms_rel(host(out), ref, p.y)
    assert errs["bf16"] <= 1e-2
    assert errs["bf16x3"] <= min(errs["bf16"], TOL_MIXED)
    K = 2
    alpha = O.alpha_schedule(K)
    e0 = O.mean_cost(p.x, p.y) / 20
    res = nat.progot_solve(dev(p.x), dev(p.y), alpha, [3 * e0, e0], [1e-3] * K, max_iter=5000, precision="bf16")
    assert res.status == nat.PROGOT_OK, nat.last_error()
    ref = O.progot(None, p.x, None, p.y, [3 * e0, e0], alpha, [1e-6] * K)
    assert map_rms_rel(host(res.x_out), ref.x_out, p.y) <= 1e-2
