"""The persistent tensor-core Sinkhorn loop (one cooperative launch per Alg. 1 solve)
against the oracle and against the per-update launches it replaces, on ragged shapes,
at the stop test's edge cases, and under an expired bounded wait."""
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
    native.set_loop_tc(True)
    native.set_wait_limit_ns(0)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def host(t):
    return t.detach().cpu().numpy().astype(np.float64)


def map_rms_rel(T_gpu, T_ref, Y):
    Y = np.asarray(Y, dtype=np.float64)
    spread = np.sqrt(np.mean(np.sum((Y - Y.mean(0)) ** 2, 1)))
    return float(np.sqrt(np.mean(np.sum((np.asarray(T_gpu) - np.asarray(T_ref)) ** 2, 1))) / spread)


def marginal_l1(X, Y, f, g, eps):
    C = O.CostOperator(X, Y)
    n, m = C.n, C.m
    return float(np.abs(O.row_marginal(C, f, g, eps) - 1.0 / n).sum() +
                 np.abs(O.col_marginal(C, f, g, eps) - 1.0 / m).sum())


SHAPES = [(300, 260, 16), (1000, 700, 64), (257, 129, 17), (129, 517, 3), (640, 384, 128), (333, 200, 256),
          (2000, 3000, 64), (5, 2, 2)]


@pytest.mark.parametrize("n,m,d", SHAPES)
def test_persistent_loop_matches_oracle_and_per_update_path(nat, n, m, d):
    """Same problem through the persistent loop and through one launch per update: both
    within the mixed-precision bars of the oracle, and the two stop within one iteration
    of each other (they compute the same iteration; only the order in which the bias
    enters each float32 t_ij differs)."""
    p = W.gmm_pair(n, m, d, seed=n + 2 * m + d, k=4)
    eps = 0.05 * O.mean_cost(p.x, p.y)
    out = {}
    for loop in (True, False):
        nat.set_loop_tc(loop)
        out[loop] = nat.sinkhorn_potentials(dev(p.x), dev(p.y), eps, 1e-4, max_iter=5000, precision="bf16x3")
        assert out[loop].status == nat.PROGOT_OK, nat.last_error()
    nat.set_loop_tc(True)
    assert abs(out[True].iters - out[False].iters) <= 1
    ref = O.sinkhorn(None, p.x, None, p.y, eps, 1e-7, max_iter=20000)
    T_ref = O.entropic_map(p.x, p.y, ref.g, eps)
    for loop in (True, False):
        f, g = host(out[loop].f), host(out[loop].g)
        assert marginal_l1(p.x, p.y, f, g, eps) <= TOL_MIXED
        assert map_rms_rel(O.entropic_map(p.x, p.y, g, eps), T_ref, p.y) <= TOL_MIXED


def test_persistent_loop_stop_test_edge_cases(nat):
    """max_iter = 0 reports the initial error without an update; a small max_iter stops
    with NOT_CONVERGED after exactly that many iterations; a warm start at the fixed point
    does no work; a NaN input stops with NUMERIC."""
    p = W.gmm_pair(600, 450, 32, seed=4, k=3)
    eps = 0.05 * O.mean_cost(p.x, p.y)
    x, y = dev(p.x), dev(p.y)
    r0 = nat.sinkhorn_potentials(x, y, eps, 1e-9, max_iter=0, precision="bf16x3")
    assert r0.status == nat.PROGOT_ERR_NOT_CONVERGED and r0.iters == 0
    err0 = O.marginal_error(O.CostOperator(p.x, p.y), np.zeros(600), np.zeros(450), eps)
    assert abs(r0.err - err0) <= 1e-3 * err0
    assert not torch.any(r0.g != 0)  # the g-update of the stopping iteration writes nothing
    r3 = nat.sinkhorn_potentials(x, y, eps, 1e-9, max_iter=3, precision="bf16x3")
    assert r3.status == nat.PROGOT_ERR_NOT_CONVERGED and r3.iters == 3
    r1 = nat.sinkhorn_potentials(x, y, eps, 1e-4, precision="bf16x3")
    assert r1.status == nat.PROGOT_OK
    r2 = nat.sinkhorn_potentials(x, y, eps, 1e-4, f=r1.f.clone(), g=r1.g.clone(), precision="bf16x3")
    assert r2.iters == 0 and r2.status == nat.PROGOT_OK
    assert torch.equal(r2.g, r1.g)
    xb = p.x.copy()
    xb[17, 2] = np.nan
    with pytest.raises(nat.ProgOTError) as ei:
        nat.sinkhorn_potentials(dev(xb), y, eps, 1e-6, max_iter=50, precision="bf16x3")
    assert ei.value.code == nat.PROGOT_ERR_NUMERIC


def test_persistent_loop_is_deterministic(nat):
    """Two runs of the same solve give the same potentials bit for bit (fixed-order
    combines, the stop test computed identically by every CTA)."""
    p = W.gmm_pair(3000, 2500, 64, seed=9, k=5)
    eps = 0.05 * O.mean_cost(p.x[:500], p.y[:500])
    a = nat.sinkhorn_potentials(dev(p.x), dev(p.y), eps, 1e-4, precision="bf16x3")
    b = nat.sinkhorn_potentials(dev(p.x), dev(p.y), eps, 1e-4, precision="bf16x3")
    assert a.iters == b.iters and torch.equal(a.f, b.f) and torch.equal(a.g, b.g)


def test_persistent_loop_bounded_wait_expires_and_context_survives(nat):
    """A wait that nothing satisfies: the host withholds the initial betas of g, so the
    first f-update's tiles poll for words that no sweep writes. With a 20 ms limit the
    launch aborts (every CTA drains its copies and products and frees its tensor
    memory) and the call returns PROGOT_ERR_TIMEOUT; afterwards, with the betas written
    and the default limit, a solve on the same context matches the oracle."""
    p = W.gmm_pair(600, 450, 32, seed=4, k=3)
    eps = 0.05 * O.mean_cost(p.x, p.y)
    x, y = dev(p.x), dev(p.y)
    nat.set_wait_limit_ns(20_000_000)
    nat.test_withhold_initial_betas(True)
    try:
        with pytest.raises(nat.ProgOTError) as ei:
            nat.sinkhorn_potentials(x, y, eps, 1e-4, precision="bf16x3")
        assert ei.value.code == nat.PROGOT_ERR_TIMEOUT
    finally:
        nat.test_withhold_initial_betas(False)
        nat.set_wait_limit_ns(0)
    r = nat.sinkhorn_potentials(x, y, eps, 1e-4, precision="bf16x3")
    assert r.status == nat.PROGOT_OK, nat.last_error()
    ref = O.sinkhorn(None, p.x, None, p.y, eps, 1e-7)
    assert marginal_l1(p.x, p.y, host(r.f), host(r.g), eps) <= TOL_MIXED
    assert map_rms_rel(O.entropic_map(p.x, p.y, host(r.g), eps), O.entropic_map(p.x, p.y, ref.g, eps),
                       p.y) <= TOL_MIXED
