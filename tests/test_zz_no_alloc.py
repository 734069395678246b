"""The allocation-free marginals entry point (coupling_marginals_noalloc).

It serves callers that cannot allocate device memory (code inside a framework or
engine callback whose memory is planned ahead, code that must avoid cudaFree's
implicit synchronisation, or memory owned by another allocator): its scratch is a
static device array inside the library. This file is collected last so that a run
stopping at the first failure has already run every other test."""
import numpy as np
import pytest

from oracle import progot_oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nat():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2406_05061_gb300 import native
    native.lib()
    return native


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def test_noalloc_marginals_match_workspace_entry_point_twice(nat):
    """Two calls in a row, on different problems: each result matches coupling_marginals
    (the workspace entry point) within the parity tolerance, so nothing of the first call
    leaks into the second through the shared static scratch."""
    from paper_2406_05061_gb300 import workloads as W
    rng = np.random.default_rng(0)
    for n, m, d, seed in ((1000, 700, 64, 1), (300, 517, 16, 2)):
        p = W.gmm_pair(n, m, d, seed=seed, k=3)
        x, y = _dev(p.x), _dev(p.y)
        eps = 0.05 * float(np.mean(np.sum((p.x[:, None, :64] - p.y[None, :64, :]) ** 2, -1)))
        sk = nat.sinkhorn_potentials(x, y, eps, 1e-4, max_iter=2000)
        a = rng.uniform(0.5, 1.5, n)
        a = a / a.sum()
        row_ref, col_ref, err_ref = nat.coupling_marginals(x, y, sk.f, sk.g, eps, a=_dev(a))
        row, col, err = nat.coupling_marginals_noalloc(x, y, sk.f, sk.g, eps, a=_dev(a))
        torch.cuda.synchronize()
        np.testing.assert_allclose(row.cpu().numpy(), row_ref.cpu().numpy(), rtol=2e-4, atol=1e-9)
        np.testing.assert_allclose(col.cpu().numpy(), col_ref.cpu().numpy(), rtol=2e-4, atol=1e-9)
        assert abs(err - err_ref) <= 1e-4 * max(err_ref, 1e-3)


def test_noalloc_rejects_sizes_beyond_its_static_scratch(nat):
    n = nat.NOALLOC_MAX_POINTS + 1
    x = torch.zeros((n, 1), dtype=torch.float32, device="cuda")
    y = torch.zeros((4, 1), dtype=torch.float32, device="cuda")
    f = torch.zeros(n, dtype=torch.float32, device="cuda")
    g = torch.zeros(4, dtype=torch.float32, device="cuda")
    with pytest.raises(nat.ProgOTError) as ei:
        nat.coupling_marginals_noalloc(x, y, f, g, 1.0)
    assert ei.value.code == nat.PROGOT_ERR_INVALID_ARG
    assert "65536" in str(ei.value)


@pytest.mark.parametrize("n,m,d", [(65536, 65536, 16), (100, 65536, 8)])
def test_noalloc_marginals_against_fp64_oracle_at_the_limits(nat, n, m, d):
    """At the 65536-point limit (one 128-row block per split, the partial buffer's
    largest use is 2 x SMs x 128 rows, below its 65664 slots) and with one row block
    against 65536 columns (the largest split count): row sums on 16 sampled rows and
    column sums on 16 sampled columns, each computed one by one by the FP64 oracle from
    the same potentials; then one call without an error output (asynchronous), read
    after a stream synchronisation, must give the same marginals."""
    from paper_2406_05061_gb300 import workloads as W
    p = W.gmm_pair(n, m, d, seed=n % 97 + d, k=4)
    x, y = _dev(p.x), _dev(p.y)
    X64, Y64 = p.x.astype(np.float64), p.y.astype(np.float64)
    sub = np.random.default_rng(1).choice(min(n, m), min(n, m, 1024), replace=False)
    eps = 0.05 * O.mean_cost(X64[sub % n], Y64[sub % m])
    sk = nat.sinkhorn_potentials(x, y, eps, 1e-3, max_iter=30)  # realistic potentials; convergence not needed
    row, col, err = nat.coupling_marginals_noalloc(x, y, sk.f, sk.g, eps)
    torch.cuda.synchronize()
    f = sk.f.cpu().numpy().astype(np.float64)
    g = sk.g.cpu().numpy().astype(np.float64)
    rng = np.random.default_rng(2)
    ri = rng.choice(n, min(n, 16), replace=False)
    cj = rng.choice(m, 16, replace=False)
    r_ref = np.exp((f[ri, None] + g[None, :] - O.cost_matrix_rows(X64[ri], Y64)) / eps).sum(1)
    c_ref = np.exp((g[cj, None] + f[None, :] - O.cost_matrix_rows(Y64[cj], X64)) / eps).sum(1)
    np.testing.assert_allclose(row.cpu().numpy()[ri], r_ref, rtol=2e-4)
    np.testing.assert_allclose(col.cpu().numpy()[cj], c_ref, rtol=2e-4)
    assert np.isfinite(err)
    row2, col2, err2 = nat.coupling_marginals_noalloc(x, y, sk.f, sk.g, eps, want_err=False)
    assert err2 is None
    torch.cuda.synchronize()
    assert torch.equal(row2, row) and torch.equal(col2, col)
