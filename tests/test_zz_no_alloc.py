"""The allocation-free marginals entry point (coupling_marginals_noalloc).

It serves callers that cannot allocate device memory (code inside a framework or
engine callback whose memory is planned ahead, code that must avoid cudaFree's
implicit synchronisation, or memory owned by another allocator): its scratch is a
static device array inside the library. This file is collected last so that a run
stopping at the first failure has already run every other test."""
import numpy as np
import pytest

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
