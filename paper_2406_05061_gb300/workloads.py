"""Seeded synthetic point clouds shaped like the paper's workloads.

This module is shared by the CUDA path, the tests and the FP64 oracle. It holds
no arithmetic of the method (no cost, no potential, no schedule): it only draws
points. Every generator draws in float64 with ``numpy.random.default_rng(seed)``
and returns float32 arrays, so both sides of a parity test read the very same
values (the oracle upcasts the float32 values to float64).

Stand-ins: the paper's datasets (sci-Plex PCA features, 4i morphology features,
CIFAR-10, the Korotin GMM benchmark; Sec. 5) are not available, so the shapes
below follow the sizes the paper reports (n ~ 1e4 with d in {16, 64, 256} in
Sec. 5.1, n ~ 11k with d = 47 in Sec. 5.2, n = 60000 in Sec. 5.3) on Gaussian,
Gaussian-mixture and normalised-mixture clouds.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

__all__ = [
    "Problem",
    "gaussian_affine",
    "gmm_pair",
    "sphere_mixture_pair",
    "heldout_target",
    "batched_problems",
    "poisson_requests",
    "random_spd",
    "haar_orthogonal",
    "synthetic_images",
    "blur_pair",
]


@dataclass
class Problem:
    """One OT problem: source cloud x (n, d), target cloud y (m, d), float32."""

    x: np.ndarray
    y: np.ndarray
    seed: int
    name: str = ""

    @property
    def n(self) -> int:
        return int(self.x.shape[0])

    @property
    def m(self) -> int:
        return int(self.y.shape[0])

    @property
    def d(self) -> int:
        return int(self.x.shape[1])


def haar_orthogonal(rng: np.random.Generator, d: int) -> np.ndarray:
    """Haar-distributed orthogonal matrix: QR of a Gaussian matrix with the sign fix."""
    z = rng.standard_normal((d, d))
    q, r = np.linalg.qr(z)
    return q * np.sign(np.diag(r))[None, :]


def random_spd(rng: np.random.Generator, d: int, lo: float = 0.5, hi: float = 2.0) -> np.ndarray:
    """Q diag(lambda) Q^T with Q Haar and lambda ~ U[lo, hi]."""
    q = haar_orthogonal(rng, d)
    lam = rng.uniform(lo, hi, size=d)
    return (q * lam[None, :]) @ q.T


def gaussian_affine(n: int = 512, m: int = 512, seed: int = 0) -> Problem:
    """x ~ N(0, I_2); y = A z + b with z ~ N(0, I_2) independent of x.

    A = [[2, 0.5], [0.5, 1]], b = (1, -1): the 2-D parity workload (plain FP32,
    K = 4 steps)."""
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((n, 2))
    z = rng.standard_normal((m, 2))
    A = np.array([[2.0, 0.5], [0.5, 1.0]])
    b = np.array([1.0, -1.0])
    y = z @ A.T + b[None, :]
    return Problem(x.astype(np.float32), y.astype(np.float32), seed, "gaussian_affine_2d")


def _gmm_law(rng: np.random.Generator, d: int, k: int, mean_scale: float, spd: bool):
    """Parameters of a k-component equal-weight mixture: means and Cholesky factors
    (None for isotropic unit components)."""
    means = rng.standard_normal((k, d)) * mean_scale
    chols = [np.linalg.cholesky(random_spd(rng, d)) for _ in range(k)] if spd else None
    return means, chols


def _gmm_sample(rng: np.random.Generator, law, n: int) -> np.ndarray:
    means, chols = law
    k, d = means.shape
    comp = rng.integers(0, k, size=n)
    z = rng.standard_normal((n, d))
    if chols is None:
        return means[comp] + z
    out = np.empty((n, d))
    for c in range(k):
        idx = comp == c
        out[idx] = means[c][None, :] + z[idx] @ chols[c].T
    return out


def _gmm_laws(seed: int, d: int, k: int):
    rng = np.random.default_rng(seed)
    src = _gmm_law(rng, d, k, 2.0, spd=False)
    tgt = _gmm_law(rng, d, k, 2.0, spd=True)
    return rng, src, tgt


def gmm_pair(n: int = 8192, m: int = 8192, d: int = 64, seed: int = 1, k: int = 8) -> Problem:
    """Source: k-component equal-weight mixture, means ~ N(0, 4 I), isotropic sigma = 1.
    Target: k components with independently drawn means ~ N(0, 4 I) and covariances
    Q diag(U[0.5, 2]) Q^T."""
    rng, src, tgt = _gmm_laws(seed, d, k)
    x = _gmm_sample(rng, src, n)
    y = _gmm_sample(rng, tgt, m)
    return Problem(x.astype(np.float32), y.astype(np.float32), seed, f"gmm{k}_d{d}")


def _sphere_laws(seed: int, d: int, k: int):
    rng = np.random.default_rng(seed)
    laws = []
    for _ in range(2):
        mu = rng.standard_normal((k, d))
        laws.append(mu / np.linalg.norm(mu, axis=1, keepdims=True))
    return rng, laws[0], laws[1]


def _sphere_sample(rng: np.random.Generator, mu: np.ndarray, n: int) -> np.ndarray:
    k, d = mu.shape
    comp = rng.integers(0, k, size=n)
    v = mu[comp] + rng.standard_normal((n, d)) / np.sqrt(d)
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def sphere_mixture_pair(n: int = 65536, m: int = 65536, d: int = 256, seed: int = 2, k: int = 32) -> Problem:
    """Two k-component 'von-Mises-Fisher-like' mixtures on the unit sphere:
    normalise(mu_c + z / sqrt(d)), mu_c = normalise(N(0, I)), z ~ N(0, I)."""
    rng, src, tgt = _sphere_laws(seed, d, k)
    x = _sphere_sample(rng, src, n)
    y = _sphere_sample(rng, tgt, m)
    return Problem(x.astype(np.float32), y.astype(np.float32), seed, f"sphere{k}_d{d}")


def heldout_target(problem: Problem, m_test: int | None = None) -> np.ndarray:
    """A held-out draw Y_test from the target law of ``problem`` (seed + 1000).

    The epsilon scheduler (Alg. 4) scores candidates on target points not used in
    the fit; this draws m_test = max(64, m // 4) fresh points (an 80/20 split)
    from the same law (same means / covariances) with a generator seeded seed + 1000."""
    mt = m_test if m_test is not None else max(64, problem.m // 4)
    name = problem.name
    rt = np.random.default_rng(problem.seed + 1000)
    if name.startswith("gaussian_affine"):
        z = rt.standard_normal((mt, 2))
        A = np.array([[2.0, 0.5], [0.5, 1.0]])
        return (z @ A.T + np.array([1.0, -1.0])[None, :]).astype(np.float32)
    if name.startswith("gmm"):
        k = int(name[3:].split("_")[0])
        _, _, tgt = _gmm_laws(problem.seed, problem.d, k)
        return _gmm_sample(rt, tgt, mt).astype(np.float32)
    if name.startswith("sphere"):
        k = int(name[6:].split("_")[0])
        _, _, tgt = _sphere_laws(problem.seed, problem.d, k)
        return _sphere_sample(rt, tgt, mt).astype(np.float32)
    raise ValueError(f"no held-out law for problem {name!r}")


def batched_problems(count: int = 256, lo: int = 128, hi: int = 4096, dims=(16, 64), seed: int = 3) -> list[Problem]:
    """``count`` independent problems, n and m log-uniform in [lo, hi], d drawn from
    ``dims``, Gaussian-mixture clouds as in :func:`gmm_pair`."""
    rng = np.random.default_rng(seed)
    out = []
    for p in range(count):
        n = int(np.exp(rng.uniform(np.log(lo), np.log(hi))))
        m = int(np.exp(rng.uniform(np.log(lo), np.log(hi))))
        d = int(dims[rng.integers(0, len(dims))])
        sub = int(rng.integers(0, 2**31 - 1))
        out.append(gmm_pair(n, m, d, seed=sub))
        out[-1].name = f"batch{p}_" + out[-1].name
    return out


def poisson_requests(count: int = 20000, rate: float = 200.0, lo: int = 256, hi: int = 32768,
                     dims=(16, 64, 256), seed: int = 4):
    """Arrival times (s) of a Poisson stream and per-request (n, m, d, subseed)."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate, size=count)
    t = np.cumsum(gaps)
    reqs = []
    for i in range(count):
        n = int(np.exp(rng.uniform(np.log(lo), np.log(hi))))
        m = int(np.exp(rng.uniform(np.log(lo), np.log(hi))))
        d = int(dims[rng.integers(0, len(dims))])
        reqs.append((float(t[i]), n, m, d, int(rng.integers(0, 2**31 - 1))))
    return reqs


def synthetic_images(n: int, side: int = 32, seed: int = 5) -> np.ndarray:
    """n grey-level images (side x side, values in [0, 1]) standing in for grey-scale
    CIFAR-10 (Sec. 5.3): a random linear shading, two to four Gaussian blobs of random
    position, width and sign, one random axis-aligned rectangle (a sharp edge) and
    small pixel noise, clipped to [0, 1]. Returns (n, side * side) float32, row-major
    pixels."""
    rng = np.random.default_rng(seed)
    out = np.empty((n, side * side), dtype=np.float32)
    u = (np.arange(side) + 0.5) / side
    gy, gx = np.meshgrid(u, u, indexing="ij")
    chunk = 2048
    for i0 in range(0, n, chunk):
        c = min(chunk, n - i0)
        img = 0.5 + 0.25 * (rng.uniform(-1, 1, (c, 1, 1)) * (gx - 0.5) + rng.uniform(-1, 1, (c, 1, 1)) * (gy - 0.5))
        nb = rng.integers(2, 5, size=c)
        for b in range(4):
            on = (nb > b)[:, None, None]
            cx, cy = rng.uniform(0, 1, (c, 1, 1)), rng.uniform(0, 1, (c, 1, 1))
            w = rng.uniform(0.05, 0.3, (c, 1, 1))
            amp = rng.uniform(-0.5, 0.5, (c, 1, 1))
            img = img + on * amp * np.exp(-((gx - cx) ** 2 + (gy - cy) ** 2) / (2 * w * w))
        x0, x1 = np.sort(rng.integers(0, side + 1, (2, c)), axis=0)
        y0, y1 = np.sort(rng.integers(0, side + 1, (2, c)), axis=0)
        idx = np.arange(side)
        rect = ((idx[None, None, :] >= x0[:, None, None]) & (idx[None, None, :] < x1[:, None, None]) &
                (idx[None, :, None] >= y0[:, None, None]) & (idx[None, :, None] < y1[:, None, None]))
        img = img + rect * rng.uniform(-0.3, 0.3, (c, 1, 1))
        img = img + 0.02 * rng.standard_normal((c, side, side))
        out[i0:i0 + c] = np.clip(img, 0.0, 1.0).reshape(c, side * side)
    return out


def blur_pair(n: int = 60000, side: int = 32, sigma: float = 2.0, seed: int = 5) -> Problem:
    """The de-blurring benchmark of Sec. 5.3 on synthetic images: x = images, y = G(x)
    with G(U) = K U K and K_ij = exp(-(i - j)^2 / sigma) on the pixel grid (a Gaussian
    blur whose width grows with sigma). G is linear, symmetric and positive definite on
    vec(U), so by Prop. 3 the optimal coupling of (x, y) under the squared Euclidean
    cost is the identity Id / n: point i of y is the image of point i of x."""
    x = synthetic_images(n, side, seed)
    idx = np.arange(side, dtype=np.float64)
    K = np.exp(-((idx[:, None] - idx[None, :]) ** 2) / float(sigma))
    y = np.empty_like(x)
    chunk = 4096
    for i0 in range(0, n, chunk):
        U = x[i0:i0 + chunk].astype(np.float64).reshape(-1, side, side)
        y[i0:i0 + chunk] = np.matmul(K, np.matmul(U, K)).reshape(-1, side * side).astype(np.float32)
    return Problem(x, y, seed, f"blur_s{sigma:g}_{side}x{side}")
