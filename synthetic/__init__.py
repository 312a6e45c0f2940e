"""Seeded synthetic workloads for the CRISP engine (arXiv 2603.05180).

This module only draws random numbers.  It holds none of the method's
arithmetic: no distances, no clustering, no rotation of the data by the index's
matrix, no collision counting.  Both the CPU oracle (through the tests) and the
CUDA library (through the tests and the benchmark) are fed from here, so the two
see identical inputs.

Workloads (the paper's datasets are not available, so these stand in for them;
shapes follow the paper's workload table, §6.1 Table 2, and the engine's
benchmark configurations):

* ``gmm``       -- 50-component Gaussian mixture, means ~ N(0, 4I), shared
                  covariance F F^T + 0.1 I with a random rank-32 factor F.
                  N=20,000, D=256, 100 queries (the small parity workload).
* ``powerlaw``  -- x = U diag(sqrt(lambda)) z, lambda_i = i^-1.2, U a Haar
                  orthogonal mix, z ~ N(0, I).  N=1,000,000, D=960 (Gist-shaped),
                  10,000 held-out queries; also N=5,000,000, D=1024 (serving).
* ``vmf``       -- unit rows from a 1,000-component von Mises-Fisher mixture,
                  kappa=200, D=3072 (Simplewiki-shaped), Wood's (1994) sampler.
* ``lowrank``   -- x = L f + 0.05 e, rank-128 N(0,1) loadings, with 5% of the
                  dimensions scaled to 10x variance, D=4096 (Trevi-shaped).
* ``mixed``     -- a correlated block (the first dims, a Haar-mixed low-rank
                  Gaussian) beside independent dims whose standard deviations
                  decay geometrically: the mixed, skewed distribution that the
                  block-wise rotation and adaptive subspace sizes (§7) target.

The random numbers the *method* draws (the covariance sample of §4.1, the
Gaussian matrix G of the rotation in §3, the k-means training sample and
initial centroids) are also drawn here, by :func:`method_draws`, and passed to
both sides as inputs.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

# sub-seed offsets: base data, queries, rotation G, k-means, covariance sample
SUB_DATA, SUB_QUERY, SUB_GAUSS, SUB_KMEANS, SUB_CEV = 0, 1, 2, 3, 4
SUB_TRAIN, SUB_VALID = 5, 6          # extra query streams of the same law (learned-depth training)


def _rng(seed: int, sub: int) -> np.random.Generator:
    return np.random.default_rng([int(seed), int(sub)])


def haar_orthogonal(D: int, seed: int) -> np.ndarray:
    """A Haar-distributed D x D orthogonal matrix (scipy's ortho_group)."""
    from scipy.stats import ortho_group

    return ortho_group.rvs(dim=D, random_state=np.random.RandomState(seed % (2**32)))


# ----------------------------------------------------------------------------- data
def gmm(N=20000, D=256, nq=100, n_comp=50, rank=32, noise_var=0.1, seed=0):
    """Gaussian mixture with a shared low-rank-plus-isotropic covariance."""
    r = _rng(seed, SUB_DATA)
    mu = r.normal(0.0, 2.0, size=(n_comp, D))           # means ~ N(0, 4 I)
    F = r.normal(0.0, 1.0, size=(D, rank))              # shared rank-32 factor

    def draw(rr, n):
        comp = rr.integers(0, n_comp, size=n)
        z = rr.normal(size=(n, rank))
        e = rr.normal(size=(n, D))
        return (mu[comp] + z @ F.T + math.sqrt(noise_var) * e).astype(np.float32)

    X = draw(r, N)
    Q = draw(_rng(seed, SUB_QUERY), nq)
    return X, Q


def powerlaw_spectrum(D: int, exponent: float = 1.2) -> np.ndarray:
    return np.arange(1, D + 1, dtype=np.float64) ** (-exponent)


def powerlaw(N=1_000_000, D=960, nq=10_000, exponent=1.2, seed=0, device="cpu", query_sub=SUB_QUERY):
    """Rows x = U diag(sqrt(lambda)) z with a power-law spectrum and a Haar mix.

    With ``device='cuda'`` the Gaussian draws and the mixing product run in
    torch on the GPU (seeded torch generator); the mixing matrix U is always
    drawn on the host.  The two devices give different (equally distributed)
    rows; callers that need the same rows on both sides copy them.
    ``query_sub`` picks the query stream (training and validation queries of
    the same law use their own streams).
    """
    U = haar_orthogonal(D, seed * 7919 + 17)
    A = (U * np.sqrt(powerlaw_spectrum(D, exponent))[None, :]).astype(np.float32)  # A = U diag(sqrt l)
    if device == "cpu":
        X = _rng(seed, SUB_DATA).standard_normal((N, D), dtype=np.float32) @ A.T
        Q = _rng(seed, query_sub).standard_normal((nq, D), dtype=np.float32) @ A.T
        return np.ascontiguousarray(X, np.float32), np.ascontiguousarray(Q, np.float32)
    import torch

    At = torch.from_numpy(A.T.copy()).to(device)
    g = torch.Generator(device=device)
    out = []
    for sub, n in ((SUB_DATA, N), (query_sub, nq)):
        g.manual_seed(seed * 1000003 + sub)
        Y = torch.empty((n, D), dtype=torch.float32, device=device)
        step = 1 << 18
        for s in range(0, n, step):
            e = min(n, s + step)
            z = torch.randn((e - s, D), generator=g, device=device, dtype=torch.float32)
            Y[s:e] = z @ At
        out.append(Y)
    return out[0], out[1]


def _wood_vmf_weights(rr, n, D, kappa):
    """Wood (1994) rejection sampler for the vMF cosine w = <x, mu>."""
    b = (-2.0 * kappa + math.sqrt(4.0 * kappa * kappa + (D - 1.0) ** 2)) / (D - 1.0)
    x0 = (1.0 - b) / (1.0 + b)
    c = kappa * x0 + (D - 1.0) * math.log(1.0 - x0 * x0)
    w = np.empty(n)
    filled = 0
    while filled < n:
        m = (n - filled) * 2 + 16
        z = rr.beta((D - 1.0) / 2.0, (D - 1.0) / 2.0, size=m)
        ww = (1.0 - (1.0 + b) * z) / (1.0 - (1.0 - b) * z)
        u = rr.uniform(size=m)
        ok = kappa * ww + (D - 1.0) * np.log(1.0 - x0 * ww) - c >= np.log(u)
        acc = ww[ok][: n - filled]
        w[filled:filled + acc.size] = acc
        filled += acc.size
    return w


def vmf(N=1_000_000, D=3072, nq=10_000, n_comp=1000, kappa=200.0, seed=0, device="cpu", query_sub=SUB_QUERY):
    """Unit rows from a vMF mixture (uniform weights, means uniform on the sphere).

    With ``device='cuda'`` the per-row scalars (component, Wood cosine) are
    drawn on the host and the D-dimensional tangent directions on the GPU with
    a seeded torch generator (other rows than the host version, same law)."""
    r = _rng(seed, SUB_DATA)
    mu = r.normal(size=(n_comp, D))
    mu /= np.linalg.norm(mu, axis=1, keepdims=True)
    if device != "cpu":
        return _vmf_device(mu, N, D, nq, n_comp, kappa, seed, device, query_sub)

    def draw(rr, n):
        comp = rr.integers(0, n_comp, size=n)
        w = _wood_vmf_weights(rr, n, D, kappa)
        v = rr.normal(size=(n, D))
        m = mu[comp]
        v -= (v * m).sum(1, keepdims=True) * m                 # tangent direction
        v /= np.linalg.norm(v, axis=1, keepdims=True)
        x = w[:, None] * m + np.sqrt(np.maximum(0.0, 1.0 - w * w))[:, None] * v
        return x.astype(np.float32)

    return draw(r, N), draw(_rng(seed, SUB_QUERY), nq)


def lowrank(N=2_000_000, D=4096, nq=10_000, rank=128, noise=0.05, boost_frac=0.05, boost_var=10.0, seed=0,
            device="cpu", query_sub=SUB_QUERY):
    """x = L f + noise*e, with a seeded 5% of dims scaled to 10x variance.

    With ``device='cuda'`` the loadings and boosted dims come from the host
    stream and the Gaussian factors and noise from a seeded torch generator on
    the GPU (other rows than the host version, same law)."""
    r = _rng(seed, SUB_DATA)
    L = r.normal(size=(D, rank)).astype(np.float32)
    nb = int(math.floor(boost_frac * D))
    boost = r.choice(D, size=nb, replace=False)
    scale = np.ones(D, np.float32)
    scale[boost] = math.sqrt(boost_var)
    if device != "cpu":
        return _lowrank_device(L, scale, N, D, nq, rank, noise, seed, device, query_sub)

    def draw(rr, n):
        f = rr.standard_normal((n, rank), dtype=np.float32)
        e = rr.standard_normal((n, D), dtype=np.float32)
        return ((f @ L.T + noise * e) * scale[None, :]).astype(np.float32)

    return draw(r, N), draw(_rng(seed, SUB_QUERY), nq)


def _vmf_device(mu, N, D, nq, n_comp, kappa, seed, device, query_sub):
    import torch

    mu_d = torch.from_numpy(mu.astype(np.float32)).to(device)
    g = torch.Generator(device=device)
    out = []
    for sub, n in ((SUB_DATA, N), (query_sub, nq)):
        rr = _rng(seed, 100 + sub)
        comp = torch.from_numpy(rr.integers(0, n_comp, size=n)).to(device)
        w = torch.from_numpy(_wood_vmf_weights(rr, n, D, kappa).astype(np.float32)).to(device)
        g.manual_seed(seed * 1000003 + 100 + sub)
        Y = torch.empty((n, D), dtype=torch.float32, device=device)
        step = 1 << 16
        for s0 in range(0, n, step):
            e = min(n, s0 + step)
            m = mu_d[comp[s0:e]]
            v = torch.randn((e - s0, D), generator=g, device=device, dtype=torch.float32)
            v -= (v * m).sum(1, keepdim=True) * m                      # tangent direction
            v /= torch.linalg.vector_norm(v, dim=1, keepdim=True)
            ws = w[s0:e, None]
            Y[s0:e] = ws * m + torch.sqrt(torch.clamp(1.0 - ws * ws, min=0.0)) * v
        out.append(Y)
    return out[0], out[1]


def _lowrank_device(L, scale, N, D, nq, rank, noise, seed, device, query_sub):
    import torch

    Lt = torch.from_numpy(L.T.copy()).to(device)
    sc = torch.from_numpy(scale).to(device)
    g = torch.Generator(device=device)
    out = []
    for sub, n in ((SUB_DATA, N), (query_sub, nq)):
        g.manual_seed(seed * 1000003 + 200 + sub)
        Y = torch.empty((n, D), dtype=torch.float32, device=device)
        step = 1 << 16
        for s0 in range(0, n, step):
            e = min(n, s0 + step)
            f = torch.randn((e - s0, rank), generator=g, device=device, dtype=torch.float32)
            z = torch.randn((e - s0, D), generator=g, device=device, dtype=torch.float32)
            Y[s0:e] = (f @ Lt + noise * z) * sc
        out.append(Y)
    return out[0], out[1]


def mixed(N=200_000, D=960, nq=1_000, corr_dims=192, rank=8, skew=8.0, noise=0.05, seed=0):
    """Rows with a correlated block and a skewed independent part.

    Dims [0, corr_dims): U_b (F z) + noise e, F a rank-``rank`` N(0,1) loading
    matrix and U_b a Haar mix of the block, so the block's spectrum is
    concentrated (block CEV near 1).  Dims [corr_dims, D): independent
    N(0, s_d^2) with s_d falling geometrically from ``skew`` to 1 across the
    part (variance skewed towards its first dims, no correlation)."""
    r = _rng(seed, SUB_DATA)
    F = r.standard_normal((corr_dims, rank))
    U = haar_orthogonal(corr_dims, seed * 7919 + 17)
    L = U @ F
    rest = D - corr_dims
    s = skew ** (1.0 - np.arange(rest) / max(rest - 1, 1))

    def draw(rr, n):
        out = np.empty((n, D), np.float32)
        for a in range(0, n, 65536):
            b = min(n, a + 65536)
            z = rr.standard_normal((b - a, rank))
            out[a:b, :corr_dims] = z @ L.T + noise * rr.standard_normal((b - a, corr_dims))
            out[a:b, corr_dims:] = s[None, :] * rr.standard_normal((b - a, rest))
        return out

    X = draw(r, N)
    Q = draw(_rng(seed, SUB_QUERY), nq)
    return X, Q


def small_gaussian(N, D, nq, seed=0, scale=1.0):
    """Plain N(0, scale^2 I) rows, for edge-case tests."""
    r = _rng(seed, SUB_DATA)
    X = (scale * r.standard_normal((N, D))).astype(np.float32)
    Q = (scale * _rng(seed, SUB_QUERY).standard_normal((nq, D))).astype(np.float32)
    return X, Q


# ------------------------------------------------------------------- method's draws
@dataclass
class Draws:
    """Random numbers the index build draws, passed to both sides as inputs."""
    cev_sample: np.ndarray      # int64 [S], sorted, without replacement (§4.1)
    gaussian: np.ndarray        # float64 [D, D], G_ij ~ N(0, 1) (§3 rotation)
    kmeans_sample: np.ndarray   # int64 [T], sorted, without replacement
    kmeans_init: np.ndarray     # int32 [M, 2, K], distinct positions in kmeans_sample


def cev_sample_size(N: int) -> int:
    """min(floor(0.1 N), 10^5), raised to 2 rows (a covariance needs two), at most N."""
    return int(min(N, max(2, min(N // 10, 100_000))))


def method_draws(N: int, D: int, M: int, K: int = 50, seed: int = 0, kmeans_train: int = 100_000) -> Draws:
    r_cev = _rng(seed, SUB_CEV)
    S = cev_sample_size(N)
    cev_sample = np.sort(r_cev.choice(N, size=S, replace=False)).astype(np.int64)
    G = _rng(seed, SUB_GAUSS).standard_normal((D, D))
    r_km = _rng(seed, SUB_KMEANS)
    T = int(min(N, kmeans_train))
    km_sample = np.sort(r_km.choice(N, size=T, replace=False)).astype(np.int64)
    if K > T:
        raise ValueError("K larger than the k-means training sample")
    init = np.stack([np.stack([r_km.choice(T, size=K, replace=False) for _ in range(2)]) for _ in range(M)])
    return Draws(cev_sample, G, km_sample, init.astype(np.int32))


def subsample_queries(nq: int, n: int, seed: int = 0) -> np.ndarray:
    """A fixed seeded subset of query positions (for bounded CPU baselines)."""
    return np.sort(_rng(seed, 99).choice(nq, size=min(n, nq), replace=False))


def mlp_weights(F: int, H: int, O: int, seed: int = 0, scale: float = 1.0) -> np.ndarray:
    """Seeded Gaussian parameters for an F -> H -> H -> O network, packed as
    W1 [F][H], b1 [H], W2 [H][H], b2 [H], W3 [H][O], b3 [O] (weights scaled by
    1/sqrt(fan_in), small random biases)."""
    r = _rng(seed, 7)
    parts = []
    for shape in ((F, H), (H,), (H, H), (H,), (H, O), (O,)):
        n = int(np.prod(shape))
        fan = shape[0] if len(shape) == 2 else 10.0
        parts.append(scale * r.standard_normal(n) / math.sqrt(fan))
    return np.concatenate(parts).astype(np.float32)
