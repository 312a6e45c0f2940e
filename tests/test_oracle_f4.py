"""Pins of the oracle's two §7 extensions: variance-aware subspace boundaries
(Adaptive Subspace Decomposition) and block-wise rotation (Partial Variance
Redistribution).

Each test checks the oracle against something other than its own formula:
hand-worked boundaries, closed-form variances and spectra built from Hadamard
columns, the QR definition of each rotated block, brute-force argmins, a
binary-search restatement of the boundary rule, and the reduction of each
extension to the already-pinned global path in its special case.
"""
import math
import struct

import numpy as np
import pytest

import oracle
import synthetic


def _hadamard(n):
    H = np.array([[1.0]])
    while H.shape[0] < n:
        H = np.block([[H, H], [H, -H]])
    return H


# ------------------------------------------------------------ equal split
@pytest.mark.parametrize("D,M", [(960, 20), (1000, 7), (64, 2), (130, 3), (3072, 16)])
def test_equal_bounds_closed_form(D, M):
    b = oracle.equal_bounds(D, M)
    assert b.tolist() == [(m * D) // M for m in range(M)] + [D]


# ------------------------------------------------------- column variance
def test_column_variance_closed_form():
    """Columns +-a_d around an offset c_d over an even number S of selected rows
    have variance a_d^2 S / (S - 1); unselected rows must not enter."""
    S, D = 16, 6
    a = np.array([1.0, 0.5, 2.0, 3.0, 0.25, 4.0])
    c = np.array([10.0, -3.0, 0.0, 7.5, 1.0, -2.0])
    H = _hadamard(S)
    sel = H[:, 1:D + 1] * a[None, :] + c[None, :]          # columns of +-1, mean 0
    X = np.full((S + 5, D), 1e6, np.float32)               # garbage rows, not selected
    rows = np.arange(5, S + 5)
    X[rows] = sel
    v = oracle.column_variance(X, rows)
    assert np.array_equal(v, a * a * S / (S - 1))


# -------------------------------------------------- adaptive boundaries
@pytest.mark.parametrize("D,M", [(960, 20), (1000, 7), (64, 2), (130, 3), (3072, 16), (4096, 16)])
@pytest.mark.parametrize("level", [1.0, 0.25, 0.0])
def test_adaptive_bounds_of_equal_variances_are_the_equal_split(D, M, level):
    assert np.array_equal(oracle.adaptive_bounds(np.full(D, level), M), oracle.equal_bounds(D, M))


def test_adaptive_bounds_hand_worked():
    # 4 dims of variance 3, 20 of variance 1: total 32, targets 32/3 and 64/3.
    # V = 0,3,6,9,12,13,...: boundary 1 is j = 3 (V_3 = 9 <= 10.67 < 12),
    # boundary 2 is j = 13 (V_13 = 21 <= 21.33 < 22).
    v = [3.0] * 4 + [1.0] * 20
    assert oracle.adaptive_bounds(v, 3).tolist() == [0, 3, 13, 24]
    # one dominant dim: every target falls at j = 0 and the 2-dim minimum decides
    assert oracle.adaptive_bounds([100.0] + [1.0] * 15, 4).tolist() == [0, 2, 4, 6, 16]
    # all variance in the first 10 of 500 dims, M = 2: the target is j = 5, but
    # the second subspace may hold at most 256 dims, so the boundary is 244
    assert oracle.adaptive_bounds([1.0] * 10 + [0.0] * 490, 2).tolist() == [0, 244, 500]


def test_adaptive_bounds_variance_at_the_end():
    # targets 25, 50, 75 all fall at j = 15 (V_15 = 0 <= t < V_16 = 100); the
    # clamps from the right give 10, 12, 14
    assert oracle.adaptive_bounds([0.0] * 15 + [100.0], 4).tolist() == [0, 10, 12, 14, 16]


def test_adaptive_bounds_against_a_binary_search():
    """Random variances: where no clamp binds, boundary m is the last j with
    V_j <= m V_D / M, found here by binary search on the cumulative sums; every
    subspace keeps 2..256 dims."""
    r = np.random.default_rng(5)
    for trial in range(200):
        D = int(r.integers(8, 1200))
        M = int(r.integers(1, D // 2 + 1))
        if D > 256 * M:
            continue
        v = r.exponential(1.0, D) ** r.uniform(0.5, 4.0)
        b = oracle.adaptive_bounds(v, M)
        w = np.diff(b)
        assert b[0] == 0 and b[-1] == D and w.min() >= 2 and w.max() <= 256
        cum = np.concatenate([[0.0], np.cumsum(v)])
        # np.cumsum adds in order, the same sums as the oracle's loop
        for m in range(1, M):
            j = int(np.searchsorted(cum, m * cum[-1] / M, side="right")) - 1
            lo = max(b[m - 1] + 2, D - 256 * (M - m))
            hi = min(b[m - 1] + 256, D - 2 * (M - m))
            assert b[m] == min(max(j, lo), hi), (trial, m)


def test_adaptive_shares_are_balanced_on_skewed_variances():
    """On a smooth skewed profile each subspace's share of the variance is
    within one dim's variance of V / M (no clamp binds for this profile), and
    high-variance subspaces are narrow."""
    D, M = 960, 40
    v = 4.0 ** (2 * (1 - np.arange(D) / (D - 1)))          # 16 .. 1
    b = oracle.adaptive_bounds(v, M)
    shares = np.array([v[b[m]:b[m + 1]].sum() for m in range(M)])
    assert np.all(np.abs(shares - v.sum() / M) <= v.max())
    w = np.diff(b)
    assert w[0] < D // M < w[-1] and np.all(np.diff(w) >= -1)


# ------------------------------------------------ block-wise rotation
def test_block_cev_closed_form():
    """Hadamard columns scaled by a_d give a sample covariance diag(a_d^2 S/(S-1))
    exactly, so a block's CEV is (top floor(0.2 w) of a_d^2) / (sum of a_d^2)."""
    S, D, b = 64, 40, 16
    a = 1.0 + (np.arange(D) % 7)
    X = (_hadamard(S)[:, 1:D + 1] * a[None, :]).astype(np.float32)
    G = np.random.default_rng(1).standard_normal((D, D))
    _, info = oracle.block_rotation(X, np.arange(S), G, b, tau_cev=2.0)
    assert [(lo, hi) for lo, hi, _, _ in info] == [(0, 16), (16, 32), (32, 40)]
    for lo, hi, c, rot in info:
        lam = np.sort(a[lo:hi] ** 2)[::-1]
        k = int(math.floor(0.2 * (hi - lo)))
        assert abs(c - lam[:k].sum() / lam.sum()) < 1e-12 and not rot


def test_block_rotation_structure_and_choice():
    """A correlated block is rotated, an isotropic one is not; R is the identity
    outside rotated blocks, and each rotated block B is the orthogonal factor of
    the QR of G_BB with a positive triangular diagonal."""
    N, cd, D, b = 4000, 32, 64, 32
    X, _ = synthetic.mixed(N, D, 1, corr_dims=cd, rank=3, skew=1.0)
    G = np.random.default_rng(3).standard_normal((D, D))
    R, info = oracle.block_rotation(X, np.arange(0, N, 3), G, b, tau_cev=0.85)
    assert [r[3] for r in info] == [True, False]
    assert info[0][2] > 0.95 and info[1][2] < 0.4
    assert np.array_equal(R[cd:, :], np.eye(D)[cd:, :]) and np.array_equal(R[:, cd:], np.eye(D)[:, cd:])
    B = R[:cd, :cd]
    assert np.max(np.abs(B.T @ B - np.eye(cd))) < 1e-12
    T = B.T @ G[:cd, :cd]                                   # G_BB = B T
    assert np.max(np.abs(np.tril(T, -1))) < 1e-10 * np.abs(G).max() and np.all(np.diag(T) > 0)
    R1, info1 = oracle.block_rotation(X, np.arange(0, N, 3), G, b, tau_cev=0.85, rotate=1)
    assert all(r[3] for r in info1) and not np.array_equal(R1[cd:, cd:], np.eye(D - cd))


def test_block_rotation_build_keeps_other_dims_and_norms():
    N, D, M, K = 3000, 64, 4, 8
    X, _ = synthetic.mixed(N, D, 1, corr_dims=32, rank=3, skew=2.0)
    dr = synthetic.method_draws(N, D, M, K, kmeans_train=N)
    ix = oracle.build_index(X, M, K, draws=dr, block_dims=32)
    assert ix.rotated == 1 and [r[3] for r in ix.blocks] == [True, False]
    assert np.array_equal(ix.Xr[:, 32:D], X[:, 32:])
    n0 = np.linalg.norm(X[:, :32].astype(np.float64), axis=1)
    n1 = np.linalg.norm(ix.Xr[:, :32].astype(np.float64), axis=1)
    assert np.allclose(n0, n1, rtol=2e-6)


def test_single_block_reduces_to_the_global_rotation():
    """b >= D: one block with the global covariance, so its CEV is the global
    CEV, and with rotate = 1 the index equals the globally rotated one."""
    N, D, M, K = 1500, 48, 3, 8
    X, _ = synthetic.small_gaussian(N, D, 1, seed=4)
    dr = synthetic.method_draws(N, D, M, K, kmeans_train=N)
    g = oracle.build_index(X, M, K, draws=dr, rotate=1)
    bl = oracle.build_index(X, M, K, draws=dr, rotate=1, block_dims=64)
    assert len(bl.blocks) == 1 and abs(bl.blocks[0][2] - g.cev) < 1e-12
    assert np.array_equal(bl.R32, g.R32) and np.array_equal(bl.Xr, g.Xr)
    assert np.array_equal(bl.cells, g.cells) and np.array_equal(bl.ids, g.ids)


# -------------------------------------------------- adaptive index build
def _adaptive_index(N=3000, D=96, M=6, K=8, seed=0):
    X, Q = synthetic.mixed(N, D, 20, corr_dims=16, rank=3, skew=8.0, seed=seed)
    dr = synthetic.method_draws(N, D, M, K, kmeans_train=N, seed=seed)
    return X, Q, dr, oracle.build_index(X, M, K, draws=dr, rotate=0, adaptive=1)


def test_adaptive_build_boundaries_and_cells():
    X, Q, dr, ix = _adaptive_index()
    b = ix.sub
    assert b is not None and not np.array_equal(b, oracle.equal_bounds(ix.D, ix.M))
    assert ix.H == max(int(w - w // 2) for w in np.diff(b))
    # the cells are brute-force argmins over each half at the index's boundaries
    Xr = ix.Xr.astype(np.float64)
    for m in range(ix.M):
        lo, w = int(b[m]), int(b[m + 1] - b[m])
        hl = w // 2
        for half, (a, h) in enumerate([(lo, hl), (lo + hl, w - hl)]):
            Cm = ix.cent[m, half, :, :h].astype(np.float64)
            d = ((Xr[:, None, a:a + h] - Cm[None]) ** 2).sum(-1)
            got = ix.cells[m] // ix.K if half == 0 else ix.cells[m] % ix.K
            assert np.all(d[np.arange(ix.N), got] <= d.min(1) * (1 + 1e-5) + 1e-12), (m, half)


def test_adaptive_half_dists_use_the_boundaries():
    X, Q, dr, ix = _adaptive_index()
    qr = oracle.query_rotate(ix, Q[:3])
    b = ix.sub
    for m in (0, ix.M - 1):
        lo, w = int(b[m]), int(b[m + 1] - b[m])
        hl = w // 2
        for half, (a, h) in enumerate([(lo, hl), (lo + hl, w - hl)]):
            d, s, p = oracle.half_dists(ix, qr[0], m, half)
            ref = ((qr[0, a:a + h].astype(np.float64) - ix.cent[m, half, :, :h].astype(np.float64)) ** 2).sum(-1)
            assert np.allclose(d, ref, rtol=1e-5)


def test_adaptive_lowers_quantisation_error_on_skewed_variances():
    """§7's motivation: with the same K per half, narrow subspaces in the
    high-variance region lower the total IMI quantisation error."""
    N, D, M, K = 4000, 96, 6, 16
    X, _ = synthetic.mixed(N, D, 1, corr_dims=2, rank=1, skew=16.0, seed=2)
    dr = synthetic.method_draws(N, D, M, K, kmeans_train=N, seed=2)

    def qerr(ix):
        b, Xr, e = ix.bounds(), ix.Xr.astype(np.float64), 0.0
        for m in range(ix.M):
            lo, w = int(b[m]), int(b[m + 1] - b[m])
            hl = w // 2
            cl, cr = ix.cells[m] // ix.K, ix.cells[m] % ix.K
            e += ((Xr[:, lo:lo + hl] - ix.cent[m, 0, cl, :hl]) ** 2).sum()
            e += ((Xr[:, lo + hl:lo + w] - ix.cent[m, 1, cr, :w - hl]) ** 2).sum()
        return e

    eq = oracle.build_index(X, M, K, draws=dr, rotate=0)
    ad = oracle.build_index(X, M, K, draws=dr, rotate=0, adaptive=1)
    assert qerr(ad) < 0.9 * qerr(eq)


def test_adaptive_search_recall_and_blob_v2():
    """On the skewed mixed workload the adaptive index finds more true
    neighbours than the equal split at the same coverage."""
    X, Q, dr, ix = _adaptive_index()
    eq = oracle.build_index(X, ix.M, ix.K, draws=dr, rotate=0)
    p = oracle.SearchParams(k=5, rho=0.2, alpha=0.2)
    gt_d2 = oracle.knn_f64(X, Q, 5)[1]
    r_ad = oracle.recall_at_k(oracle.search(ix, Q, p)[0], gt_d2, X, Q, 5)
    r_eq = oracle.recall_at_k(oracle.search(eq, Q, p)[0], gt_d2, X, Q, 5)
    assert r_ad >= 0.9 and r_ad >= r_eq + 0.1
    blob = oracle.export_blob(ix)
    v, N, D, Dp, M, K, H, rot = struct.unpack_from("<8q", blob, 8)
    assert v == 2 and (N, D, M, H) == (ix.N, ix.D, ix.M, ix.H)
    sizes = [4 * M * 2 * K * H, 4 * M * (K * K + 1), 4 * M * N, 4 * N * Dp, 4 * N * (Dp // 32), 4 * (M + 1)]
    pos = 256
    for s in sizes[:-1]:
        pos = (pos + s + 255) // 256 * 256
    assert np.array_equal(np.frombuffer(blob, np.int32, M + 1, pos), ix.sub)
    assert len(blob) == (pos + sizes[-1] + 255) // 256 * 256
    assert struct.unpack_from("<q", oracle.export_blob(eq), 8)[0] == 1
