"""Pins of the CPU oracle against what the paper and mathematics fix.

Each test compares the oracle with something other than itself: a worked
example from the paper or built by hand (tests/golden), a closed form, brute
force on a tiny input, or a second, independent formulation of the same step.
"""
import math

import numpy as np
import pytest

import oracle
import synthetic
from conftest import load_golden


def _manual_index(D, M, K, cent, offsets, ids, Xr=None, rotated=0):
    N = ids.shape[1]
    Dp = oracle.padded_dim(D)
    H = cent.shape[-1]
    Xr = np.zeros((N, Dp), np.float32) if Xr is None else np.ascontiguousarray(Xr, np.float32)
    codes = oracle.sign_codes(Xr)
    cells = np.zeros((M, N), np.uint16)
    for m in range(M):
        for c in range(K * K):
            cells[m, ids[m, offsets[m, c]:offsets[m, c + 1]]] = c
    return oracle.Index(N, D, Dp, M, K, H, rotated, 0.0, None, np.ascontiguousarray(cent, np.float32),
                        np.ascontiguousarray(offsets, np.int32), np.ascontiguousarray(ids, np.int32), Xr, codes, cells)


# ----------------------------------------------------------------- B4 CSR
def test_csr_worked_example():
    g = load_golden("csr_worked_example.txt")
    n = int(g["n_points"][0])
    cells = np.full(n, 2, np.uint16)
    cells[[int(v) for v in g["cell_j_points"]]] = 0
    cells[[int(v) for v in g["cell_i_points"]]] = 1
    off, ids = oracle.csr(cells, int(g["n_cells"][0]))
    pre = [int(v) for v in g["ids_prefix"]]
    assert ids[:len(pre)].tolist() == pre
    assert off.tolist() == [int(v) for v in g["offsets"]]


@pytest.mark.parametrize("N,K2", [(1, 4), (1000, 2500), (20000, 2500), (5000, 7)])
def test_csr_invariants(N, K2):
    rng = np.random.default_rng(N)
    cells = (rng.zipf(1.5, N) % K2).astype(np.uint16)
    off, ids = oracle.csr(cells, K2)
    assert off[0] == 0 and off[-1] == N and np.all(np.diff(off) >= 0)
    assert np.array_equal(np.sort(ids), np.arange(N))
    for c in range(K2):
        seg = ids[off[c]:off[c + 1]]
        assert np.all(np.diff(seg) > 0)
        assert np.all(cells[seg] == c)


# ----------------------------------------------------- Q2/Q3 traversal
def _grid_index(empty_cell=None):
    g = load_golden("multiseq_5x5.txt")
    K = 5
    cent = np.zeros((1, 2, K, 1), np.float32)
    cent[0, 0, :, 0] = [float(v) for v in g["left_centroids"]]
    cent[0, 1, :, 0] = [float(v) for v in g["right_centroids"]]
    sizes = np.ones(K * K, np.int64)
    if empty_cell is not None:
        sizes[empty_cell] = 0
    off = np.zeros((1, K * K + 1), np.int32)
    off[0, 1:] = np.cumsum(sizes)
    ids = np.arange(int(sizes.sum()), dtype=np.int32)[None, :]
    return _manual_index(2, 1, K, cent, off, ids), g


@pytest.mark.parametrize("impl", ["heap", "sort"])
def test_multiseq_grid_fixture(impl):
    ix, g = _grid_index()
    q = np.zeros(ix.Dp, np.float32)
    cells, w, got = oracle.activate(ix, q, 0, 1, int(g["k_size"][0]), int(g["budget"][0]), impl)
    assert cells.tolist() == [int(v) for v in g["expected_cells"]]
    assert w.tolist() == [int(v) for v in g["expected_weights_optimized"]]
    assert got == 13
    cells0, w0, _ = oracle.activate(ix, q, 0, 0, int(g["k_size"][0]), int(g["budget"][0]), impl)
    assert cells0.tolist() == cells.tolist() and set(w0.tolist()) == {1}


@pytest.mark.parametrize("impl", ["heap", "sort"])
def test_multiseq_grid_empty_cell_counts_rank(impl):
    ix, g = _grid_index(empty_cell=int(load_golden("multiseq_5x5.txt")["empty_cell"][0]))
    q = np.zeros(ix.Dp, np.float32)
    cells, w, got = oracle.activate(ix, q, 0, 1, int(g["k_size"][0]), int(g["budget"][0]), impl)
    assert cells.tolist() == [int(v) for v in g["expected_cells_empty"]]
    assert w.tolist() == [int(v) for v in g["expected_weights_empty"]]
    assert got == 13


def test_half_dists_sorted_with_index_ties():
    ix, _ = _grid_index()
    q = np.zeros(ix.Dp, np.float32)
    d, s, p = oracle.half_dists(ix, q, 0, 0)
    assert d.tolist() == [4, 0, 16, 1, 9] and s.tolist() == [0, 1, 4, 9, 16] and p.tolist() == [1, 3, 0, 4, 2]
    cent = np.zeros((1, 2, 5, 1), np.float32)
    cent[0, 0, :, 0] = [1, -1, 1, 2, -1]            # equal distances tie by centroid index
    ix.cent[:] = cent
    ix._st = None
    d, s, p = oracle.half_dists(ix, q, 0, 0)
    assert p.tolist() == [0, 1, 2, 4, 3]


@pytest.fixture(scope="module")
def gmm_index():
    X, Q = synthetic.gmm(N=6000, D=64, nq=20, n_comp=20, rank=8)
    return oracle.build_index(X, M=4), X, Q


@pytest.mark.parametrize("phi,rho", [(0, 0.01), (1, 0.01), (1, 0.2), (0, 1.0)])
def test_multiseq_heap_equals_full_sort(gmm_index, phi, rho):
    ix, X, Q = gmm_index
    qr = oracle.query_rotate(ix, Q)
    b = oracle.budget(rho, ix.N)
    for i in range(Q.shape[0]):
        for m in range(ix.M):
            a = oracle.activate(ix, qr[i], m, phi, 10, b, "heap")
            s = oracle.activate(ix, qr[i], m, phi, 10, b, "sort")
            assert a[0].tolist() == s[0].tolist() and a[1].tolist() == s[1].tolist() and a[2] == s[2]
            assert a[2] >= min(b, ix.N)
            # the last popped cell was needed: without it the budget was not reached
            sizes = np.diff(ix.offsets[m])[a[0]]
            assert sizes[:-1].sum() < b


# ------------------------------------------------------ Q4 counting
@pytest.mark.parametrize("phi", [0, 1])
def test_scores_list_walk_equals_eq1(gmm_index, phi):
    ix, X, Q = gmm_index
    qr = oracle.query_rotate(ix, Q)
    b = oracle.budget(0.03, ix.N)
    for i in range(5):
        acts = [oracle.activate(ix, qr[i], m, phi, 10, b) for m in range(ix.M)]
        V1 = oracle.scores_walk(ix, acts)
        V2 = oracle.scores_membership(ix, acts)
        assert np.array_equal(V1, V2)
        assert V1.max() <= (2 if phi else 1) * ix.M


# ------------------------------------------------------ Q5 cut
def test_cut_threshold_fallback_and_cap():
    V = np.array([0, 3, 1, 3, 2, 0, 1], np.int32)
    # plain: {V >= 2}
    C, how = oracle.cut(V, 2, 2)
    assert C.tolist() == [1, 3, 4] and how == 0
    # fallback (|C| = 0 < k = 3): top 3 by (V desc, id asc) = ids 1, 3 (V 3), 4 (V 2)
    C, how = oracle.cut(V, 4, 3)
    assert C.tolist() == [1, 3, 4] and how == 1
    # fallback asking for more than the #{V >= 1} = 5 points available
    C, how = oracle.cut(V, 4, 9)
    assert C.tolist() == [1, 2, 3, 4, 6] and how == 1
    # fallback boundary tie at V = 1: ids 2 and 6, the lower id wins
    C, how = oracle.cut(V, 4, 4)
    assert C.tolist() == [1, 2, 3, 4] and how == 1
    # cap: |{V >= 1}| = 5 > cap 3 -> keep the top 3
    C, how = oracle.cut(V, 1, 2, cap=3)
    assert C.tolist() == [1, 3, 4] and how == 2
    # tau = 0 keeps every point, even with V = 0
    C, how = oracle.cut(V, 0, 2)
    assert C.tolist() == list(range(7)) and how == 0


# ------------------------------------------------------ FP32 orders
def test_cr32_order_worked_example():
    g = load_golden("cr32_order.txt")
    x = np.zeros(32, np.float32)
    q = np.zeros(32, np.float32)
    x[:] = float(g["diff_rest"][0])
    x[0] = float(g["diff_dim0"][0])
    assert oracle.cr32(x, q) == np.float32(float(g["expected"][0]))


def test_cr32_exact_on_integers_and_error_bound():
    rng = np.random.default_rng(3)
    for Dp in (32, 64, 960, 4096):
        x = rng.integers(-8, 9, Dp).astype(np.float32)
        q = rng.integers(-8, 9, Dp).astype(np.float32)
        exact = float(np.sum((x.astype(np.float64) - q) ** 2))
        assert float(oracle.cr32(x, q)) == exact            # all partial sums exact below 2^24
        x = rng.standard_normal(Dp).astype(np.float32)
        q = rng.standard_normal(Dp).astype(np.float32)
        exact = float(np.sum((x.astype(np.float64) - q) ** 2))
        # depth of the reduction: 4 fma + 3 tree + Dp/32 sequential adds, plus the subtraction
        gamma = (4 + 3 + Dp // 32 + 2) * 2.0 ** -24
        assert abs(float(oracle.cr32(x, q)) - exact) <= gamma * exact * 1.01
        s = oracle.cr32_blocks(x, q)
        assert s.size == Dp // 32 and np.all(s >= 0)


def test_seq_sqdist_and_rotation_error_bounds():
    rng = np.random.default_rng(5)
    a = rng.standard_normal(96).astype(np.float32)
    b = rng.standard_normal(96).astype(np.float32)
    ex = float(np.sum((a.astype(np.float64) - b) ** 2))
    assert abs(float(oracle.seq_sqdist(a, b)) - ex) <= 100 * 2.0 ** -24 * ex
    D = 96
    R = oracle.rotation_from_gaussian(rng.standard_normal((D, D))).astype(np.float32)
    X = rng.standard_normal((7, D)).astype(np.float32)
    Y = oracle.rotate_rows(X, R)
    ref = X.astype(np.float64) @ R.astype(np.float64)
    bound = (D + 1) * 2.0 ** -24 * (np.abs(X).astype(np.float64) @ np.abs(R).astype(np.float64))
    assert Y.shape == (7, 96) and np.all(np.abs(Y[:, :D] - ref) <= bound)


# --------------------------------------------------- B1 covariance / CEV
def test_cev_closed_form_diagonal():
    g = load_golden("cev_diagonal.txt")
    D = int(g["D"][0])
    a = np.array([float(v) for v in g["a"]])
    X = np.zeros((2 * D, D), np.float32)
    for i in range(D):
        X[2 * i, i] = a[i]
        X[2 * i + 1, i] = -a[i]
    cov = oracle.covariance(X, np.arange(2 * D))
    assert np.allclose(cov, np.diag(2 * a * a / (2 * D - 1)), rtol=0, atol=1e-12)
    c, ev = oracle.cev(X, np.arange(2 * D))
    assert c == pytest.approx(int(g["cev_num"][0]) / int(g["cev_den"][0]), rel=1e-12)


def test_cev_isotropic_and_rank_deficient():
    rng = np.random.default_rng(7)
    X = rng.standard_normal((20000, 50)).astype(np.float32)
    c, _ = oracle.cev(X, np.arange(20000))
    assert 0.2 <= c < 0.25          # 0.2 in the limit; sampling spreads the spectrum upwards
    L = rng.standard_normal((100, 10))
    Y = (rng.standard_normal((3000, 10)) @ L.T).astype(np.float32)     # rank 10 <= 0.2 * 100
    c, _ = oracle.cev(Y, np.arange(3000))
    assert c == pytest.approx(1.0, abs=1e-9)


def test_cev_powerlaw_matches_analytic_spectrum():
    D = 100
    X, _ = synthetic.powerlaw(N=60000, D=D, nq=1, seed=1)
    c, _ = oracle.cev(X, np.arange(60000))
    lam = synthetic.powerlaw_spectrum(D)
    expected = lam[: int(0.2 * D)].sum() / lam.sum()
    assert c == pytest.approx(expected, abs=0.01)


def test_covariance_brute_force_small():
    rng = np.random.default_rng(11)
    X = rng.standard_normal((40, 6)).astype(np.float32)
    rows = np.array([0, 3, 5, 9, 17, 22, 39])
    cov = oracle.covariance(X, rows)
    assert np.allclose(cov, oracle.covariance_loops(X, rows), rtol=1e-12, atol=1e-14)
    S = X[rows].astype(np.float64)
    mu = S.mean(0)
    ref = sum(np.outer(s - mu, s - mu) for s in S) / (len(rows) - 1)
    assert np.allclose(cov, ref, rtol=1e-13, atol=1e-14)


# ------------------------------------------------------------ B2 rotation
@pytest.mark.parametrize("D", [16, 64, 256])
def test_rotation_orthogonal_and_unique(D):
    G = np.random.default_rng(D).standard_normal((D, D))
    R = oracle.rotation_from_gaussian(G)
    assert np.max(np.abs(R.T @ R - np.eye(D))) < 1e-10
    # G = R (R^T G) with R^T G upper triangular and a positive diagonal: this is
    # the unique QR factor with the sign convention R = Q diag(sign(diag R')).
    T = R.T @ G
    assert np.max(np.abs(np.tril(T, -1))) < 1e-9 * np.abs(G).max()
    assert np.all(np.diag(T) > 0)


def test_rotation_preserves_neighbours():
    rng = np.random.default_rng(2)
    X = rng.standard_normal((3000, 32)).astype(np.float32)
    Q = rng.standard_normal((10, 32)).astype(np.float32)
    R = oracle.rotation_from_gaussian(rng.standard_normal((32, 32)))
    i0, d0 = oracle.knn_f64(X, Q, 10)
    i1, d1 = oracle.knn_f64((X.astype(np.float64) @ R).astype(np.float32), (Q.astype(np.float64) @ R).astype(np.float32), 10)
    assert np.allclose(d0, d1, rtol=1e-5)
    assert np.mean(i0 == i1) > 0.99


def test_rotation_flattens_variance():
    X, _ = synthetic.powerlaw(N=20000, D=64, nq=1, seed=3)
    v0 = X.var(0)
    Dgen = np.random.default_rng(0).standard_normal((64, 64))
    Y = oracle.rotate_rows(X, oracle.rotation_from_gaussian(Dgen).astype(np.float32))
    assert Y.shape == (20000, 64)
    # a Haar mix already flattens most of it; check the rotated variance stays flat
    v1 = Y.var(0)
    assert v1.max() / v1.mean() < 3.0 and abs(v1.sum() / v0.sum() - 1) < 1e-3


# ------------------------------------------------------------- B3 k-means
def test_kmeans_hand_worked_cases():
    g = load_golden("kmeans_tiny.txt")
    for case in ("caseA", "caseB"):
        pts = np.array([[float(v)] for v in g[case + "_points"]], np.float32)
        init = np.array([int(v) for v in g[case + "_init"]], np.int32)
        C = oracle.kmeans(pts, 0, 1, 2, 1, init, int(g[case + "_iters"][0]))
        assert C[:, 0].tolist() == [float(v) for v in g[case + "_expected"]]


def test_kmeans_fixed_point_and_brute_force():
    rng = np.random.default_rng(4)
    for trial in range(20):
        pts = rng.standard_normal((8, 1)).astype(np.float32) * 3
        C = oracle.kmeans(pts, 0, 1, 2, 1, np.array([0, 1], np.int32), 50)
        d = (pts - C[:, 0][None, :]) ** 2
        asg = np.argmin(d, 1)
        for c in range(2):              # Lloyd fixed point: centroid = mean of members
            if np.any(asg == c):
                assert C[c, 0] == pytest.approx(pts[asg == c, 0].astype(np.float64).mean(), rel=1e-6, abs=1e-6)
        inertia = float(np.min(d, 1).sum())
        best = min(  # brute force over all 2-partitions
            sum(((pts[m, 0] - pts[m, 0].mean()) ** 2).sum() for m in (mask, ~mask) if m.any())
            for mask in (np.array([(b >> i) & 1 for i in range(8)], bool) for b in range(256)))
        assert best <= inertia + 1e-4


def test_assignment_is_fp64_argmin(gmm_index):
    ix, X, Q = gmm_index
    for m in range(ix.M):
        lo, hl, hr = oracle.subspace(ix.D, ix.M, m)
        for half, (o, h) in enumerate(((lo, hl), (lo + hl, hr))):
            Cm = ix.cent[m, half, :, :h].astype(np.float64)
            d = ((ix.Xr[:, None, o:o + h].astype(np.float64) - Cm[None]) ** 2).sum(-1)
            c = ix.cells[m] // ix.K if half == 0 else ix.cells[m] % ix.K
            got = d[np.arange(ix.N), c]
            assert np.all(got <= d.min(1) * (1 + 1e-5) + 1e-12)


# -------------------------------------------------------------- B5 codes
def test_sign_codes_hand_example():
    x = np.zeros((1, 64), np.float32)
    x[0, [0, 4, 31, 32, 63]] = [1.0, 2.0, 1e-30, 0.5, 3.0]
    x[0, [1, 2, 3]] = [-1.0, 0.0, -0.0]
    codes = oracle.sign_codes(x)
    assert codes[0].tolist() == [(1 << 0) | (1 << 4) | (1 << 31), (1 << 0) | (1 << 31)]


# ------------------------------------------------- Q6 Guaranteed mode
def test_guaranteed_full_coverage_is_exact_knn(gmm_index):
    ix, X, Q = gmm_index
    gt_i, gt_d = oracle.knn_f64(X, Q, 10)
    for rho, alpha in ((1.0, 0.5), (0.01, 0.0)):        # every cell, or tau = 0: C = all N
        ids, d2, st, _ = oracle.search(ix, Q, oracle.SearchParams(k=10, mode=0, rho=rho, alpha=alpha))
        assert np.all(st["n_candidates"] == ix.N)
        for i in range(Q.shape[0]):
            same = ids[i] == gt_i[i]
            # ids equal except at distance ties within 1e-5 relative
            assert np.all(same | np.isclose(d2[i], gt_d[i], rtol=1e-5))
            assert np.allclose(d2[i], gt_d[i], rtol=1e-5)


def test_guaranteed_returns_every_true_neighbour_with_enough_votes(gmm_index):
    ix, X, Q = gmm_index
    p = oracle.SearchParams(k=10, mode=0, rho=0.02, alpha=0.5)
    ids, d2, st, _ = oracle.search(ix, Q, p)
    gt_i, gt_d = oracle.knn_f64(X, Q, 10)
    for i in range(Q.shape[0]):
        det = oracle.query_detail(ix, Q[i], p)
        for j, x in enumerate(gt_i[i]):
            if det["V"][x] >= det["tau"]:
                assert x in ids[i] or np.isclose(gt_d[i, j], gt_d[i, -1], rtol=1e-5)


def test_search_equals_composed_steps(gmm_index):
    ix, X, Q = gmm_index
    for mode in (0, 1):
        p = oracle.SearchParams(k=7, mode=mode, rho=0.02, alpha=0.25)
        ids, d2, st, _ = oracle.search(ix, Q, p)
        for i in range(Q.shape[0]):
            det = oracle.query_detail(ix, Q[i], p)
            assert st["n_candidates"][i] == det["C"].size
            if mode == 0:
                i2, dd = oracle.rerank(ix, det["qr"], det["C"], 7)
            else:
                i2, dd, _, _ = oracle.verify_opt(ix, det["qr"], det["C"], 7, 2.1, 40 * 7)
            assert ids[i].tolist() == i2.tolist() and d2[i].tolist() == dd.tolist()


def test_rerank_pads_when_few_candidates(gmm_index):
    ix, X, Q = gmm_index
    qr = oracle.query_rotate(ix, Q)[0]
    ids, d2 = oracle.rerank(ix, qr, np.array([5, 2], np.int32), 4)
    assert ids[2:].tolist() == [-1, -1] and np.all(np.isinf(d2[2:]))
    assert sorted(ids[:2].tolist()) == [2, 5] and d2[0] <= d2[1]


# -------------------------------------------------- Q7 Optimized mode
def _opt_index(D, rows):
    Xr = np.zeros((len(rows), oracle.padded_dim(D)), np.float32)
    for r, v in enumerate(rows):
        Xr[r, :D] = v
    cent = np.zeros((1, 2, 2, 1), np.float32)
    off = np.zeros((1, 5), np.int32)
    off[0, 1:] = len(rows)
    ids = np.arange(len(rows), dtype=np.int32)[None, :]
    return _manual_index(D, 1, 2, cent, off, ids, Xr)


def test_verify_opt_patience_hand_example():
    g = load_golden("verify_opt_tiny.txt")
    D = 32
    rows = []
    for r, tgt in enumerate(float(v) for v in g["targets"]):
        x = np.ones(D, np.float32)
        x[:r] = -0.0
        x[D - 1] = 1.0 + math.sqrt(tgt - r)
        rows.append(x)
    ix = _opt_index(D, rows)
    q = np.ones(32, np.float32)
    C = np.arange(5, dtype=np.int32)
    ids, d2, nv, nf = oracle.verify_opt(ix, q, C, 1, float("inf"), 2)
    assert ids[0] == int(g["best_P2"][0]) and nv == 5
    ids, d2, nv, nf = oracle.verify_opt(ix, q, C, 1, float("inf"), 1)
    assert ids[0] == int(g["best_P1"][0]) and nv == int(g["processed_P1"][0])


def test_verify_opt_id_order_hand_example():
    """The ablation without Hamming re-ranking (order 1) verifies in id order.
    The rows of the hand example get their distances back, but now their
    Hamming distances fall with the id (row r has 4 - r dims flipped), so only
    order 1 walks them 0, 1, 2, 3, 4 as the hand-worked results assume; order
    0 walks them the other way round."""
    g = load_golden("verify_opt_tiny.txt")
    D = 32
    rows = []
    for r, tgt in enumerate(float(v) for v in g["targets"]):
        x = np.ones(D, np.float32)
        nneg = 4 - r
        x[:nneg] = -0.0
        x[D - 1] = 1.0 + math.sqrt(tgt - nneg)
        rows.append(x)
    ix = _opt_index(D, rows)
    q = np.ones(32, np.float32)
    C = np.arange(5, dtype=np.int32)
    ids, d2, nv, nf = oracle.verify_opt(ix, q, C, 1, float("inf"), 2, order=1)
    assert ids[0] == int(g["best_P2"][0]) and nv == 5
    ids, d2, nv, nf = oracle.verify_opt(ix, q, C, 1, float("inf"), 1, order=1)
    assert ids[0] == int(g["best_P1"][0]) and nv == int(g["processed_P1"][0])
    # exhaustive verification does not depend on the order
    a = oracle.verify_opt(ix, q, C, 3, float("inf"), 0, order=0)
    b = oracle.verify_opt(ix, q, C, 3, float("inf"), 0, order=1)
    assert a[0].tolist() == b[0].tolist() and a[1].tolist() == b[1].tolist()


def test_verify_opt_adsampling_prune_hand_example():
    D = 64
    a = np.ones(D, np.float32)
    a[D - 1] = 1.0 + math.sqrt(10.0)
    b = np.ones(D, np.float32)
    b[0] = -0.0
    b[1] = 1.0 + math.sqrt(5.0)
    ix = _opt_index(D, [a, b])
    q = np.ones(D, np.float32)
    C = np.array([0, 1], np.int32)
    assert oracle.ads_factor(32, 64, 0.0) == np.float32(0.5)
    ids, d2, nv, nf = oracle.verify_opt(ix, q, C, 1, 0.0, 0)
    assert ids[0] == 0 and nf == 1 and nv == 2
    ids, d2, nv, nf = oracle.verify_opt(ix, q, C, 1, float("inf"), 0)
    assert ids[0] == 1 and nf == 2


def test_verify_opt_without_pruning_equals_exact_rerank(gmm_index):
    ix, X, Q = gmm_index
    qr = oracle.query_rotate(ix, Q)
    p = oracle.SearchParams(k=10, mode=1, rho=0.03, alpha=0.25)
    for i in range(Q.shape[0]):
        det = oracle.query_detail(ix, Q[i], p)
        a = oracle.verify_opt(ix, qr[i], det["C"], 10, float("inf"), 0)
        b = oracle.rerank(ix, qr[i], det["C"], 10)
        assert a[0].tolist() == b[0].tolist() and a[1].tolist() == b[1].tolist()
        assert a[2] == a[3] == det["C"].size


def test_verify_opt_prunes_only_above_bound(gmm_index):
    """Every ADSampling prune rests on a partial distance above the Eq. 2 bound
    (checked in FP64 from the raw rows), and results stay within the candidates."""
    ix, X, Q = gmm_index
    qr = oracle.query_rotate(ix, Q)
    p = oracle.SearchParams(k=10, mode=1, rho=0.03, alpha=0.25)
    for i in range(Q.shape[0]):
        det = oracle.query_detail(ix, Q[i], p)
        ids, d2, nv, nf = oracle.verify_opt(ix, qr[i], det["C"], 10, 2.1, 400)
        assert set(ids[ids >= 0].tolist()) <= set(det["C"].tolist())
        assert nf <= nv <= det["C"].size
        ex = ((ix.Xr[ids[ids >= 0]].astype(np.float64) - qr[i]) ** 2).sum(1)
        assert np.allclose(ex, d2[ids >= 0], rtol=1e-5)


# ------------------------------------------------------- Theorem 1
def test_theorem1_hoeffding_bound_holds_empirically():
    """Guaranteed Mode: P(x* in C) >= 1 - exp(-2 (M p* - tau)^2 / M) (Theorem 1).

    p* is estimated per query pool as the mean single-subspace collision rate of
    the true nearest neighbour; the empirical retrieval rate must not fall below
    the bound by more than three binomial standard deviations."""
    X, Q = synthetic.gmm(N=8000, D=128, nq=200, n_comp=30, rank=16, seed=5)
    ix = oracle.build_index(X, M=8, rotate=1)
    gt_i, _ = oracle.knn_f64(X, Q, 1)
    p = oracle.SearchParams(k=1, mode=0, rho=0.05, alpha=0.25)
    hits, coll = 0, []
    for i in range(Q.shape[0]):
        det = oracle.query_detail(ix, Q[i], p)
        x = gt_i[i, 0]
        coll.append(det["V"][x] / ix.M)
        hits += det["V"][x] >= det["tau"]
    ps = float(np.mean(coll))
    t = oracle.tau(p.alpha, ix.M)
    assert ix.M * ps > t
    bound = 1 - math.exp(-2 * (ix.M * ps - t) ** 2 / ix.M)
    rate = hits / Q.shape[0]
    sd = math.sqrt(max(bound * (1 - bound), 1e-4) / Q.shape[0])
    assert rate >= bound - 3 * sd, (rate, bound)


def test_readings_tau_and_budget():
    assert oracle.tau(0.3, 10) == 3 and oracle.tau(0.25, 8) == 2 and oracle.tau(0.0, 8) == 0
    assert oracle.tau(0.31, 10) == 4 and oracle.tau(1.0, 16) == 16
    assert oracle.budget(0.01, 20000) == 200 and oracle.budget(0.07, 100) == 7
    assert oracle.budget(1e-9, 10) == 1 and oracle.budget(1.0, 12345) == 12345
    assert [oracle.subspace(960, 10, m) for m in (0, 9)] == [(0, 48, 48), (864, 48, 48)]
    assert oracle.subspace(10, 3, 1) == (3, 1, 2)


def test_ads_factor_closed_values():
    # eps0 = sqrt(t) makes (1 + eps0/sqrt(t))^2 = 4, so the factor is 4 t / D:
    # t = 64, D = 256 gives exactly 1; t = 32, D = 1024 gives exactly 1/8.
    assert oracle.ads_factor(64, 256, 8.0) == np.float32(1.0)
    assert oracle.ads_factor(32, 1024, math.sqrt(32.0)) == pytest.approx(0.125, rel=1e-7)
    # eps0 = sqrt(t) (sqrt 2 - 1) makes the square 2: t = 32, D = 128 -> 0.5
    assert oracle.ads_factor(32, 128, math.sqrt(32.0) * (math.sqrt(2.0) - 1.0)) == pytest.approx(0.5, rel=1e-6)
    assert oracle.ads_factor(32, 960, 0.0) == pytest.approx(1.0 / 30.0, rel=1e-7)
