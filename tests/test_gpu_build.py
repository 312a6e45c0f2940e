"""GPU index build (§4.1-§4.2) against the oracle.

Steps whose result is an integer or bit pattern -- cell assignment (given the
centroids), CSR lists (given the cells), sign codes (given the rows) -- must be
identical.  FP64 linear algebra (covariance, eigenvalues, QR) is compared within
tolerances set by its arithmetic; k-means from the same initial centroids within
FP32 rounding of the means.  The whole build is checked by the invariants that
define a valid index and by its recall.  The oracle's inputs never come from
the GPU side."""
import numpy as np
import pytest

import oracle
import synthetic

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2603_05180_gb300 as crisp  # noqa: E402

DEV = torch.device("cuda:0")


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


@pytest.fixture(scope="module")
def data():
    X, Q = synthetic.gmm()
    draws = synthetic.method_draws(20000, 256, 8, 50, seed=0)
    ix_o = oracle.build_index(X, M=8, draws=draws)
    return X, Q, draws, ix_o


def test_covariance_and_eigenvalues(data):
    X, Q, draws, ix_o = data
    S, D = draws.cev_sample.size, 256
    cov = torch.empty((D, D), dtype=torch.float64, device=DEV)
    crisp.crisp_covariance(dev(X), 20000, D, D, dev(draws.cev_sample), S, cov)
    ref = oracle.covariance(X, draws.cev_sample)
    c = cov.cpu().numpy()
    assert np.allclose(c, ref, rtol=1e-9, atol=1e-9 * np.abs(ref).max())
    eig = torch.empty(D, dtype=torch.float64, device=DEV)
    crisp.crisp_eigvalsh(cov, D, eig)
    ev = np.linalg.eigvalsh(ref)[::-1]
    assert np.allclose(eig.cpu().numpy(), ev, rtol=0, atol=1e-10 * ev[0])
    cev = crisp.crisp_cev(dev(X), 20000, D, D, dev(draws.cev_sample), S)
    assert abs(cev - ix_o.cev) < 1e-10


@pytest.mark.parametrize("D", [2, 33, 256])
def test_eigenvalues_of_known_spectra(D):
    r = np.random.default_rng(D)
    U = np.linalg.qr(r.standard_normal((D, D)))[0]
    lam = np.sort(r.uniform(0.1, 10.0, D))[::-1]
    A = (U * lam) @ U.T
    A = 0.5 * (A + A.T)
    eig = torch.empty(D, dtype=torch.float64, device=DEV)
    crisp.crisp_eigvalsh(dev(A), D, eig)
    assert np.allclose(eig.cpu().numpy(), lam, rtol=0, atol=1e-11 * lam[0])


@pytest.mark.parametrize("D", [1, 7, 64, 256])
def test_rotation_from_gaussian(D):
    G = np.random.default_rng(D).standard_normal((D, D))
    R = torch.empty((D, D), dtype=torch.float64, device=DEV)
    crisp.crisp_rotation_from_gaussian(dev(G), D, R)
    Rg = R.cpu().numpy()
    assert np.max(np.abs(Rg.T @ Rg - np.eye(D))) < 1e-10
    assert np.max(np.abs(Rg - oracle.rotation_from_gaussian(G))) < 1e-11
    T = Rg.T @ G                                   # upper triangular, positive diagonal
    assert np.max(np.abs(np.tril(T, -1))) < 1e-9 * np.abs(G).max() and np.all(np.diag(T) > 0)


def test_cells_csr_and_codes_bitexact(data):
    X, Q, draws, ix_o = data
    N, D, Dp, M, K, H = ix_o.N, ix_o.D, ix_o.Dp, ix_o.M, ix_o.K, ix_o.H
    cells = torch.empty((M, N), dtype=torch.int16, device=DEV)
    crisp.crisp_assign_cells(dev(ix_o.Xr), N, D, Dp, M, K, H, dev(ix_o.cent), cells)
    got = cells.cpu().numpy().view(np.uint16)
    assert np.array_equal(got, ix_o.cells)
    for m in range(M):
        off = torch.empty(K * K + 1, dtype=torch.int32, device=DEV)
        ids = torch.empty(N, dtype=torch.int32, device=DEV)
        crisp.crisp_csr_build(dev(ix_o.cells[m]), N, K * K, off, ids)
        assert np.array_equal(off.cpu().numpy(), ix_o.offsets[m])
        assert np.array_equal(ids.cpu().numpy(), ix_o.ids[m])
    codes = torch.empty((N, Dp // 32), dtype=torch.int32, device=DEV)
    crisp.crisp_sign_codes(dev(ix_o.Xr), N, Dp, codes)
    assert np.array_equal(codes.cpu().numpy().view(np.uint32), ix_o.codes)


@pytest.mark.parametrize("N,K2", [(1, 4), (4095, 2500), (4097, 7), (150000, 2500)])
def test_csr_shapes_and_ragged_chunks(N, K2):
    cells = (np.random.default_rng(N).zipf(1.4, N) % K2).astype(np.uint16)
    off = torch.empty(K2 + 1, dtype=torch.int32, device=DEV)
    ids = torch.empty(N, dtype=torch.int32, device=DEV)
    crisp.crisp_csr_build(dev(cells), N, K2, off, ids)
    ro, ri = oracle.csr(cells, K2)
    assert np.array_equal(off.cpu().numpy(), ro) and np.array_equal(ids.cpu().numpy(), ri)


def test_kmeans_from_the_same_start(data):
    X, Q, draws, ix_o = data
    T = np.ascontiguousarray(ix_o.Xr[draws.kmeans_sample])
    S, ldt, K, H = T.shape[0], ix_o.Dp, 50, ix_o.H
    for m, half in ((0, 0), (3, 1), (7, 1)):
        lo, hl, hr = oracle.subspace(ix_o.D, ix_o.M, m)
        off, h = (lo, hl) if half == 0 else (lo + hl, hr)
        init = draws.kmeans_init[m, half]
        Cg = torch.empty((K, H), dtype=torch.float32, device=DEV)
        crisp.crisp_kmeans(dev(T), S, ldt, off, h, K, H, dev(init), 20, Cg)
        Cg = Cg.cpu().numpy()
        Co = oracle.kmeans(T, off, h, K, H, init, 20)
        # same start, same FP32 assignment order; FP64 sums in another order can
        # flip a near-tie point, so compare the objective, and most centroids
        assert np.mean(np.all(np.isclose(Cg, Co, rtol=1e-4, atol=1e-4), axis=1)) > 0.9
        x = T[:, off:off + h].astype(np.float64)

        def inertia(Cc):
            return float(np.min(((x[:, None, :] - Cc[None, :, :h]) ** 2).sum(-1), 1).sum())

        assert inertia(Cg) <= inertia(Co) * 1.01


def test_build_end_to_end(data):
    X, Q, draws, ix_o = data
    ix = crisp.crisp_build(dev(X), 20000, 256, crisp.build_params(8, draws=draws, copies=3))
    info = ix.info()
    assert info.rotated == ix_o.rotated and abs(info.cev - ix_o.cev) < 1e-10
    blob = crisp.crisp_index_export(ix)
    R32 = np.frombuffer(blob, np.float32, 256 * 256, 256).reshape(256, 256)
    assert np.max(np.abs(R32 - ix_o.R32)) < 1e-6
    # invariants of the index through its own search: a rho = 1, tau = 0 search is exact kNN
    gi, gd = oracle.knn_f64(X, Q, 10)
    ids = torch.empty((100, 10), dtype=torch.int64, device=DEV)
    d2 = torch.empty((100, 10), dtype=torch.float32, device=DEV)
    crisp.crisp_search(ix, dev(Q), 100, crisp.search_params(k=10, rho=1.0, alpha=0.0), ids, d2)
    assert np.allclose(d2.cpu().numpy(), gd, rtol=2e-5)
    # recall at a normal operating point is close to the oracle index's
    p = dict(k=10, rho=0.02, alpha=0.25)
    crisp.crisp_search(ix, dev(Q), 100, crisp.search_params(**p), ids, d2)
    r_gpu = oracle.recall_at_k(ids.cpu().numpy(), gd, X, Q, 10)
    r_orc = oracle.recall_at_k(oracle.search(ix_o, Q, oracle.SearchParams(**p))[0], gd, X, Q, 10)
    assert r_gpu >= r_orc - 0.03


def test_build_cells_are_valid_argmins(data):
    """Every cell of the GPU-built index is a nearest (left, right) centroid pair
    of its row, within FP32 rounding of the FP64 minimum."""
    X, Q, draws, ix_o = data
    ix = crisp.crisp_build(dev(X), 20000, 256, crisp.build_params(8, draws=draws))
    blob = crisp.crisp_index_export(ix)
    import struct
    v, N, D, Dp, M, K, H, rot = struct.unpack_from("<8q", blob, 8)
    pos = 256
    secs = []
    for n in ([4 * D * D] if rot else []) + [4 * M * 2 * K * H, 4 * M * (K * K + 1), 4 * M * N, 4 * N * Dp]:
        secs.append((pos, n))
        pos = (pos + n + 255) // 256 * 256
    i0 = 1 if rot else 0
    cent = np.frombuffer(blob, np.float32, M * 2 * K * H, secs[i0][0]).reshape(M, 2, K, H)
    offs = np.frombuffer(blob, np.int32, M * (K * K + 1), secs[i0 + 1][0]).reshape(M, K * K + 1)
    ids = np.frombuffer(blob, np.int32, M * N, secs[i0 + 2][0]).reshape(M, N)
    Xr = np.frombuffer(blob, np.float32, N * Dp, secs[i0 + 3][0]).reshape(N, Dp)
    for m in range(M):
        assert offs[m, 0] == 0 and offs[m, -1] == N and np.all(np.diff(offs[m]) >= 0)
        assert np.array_equal(np.sort(ids[m]), np.arange(N))
        lo, hl, hr = oracle.subspace(D, M, m)
        cell_of = np.empty(N, np.int64)
        for c in range(K * K):
            seg = ids[m, offs[m, c]:offs[m, c + 1]]
            assert np.all(np.diff(seg) > 0)
            cell_of[seg] = c
        for half, (o, h) in enumerate(((lo, hl), (lo + hl, hr))):
            d = ((Xr[:, None, o:o + h].astype(np.float64) - cent[m, half, None, :, :h]) ** 2).sum(-1)
            c = cell_of // K if half == 0 else cell_of % K
            assert np.all(d[np.arange(N), c] <= d.min(1) * (1 + 1e-5) + 1e-12)


@pytest.mark.slow
def test_full_size_build_and_search_properties():
    """The benchmark's workload (1M x 960, M = 20): returned distances equal
    FP64 distances recomputed from the original rows, results are sorted, and
    recall@10 at the benchmark's point is at least 0.95.  The 2,000-query batch
    takes the grouped scorers; its first 500 queries searched on their own take
    the streaming kernels, and both must give the same bits (every distance is
    the CR32 order of its own (query, row) pair)."""
    import bench

    X, Q = synthetic.powerlaw(1_000_000, 960, 2000, device="cuda")
    ix = crisp.crisp_build(X, 1_000_000, 960, crisp.build_params(20, draws=synthetic.method_draws(1_000_000, 960, 20, 50)))
    ids = torch.empty((2000, 10), dtype=torch.int64, device=DEV)
    d2 = torch.empty((2000, 10), dtype=torch.float32, device=DEV)
    crisp.crisp_search(ix, Q, 2000, crisp.search_params(k=10, **{k: v for k, v in bench.DEFAULT_POINT.items()}), ids,
                       d2)
    _, gd = bench.ground_truth(torch, X, Q, 10)
    r = bench.recall_at_k(torch, X, Q, ids, gd[:, 9].contiguous())
    assert r >= 0.95
    sel = ids[:200]
    ex = ((X[sel].double() - Q[:200].double()[:, None, :]) ** 2).sum(-1)
    assert torch.allclose(ex, d2[:200].double(), rtol=1e-4)
    assert bool((d2[:, 1:] >= d2[:, :-1]).all())
    ids_s = torch.empty((500, 10), dtype=torch.int64, device=DEV)
    d2_s = torch.empty((500, 10), dtype=torch.float32, device=DEV)
    crisp.crisp_search(ix, Q[:500].contiguous(), 500,
                       crisp.search_params(k=10, **{k: v for k, v in bench.DEFAULT_POINT.items()}), ids_s, d2_s)
    assert torch.equal(ids_s, ids[:500]) and torch.equal(d2_s, d2[:500])


@pytest.mark.slow
def test_full_size_steps_equal_the_oracle():
    """The benchmark's workload (1M x 960, M = 20) on an index the oracle built
    from the same rows and draws: a 2,000-query batch (large enough for the
    grouped re-rank) through the library's steps, and for 200 sampled queries
    the visited cells, candidate lists, their scores and the re-ranked top-10
    equal the oracle's, element by element."""
    import bench

    N, D, M, nq = 1_000_000, 960, 20, 2000
    X, Q = synthetic.powerlaw(N, D, nq, device="cuda")
    Xh, Qh = X.cpu().numpy(), Q.cpu().numpy()
    del X
    ix_o = oracle.build_index(Xh, M=M, draws=synthetic.method_draws(N, D, M, 50))
    ix = crisp.crisp_index_import(oracle.export_blob(ix_o))
    pt = bench.DEFAULT_POINT
    p = oracle.SearchParams(k=10, mode=pt["mode"], rho=pt["rho"], alpha=pt["alpha"])
    K2 = ix_o.K * ix_o.K
    Qr = torch.empty((nq, ix_o.Dp), dtype=torch.float32, device=DEV)
    crisp.crisp_rotate_rows(Q, nq, D, D, dev(ix_o.R32), Qr, ix_o.Dp)
    act = torch.empty((nq, M, K2), dtype=torch.int32, device=DEV)
    nact = torch.empty((nq, M), dtype=torch.int32, device=DEV)
    bud = oracle.budget(p.rho, N)
    crisp.crisp_activate(ix, Qr, nq, 0, 10, bud, act, nact)
    stride = 200_000
    cand = torch.empty((nq, stride), dtype=torch.int32, device=DEV)
    ncand = torch.empty((nq,), dtype=torch.int64, device=DEV)
    score = torch.empty((nq, stride), dtype=torch.uint8, device=DEV)
    crisp.crisp_count_cut(ix, act, nact, nq, oracle.tau(p.alpha, M), 10, 0, cand, stride, ncand, score)
    ids = torch.empty((nq, 10), dtype=torch.int64, device=DEV)
    d2 = torch.empty((nq, 10), dtype=torch.float32, device=DEV)
    crisp.crisp_rerank(ix, Qr, nq, cand, stride, ncand, 10, ids, d2)
    qr_g = Qr.cpu().numpy()
    nact_g, n_g, gi, gd = nact.cpu().numpy(), ncand.cpu().numpy(), ids.cpu().numpy(), d2.cpu().numpy()
    assert int(n_g.max()) < stride
    sample = synthetic.subsample_queries(nq, 200, seed=1)
    for q in sample:
        det = oracle.query_detail(ix_o, Qh[q], p)
        assert np.array_equal(qr_g[q], det["qr"]), q
        a = act[q].cpu().numpy()
        for m in range(M):
            cells, w, _ = det["acts"][m]
            assert nact_g[q, m] == len(cells) and np.array_equal(a[m, :len(cells)] & 0xFFFF, cells), (q, m)
        C = det["C"]
        assert n_g[q] == C.size and np.array_equal(cand[q, :C.size].cpu().numpy(), C), q
        assert np.array_equal(score[q, :C.size].cpu().numpy(), det["V"][C]), q
        oi, od = oracle.rerank(ix_o, det["qr"], C, 10)
        assert np.array_equal(gi[q], oi) and np.array_equal(gd[q], od), q
    ix.free()
