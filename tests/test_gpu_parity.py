"""GPU vs oracle parity, step by step and end to end, through the C ABI.

The oracle builds the index (its own CPU code, from the seeded workload and
the seeded draws); the blob goes into the GPU library with crisp_index_import,
so both sides search the very same index.  Integer outputs (visited cells,
weights, candidate sets, scores, ids) must be identical; FP32 values computed
in the canonical orders (rotated queries, half distances, CR32 distances) must
be identical too.  No input or expected value here comes from the GPU side.
"""
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


def empty(shape, dtype):
    return torch.empty(shape, dtype=dtype, device=DEV)


@pytest.fixture(scope="module")
def c1():
    """The small parity workload: 50-component GMM, N=20,000, D=256, 100 queries, M=8."""
    X, Q = synthetic.gmm()
    ix_o = oracle.build_index(X, M=8, draws=synthetic.method_draws(20000, 256, 8, 50, seed=0))
    assert ix_o.rotated == 1
    ix = crisp.crisp_index_import(oracle.export_blob(ix_o))
    return X, Q, ix_o, ix


@pytest.fixture(scope="module")
def multitile():
    """N = 150,000 ids: three counting tiles, the last one ragged; no rotation."""
    X, Q = synthetic.gmm(N=150000, D=64, nq=24, n_comp=40, rank=8, seed=3)
    ix_o = oracle.build_index(X, M=4, rotate=0, draws=synthetic.method_draws(150000, 64, 4, 50, seed=3,
                                                                            kmeans_train=30000))
    ix = crisp.crisp_index_import(oracle.export_blob(ix_o))
    return X, Q, ix_o, ix


def gpu_qr(ix_o, ix, Q):
    nq = Q.shape[0]
    Qr = empty((nq, ix_o.Dp), torch.float32)
    if ix_o.rotated:
        crisp.crisp_rotate_rows(dev(Q), nq, ix_o.D, ix_o.D, dev(ix_o.R32), Qr, ix_o.Dp)
    else:
        Qr.zero_()
        Qr[:, :ix_o.D] = dev(Q)
    return Qr


def test_import_export_roundtrip(c1):
    X, Q, ix_o, ix = c1
    blob = oracle.export_blob(ix_o)
    assert crisp.crisp_index_export(ix) == blob
    info = ix.info()
    assert (info.N, info.D, info.Dp, info.M, info.K, info.H, info.rotated) == (20000, 256, 256, 8, 50, 16, 1)
    assert info.max_cell == int(np.diff(ix_o.offsets, axis=1).max())


def test_q1_query_rotation_bitexact(c1):
    X, Q, ix_o, ix = c1
    got = gpu_qr(ix_o, ix, Q).cpu().numpy()
    assert np.array_equal(got, oracle.query_rotate(ix_o, Q))
    # a ragged block of base rows too (several GEMM tiles)
    Y = empty((333, 256), torch.float32)
    crisp.crisp_rotate_rows(dev(X[:333]), 333, 256, 256, dev(ix_o.R32), Y, 256)
    assert np.array_equal(Y.cpu().numpy(), oracle.rotate_rows(X[:333], ix_o.R32))


def test_q2_half_distances_bitexact(c1):
    X, Q, ix_o, ix = c1
    nq = Q.shape[0]
    Qr = gpu_qr(ix_o, ix, Q)
    srt = empty((nq, 8, 2, 50), torch.float32)
    prm = empty((nq, 8, 2, 50), torch.int32)
    crisp.crisp_half_dists(ix, Qr, nq, srt, prm)
    srt, prm = srt.cpu().numpy(), prm.cpu().numpy()
    qr = oracle.query_rotate(ix_o, Q)
    for i in range(0, nq, 7):
        for m in range(8):
            for h in range(2):
                _, s, p = oracle.half_dists(ix_o, qr[i], m, h)
                assert np.array_equal(srt[i, m, h], s) and np.array_equal(prm[i, m, h], p)


def _gpu_activate(ix_o, ix, Qr, nq, phi, k, bud):
    K2 = ix_o.K * ix_o.K
    act = empty((nq, ix_o.M, K2), torch.int32)
    nact = empty((nq, ix_o.M), torch.int32)
    got = empty((nq, ix_o.M), torch.int64)
    crisp.crisp_activate(ix, Qr, nq, phi, k, bud, act, nact, got)
    return act, nact, got


@pytest.mark.parametrize("phi,rho,k", [(0, 0.01, 10), (1, 0.01, 10), (1, 0.05, 100), (0, 1.0, 10), (1, 1e-9, 3)])
def test_q3_activation_bitexact(c1, phi, rho, k):
    X, Q, ix_o, ix = c1
    nq = Q.shape[0]
    Qr = gpu_qr(ix_o, ix, Q)
    bud = oracle.budget(rho, ix_o.N)
    act, nact, got = (t.cpu().numpy() for t in _gpu_activate(ix_o, ix, Qr, nq, phi, k, bud))
    qr = oracle.query_rotate(ix_o, Q)
    for i in range(nq):
        for m in range(ix_o.M):
            cells, w, r = oracle.activate(ix_o, qr[i], m, phi, k, bud)
            n = nact[i, m]
            assert n == len(cells) and got[i, m] == r
            assert np.array_equal(act[i, m, :n] & 0xFFFF, cells)
            assert np.array_equal(act[i, m, :n] >> 16, w)


def _count_case(ix_o, ix, Q, p, stride=None, with_score=True):
    nq = Q.shape[0]
    Qr = gpu_qr(ix_o, ix, Q)
    bud = oracle.budget(p.rho, ix_o.N)
    act, nact, _ = _gpu_activate(ix_o, ix, Qr, nq, p.mode, p.k, bud)
    t = oracle.tau(p.alpha, ix_o.M)
    stride = stride or ix_o.N
    cand = empty((nq, stride), torch.int32)
    ncand = empty((nq,), torch.int64)
    score = empty((nq, stride), torch.uint8) if with_score else None
    how = empty((nq,), torch.int32)
    crisp.crisp_count_cut(ix, act, nact, nq, t, p.k, p.max_candidates, cand, stride, ncand, score, how)
    return cand.cpu().numpy(), ncand.cpu().numpy(), (score.cpu().numpy() if with_score else None), how.cpu().numpy()


def _oracle_cuts(ix_o, Q, p, cand, ncand):
    """The oracle's own rotated query and cut per query (the inputs of the
    oracle's re-rank / verification below); the GPU's lists must equal them."""
    out = []
    for i in range(Q.shape[0]):
        det = oracle.query_detail(ix_o, Q[i], p)
        assert np.array_equal(cand[i, :ncand[i]], det["C"]), i
        out.append((det["qr"], det["C"]))
    return out


@pytest.mark.parametrize("mode,rho,alpha,cap", [
    (0, 0.01, 0.3, 0),      # plain cut
    (1, 0.02, 0.25, 0),     # weighted scores
    (0, 0.002, 1.0, 0),     # tau = M: fallback for most queries
    (1, 0.003, 1.0, 0),     # weighted fallback
    (0, 0.03, 0.125, 50),   # cap binds
    (1, 0.03, 0.0, 300),    # tau = 0: every point, then the cap
])
def test_q4_q5_counts_and_candidates_bitexact(c1, mode, rho, alpha, cap):
    X, Q, ix_o, ix = c1
    p = oracle.SearchParams(k=10, mode=mode, rho=rho, alpha=alpha, max_candidates=cap)
    cand, ncand, score, how = _count_case(ix_o, ix, Q, p)
    hows = set()
    for i in range(Q.shape[0]):
        det = oracle.query_detail(ix_o, Q[i], p)
        n = ncand[i]
        assert n == det["C"].size, (i, n, det["C"].size)
        assert np.array_equal(cand[i, :n], det["C"])
        assert np.array_equal(score[i, :n], det["V"][det["C"]])
        assert how[i] == det["how"]
        hows.add(det["how"])
    if alpha == 1.0:
        assert 1 in hows
    if cap:
        assert 2 in hows


def test_q4_q5_multi_tile_ragged(multitile):
    X, Q, ix_o, ix = multitile
    assert ix_o.N > 2 * 65536
    for p in (oracle.SearchParams(k=10, mode=0, rho=0.01, alpha=0.5),
              oracle.SearchParams(k=10, mode=1, rho=0.01, alpha=0.5),
              oracle.SearchParams(k=10, mode=0, rho=0.0005, alpha=1.0)):
        cand, ncand, score, how = _count_case(ix_o, ix, Q, p)
        for i in range(Q.shape[0]):
            det = oracle.query_detail(ix_o, Q[i], p)
            assert np.array_equal(cand[i, :ncand[i]], det["C"]) and how[i] == det["how"]
            assert np.array_equal(score[i, :ncand[i]], det["V"][det["C"]])


@pytest.mark.parametrize("k", [1, 10, 100, 256])
def test_q6_rerank_bitexact(c1, k):
    X, Q, ix_o, ix = c1
    p = oracle.SearchParams(k=k, mode=0, rho=0.02, alpha=0.25)
    cand, ncand, _, _ = _count_case(ix_o, ix, Q, p, with_score=False)
    nq = Q.shape[0]
    Qr = gpu_qr(ix_o, ix, Q)
    ids = empty((nq, k), torch.int64)
    d2 = empty((nq, k), torch.float32)
    crisp.crisp_rerank(ix, Qr, nq, dev(cand), cand.shape[1], dev(ncand), k, ids, d2)
    ids, d2 = ids.cpu().numpy(), d2.cpu().numpy()
    for i, (qr, C) in enumerate(_oracle_cuts(ix_o, Q, p, cand, ncand)):
        oi, od = oracle.rerank(ix_o, qr, C, k)
        assert np.array_equal(ids[i], oi) and np.array_equal(d2[i], od)


@pytest.mark.parametrize("k,eps0,P", [(10, 2.1, 400), (10, 0.0, 400), (10, float("inf"), 0), (1, 2.1, 1),
                                      (100, 2.1, 4000), (10, 1.0, 20)])
@pytest.mark.parametrize("order", [0, 1])
def test_q7_optimized_verification_bitexact(c1, k, eps0, P, order):
    X, Q, ix_o, ix = c1
    p = oracle.SearchParams(k=k, mode=1, rho=0.03, alpha=0.25)
    cand, ncand, _, _ = _count_case(ix_o, ix, Q, p, with_score=False)
    nq = Q.shape[0]
    Qr = gpu_qr(ix_o, ix, Q)
    ids = empty((nq, k), torch.int64)
    d2 = empty((nq, k), torch.float32)
    nv = empty((nq,), torch.int64)
    nf = empty((nq,), torch.int64)
    crisp.crisp_verify_opt(ix, Qr, nq, dev(cand), cand.shape[1], dev(ncand), k, eps0, P, ids, d2, nv, nf, order=order)
    ids, d2, nv, nf = (t.cpu().numpy() for t in (ids, d2, nv, nf))
    for i, (qr, C) in enumerate(_oracle_cuts(ix_o, Q, p, cand, ncand)):
        oi, od, onv, onf = oracle.verify_opt(ix_o, qr, C, k, eps0, P, order=order)
        assert np.array_equal(ids[i], oi) and np.array_equal(d2[i], od), i
        assert (nv[i], nf[i]) == (onv, onf), (i, nv[i], nf[i], onv, onf)


SEARCH_CASES = [
    dict(k=10, mode=0, rho=0.01, alpha=0.3),
    dict(k=10, mode=1, rho=0.01, alpha=0.3),
    dict(k=10, mode=0, rho=0.05, alpha=0.25),
    dict(k=10, mode=1, rho=0.05, alpha=0.25),
    dict(k=100, mode=1, rho=0.03, alpha=0.25, patience_factor=20),
    dict(k=5, mode=0, rho=0.002, alpha=1.0),
    dict(k=10, mode=1, rho=0.04, alpha=0.125, max_candidates=400),
    dict(k=10, mode=1, rho=0.03, alpha=0.25, verify_order=1),
]


@pytest.mark.parametrize("kw", SEARCH_CASES)
def test_search_end_to_end_bitexact(c1, kw):
    X, Q, ix_o, ix = c1
    p = oracle.SearchParams(**kw)
    nq, k = Q.shape[0], p.k
    ids = empty((nq, k), torch.int64)
    d2 = empty((nq, k), torch.float32)
    st = empty((nq, 6), torch.int64)   # crisp_query_stats is 48 bytes
    crisp.crisp_search(ix, dev(Q), nq, crisp.search_params(**kw), ids, d2, st)
    oi, od, ost, _ = oracle.search(ix_o, Q, p)
    assert np.array_equal(ids.cpu().numpy(), oi)
    assert np.array_equal(d2.cpu().numpy(), od)
    s = st.cpu().numpy()
    assert np.array_equal(s[:, 0], ost["n_candidates"])
    assert np.array_equal(s[:, 1], ost["n_verified"])
    assert np.array_equal(s[:, 2], ost["n_full"])
    assert np.array_equal(s[:, 3], ost["n_retrieved"])
    flags = np.ascontiguousarray(s[:, 4]).view(np.int32).reshape(nq, 2)
    assert np.array_equal(flags[:, 0], ost["fallback"]) and np.array_equal(flags[:, 1], ost["capped"])


def test_search_multi_tile_end_to_end(multitile):
    X, Q, ix_o, ix = multitile
    for mode in (0, 1):
        p = oracle.SearchParams(k=10, mode=mode, rho=0.01, alpha=0.5)
        ids = empty((Q.shape[0], 10), torch.int64)
        d2 = empty((Q.shape[0], 10), torch.float32)
        crisp.crisp_search(ix, dev(Q), Q.shape[0], crisp.search_params(k=10, mode=mode, rho=0.01, alpha=0.5), ids, d2)
        oi, od, _, _ = oracle.search(ix_o, Q, p)
        assert np.array_equal(ids.cpu().numpy(), oi) and np.array_equal(d2.cpu().numpy(), od)


def test_search_host_equals_device_and_chunking(c1, monkeypatch):
    X, Q, ix_o, ix = c1
    sp = crisp.search_params(k=10, mode=1, rho=0.02, alpha=0.25)
    ids = np.empty((100, 10), np.int64)
    d2 = np.empty((100, 10), np.float32)
    crisp.crisp_search_host(ix, Q, 100, sp, ids, d2)
    oi, od, _, _ = oracle.search(ix_o, Q, oracle.SearchParams(k=10, mode=1, rho=0.02, alpha=0.25))
    assert np.array_equal(ids, oi) and np.array_equal(d2, od)
    # a scratch budget of a few queries forces many internal chunks
    monkeypatch.setenv("CRISP_SCRATCH_MB", "1")
    ids2 = np.empty_like(ids)
    d22 = np.empty_like(d2)
    crisp.crisp_search_host(ix, Q, 100, sp, ids2, d22)
    assert np.array_equal(ids2, oi) and np.array_equal(d22, od)


def test_search_edge_cases():
    X, Q = synthetic.small_gaussian(300, 64, 5, seed=9)
    ix_o = oracle.build_index(X, M=2, K=8, draws=synthetic.method_draws(300, 64, 2, 8, seed=9, kmeans_train=300))
    ix = crisp.crisp_index_import(oracle.export_blob(ix_o))
    # nq = 0 is a no-op
    crisp.crisp_search(ix, dev(Q), 0, crisp.search_params(k=5), empty((1, 5), torch.int64), empty((1, 5), torch.float32))
    for kw in (dict(k=256, mode=0, rho=1.0, alpha=0.0), dict(k=256, mode=1, rho=0.1, alpha=1.0),
               dict(k=1, mode=0, rho=0.001, alpha=0.5), dict(k=300, mode=0, rho=0.5, alpha=0.0)):
        if kw["k"] > 256:
            with pytest.raises(crisp.CrispError):
                crisp.crisp_search(ix, dev(Q), 5, crisp.search_params(**kw), empty((5, 300), torch.int64),
                                   empty((5, 300), torch.float32))
            continue
        k = kw["k"]
        ids = empty((5, k), torch.int64)
        d2 = empty((5, k), torch.float32)
        crisp.crisp_search(ix, dev(Q), 5, crisp.search_params(**kw), ids, d2)
        oi, od, _, _ = oracle.search(ix_o, Q, oracle.SearchParams(**kw))
        assert np.array_equal(ids.cpu().numpy(), oi) and np.array_equal(d2.cpu().numpy(), od)
    # rho = 1, tau = 0: every point is verified -> exact kNN (textbook special case)
    gi, gd = oracle.knn_f64(X, Q, 10)
    ids = empty((5, 10), torch.int64)
    d2 = empty((5, 10), torch.float32)
    crisp.crisp_search(ix, dev(Q), 5, crisp.search_params(k=10, mode=0, rho=1.0, alpha=0.0), ids, d2)
    assert np.allclose(d2.cpu().numpy(), gd, rtol=1e-5)


@pytest.mark.parametrize("kw", [dict(k=0), dict(k=257), dict(mode=2), dict(rho=0.0), dict(rho=1.5), dict(alpha=-0.1),
                                dict(mode=1, verify_order=2),
                                dict(alpha=1.1), dict(k=10, max_candidates=5)])
def test_invalid_params_raise_and_write_nothing(c1, kw):
    X, Q, ix_o, ix = c1
    base = dict(k=10, mode=0, rho=0.01, alpha=0.3)
    base.update(kw)
    ids = torch.full((4, 300), -7, dtype=torch.int64, device=DEV)
    d2 = torch.full((4, 300), -7.0, dtype=torch.float32, device=DEV)
    with pytest.raises(crisp.CrispError) as e:
        crisp.crisp_search(ix, dev(Q[:4]), 4, crisp.search_params(**base), ids, d2)
    assert e.value.status == crisp.CRISP_EINVAL
    assert bool((ids == -7).all()) and bool((d2 == -7.0).all())


# ------------------------------------------------ large batches (grouped scoring)
@pytest.fixture(scope="module")
def c1_big():
    """The parity index with 1,100 queries of the same law: batches this large
    are scored in MinHash-ordered query groups (each row read once per group)."""
    X, Q = synthetic.gmm(nq=1100)
    ix_o = oracle.build_index(X, M=8, draws=synthetic.method_draws(20000, 256, 8, 50, seed=0)).add_copies()
    ix = crisp.crisp_index_import(oracle.export_blob(ix_o))
    crisp.crisp_index_add_copies(ix, 3)
    return X, Q, ix_o, ix


@pytest.mark.parametrize("kw", [dict(k=10, mode=0, rho=0.02, alpha=0.25),
                                dict(k=100, mode=0, rho=0.05, alpha=0.125),
                                dict(k=10, mode=0, rho=0.02, alpha=0.25, precision=1, shortlist=20),
                                dict(k=10, mode=0, rho=0.03, alpha=0.25, precision=2, shortlist=40)])
def test_large_batch_search_bitexact(c1_big, kw):
    X, Q, ix_o, ix = c1_big
    nq = Q.shape[0]
    ids = empty((nq, kw["k"]), torch.int64)
    d2 = empty((nq, kw["k"]), torch.float32)
    crisp.crisp_search(ix, dev(Q), nq, crisp.search_params(**kw), ids, d2)
    oi, od, _, _ = oracle.search(ix_o, Q, oracle.SearchParams(**kw))
    assert np.array_equal(ids.cpu().numpy(), oi)
    assert np.array_equal(d2.cpu().numpy(), od)


def test_large_batch_rerank_and_shortlist_steps(c1_big):
    X, Q, ix_o, ix = c1_big
    nq, M, K2 = Q.shape[0], ix_o.M, ix_o.K * ix_o.K
    Qr = gpu_qr(ix_o, ix, Q)
    act = empty((nq, M, K2), torch.int32)
    nact = empty((nq, M), torch.int32)
    crisp.crisp_activate(ix, Qr, nq, 0, 10, crisp.budget(0.03, ix_o.N), act, nact)
    stride = ix_o.N
    cand = empty((nq, stride), torch.int32)
    ncand = empty((nq,), torch.int64)
    crisp.crisp_count_cut(ix, act, nact, nq, crisp.tau(0.25, M), 10, 0, cand, stride, ncand)
    n = ncand.cpu().numpy()
    c = cand.cpu().numpy()
    ids = empty((nq, 10), torch.int64)
    d2 = empty((nq, 10), torch.float32)
    crisp.crisp_rerank(ix, Qr, nq, cand, stride, ncand, 10, ids, d2)
    sl = empty((nq, 64), torch.int32)
    nsl = empty((nq,), torch.int64)
    crisp.crisp_shortlist(ix, Qr, nq, cand, stride, ncand, 1, 30, sl, 64, nsl)
    sl8 = empty((nq, 64), torch.int32)
    nsl8 = empty((nq,), torch.int64)
    crisp.crisp_shortlist(ix, Qr, nq, cand, stride, ncand, 2, 45, sl8, 64, nsl8)
    gi, gd, gs, gns = ids.cpu().numpy(), d2.cpu().numpy(), sl.cpu().numpy(), nsl.cpu().numpy()
    gs8, gns8 = sl8.cpu().numpy(), nsl8.cpu().numpy()
    Xb = oracle.quantize_bf16(ix_o.Xr)
    for q in range(0, nq, 53):
        # the oracle's own rotated query and cut (the GPU's list must match it)
        dq = oracle.query_detail(ix_o, Q[q], oracle.SearchParams(k=10, mode=0, rho=0.03, alpha=0.25))
        assert np.array_equal(c[q, :n[q]], dq["C"]), q
        cq = dq["C"].astype(np.int64)
        ri, rd = oracle.rerank(ix_o, dq["qr"], cq, 10)
        assert np.array_equal(gi[q], ri) and np.array_equal(gd[q], rd), q
        ro = oracle.shortlist(ix_o, dq["qr"], cq, 30, "bf16", quant=Xb)
        assert gns[q] == len(ro) and np.array_equal(gs[q, :gns[q]], ro), q
        r8 = oracle.shortlist(ix_o, dq["qr"], cq, 45, "fp8", quant=(ix_o.X8, ix_o.S8))
        assert gns8[q] == len(r8) and np.array_equal(gs8[q, :gns8[q]], r8), q
