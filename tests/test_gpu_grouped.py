"""Grouped scoring (large batches) against the oracle at the shapes the scorers
treat specially: D = 1024 (every 128-dim chunk of the FP32 warp layout and all
32 blocks in use), D = 100 and D = 33 (padded to 128 and 64, so the last blocks
and chunks are padding), D = 96 (a BF16 row ends halfway through its last
128-byte k-block of the tensor-core re-rank), and batch sizes that leave a
partial last query group (64 queries per tensor-core group, 16 / 32 per group
of the FP32 / BF16 shortlist scorers).

The oracle builds the index and the GPU searches the imported blob.  For every
sampled query the GPU's candidate list must equal the oracle's cut, and the
GPU's re-rank and shortlists (computed on the GPU's lists) must equal the
oracle's results on the oracle's own rotated query and cut, bit for bit.  No
input or expected value here comes from the GPU side.
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


@pytest.fixture(scope="module", params=[(6000, 1024, 1100, 4), (5000, 100, 1030, 5), (3000, 33, 1531, 3),
                                        (4000, 96, 600, 4)],
                ids=["D1024", "D100", "D33", "D96"])
def grouped_case(request):
    N, D, nq, M = request.param
    X, Q = synthetic.gmm(N=N, D=D, nq=nq, n_comp=30, rank=min(16, D), seed=D)
    ix_o = oracle.build_index(X, M=M, draws=synthetic.method_draws(N, D, M, 50, seed=D)).add_copies()
    ix = crisp.crisp_index_import(oracle.export_blob(ix_o))
    crisp.crisp_index_add_copies(ix, 3)
    return X, Q, ix_o, ix


def _candidates(ix_o, ix, Q, rho, alpha, k):
    nq, M, K2, Dp = Q.shape[0], ix_o.M, ix_o.K * ix_o.K, ix_o.Dp
    Qr = empty((nq, Dp), torch.float32)
    if ix_o.rotated:
        crisp.crisp_rotate_rows(dev(Q), nq, ix_o.D, ix_o.D, dev(ix_o.R32), Qr, Dp)
    else:
        Qr.zero_()
        Qr[:, :ix_o.D] = dev(Q.astype(np.float32))
    act = empty((nq, M, K2), torch.int32)
    nact = empty((nq, M), torch.int32)
    crisp.crisp_activate(ix, Qr, nq, 0, k, crisp.budget(rho, ix_o.N), act, nact)
    cand = empty((nq, ix_o.N), torch.int32)
    ncand = empty((nq,), torch.int64)
    crisp.crisp_count_cut(ix, act, nact, nq, crisp.tau(alpha, M), k, 0, cand, ix_o.N, ncand)
    return Qr, cand, ncand


def _oracle_cut(ix_o, Q, q, rho, alpha, k, cand, ncand):
    """The oracle's rotated query and cut for query q; the GPU's list must match."""
    d = oracle.query_detail(ix_o, Q[q], oracle.SearchParams(k=k, mode=0, rho=rho, alpha=alpha))
    assert np.array_equal(cand[q, :ncand[q]], d["C"]), q
    return d["qr"], d["C"]


def _sample(nq, step):
    # every query of the first and last groups, and a sample in between
    return sorted(set(range(32)) | set(range(nq - 40, nq)) | set(range(0, nq, step)))


@pytest.mark.parametrize("k", [10, 100])
@pytest.mark.parametrize("scorer", ["bf16", "tf32"])
def test_grouped_rerank_bitexact(grouped_case, k, scorer, monkeypatch):
    """The index keeps its BF16 copy, so the tensor-core bounds come from one
    BF16 pass over it; CRISP_RERANK_TF32=1 takes one TF32 pass over the FP32
    rows instead.  Either way every returned distance is exact (CR32)."""
    if scorer == "tf32":
        monkeypatch.setenv("CRISP_RERANK_TF32", "1")
    X, Q, ix_o, ix = grouped_case
    nq = Q.shape[0]
    Qr, cand, ncand = _candidates(ix_o, ix, Q, 0.05, 0.3, k)
    ids = empty((nq, k), torch.int64)
    d2 = empty((nq, k), torch.float32)
    crisp.crisp_rerank(ix, Qr, nq, cand, ix_o.N, ncand, k, ids, d2)
    gi, gd = ids.cpu().numpy(), d2.cpu().numpy()
    c, n = cand.cpu().numpy(), ncand.cpu().numpy()
    assert n.min() > 0
    for q in _sample(nq, 37):
        qr, C = _oracle_cut(ix_o, Q, q, 0.05, 0.3, k, c, n)
        ri, rd = oracle.rerank(ix_o, qr, C, k)
        assert np.array_equal(gi[q], ri) and np.array_equal(gd[q], rd), q


@pytest.mark.parametrize("precision,S", [(1, 40), (2, 60), (1, 300)])
def test_grouped_shortlist_bitexact(grouped_case, precision, S):
    X, Q, ix_o, ix = grouped_case
    nq = Q.shape[0]
    Qr, cand, ncand = _candidates(ix_o, ix, Q, 0.05, 0.3, 10)
    out = empty((nq, S), torch.int32)
    nout = empty((nq,), torch.int64)
    crisp.crisp_shortlist(ix, Qr, nq, cand, ix_o.N, ncand, precision, S, out, S, nout)
    go, gn = out.cpu().numpy(), nout.cpu().numpy()
    c, n = cand.cpu().numpy(), ncand.cpu().numpy()
    quant = ix_o.Xb if precision == 1 else (ix_o.X8, ix_o.S8)
    for q in _sample(nq, 41):
        qr, C = _oracle_cut(ix_o, Q, q, 0.05, 0.3, 10, c, n)
        ref = oracle.shortlist(ix_o, qr, C, S, "bf16" if precision == 1 else "fp8", quant)
        assert gn[q] == ref.size and np.array_equal(go[q, :gn[q]], ref), q


def test_duplicate_rows_select_by_id():
    """4,000 copies of one row among 2,000 others, 300 queries near it: every
    copy is a candidate at the same distance, so the selection's 16-bit bin
    holds more keys than its shared-memory buffer (the four-pass path), and
    the top-k among equal distances must be the lowest ids, as in the oracle."""
    r = np.random.default_rng(17)
    N, D, nq, M = 6000, 64, 300, 4
    X = r.standard_normal((N, D)).astype(np.float32)
    v = r.standard_normal(D).astype(np.float32)
    dup = np.sort(r.choice(N, 4000, replace=False))
    X[dup] = v
    Q = (v[None, :] + 0.01 * r.standard_normal((nq, D))).astype(np.float32)
    ix_o = oracle.build_index(X, M=M, K=16, draws=synthetic.method_draws(N, D, M, 16, seed=17, kmeans_train=N))
    ix = crisp.crisp_index_import(oracle.export_blob(ix_o))
    crisp.crisp_index_add_copies(ix, 1)
    for kw in (dict(k=10, mode=0, rho=0.5, alpha=0.5), dict(k=100, mode=0, rho=0.5, alpha=0.25)):
        k = kw["k"]
        ids = empty((nq, k), torch.int64)
        d2 = empty((nq, k), torch.float32)
        crisp.crisp_search(ix, dev(Q), nq, crisp.search_params(**kw), ids, d2)
        oi, od, _, _ = oracle.search(ix_o, Q, oracle.SearchParams(**kw))
        assert np.array_equal(ids.cpu().numpy(), oi) and np.array_equal(d2.cpu().numpy(), od)
        assert np.all(np.isin(oi[:, 0], dup))
