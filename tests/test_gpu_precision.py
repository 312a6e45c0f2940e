"""GPU vs oracle parity of the low-precision coarse scoring (BF16 / FP8 E4M3
row copies, coarse-score shortlist, FP32 re-rank of the shortlist).

The quantised copies are compared bit for bit (codes and per-row scales), the
shortlists as exact id lists, and whole searches as exact ids and FP32
distances, on an index and copies the oracle built."""
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
def c1q():
    X, Q = synthetic.gmm(N=20000, D=256, nq=60, seed=6)
    ix_o = oracle.build_index(X, M=8, draws=synthetic.method_draws(20000, 256, 8, 50, seed=6)).add_copies()
    ix = crisp.crisp_index_import(oracle.export_blob(ix_o))
    crisp.crisp_index_add_copies(ix, 3)
    return X, Q, ix_o, ix


def test_quantised_copies_bitexact(c1q):
    X, Q, ix_o, ix = c1q
    info = ix.info()
    assert info.Xb and info.X8 and info.S8
    N, Dp = ix_o.N, ix_o.Dp
    Xb = torch.empty((N, Dp), dtype=torch.int16, device=DEV)
    X8 = torch.empty((N, Dp), dtype=torch.uint8, device=DEV)
    S8 = torch.empty((N,), dtype=torch.float32, device=DEV)
    Xr = dev(ix_o.Xr)
    crisp.crisp_quantize_bf16(Xr, N, Dp, Xb)
    crisp.crisp_quantize_e4m3(Xr, N, Dp, X8, S8)
    assert np.array_equal(Xb.cpu().numpy().view(np.uint16), ix_o.Xb)
    assert np.array_equal(X8.cpu().numpy(), ix_o.X8)
    assert np.array_equal(S8.cpu().numpy(), ix_o.S8)
    # the index's own copies (crisp_index_add_copies) feed the shortlist tests below


def _cands(ix_o, ix, Q, rho, alpha, k):
    nq, M, K2, Dp = Q.shape[0], ix_o.M, ix_o.K * ix_o.K, ix_o.Dp
    Qr = torch.empty((nq, Dp), dtype=torch.float32, device=DEV)
    crisp.crisp_rotate_rows(dev(Q), nq, ix_o.D, ix_o.D, dev(ix_o.R32), Qr, Dp)
    act = torch.empty((nq, M, K2), dtype=torch.int32, device=DEV)
    nact = torch.empty((nq, M), dtype=torch.int32, device=DEV)
    crisp.crisp_activate(ix, Qr, nq, 0, k, crisp.budget(rho, ix_o.N), act, nact)
    cand = torch.empty((nq, ix_o.N), dtype=torch.int32, device=DEV)
    ncand = torch.empty((nq,), dtype=torch.int64, device=DEV)
    crisp.crisp_count_cut(ix, act, nact, nq, crisp.tau(alpha, M), k, 0, cand, ix_o.N, ncand)
    return Qr, cand, ncand


@pytest.mark.parametrize("precision,S", [(1, 10), (1, 100), (1, 5000), (2, 10), (2, 250), (2, 20000)])
def test_shortlist_bitexact(c1q, precision, S):
    X, Q, ix_o, ix = c1q
    Qr, cand, ncand = _cands(ix_o, ix, Q, 0.02, 0.25, 10)
    nq = Q.shape[0]
    out = torch.empty((nq, S), dtype=torch.int32, device=DEV)
    nout = torch.empty((nq,), dtype=torch.int64, device=DEV)
    crisp.crisp_shortlist(ix, Qr, nq, cand, ix_o.N, ncand, precision, S, out, S, nout)
    out, nout, cand, ncand = out.cpu().numpy(), nout.cpu().numpy(), cand.cpu().numpy(), ncand.cpu().numpy()
    quant = ix_o.Xb if precision == 1 else (ix_o.X8, ix_o.S8)
    p = oracle.SearchParams(k=10, mode=0, rho=0.02, alpha=0.25)
    for i in range(nq):
        # the oracle's own rotated query and cut (the GPU's list must match it)
        det = oracle.query_detail(ix_o, Q[i], p)
        assert np.array_equal(cand[i, :ncand[i]], det["C"]), i
        ref = oracle.shortlist(ix_o, det["qr"], det["C"], S, "bf16" if precision == 1 else "fp8", quant)
        assert nout[i] == ref.size and np.array_equal(out[i, :nout[i]], ref), i


@pytest.mark.parametrize("precision,S,k", [(1, 64, 10), (1, 400, 10), (2, 64, 10), (2, 1000, 100), (1, 10, 10)])
def test_search_with_coarse_scoring_bitexact(c1q, precision, S, k):
    X, Q, ix_o, ix = c1q
    kw = dict(k=k, mode=0, rho=0.03, alpha=0.25, precision=precision, shortlist=S)
    nq = Q.shape[0]
    ids = torch.empty((nq, k), dtype=torch.int64, device=DEV)
    d2 = torch.empty((nq, k), dtype=torch.float32, device=DEV)
    st = torch.empty((nq, 6), dtype=torch.int64, device=DEV)
    crisp.crisp_search(ix, dev(Q), nq, crisp.search_params(**kw), ids, d2, st)
    oi, od, ost, _ = oracle.search(ix_o, Q, oracle.SearchParams(**kw))
    assert np.array_equal(ids.cpu().numpy(), oi) and np.array_equal(d2.cpu().numpy(), od)
    s = st.cpu().numpy()
    assert np.array_equal(s[:, 0], ost["n_candidates"]) and np.array_equal(s[:, 2], ost["n_full"])


@pytest.mark.parametrize("kw", [dict(precision=3, shortlist=50), dict(precision=1, shortlist=5),
                                dict(precision=1, shortlist=50, mode=1)])
def test_coarse_scoring_argument_errors(c1q, kw):
    X, Q, ix_o, ix = c1q
    base = dict(k=10, mode=0, rho=0.03, alpha=0.25)
    base.update(kw)
    ids = torch.empty((4, 10), dtype=torch.int64, device=DEV)
    d2 = torch.empty((4, 10), dtype=torch.float32, device=DEV)
    with pytest.raises(crisp.CrispError) as e:
        crisp.crisp_search(ix, dev(Q[:4]), 4, crisp.search_params(**base), ids, d2)
    assert e.value.status == crisp.CRISP_EINVAL


def test_coarse_scoring_needs_the_copy():
    X, Q = synthetic.small_gaussian(300, 64, 4, seed=9)
    ix_o = oracle.build_index(X, M=2, K=8, draws=synthetic.method_draws(300, 64, 2, 8, seed=9, kmeans_train=300))
    ix = crisp.crisp_index_import(oracle.export_blob(ix_o))
    ids = torch.empty((4, 5), dtype=torch.int64, device=DEV)
    d2 = torch.empty((4, 5), dtype=torch.float32, device=DEV)
    with pytest.raises(crisp.CrispError) as e:
        crisp.crisp_search(ix, dev(Q), 4, crisp.search_params(k=5, precision=2, shortlist=20), ids, d2)
    assert "FP8 copy" in str(e.value)
