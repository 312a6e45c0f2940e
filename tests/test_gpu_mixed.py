"""One crisp_search call with a parameter set per query (p_count = nq): every
query may have its own k, mode (Guaranteed, Optimized, Learned), precision,
coverage, threshold and verification settings.  Each row must equal the same
query searched alone with its own parameters, and the oracle, bit for bit; rows
are padded -1 / +inf past the query's k up to kmax.  Batches large enough for the
tensor-core re-rank keep that path for their Guaranteed queries.  No input or
expected value comes from the GPU side."""
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
def ix_mixed():
    X, Q = synthetic.gmm(N=20000, D=256, nq=1200, seed=13)
    ix_o = oracle.build_index(X, M=8, draws=synthetic.method_draws(20000, 256, 8, 50, seed=13)).add_copies()
    F, H = 2 * 8 + 68, 64
    P = synthetic.mlp_weights(F, H, 2, seed=14)
    P[-2:] += np.float32(6.0)
    ix_o.set_model(P, H)
    ix = crisp.crisp_index_import(oracle.export_blob(ix_o))
    crisp.crisp_index_add_copies(ix, 3)
    crisp.crisp_index_set_model(ix, dev(P), H)
    yield X, Q, ix_o, ix
    ix.free()


# a menu of parameter sets covering every stage-3 class and per-query value
MENU = [
    dict(k=10, mode=0, rho=0.02, alpha=0.25),
    dict(k=1, mode=0, rho=0.01, alpha=0.5),
    dict(k=100, mode=0, rho=0.05, alpha=0.125),
    dict(k=37, mode=0, rho=0.03, alpha=0.25, max_candidates=300),
    dict(k=10, mode=1, rho=0.03, alpha=0.25),
    dict(k=20, mode=1, rho=0.02, alpha=0.375, eps0=0.5, patience_factor=10),
    dict(k=10, mode=1, rho=0.03, alpha=0.25, verify_order=1),
    dict(k=10, mode=0, rho=0.02, alpha=0.25, precision=1, shortlist=30),
    dict(k=5, mode=0, rho=0.03, alpha=0.25, precision=2, shortlist=45),
    dict(k=10, mode=2, rho=0.02, alpha=0.25, depth_margin=0.5, short_margin=0.25),
    dict(k=3, mode=0, rho=0.002, alpha=1.0),
]


def _alone(ix, q, kw):
    k = kw["k"]
    ids = torch.empty((1, k), dtype=torch.int64, device=DEV)
    d2 = torch.empty((1, k), dtype=torch.float32, device=DEV)
    crisp.crisp_search(ix, dev(q[None]), 1, crisp.search_params(**kw), ids, d2)
    return ids.cpu().numpy()[0], d2.cpu().numpy()[0]


def test_mixed_batch_equals_alone_and_oracle(ix_mixed):
    X, Q, ix_o, ix = ix_mixed
    nq = 110
    pick = np.random.default_rng(3).integers(0, len(MENU), nq)
    kws = [MENU[i] for i in pick]
    kmax = 128
    ids = torch.full((nq, kmax), -7, dtype=torch.int64, device=DEV)
    d2 = torch.full((nq, kmax), -7.0, dtype=torch.float32, device=DEV)
    st = torch.empty((nq, 6), dtype=torch.int64, device=DEV)
    crisp.crisp_search(ix, dev(Q[:nq]), nq, [crisp.search_params(**kw) for kw in kws], ids, d2, st)
    ids, d2, st = ids.cpu().numpy(), d2.cpu().numpy(), st.cpu().numpy()
    for i, kw in enumerate(kws):
        k = kw["k"]
        assert np.all(ids[i, k:] == -1) and np.all(np.isinf(d2[i, k:])), i
        ai, ad = _alone(ix, Q[i], kw)
        assert np.array_equal(ids[i, :k], ai) and np.array_equal(d2[i, :k], ad), (i, kw)
        oi, od, ost, _ = oracle.search(ix_o, Q[i:i + 1], oracle.SearchParams(**kw))
        assert np.array_equal(ids[i, :k], oi[0]) and np.array_equal(d2[i, :k], od[0]), (i, kw)
        assert st[i, 0] == ost["n_candidates"][0] and st[i, 1] == ost["n_verified"][0], (i, kw)
        assert st[i, 2] == ost["n_full"][0] and st[i, 3] == ost["n_retrieved"][0], (i, kw)


def test_per_query_array_of_one_class_equals_shared(ix_mixed):
    """p_count = nq with the same set everywhere gives the shared call's bits."""
    X, Q, ix_o, ix = ix_mixed
    nq = 64
    kw = dict(k=10, mode=1, rho=0.03, alpha=0.25)
    a_i = torch.empty((nq, 10), dtype=torch.int64, device=DEV)
    a_d = torch.empty((nq, 10), dtype=torch.float32, device=DEV)
    b_i, b_d = torch.empty_like(a_i), torch.empty_like(a_d)
    crisp.crisp_search(ix, dev(Q[:nq]), nq, crisp.search_params(**kw), a_i, a_d)
    crisp.crisp_search(ix, dev(Q[:nq]), nq, [crisp.search_params(**kw)] * nq, b_i, b_d)
    assert torch.equal(a_i, b_i) and torch.equal(a_d, b_d)


def test_large_mixed_batch(ix_mixed):
    """1,200 queries, most of them Guaranteed with FP32 re-rank (a class segment
    of more than 1,024 queries takes the tensor-core path) and varied k, the
    rest in the other classes; sampled rows against the oracle."""
    X, Q, ix_o, ix = ix_mixed
    nq = Q.shape[0]
    r = np.random.default_rng(5)
    kws = []
    for i in range(nq):
        if i % 12 == 0:
            kws.append(MENU[4 + (i // 12) % 7])
        else:
            kws.append(dict(k=int(r.choice([1, 10, 50, 100])), mode=0, rho=0.03, alpha=0.25))
    kmax = 100
    ids = torch.empty((nq, kmax), dtype=torch.int64, device=DEV)
    d2 = torch.empty((nq, kmax), dtype=torch.float32, device=DEV)
    crisp.crisp_search(ix, dev(Q), nq, [crisp.search_params(**kw) for kw in kws], ids, d2)
    ids, d2 = ids.cpu().numpy(), d2.cpu().numpy()
    for i in list(range(0, nq, 29)) + [j for j in range(0, nq, 12)][:25]:
        kw = kws[i]
        k = kw["k"]
        oi, od, _, _ = oracle.search(ix_o, Q[i:i + 1], oracle.SearchParams(**kw))
        assert np.array_equal(ids[i, :k], oi[0]) and np.array_equal(d2[i, :k], od[0]), (i, kw)
        assert np.all(ids[i, k:] == -1), i


def test_per_query_argument_errors(ix_mixed):
    X, Q, ix_o, ix = ix_mixed
    ids = torch.full((4, 16), -7, dtype=torch.int64, device=DEV)
    d2 = torch.full((4, 16), -7.0, dtype=torch.float32, device=DEV)
    ps = [crisp.search_params(k=10)] * 3
    with pytest.raises(crisp.CrispError) as e:                # p_count neither 1 nor nq
        crisp.crisp_search(ix, dev(Q[:4]), 4, ps, ids, d2)
    assert e.value.status == crisp.CRISP_EINVAL
    with pytest.raises(crisp.CrispError) as e:                # kmax below a query's k
        crisp.crisp_search(ix, dev(Q[:4]), 4, [crisp.search_params(k=10)] * 3 + [crisp.search_params(k=20)],
                           ids, d2)
    assert e.value.status == crisp.CRISP_EINVAL
    with pytest.raises(crisp.CrispError) as e:                # one invalid set among valid ones
        crisp.crisp_search(ix, dev(Q[:4]), 4, [crisp.search_params(k=10)] * 3 + [crisp.search_params(rho=0.0)],
                           ids, d2)
    assert e.value.status == crisp.CRISP_EINVAL
    assert bool((ids == -7).all()) and bool((d2 == -7.0).all())
