"""The continuous-batching server: requests with mixed k and modes, submitted
from several threads while earlier batches are on the GPU, must each return
exactly what a search of that query alone returns; batching and stream overlap
must actually happen; the scratch budget must throttle admission without
deadlock."""
import threading

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


@pytest.fixture(scope="module")
def served():
    X, Q = synthetic.gmm(N=20000, D=256, nq=240, seed=21)
    ix_o = oracle.build_index(X, M=8, draws=synthetic.method_draws(20000, 256, 8, 50, seed=21))
    ix = crisp.crisp_index_import(oracle.export_blob(ix_o))
    crisp.crisp_index_add_copies(ix, 1)
    F, H = 2 * 8 + 68, 64
    P = synthetic.mlp_weights(F, H, 2, seed=5)
    P[-2:] += np.float32(7.0)
    crisp.crisp_index_set_model(ix, torch.from_numpy(P).to(DEV), H)
    return X, Q, ix


def _params(i):
    k = (1, 10, 100)[i % 3]
    mode = (0, 1, 1, 2, 2)[i % 5]
    return crisp.search_params(k=k, mode=mode, rho=0.02, alpha=0.25, max_candidates=4000 if mode == 1 else 0)


def _alone(ix, q, p):
    ids = torch.empty((1, p.k), dtype=torch.int64, device=DEV)
    d2 = torch.empty((1, p.k), dtype=torch.float32, device=DEV)
    crisp.crisp_search(ix, torch.from_numpy(q[None, :].copy()).to(DEV), 1, p, ids, d2)
    torch.cuda.synchronize()
    return ids.cpu().numpy()[0], d2.cpu().numpy()[0]


def test_results_same_alone_and_in_the_mix(served):
    X, Q, ix = served
    sv = crisp.crisp_server_create(ix, streams=3, max_batch=32)
    tickets = {}
    lock = threading.Lock()

    def submitter(part):
        for i in range(part, Q.shape[0], 4):
            t = crisp.crisp_server_submit(sv, np.ascontiguousarray(Q[i]), _params(i))
            with lock:
                tickets[i] = t

    th = [threading.Thread(target=submitter, args=(j,)) for j in range(4)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    got = {}
    for i, t in tickets.items():
        got[i] = crisp.crisp_server_wait(sv, t, _params(i).k, timeout_ms=60000)
    st = crisp.crisp_server_get_stats(sv)
    sv.free()
    assert st.completed == Q.shape[0] and st.failed == 0
    assert st.batches < Q.shape[0] and st.mean_batch > 1.0        # requests were batched
    assert 0 < st.p50_us <= st.p99_us <= st.max_us
    for i in range(Q.shape[0]):
        ids, d2 = _alone(ix, Q[i], _params(i))
        assert np.array_equal(got[i][0], ids) and np.array_equal(got[i][1], d2), i


def test_scratch_budget_throttles_without_deadlock(served):
    X, Q, ix = served
    p = crisp.search_params(k=10, mode=0, rho=0.05, alpha=0.25)
    one = crisp.crisp_search_scratch_bytes(ix, 8, p)
    sv = crisp.crisp_server_create(ix, streams=4, max_batch=8, scratch_budget=one)   # one batch in flight
    ts = [crisp.crisp_server_submit(sv, np.ascontiguousarray(Q[i]), p) for i in range(64)]
    res = [crisp.crisp_server_wait(sv, t, 10, timeout_ms=60000) for t in ts]
    st = crisp.crisp_server_get_stats(sv)
    sv.free()
    assert st.completed == 64 and st.scratch_peak <= one
    for i in (0, 17, 63):
        ids, d2 = _alone(ix, Q[i], p)
        assert np.array_equal(res[i][0], ids)


def test_submit_validates_and_wait_times_out(served):
    X, Q, ix = served
    sv = crisp.crisp_server_create(ix, streams=1, max_batch=4)
    with pytest.raises(crisp.CrispError) as e:
        crisp.crisp_server_submit(sv, np.ascontiguousarray(Q[0]), crisp.search_params(k=0))
    assert e.value.status == crisp.CRISP_EINVAL
    t = crisp.crisp_server_submit(sv, np.ascontiguousarray(Q[0]), crisp.search_params(k=5, rho=0.02, alpha=0.25))
    ids, d2, lat = crisp.crisp_server_wait(sv, t, 5, timeout_ms=60000)
    assert lat > 0 and ids[0] >= 0
    with pytest.raises(crisp.CrispError):
        crisp.crisp_server_wait(sv, t, 5, timeout_ms=10)        # consumed ticket
    sv.free()


def test_replay_open_loop_matches_alone(served):
    """A Poisson trace (20k requests/s offered) of mixed k and modes through the
    native replay: every result equals the query searched alone, latencies are
    finite and counted from the scheduled arrivals."""
    X, Q, ix = served
    n = 400
    r = np.random.default_rng(3)
    arrival = np.cumsum(r.exponential(1e6 / 20000.0, n))
    params = [_params(i) for i in range(15)]
    pidx = r.integers(0, 15, n).astype(np.int32)
    qidx = r.integers(0, Q.shape[0], n).astype(np.int32)
    sv = crisp.crisp_server_create(ix, streams=4, max_batch=64)
    ids, d2, lat, wall = crisp.crisp_server_replay(sv, Q, qidx, params, pidx, arrival, 100)
    st = crisp.crisp_server_get_stats(sv)
    sv.free()
    assert st.completed == n and st.failed == 0
    assert np.all(np.isfinite(lat)) and np.all(lat > 0) and wall >= arrival[-1]
    for i in range(0, n, 7):
        p = params[pidx[i]]
        a_ids, a_d2 = _alone(ix, Q[qidx[i]], p)
        assert np.array_equal(ids[i, :p.k], a_ids) and np.array_equal(d2[i, :p.k], a_d2), i
        assert np.all(ids[i, p.k:] == -1)


def test_replay_rejects_bad_traces(served):
    X, Q, ix = served
    sv = crisp.crisp_server_create(ix, streams=1, max_batch=4)
    p = [crisp.search_params(k=10, rho=0.02, alpha=0.25)]
    with pytest.raises(crisp.CrispError):          # unsorted arrivals
        crisp.crisp_server_replay(sv, Q, [0, 1], p, [0, 0], [5.0, 1.0], 10)
    with pytest.raises(crisp.CrispError):          # query index out of range
        crisp.crisp_server_replay(sv, Q, [Q.shape[0]], p, [0], [0.0], 10)
    with pytest.raises(crisp.CrispError):          # k > kmax
        crisp.crisp_server_replay(sv, Q, [0], p, [0], [0.0], 5)
    with pytest.raises(crisp.CrispError):          # parameter index out of range
        crisp.crisp_server_replay(sv, Q, [0], p, [1], [0.0], 10)
    st = crisp.crisp_server_get_stats(sv)
    sv.free()
    assert st.submitted == 0
