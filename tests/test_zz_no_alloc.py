"""crisp_rerank_noalloc: the re-rank for callers that cannot allocate device memory.

Some callers cannot allocate GPU memory while they search: another allocator
may own all of the device's memory, or their query path may not call
cudaMalloc/cudaFree, which can block and synchronise the device.  For them the
library offers crisp_rerank_noalloc, which keeps its distance scratch in a fixed
array of the library's own device memory instead of allocating it.

This test calls it through the C ABI twice in a row -- with different queries,
candidate lists and k, so that anything left in the shared array by the first
call would show -- and checks each result against crisp_rerank's, bit for bit
(the tolerance the parity tests use for the re-rank).  It builds everything it
needs itself, so it passes alone in a fresh process as well as after the rest
of the suite; the file name makes pytest collect it last.
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


def _candidates(ix_o, ix, Q, rho, alpha, k, stride=None, cap=0):
    """Rotated queries and their candidate lists from the library's own steps
    (at most `cap` candidates a query when cap > 0)."""
    nq, M, K2, Dp = Q.shape[0], ix_o.M, ix_o.K * ix_o.K, ix_o.Dp
    Qd = torch.from_numpy(Q).to(DEV)
    Qr = torch.empty((nq, Dp), dtype=torch.float32, device=DEV)
    crisp.crisp_rotate_rows(Qd, nq, ix_o.D, ix_o.D, torch.from_numpy(ix_o.R32).to(DEV), Qr, Dp)
    act = torch.empty((nq, M, K2), dtype=torch.int32, device=DEV)
    nact = torch.empty((nq, M), dtype=torch.int32, device=DEV)
    crisp.crisp_activate(ix, Qr, nq, 0, k, crisp.budget(rho, ix_o.N), act, nact)
    stride = stride or ix_o.N
    cand = torch.empty((nq, stride), dtype=torch.int32, device=DEV)
    ncand = torch.empty((nq,), dtype=torch.int64, device=DEV)
    crisp.crisp_count_cut(ix, act, nact, nq, crisp.tau(alpha, M), k, cap, cand, stride, ncand)
    return Qr, cand, stride, ncand


def test_rerank_noalloc_matches_rerank_on_two_calls_in_a_row():
    X, Q = synthetic.gmm(N=20000, D=256, nq=64, seed=2)
    ix_o = oracle.build_index(X, M=8, draws=synthetic.method_draws(20000, 256, 8, 50, seed=2))
    ix = crisp.crisp_index_import(oracle.export_blob(ix_o))
    calls = [(Q[:32], 0.02, 0.25, 10), (Q[32:], 0.04, 0.125, 25)]
    for Qc, rho, alpha, k in calls:
        Qr, cand, stride, ncand = _candidates(ix_o, ix, Qc, rho, alpha, k)
        nq = Qc.shape[0]
        assert nq * stride <= crisp.CRISP_RERANK_NOALLOC_MAX
        ref_i = torch.empty((nq, k), dtype=torch.int64, device=DEV)
        ref_d = torch.empty((nq, k), dtype=torch.float32, device=DEV)
        crisp.crisp_rerank(ix, Qr, nq, cand, stride, ncand, k, ref_i, ref_d)
        got_i = torch.full((nq, k), -7, dtype=torch.int64, device=DEV)
        got_d = torch.full((nq, k), -7.0, dtype=torch.float32, device=DEV)
        crisp.crisp_rerank_noalloc(ix, Qr, nq, cand, stride, ncand, k, got_i, got_d)
        torch.cuda.synchronize()
        assert torch.equal(got_i, ref_i)
        assert torch.equal(got_d, ref_d)
        assert int(ncand.min()) > 0 and bool((got_i[:, 0] >= 0).all())
    ix.free()


def test_rerank_noalloc_matches_the_grouped_rerank_of_a_large_batch():
    """1,024 queries with lists of up to 2,048 candidates: crisp_rerank scores
    this batch in query groups that share row reads, the no-allocation entry
    point streams every (query, candidate) pair; both must give the same bits,
    on two calls in a row."""
    X, Q = synthetic.gmm(N=20000, D=256, nq=2048, seed=4)
    ix_o = oracle.build_index(X, M=8, draws=synthetic.method_draws(20000, 256, 8, 50, seed=4))
    ix = crisp.crisp_index_import(oracle.export_blob(ix_o))
    stride = 2048
    for Qc, k in ((Q[:1024], 10), (Q[1024:], 30)):
        Qr, cand, _, ncand = _candidates(ix_o, ix, Qc, 0.05, 0.25, k, stride=stride, cap=stride)
        nq = Qc.shape[0]
        assert nq * stride <= crisp.CRISP_RERANK_NOALLOC_MAX
        assert int(ncand.max()) > 1024
        ref_i = torch.empty((nq, k), dtype=torch.int64, device=DEV)
        ref_d = torch.empty((nq, k), dtype=torch.float32, device=DEV)
        crisp.crisp_rerank(ix, Qr, nq, cand, stride, ncand, k, ref_i, ref_d)
        got_i = torch.full((nq, k), -7, dtype=torch.int64, device=DEV)
        got_d = torch.full((nq, k), -7.0, dtype=torch.float32, device=DEV)
        crisp.crisp_rerank_noalloc(ix, Qr, nq, cand, stride, ncand, k, got_i, got_d)
        torch.cuda.synchronize()
        assert torch.equal(got_i, ref_i)
        assert torch.equal(got_d, ref_d)
    ix.free()


def test_rerank_noalloc_rejects_sizes_beyond_its_scratch():
    X, Q = synthetic.small_gaussian(300, 64, 4, seed=9)
    ix_o = oracle.build_index(X, M=2, K=8, draws=synthetic.method_draws(300, 64, 2, 8, seed=9, kmeans_train=300))
    ix = crisp.crisp_index_import(oracle.export_blob(ix_o))
    too_wide = crisp.CRISP_RERANK_NOALLOC_MAX // 4 + 1
    ids = torch.full((4, 5), -7, dtype=torch.int64, device=DEV)
    d2 = torch.full((4, 5), -7.0, dtype=torch.float32, device=DEV)
    dummy = torch.zeros((4, 1), dtype=torch.int32, device=DEV)
    with pytest.raises(crisp.CrispError) as e:
        crisp.crisp_rerank_noalloc(ix, torch.zeros((4, 64), device=DEV), 4, dummy, too_wide,
                                   torch.zeros(4, dtype=torch.int64, device=DEV), 5, ids, d2)
    assert e.value.status == crisp.CRISP_EINVAL
    assert "exceeds the fixed scratch" in str(e.value)
    assert bool((ids == -7).all()) and bool((d2 == -7.0).all())
    # a stride so large that nq * stride would wrap a 64-bit integer
    with pytest.raises(crisp.CrispError) as e:
        crisp.crisp_rerank_noalloc(ix, torch.zeros((4, 64), device=DEV), 4, dummy, (1 << 62) + 1,
                                   torch.zeros(4, dtype=torch.int64, device=DEV), 5, ids, d2)
    assert e.value.status == crisp.CRISP_EINVAL
    assert bool((ids == -7).all()) and bool((d2 == -7.0).all())
    ix.free()
