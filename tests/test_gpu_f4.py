"""The §7 build extensions on the GPU against the oracle: variance-aware
subspace boundaries and block-wise rotation.

Integer results (boundaries, cells given the centroids, search ids on an
imported index) must be identical; FP64 statistics within their rounding; the
block rotation of the rows (tensor cores, 3xTF32) within the two products'
error bounds (w 2^-24 |x_B| for the oracle's FP32 chain of w terms, 4e-6 |x_B|
for the split product), with every column outside the rotated blocks copied
exactly.  The oracle's inputs never come from the GPU side."""
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
def mixed():
    """Skewed mixed workload: a 48-dim correlated block beside 208 independent
    dims with standard deviations from 8 down to 1; N = 20,000, D = 256, M = 8."""
    N, D, M, K = 20000, 256, 8, 50
    X, Q = synthetic.mixed(N, D, 64, corr_dims=48, rank=4, skew=8.0, seed=11)
    draws = synthetic.method_draws(N, D, M, K, seed=11, kmeans_train=20000)
    return X, Q, draws, N, D, M, K


def test_column_variance_equals_the_oracle(mixed):
    X, Q, draws, N, D, M, K = mixed
    var = empty((D,), torch.float64)
    crisp.crisp_column_variance(dev(X), N, D, D, dev(draws.cev_sample), draws.cev_sample.size, var)
    ref = oracle.column_variance(X, draws.cev_sample)
    assert np.allclose(var.cpu().numpy(), ref, rtol=1e-12, atol=0)


def test_assign_cells_with_boundaries_bitexact(mixed):
    X, Q, draws, N, D, M, K = mixed
    ix_o = oracle.build_index(X, M, K, draws=draws, rotate=0, adaptive=1)
    assert not np.array_equal(ix_o.sub, oracle.equal_bounds(D, M))
    for fn in (crisp.crisp_assign_cells, crisp.crisp_assign_cells_tc):
        cells = empty((M, N), torch.int16)
        fn(dev(ix_o.Xr), N, D, ix_o.Dp, M, K, ix_o.H, dev(ix_o.cent), cells, sub=ix_o.sub)
        assert np.array_equal(cells.cpu().numpy().view(np.uint16), ix_o.cells), fn.__name__


@pytest.mark.parametrize("mode", [0, 1])
def test_adaptive_index_search_bitexact(mixed, mode):
    """An oracle index with variance-aware boundaries, imported (blob version
    2): every search step reads the boundaries, and the results are the oracle's."""
    X, Q, draws, N, D, M, K = mixed
    ix_o = oracle.build_index(X, M, K, draws=draws, rotate=0, adaptive=1)
    blob = oracle.export_blob(ix_o)
    ix = crisp.crisp_index_import(blob)
    assert crisp.crisp_index_export(ix) == blob
    info = ix.info()
    nq, k = Q.shape[0], 10
    kw = dict(k=k, mode=mode, rho=0.05, alpha=0.25)
    ids = empty((nq, k), torch.int64)
    d2 = empty((nq, k), torch.float32)
    crisp.crisp_search(ix, dev(Q), nq, crisp.search_params(**kw), ids, d2)
    oi, od, _, _ = oracle.search(ix_o, Q, oracle.SearchParams(**kw))
    assert np.array_equal(ids.cpu().numpy(), oi) and np.array_equal(d2.cpu().numpy(), od)
    assert info.H == ix_o.H


def test_build_adaptive_equals_the_oracle(mixed):
    X, Q, draws, N, D, M, K = mixed
    ix_o = oracle.build_index(X, M, K, draws=draws, rotate=0, adaptive=1)
    ix = crisp.crisp_build(dev(X), N, D, crisp.build_params(M, K, rotate=0, draws=draws, adaptive=1))
    blob = crisp.crisp_index_export(ix)
    v = np.frombuffer(blob, np.int64, 1, 8)[0]
    assert v == 2
    info = ix.info()
    assert info.H == ix_o.H
    sub = np.frombuffer(blob[-((4 * (M + 1) + 255) // 256 * 256):], np.int32, M + 1)
    assert np.array_equal(sub, ix_o.sub) and np.array_equal(crisp.crisp_index_get_bounds(ix), ix_o.sub)
    assert info.sub
    # the stored rows are the padded input; cells from the same rows and boundaries
    # are checked bit-exact above, so here the build's own invariants: recall
    gi, gd = oracle.knn_f64(X, Q, 10)
    kw = dict(k=10, rho=0.05, alpha=0.25)
    ids = empty((Q.shape[0], 10), torch.int64)
    d2 = empty((Q.shape[0], 10), torch.float32)
    crisp.crisp_search(ix, dev(Q), Q.shape[0], crisp.search_params(**kw), ids, d2)
    r_gpu = oracle.recall_at_k(ids.cpu().numpy(), gd, X, Q, 10)
    r_orc = oracle.recall_at_k(oracle.search(ix_o, Q, oracle.SearchParams(**kw))[0], gd, X, Q, 10)
    assert r_gpu >= r_orc - 0.03


@pytest.mark.parametrize("block_dims,rotate", [(48, -1), (64, 1), (100, 1)])
def test_build_block_rotation_against_the_oracle(mixed, block_dims, rotate):
    """Blocks of 48 (the test picks the correlated block alone; the last block
    of 16 dims ragged), 64 (every block, rotate = 1) and 100 (every block, the
    last one of 56 dims ragged and not a multiple of 32)."""
    X, Q, draws, N, D, M, K = mixed
    ix_o = oracle.build_index(X, M, K, draws=draws, rotate=rotate, block_dims=block_dims)
    ix = crisp.crisp_build(dev(X), N, D, crisp.build_params(M, K, rotate=rotate, draws=draws, block_dims=block_dims))
    info = ix.info()
    n_rot = sum(b[3] for b in ix_o.blocks)
    assert info.rotated == ix_o.rotated and info.rotated_blocks == n_rot and n_rot >= 1
    assert info.block_dims == block_dims
    blob = crisp.crisp_index_export(ix)
    R32 = np.frombuffer(blob, np.float32, D * D, 256).reshape(D, D)
    assert np.max(np.abs(R32 - ix_o.R32)) < 1e-6
    # the stored rows through the exported blob (Xr is the fifth section)
    K2 = K * K
    pos = 256
    for s in (4 * D * D, 4 * M * 2 * K * info.H, 4 * M * (K2 + 1), 4 * M * N):
        pos = (pos + s + 255) // 256 * 256
    xr = np.frombuffer(blob, np.float32, N * ix_o.Dp, pos).reshape(N, ix_o.Dp)
    keep = np.ones(D, bool)
    for lo, hi, _, rot in ix_o.blocks:
        if rot:
            keep[lo:hi] = False
            # the oracle's FP32 GEMV chain over w terms is within w 2^-24 |x_B| of the exact
            # product (sum |x_i R_ij| <= |x_B| for a unit column), the tensor-core split
            # product within 4e-6 |x_B|
            scale = np.linalg.norm(X[:, lo:hi].astype(np.float64), axis=1, keepdims=True)
            tol = ((hi - lo) * 2.0 ** -24 + 4e-6) * scale
            assert np.all(np.abs(xr[:, lo:hi] - ix_o.Xr[:, lo:hi]) <= tol)
    assert np.array_equal(xr[:, :D][:, keep], X[:, keep])
    assert np.all(xr[:, D:] == 0)
    gi, gd = oracle.knn_f64(X, Q, 10)
    kw = dict(k=10, rho=0.05, alpha=0.25)
    ids = empty((Q.shape[0], 10), torch.int64)
    d2 = empty((Q.shape[0], 10), torch.float32)
    crisp.crisp_search(ix, dev(Q), Q.shape[0], crisp.search_params(**kw), ids, d2)
    r_gpu = oracle.recall_at_k(ids.cpu().numpy(), gd, X, Q, 10)
    r_orc = oracle.recall_at_k(oracle.search(ix_o, Q, oracle.SearchParams(**kw))[0], gd, X, Q, 10)
    assert r_gpu >= r_orc - 0.03


def test_block_and_adaptive_argument_errors(mixed):
    X, Q, draws, N, D, M, K = mixed
    with pytest.raises(crisp.CrispError):
        crisp.crisp_build(dev(X), N, D, crisp.build_params(M, K, draws=draws, block_dims=30))
    with pytest.raises(crisp.CrispError):
        crisp.crisp_build(dev(X), N, D, crisp.build_params(M, K, draws=draws, adaptive=2))
    X6, _ = synthetic.small_gaussian(1000, 600, 1, seed=2)
    with pytest.raises(crisp.CrispError):   # D > 256 M
        crisp.crisp_build(dev(X6), 1000, 600, crisp.build_params(2, 8, adaptive=1,
                                                               draws=synthetic.method_draws(1000, 600, 2, 8,
                                                                                            kmeans_train=1000)))
    cells = empty((M, N), torch.int16)
    ix_o = oracle.build_index(X[:2000], M, 8, draws=synthetic.method_draws(2000, D, M, 8, kmeans_train=2000), rotate=0)
    bad = oracle.equal_bounds(D, M).copy()
    bad[1] = bad[0] + 1                      # a 1-dim subspace
    with pytest.raises(crisp.CrispError):
        crisp.crisp_assign_cells(dev(ix_o.Xr), 2000, D, ix_o.Dp, M, 8, ix_o.H, dev(ix_o.cent), cells, sub=bad)
