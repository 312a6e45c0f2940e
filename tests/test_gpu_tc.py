"""Tensor-core (tcgen05) rotation of the build (§4.1, X' = X R) against an FP64
product of the same FP32 inputs.

The kernel splits every FP32 operand into a TF32 head and an FP32 tail and
sums three TF32 products, so each output must lie within a few 1e-6 of
|x| |R e_j| of the exact product of the FP32 inputs; padding columns must be
exact zeros.  Shapes cover one row, ragged row tiles, a contraction that is not
a multiple of 32, row pitches wider than D, and several column tiles."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2603_05180_gb300 as crisp  # noqa: E402

DEV = torch.device("cuda:0")


def _orth(D, seed):
    q, r = np.linalg.qr(np.random.default_rng(seed).standard_normal((D, D)))
    return (q * np.sign(np.diag(r))).astype(np.float32)


@pytest.mark.parametrize("N,D,ldx,ldy", [(1, 32, 32, 32), (300, 960, 960, 960), (4096, 960, 960, 960),
                                         (1000, 36, 36, 64), (257, 256, 256, 288), (130, 33, 36, 33),
                                         (517, 1024, 1024, 1024), (64, 600, 600, 608)])
def test_rotate_tc_matches_fp64(N, D, ldx, ldy):
    r = np.random.default_rng(N * 7 + D)
    X = np.zeros((N, ldx), np.float32)
    X[:, :D] = (r.standard_normal((N, D)) * r.uniform(0.1, 10.0, (N, 1))).astype(np.float32)
    R = _orth(D, D)
    Y = torch.full((N, ldy), np.nan, dtype=torch.float32, device=DEV)
    crisp.crisp_rotate_rows_tc(torch.from_numpy(X).to(DEV), N, D, ldx, torch.from_numpy(R).to(DEV), Y, ldy)
    Yg = Y.cpu().numpy()
    exact = X[:, :D].astype(np.float64) @ R.astype(np.float64)
    bound = 4e-6 * np.linalg.norm(X[:, :D].astype(np.float64), axis=1, keepdims=True)
    err = np.abs(Yg[:, :D] - exact)
    assert np.all(err <= bound), float((err / bound).max())
    assert np.all(Yg[:, D:] == 0.0)
    # the rotation keeps row norms (up to the FP32 rounding of R)
    assert np.allclose(np.linalg.norm(Yg[:, :D].astype(np.float64), axis=1),
                       np.linalg.norm(X[:, :D].astype(np.float64), axis=1), rtol=2e-5)


def test_rotate_tc_against_the_fp32_gemv_path():
    N, D = 2048, 960
    r = np.random.default_rng(5)
    X = torch.from_numpy(r.standard_normal((N, D)).astype(np.float32)).to(DEV)
    R = torch.from_numpy(r.standard_normal((D, D)).astype(np.float32) / np.float32(np.sqrt(D))).to(DEV)  # not orthogonal
    Yt = torch.empty((N, D), dtype=torch.float32, device=DEV)
    Ys = torch.empty((N, D), dtype=torch.float32, device=DEV)
    crisp.crisp_rotate_rows_tc(X, N, D, D, R, Yt, D)
    crisp.crisp_rotate_rows(X, N, D, D, R, Ys, D)
    scale = X.double().norm(dim=1, keepdim=True) * R.double().norm(dim=0, keepdim=True)
    assert bool(((Yt.double() - Ys.double()).abs() <= 4e-6 * scale).all())


def test_rotate_tc_rejects_unaligned_rows():
    X = torch.zeros((8, 33), dtype=torch.float32, device=DEV)
    R = torch.zeros((33, 33), dtype=torch.float32, device=DEV)
    Y = torch.zeros((8, 64), dtype=torch.float32, device=DEV)
    with pytest.raises(crisp.CrispError) as e:
        crisp.crisp_rotate_rows_tc(X, 8, 33, 33, R, Y, 64)
    assert e.value.status == crisp.CRISP_EINVAL


# ------------------------------------------------------------ B3 cell assignment
def _assign_both(Xr, N, D, Dp, M, K, H, cent):
    """Cells from the tensor-core kernel with one TF32 pass and with one BF16
    pass (its BF16 copy of the rows made by the oracle's rounding), both
    checked against the SIMT kernel; returns (tensor cores, SIMT)."""
    import oracle

    dX = torch.from_numpy(np.ascontiguousarray(Xr)).to(DEV)
    dXb = torch.from_numpy(oracle.quantize_bf16(np.ascontiguousarray(Xr, np.float32)).view(np.int16)).to(DEV)
    dC = torch.from_numpy(np.ascontiguousarray(cent)).to(DEV)
    a = torch.empty((M, N), dtype=torch.int16, device=DEV)
    b = torch.empty((M, N), dtype=torch.int16, device=DEV)
    c = torch.empty((M, N), dtype=torch.int16, device=DEV)
    crisp.crisp_assign_cells_tc(dX, N, D, Dp, M, K, H, dC, a)
    crisp.crisp_assign_cells(dX, N, D, Dp, M, K, H, dC, b)
    crisp.crisp_assign_cells_tc(dX, N, D, Dp, M, K, H, dC, c, Xb=dXb)
    a, b, c = (t.cpu().numpy().view(np.uint16) for t in (a, b, c))
    assert np.array_equal(c, b), "BF16 pass"
    return a, b


def test_assign_tc_bitexact_with_the_oracle():
    import oracle
    import synthetic

    X, Q = synthetic.gmm()
    ix = oracle.build_index(X, M=8, draws=synthetic.method_draws(20000, 256, 8, 50, seed=0))
    a, b = _assign_both(ix.Xr, ix.N, ix.D, ix.Dp, ix.M, ix.K, ix.H, ix.cent)
    assert np.array_equal(a, ix.cells) and np.array_equal(b, ix.cells)


@pytest.mark.parametrize("N,D,M,K", [(1, 64, 2, 50), (5000, 960, 20, 50), (3001, 33, 4, 7), (777, 600, 7, 64),
                                     (2048, 1024, 8, 50)])
def test_assign_tc_equals_the_simt_kernel(N, D, M, K):
    """Subspaces that start off the 32-column grid, odd widths, K < 64 and
    K = 64, a ragged last row tile; centroids drawn from the rows."""
    r = np.random.default_rng(N + D)
    Dp = (D + 31) // 32 * 32
    Xr = np.zeros((N, Dp), np.float32)
    Xr[:, :D] = (r.standard_normal((N, D)) * (1.0 + np.arange(D) % 7)).astype(np.float32)
    H = max((D // M + 1) // 2 + 1, 1)
    cent = np.zeros((M, 2, K, H), np.float32)
    for m in range(M):
        lo, hi = m * D // M, (m + 1) * D // M
        hl = (hi - lo) // 2
        for half, (o, h) in enumerate(((lo, hl), (lo + hl, hi - lo - hl))):
            pick = r.choice(N, size=K, replace=N < K)
            cent[m, half, :, :h] = Xr[pick, o:o + h] + r.standard_normal((K, h)).astype(np.float32) * 0.1
    a, b = _assign_both(Xr, N, D, Dp, M, K, H, cent)
    assert np.array_equal(a, b)


def test_assign_tc_exact_ties_go_to_the_lowest_index():
    """Rows equidistant from two centroids (and duplicated centroids): the
    tensor-core scores cannot separate them, the SEQ re-measure must pick the
    lower index exactly as the plain kernel does."""
    N, D, M, K = 4096, 64, 2, 8
    r = np.random.default_rng(1)
    H = 16
    cent = np.zeros((M, 2, K, H), np.float32)
    cent[:, :, :, :] = r.integers(-4, 5, (M, 2, K, H)).astype(np.float32)
    cent[:, :, 5] = cent[:, :, 2]                        # duplicate centroid
    Xr = np.zeros((N, D), np.float32)
    for m in range(M):
        for half in range(2):
            o = m * 32 + half * 16
            i, j = r.integers(0, K, N), r.integers(0, K, N)
            Xr[:, o:o + 16] = 0.5 * (cent[m, half, i] + cent[m, half, j])   # exact midpoints (small integers)
    a, b = _assign_both(Xr, N, D, D, M, K, H, cent)
    assert np.array_equal(a, b)
    assert not np.any((a // K == 5) | (a % K == 5))     # the duplicate never wins over index 2
