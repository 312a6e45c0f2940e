"""CPU oracle of CRISP (arXiv 2603.05180) -- TEST INFRASTRUCTURE ONLY.

A plain, slow, obviously-correct restatement of what the GPU engine computes,
written from the paper: the index build of §4.1-§4.2 (covariance and CEV test,
random orthogonal rotation, IMI k-means per subspace half, cell assignment,
CSR, sign codes), the two build extensions of §7 (block-wise rotation of the
correlated blocks only, variance-aware subspace boundaries) and the query
pipeline of Algorithm 1 / §4.3 (partial
distances, multi-sequence traversal, collision counting, threshold cut with
fallback, exact re-rank or Hamming-ordered ADSampling with patience).

Only the test suite, ``__graft_entry__.smoke()`` and the benchmark's CPU
baseline leg may import this package.  It shares no code with the CUDA library
and never imports it; the only module both sides are fed from is ``synthetic``.

The per-query loops live in ``crisp_oracle.c`` (plain C11); this module adds
the steps that are library primitives (a symmetric eigenvalue routine and a QR
factorisation from numpy/LAPACK) and writes the index blob the CUDA library
can import, so that both sides search the very same index.

Parity status: every function here is pinned by a ``-m "not gpu"`` test
(tests/test_oracle_*.py) against closed forms, brute force, worked examples or
a second independent implementation.
"""
from __future__ import annotations

import ctypes as C
import math
import struct
from dataclasses import dataclass, field

import numpy as np

from . import build as _build

_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(_build.build())
        _declare(_lib)
    return _lib


class _OrIndex(C.Structure):
    _fields_ = [("N", C.c_int64), ("D", C.c_int32), ("Dp", C.c_int32), ("M", C.c_int32), ("K", C.c_int32),
                ("H", C.c_int32), ("rotated", C.c_int32), ("_pad", C.c_int32),
                ("R32", C.c_void_p), ("cent", C.c_void_p), ("offsets", C.c_void_p), ("ids", C.c_void_p),
                ("Xr", C.c_void_p), ("codes", C.c_void_p), ("Xb", C.c_void_p), ("X8", C.c_void_p),
                ("S8", C.c_void_p), ("mlp", C.c_void_p), ("mlp_H", C.c_int32), ("_pad2", C.c_int32),
                ("sub", C.c_void_p)]


class _OrParams(C.Structure):
    _fields_ = [("k", C.c_int32), ("mode", C.c_int32), ("rho", C.c_double), ("alpha", C.c_double),
                ("patience_factor", C.c_int32), ("eps0", C.c_float), ("max_candidates", C.c_int64),
                ("precision", C.c_int32), ("shortlist", C.c_int32), ("depth_margin", C.c_float),
                ("short_margin", C.c_float), ("verify_order", C.c_int32), ("_pad", C.c_int32)]


STATS_DTYPE = np.dtype([("n_candidates", np.int64), ("n_verified", np.int64), ("n_full", np.int64),
                        ("n_retrieved", np.int64), ("fallback", np.int32), ("capped", np.int32),
                        ("tau", np.int32), ("_pad", np.int32)])

_P = C.c_void_p
_I64, _I32, _F, _D = C.c_int64, C.c_int32, C.c_float, C.c_double


def _declare(L):
    sig = {
        "or_subspace": (None, [_I32, _I32, _I32, _P, _P, _P]),
        "or_tau": (_I32, [_D, _I32]),
        "or_budget": (_I64, [_D, _I64]),
        "or_seq_sqdist": (_F, [_P, _P, _I32]),
        "or_cr32_blocks": (None, [_P, _P, _I32, _P]),
        "or_cr32": (_F, [_P, _P, _I32]),
        "or_rotate_rows": (None, [_P, _I64, _I32, _I32, _P, _I32, _P]),
        "or_pad_rows": (None, [_P, _I64, _I32, _I32, _I32, _P]),
        "or_covariance": (None, [_P, _I64, _I32, _I32, _P, _I64, _P]),
        "or_kmeans": (None, [_P, _I64, _I32, _I32, _I32, _I32, _I32, _P, _I32, _P]),
        "or_assign_cells": (None, [_P, _I64, _I32, _I32, _I32, _I32, _I32, _P, _P, _P]),
        "or_csr": (None, [_P, _I64, _I32, _P, _P]),
        "or_sign_codes": (None, [_P, _I64, _I32, _P]),
        "or_half_dists": (None, [_P, _P, _I32, _I32, _P, _P, _P]),
        "or_activate_heap": (_I32, [_P, _P, _I32, _I32, _I32, _I64, _P, _P, _P]),
        "or_activate_sorted": (_I32, [_P, _P, _I32, _I32, _I32, _I64, _P, _P, _P]),
        "or_scores_walk": (None, [_P, _P, _P, _P, _P]),
        "or_scores_membership": (None, [_P, _P, _P, _P, _P, _P]),
        "or_cut": (_I64, [_P, _I64, _I32, _I32, _I64, _P, _P]),
        "or_rerank": (_I32, [_P, _P, _P, _I64, _I32, _P, _P]),
        "or_ads_factor": (_F, [_I32, _I32, _F]),
        "or_verify_opt": (_I32, [_P, _P, _P, _P, _I64, _I32, _F, _I64, _I32, _P, _P, _P, _P]),
        "or_search_batch": (_I32, [_P, _P, _I64, _I32, _P, _P, _P, _P, _I32]),
        "or_knn_f64": (None, [_P, _I64, _I32, _I32, _P, _I64, _I32, _I32, _P, _P]),
        "or_bf16_rne": (C.c_uint16, [_F]),
        "or_bf16_to_f32": (_F, [C.c_uint16]),
        "or_e4m3_rne": (C.c_uint8, [_F]),
        "or_e4m3_to_f32": (_F, [C.c_uint8]),
        "or_quantize_bf16": (None, [_P, _I64, _I32, _P]),
        "or_quantize_e4m3": (None, [_P, _I64, _I32, _P, _P]),
        "or_prescore": (_F, [_P, _P, _F, _P, _I32]),
        "or_shortlist": (_I64, [_P, _P, _P, _I32, _P, _P, _I64, _I64, _P]),
        "or_erf_as": (_F, [_F]),
        "or_gelu": (_F, [_F]),
        "or_mlp_infer": (None, [_P, _I32, _I32, _I32, _P, _P]),
        "or_features": (None, [_P, _P, _I64, _I64, _P, _P, _I32, _I32, _I32, _P]),
        "or_depth": (_I64, [_F, _F, _I64, _I64]),
        "or_select_by_score": (_I64, [_P, _P, _I64, _I64, _P]),
        "or_activate_heap_costs": (_I32, [_P, _P, _I32, _I32, _I32, _I64, _P, _P, _P, _P, _P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


# ------------------------------------------------------------------ readings
def tau(alpha: float, M: int) -> int:
    """tau = ceil(alpha M) (Theorem 1)."""
    return int(lib().or_tau(float(alpha), int(M)))


def budget(rho: float, N: int) -> int:
    """max(1, ceil(rho N)) ids per subspace (Algorithm 1)."""
    return int(lib().or_budget(float(rho), int(N)))


def subspace(D: int, M: int, m: int):
    lo, hl, hr = C.c_int(), C.c_int(), C.c_int()
    lib().or_subspace(D, M, m, C.byref(lo), C.byref(hl), C.byref(hr))
    return lo.value, hl.value, hr.value


def padded_dim(D: int) -> int:
    return (D + 31) // 32 * 32


def half_width_max(D: int, M: int) -> int:
    return max(max(subspace(D, M, m)[1:]) for m in range(M))


def equal_bounds(D: int, M: int) -> np.ndarray:
    """Boundaries of the equal split of §3: sub[m] = floor(mD/M), sub[M] = D."""
    return np.array([subspace(D, M, m)[0] for m in range(M)] + [D], np.int32)


def bounds_half_max(sub) -> int:
    """Widest subspace half (the centroid row length H) for boundaries sub[0..M]."""
    w = np.diff(np.asarray(sub, np.int64))
    return int(np.max(w - w // 2))


# ------------------------------------- §7 adaptive subspace decomposition
def column_variance(X, rows) -> np.ndarray:
    """Per-dimension sample variance of X[rows] over the first D columns, FP64,
    mean-centred with 1/(S-1): the statistic the adaptive decomposition of §7
    balances across subspaces.  X may carry padding columns past D (pass D)."""
    Xs = np.asarray(X)[np.asarray(rows, np.int64)].astype(np.float64)
    S = Xs.shape[0]
    mean = Xs.sum(axis=0) / S
    c = Xs - mean[None, :]
    return (c * c).sum(axis=0) / (S - 1)


SUB_MIN, SUB_MAX = 2, 256   # a subspace needs two non-empty halves of at most 128 dims


def adaptive_bounds(var, M: int) -> np.ndarray:
    """Variance-aware subspace boundaries (§7 Adaptive Subspace Decomposition).

    Subspaces stay contiguous in dimension order and get (near) equal shares of
    the total variance, so a high-variance region is split into narrow
    subspaces and a low-variance region grouped into wide ones.  With the
    cumulative variance V_j = var[0] + ... + var[j-1] (FP64, summed in order),
    boundary m (0 < m < M) is the largest j with V_j <= m V_D / M, clamped so
    that every subspace keeps between 2 and 256 dims.  Zero total variance
    gives the equal split."""
    var = [float(v) for v in var]
    D = len(var)
    cum = [0.0]
    for v in var:
        cum.append(cum[-1] + v)
    tot = cum[D]
    b = [0]
    for m in range(1, M):
        if tot > 0.0:
            t = float(m) * tot / float(M)
            j = 0
            while j < D and cum[j + 1] <= t:
                j += 1
        else:
            j = (m * D) // M
        lo = max(b[-1] + SUB_MIN, D - SUB_MAX * (M - m))
        hi = min(b[-1] + SUB_MAX, D - SUB_MIN * (M - m))
        b.append(min(max(j, lo), hi))
    b.append(D)
    return np.array(b, np.int32)


# ------------------------------------------------------------ FP32 orders
def seq_sqdist(a, b) -> np.float32:
    a, b = _c(a, np.float32), _c(b, np.float32)
    return np.float32(lib().or_seq_sqdist(_p(a), _p(b), a.size))


def cr32_blocks(x, q) -> np.ndarray:
    x, q = _c(x, np.float32), _c(q, np.float32)
    assert x.size % 32 == 0 and x.size == q.size
    s = np.empty(x.size // 32, np.float32)
    lib().or_cr32_blocks(_p(x), _p(q), x.size, _p(s))
    return s


def cr32(x, q) -> np.float32:
    x, q = _c(x, np.float32), _c(q, np.float32)
    return np.float32(lib().or_cr32(_p(x), _p(q), x.size))


# ------------------------------------------------------- B1 covariance + CEV
def covariance(X, rows) -> np.ndarray:
    """Sample covariance of X[rows] in FP64, mean-centred, 1/(S-1) (§4.1).

    The centred product Xc^T Xc is a library matmul (numpy/BLAS)."""
    Xs = np.asarray(X)[np.asarray(rows, np.int64)].astype(np.float64)
    Xs -= Xs.mean(axis=0, keepdims=True)
    cov = (Xs.T @ Xs) / float(Xs.shape[0] - 1)
    return 0.5 * (cov + cov.T)


def covariance_loops(X, rows) -> np.ndarray:
    """The same covariance written as plain loops in C (a second form, for small inputs)."""
    X = _c(X, np.float32)
    rows = _c(rows, np.int64)
    D = X.shape[1]
    cov = np.empty((D, D), np.float64)
    lib().or_covariance(_p(X), X.shape[0], D, D, _p(rows), rows.size, _p(cov))
    return cov


def cev_from_eigenvalues(eig_desc: np.ndarray) -> float:
    """CEV = sum of the top floor(0.2 D) eigenvalues over the sum of all (§4.1)."""
    D = eig_desc.size
    k = int(math.floor(0.2 * D))
    tot = float(np.sum(eig_desc))
    return float(np.sum(eig_desc[:k]) / tot) if tot > 0 else 0.0


def cev(X, rows):
    """(CEV, eigenvalues descending) of the sample covariance (§4.1).

    The eigenvalues come from LAPACK's symmetric eigenvalue routine (numpy)."""
    ev = np.linalg.eigvalsh(covariance(X, rows))[::-1].copy()
    return cev_from_eigenvalues(ev), ev


# ------------------------------------------------------------ B2 rotation
def rotation_from_gaussian(G: np.ndarray) -> np.ndarray:
    """R from G = Q R' (§3 Randomized Orthogonal Rotation): R = Q diag(sign(diag R')).

    The sign fix makes Q unique (and Haar when G is Gaussian); the QR itself is
    LAPACK's Householder factorisation (numpy)."""
    Q, Rp = np.linalg.qr(np.asarray(G, np.float64))
    s = np.where(np.diag(Rp) < 0, -1.0, 1.0)
    return Q * s[None, :]


def rotation_blocks(D: int, b: int):
    """Contiguous blocks of b dims, [jb, min((j+1)b, D)), the last one ragged."""
    return [(lo, min(lo + b, D)) for lo in range(0, D, b)]


def block_rotation(X, rows, G, b: int, tau_cev: float, rotate: int = -1):
    """Block-wise variance redistribution (§7 Partial Variance Redistribution).

    The dimensions are cut into contiguous blocks of b dims.  Each block takes
    the §4.1 test on its own: its CEV is computed from the eigenvalues of the
    sample covariance restricted to the block (top floor(0.2 w) of w), and a
    block whose CEV exceeds tau_cev (every block for rotate = 1, none for 0) is
    rotated by its own Haar rotation, R_B = rotation_from_gaussian(G_BB) with
    G_BB the block's diagonal block of the Gaussian draws.  R is block-diagonal,
    the identity outside rotated blocks, so X R costs O(N sum w^2) <= O(N D b).

    Returns (R64 [D][D], [(lo, hi, cev, rotated) per block])."""
    G = np.asarray(G, np.float64)
    D = G.shape[0]
    cov = covariance(X, rows)
    R = np.eye(D)
    info = []
    for lo, hi in rotation_blocks(D, b):
        ev = np.linalg.eigvalsh(cov[lo:hi, lo:hi])[::-1].copy()
        c = cev_from_eigenvalues(ev)
        rot = rotate == 1 or (rotate == -1 and c > tau_cev)
        if rot:
            R[lo:hi, lo:hi] = rotation_from_gaussian(G[lo:hi, lo:hi])
        info.append((lo, hi, c, bool(rot)))
    return R, info


def rotate_rows(X, R32, Dp=None) -> np.ndarray:
    """X' = X R in FP32, each output an fmaf chain over d = 0..D-1 (Q1 / B2)."""
    X = _c(X, np.float32)
    R32 = _c(R32, np.float32)
    N, D = X.shape
    Dp = padded_dim(D) if Dp is None else Dp
    Y = np.empty((N, Dp), np.float32)
    lib().or_rotate_rows(_p(X), N, D, D, _p(R32), Dp, _p(Y))
    return Y


def pad_rows(X, Dp=None) -> np.ndarray:
    X = _c(X, np.float32)
    N, D = X.shape
    Dp = padded_dim(D) if Dp is None else Dp
    Y = np.zeros((N, Dp), np.float32)
    Y[:, :D] = X
    return Y


# ------------------------------------------------------------- B3 k-means
def kmeans(T, off, h, K, H, init, iters) -> np.ndarray:
    """Lloyd's k-means over dims [off, off+h) of the training rows (§4.2 IMI, K centroids)."""
    T = _c(T, np.float32)
    init = _c(init, np.int32)
    Cc = np.zeros((K, H), np.float32)
    lib().or_kmeans(_p(T), T.shape[0], T.shape[1], off, h, K, H, _p(init), iters, _p(Cc))
    return Cc


def assign_cells(Xr, D, M, K, H, cent, sub=None) -> np.ndarray:
    """u_m(x) = cL*K + cR for all rows and subspaces, [M][N] uint16 (§3, §4.2);
    ``sub`` gives the subspace boundaries (None: the equal split)."""
    Xr = _c(Xr, np.float32)
    cent = _c(cent, np.float32)
    N, Dp = Xr.shape
    cells = np.empty((M, N), np.uint16)
    sb = _c(sub, np.int32) if sub is not None else None
    lib().or_assign_cells(_p(Xr), N, D, Dp, M, K, H, _p(cent), _p(sb) if sb is not None else None, _p(cells))
    return cells


def csr(cells_m, K2):
    """(Offsets[K^2+1], ids[N]) of one subspace (§4.2)."""
    cells_m = _c(cells_m, np.uint16)
    off = np.empty(K2 + 1, np.int32)
    ids = np.empty(cells_m.size, np.int32)
    lib().or_csr(_p(cells_m), cells_m.size, K2, _p(off), _p(ids))
    return off, ids


def sign_codes(Xr) -> np.ndarray:
    """b(x): bit d of word d/32 is (x'_d > 0) (§3 Binary Quantization)."""
    Xr = _c(Xr, np.float32)
    N, Dp = Xr.shape
    codes = np.empty((N, Dp // 32), np.uint32)
    lib().or_sign_codes(_p(Xr), N, Dp, _p(codes))
    return codes


# ---------------------------------------------------------------- index
@dataclass
class Index:
    N: int
    D: int
    Dp: int
    M: int
    K: int
    H: int
    rotated: int
    cev: float
    R32: np.ndarray | None
    cent: np.ndarray          # [M][2][K][H] float32
    offsets: np.ndarray       # [M][K*K+1] int32
    ids: np.ndarray           # [M][N] int32
    Xr: np.ndarray            # [N][Dp] float32
    codes: np.ndarray         # [N][Dp/32] uint32
    cells: np.ndarray         # [M][N] uint16 (u_m(x), kept for the Eq. 1 check)
    R64: np.ndarray | None = None
    eig: np.ndarray | None = None
    Xb: np.ndarray | None = None          # [N][Dp] BF16 bits (F2)
    X8: np.ndarray | None = None          # [N][Dp] FP8 E4M3 codes (F2)
    S8: np.ndarray | None = None          # [N] FP8 row scales
    mlp: np.ndarray | None = None         # learned depth model, packed FP32 parameters
    mlp_H: int = 0
    sub: np.ndarray | None = None         # [M+1] subspace boundaries (None: the equal split)
    blocks: list | None = None            # block-wise rotation: (lo, hi, cev, rotated) per block
    _st: _OrIndex | None = field(default=None, repr=False)

    def bounds(self) -> np.ndarray:
        return self.sub if self.sub is not None else equal_bounds(self.D, self.M)

    def set_model(self, params, H):
        self.mlp = np.ascontiguousarray(params, np.float32)
        self.mlp_H = int(H)
        self._st = None
        return self

    def add_copies(self, bf16=True, fp8=True):
        if bf16 and self.Xb is None:
            self.Xb = quantize_bf16(self.Xr)
        if fp8 and self.X8 is None:
            self.X8, self.S8 = quantize_e4m3(self.Xr)
        self._st = None
        return self

    def st(self) -> _OrIndex:
        if self._st is None:
            pv = lambda a: _p(a).value if a is not None else None
            self._st = _OrIndex(self.N, self.D, self.Dp, self.M, self.K, self.H, self.rotated, 0,
                                pv(self.R32), pv(self.cent), pv(self.offsets), pv(self.ids), pv(self.Xr),
                                pv(self.codes), pv(self.Xb), pv(self.X8), pv(self.S8), pv(self.mlp), self.mlp_H, 0,
                                pv(self.sub))
        return self._st


def build_index(X, M, K=50, draws=None, tau_cev=0.85, rotate=-1, kmeans_iters=20, seed=0, adaptive=0,
                block_dims=0) -> Index:
    """The index build of §4.1-§4.2 in order: CEV test, optional rotation,
    k-means per subspace half, cell assignment, CSR per subspace, sign codes.

    ``draws`` holds the random numbers the build uses (synthetic.method_draws);
    ``rotate`` is -1 (decide by CEV > tau_cev), 0 (never) or 1 (always).
    The two extensions of §7: ``block_dims`` = b > 0 replaces the global test
    and rotation by the block-wise one (block_rotation); ``adaptive`` = 1 sets
    the subspace boundaries by adaptive_bounds from the per-dimension variance
    of the stored rows over the covariance sample (else the equal split)."""
    import synthetic

    X = _c(X, np.float32)
    N, D = X.shape
    if draws is None:
        draws = synthetic.method_draws(N, D, M, K, seed)
    Dp = padded_dim(D)
    cval, eig = cev(X, draws.cev_sample)
    blocks = None
    if block_dims > 0:
        R64, blocks = block_rotation(X, draws.cev_sample, draws.gaussian, block_dims, tau_cev, rotate)
        do_rot = any(b[3] for b in blocks)
        if not do_rot:
            R64 = None
    else:
        do_rot = (rotate == 1) or (rotate == -1 and cval > tau_cev)
        R64 = rotation_from_gaussian(draws.gaussian) if do_rot else None
    R32 = None
    if do_rot:
        R32 = R64.astype(np.float32)
        Xr = rotate_rows(X, R32, Dp)
    else:
        Xr = pad_rows(X, Dp)
    sub = adaptive_bounds(column_variance(Xr[:, :D], draws.cev_sample), M) if adaptive else equal_bounds(D, M)
    H = bounds_half_max(sub)
    T = np.ascontiguousarray(Xr[draws.kmeans_sample])
    cent = np.zeros((M, 2, K, H), np.float32)
    for m in range(M):
        lo, w = int(sub[m]), int(sub[m + 1] - sub[m])
        hl, hr = w // 2, w - w // 2
        cent[m, 0] = kmeans(T, lo, hl, K, H, draws.kmeans_init[m, 0], kmeans_iters)
        cent[m, 1] = kmeans(T, lo + hl, hr, K, H, draws.kmeans_init[m, 1], kmeans_iters)
    cells = assign_cells(Xr, D, M, K, H, cent, sub)
    offsets = np.empty((M, K * K + 1), np.int32)
    ids = np.empty((M, N), np.int32)
    for m in range(M):
        offsets[m], ids[m] = csr(cells[m], K * K)
    codes = sign_codes(Xr)
    ix = Index(N, D, Dp, M, K, H, int(do_rot), float(cval), R32, cent, offsets, ids, Xr, codes, cells, R64, eig)
    if adaptive:
        ix.sub = sub
    ix.blocks = blocks
    return ix


# Index blob: a 256-byte header (magic "CRISPIX1", then int64 version, N, D,
# Dp, M, K, H, rotated, and the CEV as a float64), then sections R32 (only if
# rotated), cent, offsets, ids, Xr, codes, each starting at a multiple of 256.
# Version 2 adds a last section, the int32 subspace boundaries [M+1], for an
# index whose boundaries are not the equal split; version 1 has the equal split.
BLOB_MAGIC = b"CRISPIX1"


def export_blob(ix: Index) -> bytes:
    sub = ix.bounds()
    v2 = not np.array_equal(sub, equal_bounds(ix.D, ix.M))
    hdr = bytearray(256)
    hdr[0:8] = BLOB_MAGIC
    struct.pack_into("<8q", hdr, 8, 2 if v2 else 1, ix.N, ix.D, ix.Dp, ix.M, ix.K, ix.H, ix.rotated)
    struct.pack_into("<d", hdr, 72, ix.cev)
    parts = [bytes(hdr)]
    secs = ([ix.R32.astype(np.float32)] if ix.rotated else []) + [
        ix.cent.astype(np.float32), ix.offsets.astype(np.int32), ix.ids.astype(np.int32),
        ix.Xr.astype(np.float32), ix.codes.astype(np.uint32)] + ([sub.astype(np.int32)] if v2 else [])
    pos = 256
    for a in secs:
        b = np.ascontiguousarray(a).tobytes()
        parts.append(b)
        pos += len(b)
        pad = (-pos) % 256
        parts.append(b"\0" * pad)
        pos += pad
    return b"".join(parts)


# ----------------------------------------------------------------- query side
@dataclass
class SearchParams:
    k: int = 10
    mode: int = 0                 # 0 Guaranteed, 1 Optimized
    rho: float = 0.01
    alpha: float = 0.3
    patience_factor: int = 40
    eps0: float = 2.1
    max_candidates: int = 0
    precision: int = 0            # Guaranteed mode coarse scoring: 0 none, 1 BF16, 2 FP8 E4M3
    shortlist: int = 0            # candidates kept for the FP32 re-rank when precision > 0
    depth_margin: float = 0.0     # learned mode (2): margins on the predicted log2 depths
    short_margin: float = 0.0
    verify_order: int = 0         # Optimized mode: 0 (Hamming, id) order, 1 id order (ablation)

    def st(self) -> _OrParams:
        return _OrParams(self.k, self.mode, self.rho, self.alpha, self.patience_factor, self.eps0,
                         self.max_candidates, self.precision, self.shortlist, self.depth_margin, self.short_margin,
                         self.verify_order, 0)


def query_rotate(ix: Index, Q) -> np.ndarray:
    Q = np.atleast_2d(_c(Q, np.float32))
    return rotate_rows(Q, ix.R32, ix.Dp) if ix.rotated else pad_rows(Q, ix.Dp)


def half_dists(ix: Index, qr, m, half):
    qr = _c(qr, np.float32)
    d = np.empty(ix.K, np.float32)
    s = np.empty(ix.K, np.float32)
    p = np.empty(ix.K, np.int32)
    lib().or_half_dists(C.byref(ix.st()), _p(qr), m, half, _p(d), _p(s), _p(p))
    return d, s, p


def activate(ix: Index, qr, m, phi, k, bud, impl="heap"):
    """Popped cells (pop order), their weights, and the ids retrieved (Algorithm 1)."""
    qr = _c(qr, np.float32)
    K2 = ix.K * ix.K
    cells = np.empty(K2, np.int32)
    w = np.empty(K2, np.uint8)
    got = C.c_int64()
    f = lib().or_activate_heap if impl == "heap" else lib().or_activate_sorted
    n = f(C.byref(ix.st()), _p(qr), m, phi, k, bud, _p(cells), _p(w), C.byref(got))
    return cells[:n].copy(), w[:n].copy(), got.value


def _act_arrays(ix, acts):
    K2 = ix.K * ix.K
    nc = np.array([len(a[0]) for a in acts], np.int32)
    cells = np.zeros((ix.M, K2), np.int32)
    w = np.zeros((ix.M, K2), np.uint8)
    for m, (c, ww, _) in enumerate(acts):
        cells[m, :len(c)] = c
        w[m, :len(c)] = ww
    return nc, cells, w


def scores_walk(ix: Index, acts) -> np.ndarray:
    nc, cells, w = _act_arrays(ix, acts)
    V = np.empty(ix.N, np.int32)
    lib().or_scores_walk(C.byref(ix.st()), _p(nc), _p(cells), _p(w), _p(V))
    return V


def scores_membership(ix: Index, acts) -> np.ndarray:
    nc, cells, w = _act_arrays(ix, acts)
    V = np.empty(ix.N, np.int32)
    pc = _c(ix.cells, np.uint16)
    lib().or_scores_membership(C.byref(ix.st()), _p(pc), _p(nc), _p(cells), _p(w), _p(V))
    return V


def cut(V, t, k, cap=0):
    V = _c(V, np.int32)
    Cc = np.empty(max(1, V.size), np.int32)
    how = C.c_int()
    n = lib().or_cut(_p(V), V.size, int(t), int(k), int(cap), _p(Cc), C.byref(how))
    return Cc[:n].copy(), how.value


def rerank(ix: Index, qr, Cand, k):
    qr = _c(qr, np.float32)
    Cand = _c(Cand, np.int32)
    ids = np.empty(k, np.int64)
    d2 = np.empty(k, np.float32)
    lib().or_rerank(C.byref(ix.st()), _p(qr), _p(Cand), Cand.size, k, _p(ids), _p(d2))
    return ids, d2


def ads_factor(t, D, eps0) -> np.float32:
    return np.float32(lib().or_ads_factor(int(t), int(D), float(eps0)))


def verify_opt(ix: Index, qr, Cand, k, eps0=2.1, P=400, order=0):
    qr = _c(qr, np.float32)
    Cand = _c(Cand, np.int32)
    qcode = sign_codes(qr.reshape(1, -1))[0]
    ids = np.empty(k, np.int64)
    d2 = np.empty(k, np.float32)
    nv, nf = C.c_int64(), C.c_int64()
    lib().or_verify_opt(C.byref(ix.st()), _p(qr), _p(qcode), _p(Cand), Cand.size, k, float(eps0), int(P), int(order),
                        _p(ids), _p(d2), C.byref(nv), C.byref(nf))
    return ids, d2, nv.value, nf.value


def search(ix: Index, Q, params: SearchParams, nthreads: int = 0):
    """Algorithm 1 for a batch of queries: (ids [nq,k] int64, d2 [nq,k] f32, stats, threads used)."""
    Q = np.atleast_2d(_c(Q, np.float32))
    if params.precision == 1 and ix.Xb is None:
        raise ValueError("search: precision 1 needs the index's BF16 copy (Index.add_copies)")
    if params.precision == 2 and ix.X8 is None:
        raise ValueError("search: precision 2 needs the index's FP8 copy (Index.add_copies)")
    if params.mode == 2 and (getattr(ix, "mlp", None) is None or ix.Xb is None):
        raise ValueError("search: mode 2 needs a model (Index.set_model) and the BF16 copy (Index.add_copies)")
    nq = Q.shape[0]
    ids = np.empty((nq, params.k), np.int64)
    d2 = np.empty((nq, params.k), np.float32)
    st = np.zeros(nq, STATS_DTYPE)
    used = lib().or_search_batch(C.byref(ix.st()), _p(Q), nq, Q.shape[1], C.byref(params.st()), _p(ids), _p(d2),
                                 _p(st), int(nthreads))
    return ids, d2, st, used


def query_detail(ix: Index, q, params: SearchParams):
    """Every intermediate of one query (for step-by-step parity tests)."""
    qr = query_rotate(ix, q)[0]
    bud = budget(params.rho, ix.N)
    acts = [activate(ix, qr, m, int(params.mode == 1), params.k, bud) for m in range(ix.M)]
    V = scores_walk(ix, acts)
    t = tau(params.alpha, ix.M)
    Cand, how = cut(V, t, params.k, params.max_candidates)
    return dict(qr=qr, acts=acts, V=V, tau=t, C=Cand, how=how, budget=bud)


def knn_f64(X, Q, k):
    """Exact kNN by FP64 squared L2, ties by id (ground truth)."""
    X = _c(X, np.float32)
    Q = np.atleast_2d(_c(Q, np.float32))
    ids = np.empty((Q.shape[0], k), np.int64)
    d2 = np.empty((Q.shape[0], k), np.float64)
    lib().or_knn_f64(_p(X), X.shape[0], X.shape[1], X.shape[1], _p(Q), Q.shape[0], Q.shape[1], k, _p(ids), _p(d2))
    return ids, d2


def recall_at_k(found_ids: np.ndarray, gt_d2: np.ndarray, X: np.ndarray, Q: np.ndarray, k: int, rel=1e-5) -> float:
    """Tie-aware recall@k: a returned id counts if its FP64 distance is within
    (1 + rel) of the true k-th distance; at most k per query."""
    hits = 0
    for i in range(found_ids.shape[0]):
        ids = found_ids[i][found_ids[i] >= 0][:k]
        if ids.size == 0:
            continue
        d = ((X[ids].astype(np.float64) - Q[i].astype(np.float64)) ** 2).sum(1)
        hits += int(np.sum(d <= gt_d2[i, k - 1] * (1 + rel)))
    return hits / (found_ids.shape[0] * k)


# ------------------------------------------- F2: low-precision coarse scoring
def bf16_rne(x: float) -> int:
    """BF16 bits of x, round to nearest even."""
    return int(lib().or_bf16_rne(float(x)))


def bf16_to_f32(b: int) -> float:
    return float(lib().or_bf16_to_f32(int(b)))


def e4m3_rne(x: float) -> int:
    """OCP FP8 E4M3 (fn) bits of x: round to nearest even, saturating to +-448."""
    return int(lib().or_e4m3_rne(float(x)))


def e4m3_to_f32(c: int) -> float:
    return float(lib().or_e4m3_to_f32(int(c)))


def quantize_bf16(Xr) -> np.ndarray:
    Xr = _c(Xr, np.float32)
    out = np.empty(Xr.shape, np.uint16)
    lib().or_quantize_bf16(_p(Xr), Xr.shape[0], Xr.shape[1], _p(out))
    return out


def quantize_e4m3(Xr):
    """(codes [N][Dp] uint8, per-row scales [N] float32): s = max|x| / 448, code = e4m3(x / s)."""
    Xr = _c(Xr, np.float32)
    codes = np.empty(Xr.shape, np.uint8)
    sc = np.empty(Xr.shape[0], np.float32)
    lib().or_quantize_e4m3(_p(Xr), Xr.shape[0], Xr.shape[1], _p(codes), _p(sc))
    return codes, sc


def prescore(qr, xb=None, x8=None, s8=0.0) -> np.float32:
    """CR32 distance of q to a row's dequantised BF16 or E4M3 copy."""
    qr = _c(qr, np.float32)
    if xb is not None:
        xb = _c(xb, np.uint16)
        return np.float32(lib().or_prescore(_p(xb), None, 0.0, _p(qr), qr.size))
    x8 = _c(x8, np.uint8)
    return np.float32(lib().or_prescore(None, _p(x8), float(s8), _p(qr), qr.size))


def shortlist(ix: Index, qr, Cand, S, precision="bf16", quant=None):
    """The S candidates of smallest (coarse distance, id), ascending id."""
    qr = _c(qr, np.float32)
    Cand = _c(Cand, np.int32)
    out = np.empty(max(1, Cand.size), np.int32)
    if precision == "bf16":
        Xb = quant if quant is not None else quantize_bf16(ix.Xr)
        n = lib().or_shortlist(_p(Xb), None, None, ix.Dp, _p(qr), _p(Cand), Cand.size, int(S), _p(out))
    else:
        X8, S8 = quant if quant is not None else quantize_e4m3(ix.Xr)
        n = lib().or_shortlist(None, _p(X8), _p(S8), ix.Dp, _p(qr), _p(Cand), Cand.size, int(S), _p(out))
    return out[:n].copy()


# --------------------------------------- F1: learned re-rank depth (small MLP)
def erf_as(u: float) -> np.float32:
    """erf by Abramowitz & Stegun 7.1.28, evaluated in FP32 in the fixed order."""
    return np.float32(lib().or_erf_as(float(u)))


def gelu(z: float) -> np.float32:
    return np.float32(lib().or_gelu(float(z)))


def mlp_param_count(F, H, O):
    return F * H + H + H * H + H + H * O + O


def mlp_unpack(P, F, H, O):
    P = np.asarray(P)
    o = 0
    out = []
    for shape in ((F, H), (H,), (H, H), (H,), (H, O), (O,)):
        n = int(np.prod(shape))
        out.append(P[o:o + n].reshape(shape))
        o += n
    return out


def mlp_infer(P, F, H, O, x) -> np.ndarray:
    """The MLP in the engine's FP32 order (fmaf chains, A&S GELU)."""
    P = _c(P, np.float32)
    x = _c(x, np.float32)
    y = np.empty(O, np.float32)
    lib().or_mlp_infer(_p(P), F, H, O, _p(x), _p(y))
    return y


def _gelu64(z):
    """GELU with the A&S 7.1.28 erf in FP64, and its derivative."""
    a1, a2, a3, a4, a5, a6 = 0.0705230784, 0.0422820123, 0.0092705272, 0.0001520143, 0.0002765672, 0.0000430638
    u = z / np.sqrt(2.0)
    a = np.abs(u)
    p = 1 + a * (a1 + a * (a2 + a * (a3 + a * (a4 + a * (a5 + a * a6)))))
    dp = a1 + a * (2 * a2 + a * (3 * a3 + a * (4 * a4 + a * (5 * a5 + a * 6 * a6))))
    e = 1 - p ** -16
    erf = np.sign(u) * e
    derf = 16 * p ** -17 * dp                  # d erf(u) / du (even in u)
    g = 0.5 * z * (1 + erf)
    dg = 0.5 * (1 + erf) + 0.5 * z * derf / np.sqrt(2.0)
    return g, dg


def mlp_forward64(P, F, H, O, X):
    """FP64 forward of a batch; returns outputs and the cache for mlp_backward64."""
    W1, b1, W2, b2, W3, b3 = (np.asarray(a, np.float64) for a in mlp_unpack(P, F, H, O))
    X = np.asarray(X, np.float64)
    Z1 = X @ W1 + b1
    H1, dH1 = _gelu64(Z1)
    Z2 = H1 @ W2 + b2
    H2, dH2 = _gelu64(Z2)
    Y = H2 @ W3 + b3
    return Y, (X, H1, dH1, H2, dH2)


def mlp_loss_grad64(P, F, H, O, X, T):
    """Mean squared error over all outputs and its gradient (FP64, packed like P)."""
    W1, b1, W2, b2, W3, b3 = (np.asarray(a, np.float64) for a in mlp_unpack(P, F, H, O))
    Y, (X, H1, dH1, H2, dH2) = mlp_forward64(P, F, H, O, X)
    B = X.shape[0]
    dY = 2.0 * (Y - T) / (B * O)
    loss = float(np.mean((Y - T) ** 2))
    gW3 = H2.T @ dY
    gb3 = dY.sum(0)
    dZ2 = (dY @ W3.T) * dH2
    gW2 = H1.T @ dZ2
    gb2 = dZ2.sum(0)
    dZ1 = (dZ2 @ W2.T) * dH1
    gW1 = X.T @ dZ1
    gb1 = dZ1.sum(0)
    return loss, np.concatenate([g.ravel() for g in (gW1, gb1, gW2, gb2, gW3, gb3)])


def features(V, Cand, N, first_cost, last_cost, M, k, t):
    V = _c(V, np.int32)
    Cand = _c(Cand, np.int32)
    fc = _c(first_cost, np.float32)
    lc = _c(last_cost, np.float32)
    f = np.empty(2 * M + 68, np.float32)
    lib().or_features(_p(V), _p(Cand), Cand.size, int(N), _p(fc), _p(lc), M, k, t, _p(f))
    return f


def depth(y, margin, lo, hi) -> int:
    return int(lib().or_depth(float(y), float(margin), int(lo), int(hi)))


def select_by_score(V, Cand, d):
    V = _c(V, np.int32)
    Cand = _c(Cand, np.int32)
    out = np.empty(max(1, Cand.size), np.int32)
    n = lib().or_select_by_score(_p(V), _p(Cand), Cand.size, int(d), _p(out))
    return out[:n].copy()


def activate_costs(ix: Index, qr, m, phi, k, bud):
    qr = _c(qr, np.float32)
    K2 = ix.K * ix.K
    cells = np.empty(K2, np.int32)
    w = np.empty(K2, np.uint8)
    got = C.c_int64()
    cf, cl = C.c_float(0.0), C.c_float(0.0)
    n = lib().or_activate_heap_costs(C.byref(ix.st()), _p(qr), m, phi, k, bud, _p(cells), _p(w), C.byref(got),
                                      C.byref(cf), C.byref(cl))
    return cells[:n].copy(), w[:n].copy(), got.value, np.float32(cf.value), np.float32(cl.value)


def learned_labels(ix: Index, Q, p: SearchParams):
    """Features and depth labels of each query, from the plain Guaranteed search:
    the minimal prefix of C by (V desc, id asc) holding the exact top-k over C,
    and the minimal coarse-score (BF16) prefix of that prefix holding them."""
    Q = np.atleast_2d(_c(Q, np.float32))
    if ix.Xb is None:
        ix.add_copies(bf16=True, fp8=False)
    F = 2 * ix.M + 68
    feats = np.empty((Q.shape[0], F), np.float32)
    labels = np.empty((Q.shape[0], 2), np.int64)
    for i in range(Q.shape[0]):
        qr = query_rotate(ix, Q[i])[0]
        bud = budget(p.rho, ix.N)
        acts, cf, cl = [], np.zeros(ix.M, np.float32), np.zeros(ix.M, np.float32)
        for m in range(ix.M):
            cells, w, got, a, b = activate_costs(ix, qr, m, 0, p.k, bud)
            acts.append((cells, w, got))
            cf[m], cl[m] = a, b
        V = scores_walk(ix, acts)
        t = tau(p.alpha, ix.M)
        Cand, _ = cut(V, t, p.k, p.max_candidates)
        feats[i] = features(V, Cand, ix.N, cf, cl, ix.M, p.k, t)
        top, _ = rerank(ix, qr, Cand, p.k)
        top = top[top >= 0]
        order = Cand[np.lexsort((Cand, -V[Cand]))]          # (V desc, id asc)
        pos = {int(c): j for j, c in enumerate(order)}
        dV = max(pos[int(r)] for r in top) + 1 if top.size else p.k
        P = np.sort(order[:dV])
        sc = np.array([prescore(qr, xb=ix.Xb[c]) for c in P], np.float32)
        co = P[np.lexsort((P, sc))]
        posS = {int(c): j for j, c in enumerate(co)}
        dS = max(posS[int(r)] for r in top) + 1 if top.size else p.k
        labels[i] = (dV, dS)
    return feats, labels
