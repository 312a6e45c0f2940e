"""CPU oracle of CRISP (arXiv 2603.05180) -- TEST INFRASTRUCTURE ONLY.

A plain, slow, obviously-correct restatement of what the GPU engine computes,
written from the paper: the index build of §4.1-§4.2 (covariance and CEV test,
random orthogonal rotation, IMI k-means per subspace half, cell assignment,
CSR, sign codes) and the query pipeline of Algorithm 1 / §4.3 (partial
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
                ("Xr", C.c_void_p), ("codes", C.c_void_p)]


class _OrParams(C.Structure):
    _fields_ = [("k", C.c_int32), ("mode", C.c_int32), ("rho", C.c_double), ("alpha", C.c_double),
                ("patience_factor", C.c_int32), ("eps0", C.c_float), ("max_candidates", C.c_int64)]


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
        "or_assign_cells": (None, [_P, _I64, _I32, _I32, _I32, _I32, _I32, _P, _P]),
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
        "or_verify_opt": (_I32, [_P, _P, _P, _P, _I64, _I32, _F, _I64, _P, _P, _P, _P]),
        "or_search_batch": (_I32, [_P, _P, _I64, _I32, _P, _P, _P, _P, _I32]),
        "or_knn_f64": (None, [_P, _I64, _I32, _I32, _P, _I64, _I32, _I32, _P, _P]),
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


def assign_cells(Xr, D, M, K, H, cent) -> np.ndarray:
    """u_m(x) = cL*K + cR for all rows and subspaces, [M][N] uint16 (§3, §4.2)."""
    Xr = _c(Xr, np.float32)
    cent = _c(cent, np.float32)
    N, Dp = Xr.shape
    cells = np.empty((M, N), np.uint16)
    lib().or_assign_cells(_p(Xr), N, D, Dp, M, K, H, _p(cent), _p(cells))
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
    _st: _OrIndex | None = field(default=None, repr=False)

    def st(self) -> _OrIndex:
        if self._st is None:
            self._st = _OrIndex(self.N, self.D, self.Dp, self.M, self.K, self.H, self.rotated, 0,
                                _p(self.R32).value if self.R32 is not None else None,
                                _p(self.cent).value, _p(self.offsets).value, _p(self.ids).value,
                                _p(self.Xr).value, _p(self.codes).value)
        return self._st


def build_index(X, M, K=50, draws=None, tau_cev=0.85, rotate=-1, kmeans_iters=20, seed=0) -> Index:
    """The index build of §4.1-§4.2 in order: CEV test, optional rotation,
    k-means per subspace half, cell assignment, CSR per subspace, sign codes.

    ``draws`` holds the random numbers the build uses (synthetic.method_draws);
    ``rotate`` is -1 (decide by CEV > tau_cev), 0 (never) or 1 (always)."""
    import synthetic

    X = _c(X, np.float32)
    N, D = X.shape
    if draws is None:
        draws = synthetic.method_draws(N, D, M, K, seed)
    Dp = padded_dim(D)
    H = half_width_max(D, M)
    cval, eig = cev(X, draws.cev_sample)
    do_rot = (rotate == 1) or (rotate == -1 and cval > tau_cev)
    R64 = R32 = None
    if do_rot:
        R64 = rotation_from_gaussian(draws.gaussian)
        R32 = R64.astype(np.float32)
        Xr = rotate_rows(X, R32, Dp)
    else:
        Xr = pad_rows(X, Dp)
    T = np.ascontiguousarray(Xr[draws.kmeans_sample])
    cent = np.zeros((M, 2, K, H), np.float32)
    for m in range(M):
        lo, hl, hr = subspace(D, M, m)
        cent[m, 0] = kmeans(T, lo, hl, K, H, draws.kmeans_init[m, 0], kmeans_iters)
        cent[m, 1] = kmeans(T, lo + hl, hr, K, H, draws.kmeans_init[m, 1], kmeans_iters)
    cells = assign_cells(Xr, D, M, K, H, cent)
    offsets = np.empty((M, K * K + 1), np.int32)
    ids = np.empty((M, N), np.int32)
    for m in range(M):
        offsets[m], ids[m] = csr(cells[m], K * K)
    codes = sign_codes(Xr)
    return Index(N, D, Dp, M, K, H, int(do_rot), float(cval), R32, cent, offsets, ids, Xr, codes, cells, R64, eig)


# Index blob: a 256-byte header (magic "CRISPIX1", then int64 version, N, D,
# Dp, M, K, H, rotated, and the CEV as a float64), then sections R32 (only if
# rotated), cent, offsets, ids, Xr, codes, each starting at a multiple of 256.
BLOB_MAGIC = b"CRISPIX1"
BLOB_VERSION = 1


def export_blob(ix: Index) -> bytes:
    hdr = bytearray(256)
    hdr[0:8] = BLOB_MAGIC
    struct.pack_into("<8q", hdr, 8, BLOB_VERSION, ix.N, ix.D, ix.Dp, ix.M, ix.K, ix.H, ix.rotated)
    struct.pack_into("<d", hdr, 72, ix.cev)
    parts = [bytes(hdr)]
    secs = ([ix.R32.astype(np.float32)] if ix.rotated else []) + [
        ix.cent.astype(np.float32), ix.offsets.astype(np.int32), ix.ids.astype(np.int32),
        ix.Xr.astype(np.float32), ix.codes.astype(np.uint32)]
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

    def st(self) -> _OrParams:
        return _OrParams(self.k, self.mode, self.rho, self.alpha, self.patience_factor, self.eps0,
                         self.max_candidates)


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


def verify_opt(ix: Index, qr, Cand, k, eps0=2.1, P=400):
    qr = _c(qr, np.float32)
    Cand = _c(Cand, np.int32)
    qcode = sign_codes(qr.reshape(1, -1))[0]
    ids = np.empty(k, np.int64)
    d2 = np.empty(k, np.float32)
    nv, nf = C.c_int64(), C.c_int64()
    lib().or_verify_opt(C.byref(ix.st()), _p(qr), _p(qcode), _p(Cand), Cand.size, k, float(eps0), int(P),
                        _p(ids), _p(d2), C.byref(nv), C.byref(nf))
    return ids, d2, nv.value, nf.value


def search(ix: Index, Q, params: SearchParams, nthreads: int = 0):
    """Algorithm 1 for a batch of queries: (ids [nq,k] int64, d2 [nq,k] f32, stats, threads used)."""
    Q = np.atleast_2d(_c(Q, np.float32))
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
