"""Python binding of the CRISP GB300 engine (arXiv 2603.05180).

A thin ctypes layer over ``libcrisp_gb300.so`` (built in-tree by
``_build.build()``): the functions below carry the C ABI's names
(include/crisp.h) and only marshal arguments.  Every step of the method runs in
the library's CUDA kernels; there is no CPU fallback, and every call fails
loudly when the library is missing.

Device buffers may be passed as torch CUDA tensors or as raw integer device
addresses; ``stream`` is a torch.cuda.Stream, a raw cudaStream_t integer, or
None (the current torch stream when torch is loaded, else the default stream).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libcrisp_gb300.so")
_lib = None

CRISP_OK, CRISP_EINVAL, CRISP_ENOMEM, CRISP_ECUDA, CRISP_ETIMEOUT, CRISP_EUNSUPPORTED = 0, -1, -2, -3, -4, -5
_STATUS = {0: "CRISP_OK", -1: "CRISP_EINVAL", -2: "CRISP_ENOMEM", -3: "CRISP_ECUDA", -4: "CRISP_ETIMEOUT",
           -5: "CRISP_EUNSUPPORTED"}


class CrispError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class BuildParams(C.Structure):
    _fields_ = [("M", C.c_int32), ("K", C.c_int32), ("tau_cev", C.c_double), ("rotate", C.c_int32),
                ("kmeans_iters", C.c_int32), ("kmeans_train", C.c_int64), ("seed", C.c_uint64),
                ("cev_sample", C.c_void_p), ("cev_sample_n", C.c_int64), ("gaussian", C.c_void_p),
                ("kmeans_sample", C.c_void_p), ("kmeans_sample_n", C.c_int64), ("kmeans_init", C.c_void_p),
                ("copies", C.c_uint32), ("adaptive", C.c_int32), ("block_dims", C.c_int32)]


class SearchParams(C.Structure):
    _fields_ = [("k", C.c_int32), ("mode", C.c_int32), ("rho", C.c_double), ("alpha", C.c_double),
                ("patience_factor", C.c_int32), ("eps0", C.c_float), ("max_candidates", C.c_int64),
                ("precision", C.c_int32), ("shortlist", C.c_int32), ("depth_margin", C.c_float),
                ("short_margin", C.c_float), ("verify_order", C.c_int32), ("reserved", C.c_int32)]


class QueryStats(C.Structure):
    _fields_ = [("n_candidates", C.c_int64), ("n_verified", C.c_int64), ("n_full", C.c_int64),
                ("n_retrieved", C.c_int64), ("fallback", C.c_int32), ("capped", C.c_int32), ("tau", C.c_int32),
                ("_pad", C.c_int32)]


class ServerParams(C.Structure):
    _fields_ = [("streams", C.c_int32), ("max_batch", C.c_int32), ("scratch_budget", C.c_int64)]


class ServerStats(C.Structure):
    _fields_ = [("submitted", C.c_uint64), ("completed", C.c_uint64), ("failed", C.c_uint64), ("batches", C.c_uint64),
                ("mean_batch", C.c_double), ("p50_us", C.c_double), ("p99_us", C.c_double), ("max_us", C.c_double),
                ("mean_us", C.c_double), ("scratch_peak", C.c_int64)]


class IndexInfo(C.Structure):
    _fields_ = [("N", C.c_int64), ("D", C.c_int32), ("Dp", C.c_int32), ("M", C.c_int32), ("K", C.c_int32),
                ("H", C.c_int32), ("rotated", C.c_int32), ("cev", C.c_double), ("max_cell", C.c_int32),
                ("id_tile_log2", C.c_int32), ("device_bytes", C.c_int64), ("R32", C.c_void_p),
                ("cent", C.c_void_p), ("offsets", C.c_void_p), ("ids", C.c_void_p), ("Xr", C.c_void_p),
                ("codes", C.c_void_p), ("Xb", C.c_void_p), ("X8", C.c_void_p), ("S8", C.c_void_p),
                ("sub", C.c_void_p), ("block_dims", C.c_int32), ("rotated_blocks", C.c_int32)]


class RerankProfile(C.Structure):
    _fields_ = [("launches", C.c_int64), ("ms", C.c_double), ("rows", C.c_int64), ("pairs", C.c_int64),
                ("Dp", C.c_int32), ("group", C.c_int32), ("elem_bytes", C.c_int32), ("_pad", C.c_int32)]


_P, _I32, _I64, _F, _D, _S = C.c_void_p, C.c_int32, C.c_int64, C.c_float, C.c_double, C.c_size_t
_SIGS = {
    "crisp_build": [_P, _I64, _I32, C.POINTER(BuildParams), _P, C.POINTER(_P)],
    "crisp_index_export": [_P, _P, C.POINTER(_S)],
    "crisp_index_import": [_P, _S, _P, C.POINTER(_P)],
    "crisp_index_get_info": [_P, C.POINTER(IndexInfo)],
    "crisp_index_get_bounds": [_P, _P],
    "crisp_index_add_copies": [_P, C.c_uint32, _P],
    "crisp_quantize_bf16": [_P, _I64, _I32, _P, _P],
    "crisp_quantize_e4m3": [_P, _I64, _I32, _P, _P, _P],
    "crisp_shortlist": [_P, _P, _I32, _P, _I64, _P, _I32, _I32, _P, _I64, _P, _P],
    "crisp_search": [_P, _P, _I32, _P, _I32, _P, _P, _I32, _P, _P],
    "crisp_search_host": [_P, _P, _I32, _P, _I32, _P, _P, _I32, _P, _P],
    "crisp_search_scratch_bytes": [_P, _I32, _P, _I32, C.POINTER(_S)],
    "crisp_search_tau": [_D, _I32],
    "crisp_rerank_profile_enable": [_I32],
    "crisp_rerank_profile_read": [C.POINTER(RerankProfile)],
    "crisp_search_budget": [_D, _I64],
    "crisp_covariance": [_P, _I64, _I32, _I32, _P, _I64, _P, _P],
    "crisp_eigvalsh": [_P, _I32, _P, _P],
    "crisp_cev": [_P, _I64, _I32, _I32, _P, _I64, C.POINTER(_D), _P],
    "crisp_rotation_from_gaussian": [_P, _I32, _P, _P],
    "crisp_rotate_rows": [_P, _I64, _I32, _I32, _P, _P, _I32, _P],
    "crisp_rotate_rows_tc": [_P, _I64, _I32, _I32, _P, _P, _I32, _P],
    "crisp_query_order": [_P, _I32, _I32, _I32, _P, _P],
    "crisp_kmeans": [_P, _I64, _I32, _I32, _I32, _I32, _I32, _P, _I32, _P, _P],
    "crisp_assign_cells": [_P, _I64, _I32, _I32, _I32, _I32, _I32, _P, _P, _P, _P],
    "crisp_assign_cells_tc": [_P, _P, _I64, _I32, _I32, _I32, _I32, _I32, _P, _P, _P, _P],
    "crisp_column_variance": [_P, _I64, _I32, _I32, _P, _I64, _P, _P],
    "crisp_adaptive_bounds": [_P, _I32, _I32, _P],
    "crisp_csr_build": [_P, _I64, _I32, _P, _P, _P],
    "crisp_sign_codes": [_P, _I64, _I32, _P, _P],
    "crisp_half_dists": [_P, _P, _I32, _P, _P, _P],
    "crisp_activate": [_P, _P, _I32, _I32, _I32, _I64, _P, _P, _P, _P],
    "crisp_count_cut": [_P, _P, _P, _I32, _I32, _I32, _I64, _P, _I64, _P, _P, _P, _P],
    "crisp_rerank": [_P, _P, _I32, _P, _I64, _P, _I32, _P, _P, _P],
    "crisp_rerank_noalloc": [_P, _P, _I32, _P, _I64, _P, _I32, _P, _P, _P],
    "crisp_activate_costs": [_P, _P, _I32, _I32, _I32, _I64, _P, _P, _P, _P, _P, _P],
    "crisp_mlp_init": [_P, _I32, _I32, _I32, C.c_uint64, _P],
    "crisp_mlp_infer": [_P, _I32, _I32, _I32, _P, _I64, _P, _P],
    "crisp_mlp_loss_grad": [_P, _I32, _I32, _I32, _P, _P, _I64, _P, _P, _P],
    "crisp_mlp_adam": [_P, _P, _P, _P, _I64, _F, _F, _F, _F, _I32, _P],
    "crisp_mlp_train": [_P, _I32, _I32, _I32, _P, _P, _I64, _I32, _I32, _F, C.c_uint64, _P, _P],
    "crisp_index_set_model": [_P, _P, _I32, _P],
    "crisp_learned_data": [_P, _P, _I32, C.POINTER(SearchParams), _P, _P, _P, _P],
    "crisp_server_create": [_P, C.POINTER(ServerParams), C.POINTER(_P)],
    "crisp_server_submit": [_P, _P, C.POINTER(SearchParams), C.POINTER(C.c_uint64)],
    "crisp_server_wait": [_P, C.c_uint64, _I32, _P, _P, _P, C.POINTER(C.c_double)],
    "crisp_server_get_stats": [_P, C.POINTER(ServerStats)],
    "crisp_server_reset_stats": [_P],
    "crisp_server_replay": [_P, _P, _I32, _I64, _P, _P, _I32, _P, _P, _I32, _P, _P, _P, C.POINTER(C.c_double)],
    "crisp_verify_opt": [_P, _P, _I32, _P, _I64, _P, _I32, _F, _I64, _I32, _P, _P, _P, _P, _P, _P],
}


def lib():
    """Load the CUDA library (raises if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CRISP CUDA library missing ({LIB_PATH}); build it with __graft_entry__.build()")
        L = C.CDLL(LIB_PATH)
        for name, args in _SIGS.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = C.c_int
        L.crisp_mlp_param_count.argtypes = [_I32, _I32, _I32]
        L.crisp_mlp_param_count.restype = C.c_int64
        L.crisp_server_destroy.argtypes = [_P]
        L.crisp_server_destroy.restype = None
        L.crisp_free.argtypes = [_P]
        L.crisp_free.restype = None
        L.crisp_last_error.argtypes = []
        L.crisp_last_error.restype = C.c_char_p
        L.crisp_search_tau.restype = C.c_int32
        L.crisp_search_budget.restype = C.c_int64
        _lib = L
    return _lib


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if hasattr(x, "ctypes"):          # numpy array (host)
        return x.ctypes.data
    raise TypeError(f"cannot pass {type(x)} as a pointer")


def _stream(s):
    if s is None:
        import sys

        if "torch" in sys.modules:
            import torch

            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        return None
    if isinstance(s, int):
        return s
    return s.cuda_stream


def _check(st):
    if st != 0:
        raise CrispError(st, lib().crisp_last_error().decode(errors="replace"))


def _call(name, *args):
    _check(getattr(lib(), name)(*args))


# ------------------------------------------------------------------ index
class Index:
    """Owner of a crisp_index handle (freed with crisp_free)."""

    def __init__(self, handle: int):
        self.handle = handle

    def info(self) -> IndexInfo:
        return crisp_index_get_info(self)

    def free(self):
        if self.handle:
            lib().crisp_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    @property
    def _as_parameter_(self):
        return C.c_void_p(self.handle)


def crisp_build(X, N, D, params: BuildParams, stream=None) -> Index:
    out = C.c_void_p()
    _call("crisp_build", _ptr(X), N, D, C.byref(params), _stream(stream), C.byref(out))
    return Index(out.value)


def crisp_free(index: Index):
    index.free()


def crisp_index_export(index: Index) -> bytes:
    n = C.c_size_t(0)
    _call("crisp_index_export", index, None, C.byref(n))
    buf = C.create_string_buffer(n.value)
    _call("crisp_index_export", index, buf, C.byref(n))
    return buf.raw[: n.value]


def crisp_index_import(blob: bytes, stream=None) -> Index:
    out = C.c_void_p()
    buf = C.create_string_buffer(blob, len(blob))
    _call("crisp_index_import", buf, len(blob), _stream(stream), C.byref(out))
    return Index(out.value)


def crisp_index_get_info(index: Index) -> IndexInfo:
    info = IndexInfo()
    _call("crisp_index_get_info", index, C.byref(info))
    return info


def crisp_index_get_bounds(index: Index) -> np.ndarray:
    """Subspace boundaries [M+1] of an index (host int32)."""
    out = np.empty(crisp_index_get_info(index).M + 1, np.int32)
    _call("crisp_index_get_bounds", index, _ptr(out))
    return out


def crisp_index_add_copies(index, copies, stream=None):
    """Add BF16 (bit 0) and/or FP8 E4M3 (bit 1) copies of the stored rows."""
    _call("crisp_index_add_copies", index, copies, _stream(stream))


def crisp_quantize_bf16(Xr, N, Dp, Xb, stream=None):
    _call("crisp_quantize_bf16", _ptr(Xr), N, Dp, _ptr(Xb), _stream(stream))


def crisp_quantize_e4m3(Xr, N, Dp, X8, scale, stream=None):
    _call("crisp_quantize_e4m3", _ptr(Xr), N, Dp, _ptr(X8), _ptr(scale), _stream(stream))


def crisp_shortlist(index, Qr, nq, cand, cand_stride, ncand, precision, S, out, out_stride, nout, stream=None):
    _call("crisp_shortlist", index, _ptr(Qr), nq, _ptr(cand), cand_stride, _ptr(ncand), precision, S, _ptr(out),
          out_stride, _ptr(nout), _stream(stream))


def _param_array(params):
    """One SearchParams (shared by every query) or a sequence of them (one per query)."""
    if isinstance(params, SearchParams):
        return (SearchParams * 1)(params), 1, params.k
    arr = (SearchParams * len(params))(*params)
    return arr, len(params), max((p.k for p in params), default=1)


def _kmax(ids, kbig, kmax):
    if kmax is not None:
        return int(kmax)
    shape = getattr(ids, "shape", None)
    return int(shape[1]) if shape is not None and len(shape) == 2 else kbig


def crisp_search(index, Q, nq, params, ids, sqdist, stats=None, stream=None, kmax=None):
    """params: one SearchParams for every query, or one per query (p_count = nq);
    ids / sqdist rows of kmax entries (default: their second dimension)."""
    arr, n, kbig = _param_array(params)
    _call("crisp_search", index, _ptr(Q), nq, C.cast(arr, C.c_void_p), n, _ptr(ids), _ptr(sqdist),
          _kmax(ids, kbig, kmax), _ptr(stats), _stream(stream))


def crisp_search_host(index, Q, nq, params, ids, sqdist, stats=None, stream=None, kmax=None):
    arr, n, kbig = _param_array(params)
    _call("crisp_search_host", index, _ptr(Q), nq, C.cast(arr, C.c_void_p), n, _ptr(ids), _ptr(sqdist),
          _kmax(ids, kbig, kmax), _ptr(stats), _stream(stream))


def crisp_search_scratch_bytes(index, nq, params) -> int:
    arr, n, _ = _param_array(params)
    out = C.c_size_t(0)
    _call("crisp_search_scratch_bytes", index, nq, C.cast(arr, C.c_void_p), n, C.byref(out))
    return int(out.value)


def crisp_covariance(X, N, D, ldx, rows, S, cov, stream=None):
    _call("crisp_covariance", _ptr(X), N, D, ldx, _ptr(rows), S, _ptr(cov), _stream(stream))


def crisp_eigvalsh(A, D, eig, stream=None):
    _call("crisp_eigvalsh", _ptr(A), D, _ptr(eig), _stream(stream))


def crisp_cev(X, N, D, ldx, rows, S, stream=None) -> float:
    out = C.c_double(0.0)
    _call("crisp_cev", _ptr(X), N, D, ldx, _ptr(rows), S, C.byref(out), _stream(stream))
    return out.value


def crisp_rotation_from_gaussian(G, D, R, stream=None):
    _call("crisp_rotation_from_gaussian", _ptr(G), D, _ptr(R), _stream(stream))


def crisp_rotate_rows(X, N, D, ldx, R, Y, ldy, stream=None):
    _call("crisp_rotate_rows", _ptr(X), N, D, ldx, _ptr(R), _ptr(Y), ldy, _stream(stream))


def crisp_rotate_rows_tc(X, N, D, ldx, R, Y, ldy, stream=None):
    _call("crisp_rotate_rows_tc", _ptr(X), N, D, ldx, _ptr(R), _ptr(Y), ldy, _stream(stream))


def crisp_query_order(Qr, nq, Dp, G, qord, stream=None):
    _call("crisp_query_order", _ptr(Qr), nq, Dp, G, _ptr(qord), _stream(stream))


def crisp_kmeans(T, S, ldt, off, h, K, H, init, iters, Cout, stream=None):
    _call("crisp_kmeans", _ptr(T), S, ldt, off, h, K, H, _ptr(init), iters, _ptr(Cout), _stream(stream))


def _host_i32(a):
    return None if a is None else np.ascontiguousarray(np.asarray(a), dtype=np.int32)


def crisp_assign_cells(Xr, N, D, Dp, M, K, H, cent, cells, stream=None, sub=None):
    """``sub``: host subspace boundaries [M+1] (None: the equal split)."""
    sb = _host_i32(sub)
    _call("crisp_assign_cells", _ptr(Xr), N, D, Dp, M, K, H, _ptr(sb), _ptr(cent), _ptr(cells), _stream(stream))


def crisp_assign_cells_tc(Xr, N, D, Dp, M, K, H, cent, cells, stream=None, sub=None, Xb=None):
    """``Xb``: the BF16 copy of ``Xr`` (device) for the BF16 pass; None: one TF32 pass."""
    sb = _host_i32(sub)
    _call("crisp_assign_cells_tc", _ptr(Xr), _ptr(Xb), N, D, Dp, M, K, H, _ptr(sb), _ptr(cent), _ptr(cells),
          _stream(stream))


def crisp_column_variance(X, N, D, ldx, rows, S, var, stream=None):
    _call("crisp_column_variance", _ptr(X), N, D, ldx, _ptr(rows), S, _ptr(var), _stream(stream))


def crisp_adaptive_bounds(var, M) -> np.ndarray:
    """Variance-aware boundaries [M+1] from host per-dimension variances."""
    v = np.ascontiguousarray(np.asarray(var), dtype=np.float64)
    out = np.empty(M + 1, np.int32)
    _call("crisp_adaptive_bounds", _ptr(v), v.size, M, _ptr(out))
    return out


def crisp_csr_build(cells, N, K2, offsets, ids, stream=None):
    _call("crisp_csr_build", _ptr(cells), N, K2, _ptr(offsets), _ptr(ids), _stream(stream))


def crisp_sign_codes(Xr, N, Dp, codes, stream=None):
    _call("crisp_sign_codes", _ptr(Xr), N, Dp, _ptr(codes), _stream(stream))


def crisp_half_dists(index, Qr, nq, sorted_out, perm, stream=None):
    _call("crisp_half_dists", index, _ptr(Qr), nq, _ptr(sorted_out), _ptr(perm), _stream(stream))


def crisp_activate(index, Qr, nq, phi, k, budget, act, nact, retrieved=None, stream=None):
    _call("crisp_activate", index, _ptr(Qr), nq, phi, k, budget, _ptr(act), _ptr(nact), _ptr(retrieved),
          _stream(stream))


def crisp_count_cut(index, act, nact, nq, tau, k, cap, cand, cand_stride, ncand, score=None, how=None, stream=None):
    _call("crisp_count_cut", index, _ptr(act), _ptr(nact), nq, tau, k, cap, _ptr(cand), cand_stride, _ptr(ncand),
          _ptr(score), _ptr(how), _stream(stream))


def crisp_rerank(index, Qr, nq, cand, cand_stride, ncand, k, ids, sqdist, stream=None):
    _call("crisp_rerank", index, _ptr(Qr), nq, _ptr(cand), cand_stride, _ptr(ncand), k, _ptr(ids), _ptr(sqdist),
          _stream(stream))


def crisp_rerank_noalloc(index, Qr, nq, cand, cand_stride, ncand, k, ids, sqdist, stream=None):
    """crisp_rerank without any device allocation (fixed 16 MiB scratch; see include/crisp.h)."""
    _call("crisp_rerank_noalloc", index, _ptr(Qr), nq, _ptr(cand), cand_stride, _ptr(ncand), k, _ptr(ids),
          _ptr(sqdist), _stream(stream))


CRISP_RERANK_NOALLOC_MAX = 4 * 1024 * 1024


def crisp_verify_opt(index, Qr, nq, cand, cand_stride, ncand, k, eps0, patience, ids, sqdist, n_verified=None,
                     n_full=None, n_blocks=None, stream=None, order=0):
    _call("crisp_verify_opt", index, _ptr(Qr), nq, _ptr(cand), cand_stride, _ptr(ncand), k, float(eps0), patience,
          order, _ptr(ids), _ptr(sqdist), _ptr(n_verified), _ptr(n_full), _ptr(n_blocks), _stream(stream))


# ------------------------------------------------------------ conveniences
def crisp_search_tau(alpha: float, M: int) -> int:
    """The library's tau for a minimum collision fraction alpha (Theorem 1's tau = alpha M)."""
    return int(lib().crisp_search_tau(float(alpha), int(M)))


def crisp_search_budget(rho: float, N: int) -> int:
    """The library's per-subspace retrieval budget for coverage rho (Algorithm 1)."""
    return int(lib().crisp_search_budget(float(rho), int(N)))


tau = crisp_search_tau
budget = crisp_search_budget


def search_params(k=10, mode=0, rho=0.01, alpha=0.3, patience_factor=40, eps0=2.1, max_candidates=0, precision=0,
                  shortlist=0, depth_margin=0.0, short_margin=0.0, verify_order=0) -> SearchParams:
    return SearchParams(k, mode, rho, alpha, patience_factor, eps0, max_candidates, precision, shortlist, depth_margin,
                        short_margin, verify_order, 0)


def build_params(M, K=50, tau_cev=0.85, rotate=-1, kmeans_iters=20, kmeans_train=100000, seed=0, draws=None,
                 copies=0, adaptive=0, block_dims=0):
    """BuildParams; ``draws`` (host numpy arrays: cev_sample, gaussian,
    kmeans_sample, kmeans_init) are referenced by the returned struct."""
    p = BuildParams(M, K, tau_cev, rotate, kmeans_iters, kmeans_train, seed, None, 0, None, None, 0, None, copies,
                    adaptive, block_dims)
    p._draws = draws          # the struct holds raw pointers into these arrays: keep them alive with it
    if draws is not None:
        p.cev_sample = draws.cev_sample.ctypes.data
        p.cev_sample_n = draws.cev_sample.size
        p.gaussian = draws.gaussian.ctypes.data
        p.kmeans_sample = draws.kmeans_sample.ctypes.data
        p.kmeans_sample_n = draws.kmeans_sample.size
        p.kmeans_init = draws.kmeans_init.ctypes.data
    return p


def crisp_kernel_launches() -> int:
    f = lib().crisp_kernel_launches
    f.restype = C.c_uint64
    return int(f())


def crisp_last_error() -> str:
    return lib().crisp_last_error().decode(errors="replace")


def crisp_activate_costs(index, Qr, nq, phi, k, budget, act, nact, retrieved=None, cost_first=None, cost_last=None,
                         stream=None):
    _call("crisp_activate_costs", index, _ptr(Qr), nq, phi, k, budget, _ptr(act), _ptr(nact), _ptr(retrieved),
          _ptr(cost_first), _ptr(cost_last), _stream(stream))


# ------------------------------------------------- learned re-rank depth (F1)
def crisp_mlp_param_count(F, H, O) -> int:
    return int(lib().crisp_mlp_param_count(F, H, O))


def crisp_mlp_init(params, F, H, O, seed=0, stream=None):
    _call("crisp_mlp_init", _ptr(params), F, H, O, seed, _stream(stream))


def crisp_mlp_infer(params, F, H, O, X, B, Y, stream=None):
    _call("crisp_mlp_infer", _ptr(params), F, H, O, _ptr(X), B, _ptr(Y), _stream(stream))


def crisp_mlp_loss_grad(params, F, H, O, X, T, B, grads, loss, stream=None):
    _call("crisp_mlp_loss_grad", _ptr(params), F, H, O, _ptr(X), _ptr(T), B, _ptr(grads), _ptr(loss), _stream(stream))


def crisp_mlp_adam(params, grads, m, v, n, lr, beta1, beta2, eps, t, stream=None):
    _call("crisp_mlp_adam", _ptr(params), _ptr(grads), _ptr(m), _ptr(v), n, lr, beta1, beta2, eps, t, _stream(stream))


def crisp_mlp_train(params, F, H, O, X, T, n, epochs, batch, lr, seed=0, stream=None):
    """Train in place; returns the mean loss of each epoch."""
    losses = (C.c_float * max(1, epochs))()
    _call("crisp_mlp_train", _ptr(params), F, H, O, _ptr(X), _ptr(T), n, epochs, batch, lr, seed, losses,
          _stream(stream))
    return [float(x) for x in losses[:epochs]]


def crisp_index_set_model(index, params, H, stream=None):
    _call("crisp_index_set_model", index, _ptr(params), H, _stream(stream))


def crisp_learned_data(index, Q, nq, params: SearchParams, features, labels, targets=None, stream=None):
    _call("crisp_learned_data", index, _ptr(Q), nq, C.byref(params), _ptr(features), _ptr(labels), _ptr(targets),
          _stream(stream))


# ------------------------------------------------------------ serving (F3)
class Server:
    """Owner of a crisp_server handle (crisp_server_destroy on free)."""

    def __init__(self, handle, D):
        self.handle = handle
        self.D = D

    def free(self):
        if self.handle:
            lib().crisp_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    @property
    def _as_parameter_(self):
        return C.c_void_p(self.handle)


def crisp_server_create(index, streams=2, max_batch=256, scratch_budget=0) -> Server:
    out = C.c_void_p()
    _call("crisp_server_create", index, C.byref(ServerParams(streams, max_batch, scratch_budget)), C.byref(out))
    return Server(out.value, index.info().D)


def crisp_server_submit(server, q, params: SearchParams) -> int:
    """q: host float32 array of D values."""
    t = C.c_uint64(0)
    _call("crisp_server_submit", server, _ptr(q), C.byref(params), C.byref(t))
    return t.value


def crisp_server_wait(server, ticket, k, timeout_ms=-1, with_stats=False):
    """(ids int64 [k], sqdist float32 [k], latency_us[, stats])."""
    import numpy as np

    ids = np.empty(k, np.int64)
    d2 = np.empty(k, np.float32)
    st = QueryStats()
    lat = C.c_double(0.0)
    _call("crisp_server_wait", server, ticket, timeout_ms, _ptr(ids), _ptr(d2), C.byref(st), C.byref(lat))
    return (ids, d2, lat.value, st) if with_stats else (ids, d2, lat.value)


def crisp_server_get_stats(server) -> ServerStats:
    s = ServerStats()
    _call("crisp_server_get_stats", server, C.byref(s))
    return s


def crisp_server_reset_stats(server):
    _call("crisp_server_reset_stats", server)


def crisp_server_replay(server, Q, qidx, params, pidx, arrival_us, kmax):
    """Open-loop replay of a request trace (host arrays): request i asks
    Q[qidx[i]] with params[pidx[i]] at arrival_us[i].  Returns
    (ids int64 [n][kmax], sqdist float32 [n][kmax], latency_us float64 [n], wall_us)."""
    import numpy as np

    Q = np.ascontiguousarray(Q, np.float32)
    qidx = np.ascontiguousarray(qidx, np.int32)
    pidx = np.ascontiguousarray(pidx, np.int32)
    arr = np.ascontiguousarray(arrival_us, np.float64)
    n = qidx.shape[0]
    P = (SearchParams * max(1, len(params)))(*params)
    ids = np.empty((n, kmax), np.int64)
    d2 = np.empty((n, kmax), np.float32)
    lat = np.empty(n, np.float64)
    wall = C.c_double(0.0)
    _call("crisp_server_replay", server, _ptr(Q), Q.shape[0], n, _ptr(qidx), C.cast(P, C.c_void_p), len(params),
          _ptr(pidx),
          _ptr(arr), kmax, _ptr(ids), _ptr(d2), _ptr(lat), C.byref(wall))
    return ids, d2, lat, wall.value


def crisp_server_destroy(server):
    server.free()


def crisp_rerank_profile_enable(on=True):
    """Record CUDA events around the tensor-core re-rank's scoring kernel (profiling aid)."""
    _call("crisp_rerank_profile_enable", int(bool(on)))


def crisp_rerank_profile_read() -> RerankProfile:
    """Launches, summed duration (ms) and work counts of the scoring kernel since the last read."""
    out = RerankProfile()
    _call("crisp_rerank_profile_read", C.byref(out))
    return out
