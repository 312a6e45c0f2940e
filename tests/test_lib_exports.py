"""The C-ABI library loads without a GPU and exports every entry point that
include/crisp.h declares; argument errors are reported without touching a GPU."""
import ctypes
import os
import re

import pytest

from conftest import ROOT


def _declared():
    src = open(os.path.join(ROOT, "include", "crisp.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(crisp_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libc():
    import paper_2603_05180_gb300 as crisp
    from paper_2603_05180_gb300 import _build

    _build.build()
    return crisp.lib()


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("crisp_build", "crisp_search", "crisp_free", "crisp_index_export", "crisp_index_import",
              "crisp_activate", "crisp_count_cut", "crisp_rerank", "crisp_verify_opt", "crisp_cev"):
        assert n in names


def test_library_exports_every_declared_symbol(libc):
    missing = [n for n in _declared() if not hasattr(libc, n)]
    assert not missing, missing


def test_python_binding_wraps_every_symbol():
    import paper_2603_05180_gb300 as crisp

    for n in _declared():
        assert hasattr(crisp, n), n


def test_argument_errors_without_gpu(libc):
    import paper_2603_05180_gb300 as crisp

    with pytest.raises(crisp.CrispError) as e:
        crisp.crisp_index_import(b"not an index blob" * 20)
    assert e.value.status == crisp.CRISP_EINVAL
    with pytest.raises(crisp.CrispError) as e:
        crisp.crisp_search_scratch_bytes(crisp.Index(0), 10, crisp.search_params())
    assert e.value.status == crisp.CRISP_EINVAL
    assert libc.crisp_last_error() != b""
    for nq, G in ((16385, 64), (100, 0)):     # refused before any launch
        with pytest.raises(crisp.CrispError) as e:
            crisp.crisp_query_order(None, nq, 8, G, None)
        assert e.value.status == crisp.CRISP_EINVAL
    libc.crisp_free(None)   # NULL is a no-op


def test_oracle_blob_header_matches_documented_layout():
    import numpy as np
    import struct

    import oracle
    import synthetic

    X, _ = synthetic.small_gaussian(300, 64, 1)
    ix = oracle.build_index(X, M=2, K=8, draws=synthetic.method_draws(300, 64, 2, 8, kmeans_train=300))
    b = oracle.export_blob(ix)
    assert b[:8] == b"CRISPIX1"
    v, N, D, Dp, M, K, H, rot = struct.unpack_from("<8q", b, 8)
    assert (v, N, D, Dp, M, K, H) == (1, 300, 64, 64, 2, 8, 16)
    sizes = ([4 * D * D] if rot else []) + [4 * M * 2 * K * H, 4 * M * (K * K + 1), 4 * M * N, 4 * N * Dp,
                                            4 * N * (Dp // 32)]
    pos = 256
    for s in sizes:
        pos = (pos + s + 255) // 256 * 256
    assert len(b) == pos
    assert np.isclose(struct.unpack_from("<d", b, 72)[0], ix.cev)


def test_binding_constants_match_the_header():
    """Constants the binding restates must equal the header's #define values."""
    import paper_2603_05180_gb300 as crisp

    src = open(os.path.join(ROOT, "include", "crisp.h")).read()
    m = re.search(r"#define\s+CRISP_RERANK_NOALLOC_MAX\s+\(([^)]*)\)", src)
    assert m, "CRISP_RERANK_NOALLOC_MAX not found in include/crisp.h"
    assert eval(m.group(1), {"__builtins__": {}}) == crisp.CRISP_RERANK_NOALLOC_MAX


def test_library_readings_of_tau_and_budget_equal_the_oracle(libc):
    """The binding takes tau and the budget from the library (no copy of the
    arithmetic); they must equal the oracle's readings, including the exact
    products such as 0.3 x 10 = 3 that a plain ceil would round up."""
    import oracle
    import paper_2603_05180_gb300 as crisp

    for alpha in (0.0, 0.1, 0.125, 0.2, 0.25, 0.3, 0.5, 0.7, 1.0):
        for M in (1, 8, 10, 16, 20, 32, 127):
            assert crisp.tau(alpha, M) == oracle.tau(alpha, M), (alpha, M)
    for rho in (1e-9, 0.001, 0.002, 0.01, 0.03, 0.06, 0.3, 1.0):
        for N in (1, 300, 20000, 1_000_000, 5_000_000):
            assert crisp.budget(rho, N) == oracle.budget(rho, N), (rho, N)


def test_library_adaptive_bounds_equal_the_oracle(libc):
    """The library's variance-aware boundaries (host arithmetic) equal the
    oracle's reading on random, skewed, flat and zero variance profiles."""
    import numpy as np

    import oracle
    import paper_2603_05180_gb300 as crisp

    r = np.random.default_rng(8)
    cases = [(np.ones(960), 20), (np.zeros(300), 7), ([0.0] * 15 + [100.0], 4), ([1.0] * 10 + [0.0] * 490, 2)]
    for _ in range(150):
        D = int(r.integers(8, 1500))
        M = int(r.integers(max(1, -(-D // 256)), D // 2 + 1))
        cases.append((r.exponential(1.0, D) ** r.uniform(0.3, 5.0), M))
    for v, M in cases:
        assert np.array_equal(crisp.crisp_adaptive_bounds(v, M), oracle.adaptive_bounds(v, M))
    with pytest.raises(crisp.CrispError):
        crisp.crisp_adaptive_bounds(np.ones(600), 2)      # D > 256 M
