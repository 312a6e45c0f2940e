"""Pins of the oracle's low-precision coarse scoring (the engine's BF16 / FP8
extension): hand-worked rounding cases, library conversions, and the special
cases where the coarse pass cannot change the result."""
import struct

import numpy as np
import pytest

import oracle
import synthetic
from conftest import load_golden


def _f32(bits):
    return struct.unpack("<f", struct.pack("<I", bits))[0]


def test_bf16_hand_worked_rounding():
    g = load_golden("bf16_e4m3_rounding.txt")
    for i, o in zip(g["bf16_in"], g["bf16_out"]):
        assert oracle.bf16_rne(_f32(int(i, 16))) == int(o, 16), i


def test_e4m3_hand_worked_rounding():
    g = load_golden("bf16_e4m3_rounding.txt")
    for i, o in zip(g["e4m3_in"], g["e4m3_out"]):
        assert oracle.e4m3_rne(float(i)) == int(o, 16), i


def test_conversions_agree_with_library_routines():
    torch = pytest.importorskip("torch")
    r = np.random.default_rng(0)
    xs = (r.standard_normal(20000) * 10.0 ** r.uniform(-7, 3, 20000)).astype(np.float32)
    tb = torch.from_numpy(xs).to(torch.bfloat16).view(torch.int16).numpy().astype(np.uint16)
    assert np.array_equal(tb, np.array([oracle.bf16_rne(x) for x in xs], np.uint16))
    inr = xs[np.abs(xs) < 448]
    t8 = torch.from_numpy(inr).to(torch.float8_e4m3fn).view(torch.uint8).numpy()
    assert np.array_equal(t8, np.array([oracle.e4m3_rne(x) for x in inr], np.uint8))
    for c in range(256):
        if c in (0x7F, 0xFF):
            continue
        ref = torch.tensor([c], dtype=torch.uint8).view(torch.float8_e4m3fn).float().item()
        assert oracle.e4m3_to_f32(c) == ref


def test_e4m3_row_scale_and_codes():
    x = np.zeros((2, 32), np.float32)
    x[0, :4] = [448.0, -224.0, 1.0, 0.0]          # max 448 -> scale 1, codes exact
    codes, sc = oracle.quantize_e4m3(x)
    assert sc[0] == 1.0 and sc[1] == 1.0            # the zero row keeps scale 1
    assert codes[0, :4].tolist() == [0x7E, 0xF6, 0x38, 0x00] and not codes[1].any()
    y = np.full((1, 32), 0.5, np.float32)
    y[0, 0] = 896.0                                 # scale 2: 896/2 = 448, 0.5/2 = 0.25 = 0x28
    codes, sc = oracle.quantize_e4m3(y)
    assert sc[0] == 2.0 and codes[0, 0] == 0x7E and codes[0, 1] == 0x28


def test_prescore_is_cr32_of_the_dequantised_row():
    r = np.random.default_rng(1)
    x = r.standard_normal((3, 64)).astype(np.float32)
    q = r.standard_normal(64).astype(np.float32)
    xb = oracle.quantize_bf16(x)
    x8, s8 = oracle.quantize_e4m3(x)
    for i in range(3):
        wide = (xb[i].astype(np.uint32) << 16).view(np.float32)
        assert oracle.prescore(q, xb=xb[i]) == oracle.cr32(wide, q)
        deq = np.array([oracle.e4m3_to_f32(c) for c in x8[i]], np.float32) * np.float32(s8[i])
        assert oracle.prescore(q, x8=x8[i], s8=s8[i]) == oracle.cr32(deq, q)
        # both stay close to the exact FP32 distance (2^-8 / 2^-4 relative per element)
        ex = float(np.sum((x[i].astype(np.float64) - q) ** 2))
        assert abs(float(oracle.prescore(q, xb=xb[i])) - ex) < 0.02 * ex
        assert abs(float(oracle.prescore(q, x8=x8[i], s8=s8[i])) - ex) < 0.25 * ex


@pytest.fixture(scope="module")
def gmm_q():
    X, Q = synthetic.gmm(N=6000, D=64, nq=20, n_comp=20, rank=8, seed=4)
    ix = oracle.build_index(X, M=4, draws=synthetic.method_draws(6000, 64, 4, 50, seed=4)).add_copies()
    return ix, X, Q


@pytest.mark.parametrize("precision", [1, 2])
def test_shortlist_covering_all_candidates_changes_nothing(gmm_q, precision):
    ix, X, Q = gmm_q
    base = oracle.SearchParams(k=10, mode=0, rho=0.03, alpha=0.25)
    i0, d0, s0, _ = oracle.search(ix, Q, base)
    p = oracle.SearchParams(k=10, mode=0, rho=0.03, alpha=0.25, precision=precision, shortlist=ix.N)
    i1, d1, s1, _ = oracle.search(ix, Q, p)
    assert np.array_equal(i0, i1) and np.array_equal(d0, d1)
    assert np.array_equal(s1["n_full"], s0["n_candidates"])


@pytest.mark.parametrize("precision", [1, 2])
def test_shortlist_is_the_coarse_top_s(gmm_q, precision):
    ix, X, Q = gmm_q
    p = oracle.SearchParams(k=10, mode=0, rho=0.03, alpha=0.25)
    quant = ix.Xb if precision == 1 else (ix.X8, ix.S8)
    for i in range(5):
        det = oracle.query_detail(ix, Q[i], p)
        C = det["C"]
        S = max(10, C.size // 3)
        sl = oracle.shortlist(ix, det["qr"], C, S, "bf16" if precision == 1 else "fp8", quant)
        assert sl.size == min(S, C.size) and np.all(np.diff(sl) > 0) and set(sl) <= set(C)
        if precision == 1:
            sc = np.array([oracle.prescore(det["qr"], xb=ix.Xb[c]) for c in C])
        else:
            sc = np.array([oracle.prescore(det["qr"], x8=ix.X8[c], s8=ix.S8[c]) for c in C])
        order = np.lexsort((C, sc))                  # (coarse distance, id)
        assert set(sl.tolist()) == set(C[order[:S]].tolist())


def test_bf16_shortlist_keeps_recall(gmm_q):
    ix, X, Q = gmm_q
    gi, gd = oracle.knn_f64(X, Q, 10)
    p0 = oracle.SearchParams(k=10, mode=0, rho=0.05, alpha=0.25)
    p1 = oracle.SearchParams(k=10, mode=0, rho=0.05, alpha=0.25, precision=1, shortlist=40)
    r0 = oracle.recall_at_k(oracle.search(ix, Q, p0)[0], gd, X, Q, 10)
    r1 = oracle.recall_at_k(oracle.search(ix, Q, p1)[0], gd, X, Q, 10)
    assert r1 >= r0 - 0.02


def test_search_rejects_missing_copies_and_model():
    """Asking for coarse scores or learned depths without the copy or the model
    is an error on the host, not a read through a null pointer."""
    import oracle as o
    import synthetic as sy

    X, Q = sy.small_gaussian(400, 64, 3, seed=4)
    ix = o.build_index(X, M=2, K=8, draws=sy.method_draws(400, 64, 2, 8, seed=4, kmeans_train=400))
    for kw in (dict(precision=1, shortlist=5), dict(precision=2, shortlist=5), dict(mode=2)):
        with pytest.raises(ValueError):
            o.search(ix, Q, o.SearchParams(k=3, rho=0.5, alpha=0.5, **kw))
