"""Pins of the oracle's learned re-rank depth (the engine's MLP extension):
the published erf error bound, the FP32 forward against an FP64 forward, FP64
gradients against central finite differences, hand-worked depth and selection
cases, and the special case where the learned mode reduces to plain search."""
import math

import numpy as np
import pytest

import oracle
import synthetic


def test_erf_as_within_published_bound():
    us = np.linspace(-6, 6, 4001)
    err = max(abs(float(oracle.erf_as(u)) - math.erf(u)) for u in us)
    assert err <= 2e-6        # A&S 7.1.28 bound (3e-7) plus the FP32 evaluation (16 ulp through the squarings)
    assert oracle.erf_as(0.0) == 0.0 and oracle.erf_as(-1.0) == -oracle.erf_as(1.0)


def test_gelu_matches_definition():
    for z in np.linspace(-8, 8, 321):
        ref = 0.5 * z * (1 + math.erf(z / math.sqrt(2)))
        assert abs(float(oracle.gelu(z)) - ref) <= 1e-6 * max(1.0, abs(z))


def _rand_model(F, H, O, seed):
    r = np.random.default_rng(seed)
    sizes = [(F, H), (H,), (H, H), (H,), (H, O), (O,)]
    parts = []
    for s in sizes:
        fan = s[0] if len(s) == 2 else 1
        parts.append((r.standard_normal(int(np.prod(s))) / math.sqrt(fan)).astype(np.float32))
    return np.concatenate(parts)


def test_fp32_forward_matches_fp64_forward():
    F, H, O = 36, 64, 2
    P = _rand_model(F, H, O, 0)
    X = np.random.default_rng(1).standard_normal((20, F)).astype(np.float32)
    Y64, _ = oracle.mlp_forward64(P, F, H, O, X)
    for i in range(20):
        y = oracle.mlp_infer(P, F, H, O, X[i])
        assert np.allclose(y, Y64[i], rtol=1e-4, atol=1e-4)


def test_gradients_match_finite_differences():
    F, H, O = 7, 9, 2
    P = _rand_model(F, H, O, 2).astype(np.float64)
    r = np.random.default_rng(3)
    X = r.standard_normal((11, F))
    T = r.standard_normal((11, O))
    loss, g = oracle.mlp_loss_grad64(P, F, H, O, X, T)
    h = 1e-6
    for j in range(P.size):
        e = np.zeros_like(P)
        e[j] = h
        fd = (oracle.mlp_loss_grad64(P + e, F, H, O, X, T)[0] - oracle.mlp_loss_grad64(P - e, F, H, O, X, T)[0]) / (2 * h)
        assert abs(fd - g[j]) <= 1e-6 + 1e-5 * abs(g[j]), j


def test_depth_quantisation_hand_values():
    assert oracle.depth(3.0, 0.0, 1, 10**9) == 8             # 4*3 = 12 -> 2^3
    assert oracle.depth(3.1, 0.0, 1, 10**9) == 10            # ceil(12.4) = 13 -> ceil(8 * 2^0.25 = 9.51)
    assert oracle.depth(3.0, 0.5, 1, 10**9) == 12            # 14 -> ceil(8 * sqrt 2 = 11.31)
    assert oracle.depth(10.0, 0.0, 1, 500) == 500            # clamped to hi
    assert oracle.depth(-5.0, 0.0, 10, 500) == 10            # clamped to lo
    assert oracle.depth(float("nan"), 0.0, 10, 500) == 500


def test_select_by_score_hand_example():
    V = np.array([0, 3, 1, 3, 2, 3], np.int32)
    C = np.array([1, 2, 3, 4, 5], np.int32)
    # (V desc, id asc): 1 (3), 3 (3), 5 (3), 4 (2), 2 (1)
    assert oracle.select_by_score(V, C, 2).tolist() == [1, 3]
    assert oracle.select_by_score(V, C, 4).tolist() == [1, 3, 4, 5]
    assert oracle.select_by_score(V, C, 9).tolist() == [1, 2, 3, 4, 5]


def test_features_hand_example():
    V = np.array([0, 2, 2, 5, 70], np.int32)
    C = np.array([1, 2, 3, 4], np.int32)
    f = oracle.features(V, C, 5, np.array([1.0, 2.0], np.float32), np.array([3.0, 5.0], np.float32), 2, 10, 2)
    assert f.size == 2 * 2 + 68
    assert f[2] == 0.5 and f[5] == 0.25 and f[63] == 0.25 and f[:64].sum() == 1.0
    assert np.allclose(f[64:68], [1 / 8, 2 / 8, 3 / 8, 5 / 8])
    assert np.allclose(f[68:], [4 / 5, 2 / 32, 10 / 256, 2 / 2])   # floor(log2 5) = 2


@pytest.fixture(scope="module")
def small():
    X, Q = synthetic.gmm(N=6000, D=64, nq=16, n_comp=20, rank=8, seed=7)
    ix = oracle.build_index(X, M=4, draws=synthetic.method_draws(6000, 64, 4, 50, seed=7)).add_copies(fp8=False)
    return ix, X, Q


def test_learned_with_full_depths_equals_plain(small):
    ix, X, Q = small
    F, H = 2 * ix.M + 68, 16
    P = _rand_model(F, H, 2, 4)
    ix.set_model(P, H)
    base = dict(k=10, rho=0.03, alpha=0.25)
    i0, d0, _, _ = oracle.search(ix, Q, oracle.SearchParams(mode=0, **base))
    i1, d1, s1, _ = oracle.search(ix, Q, oracle.SearchParams(mode=2, depth_margin=64.0, short_margin=64.0, **base))
    assert np.array_equal(i0, i1) and np.array_equal(d0, d1)


def test_labels_are_minimal_and_sufficient(small):
    ix, X, Q = small
    p = oracle.SearchParams(k=10, mode=0, rho=0.03, alpha=0.25)
    feats, labels = oracle.learned_labels(ix, Q, p)
    assert feats.shape == (Q.shape[0], 2 * ix.M + 68) and np.all(labels >= 1)
    plain = oracle.search(ix, Q, p)[0]
    for i in range(Q.shape[0]):
        det = oracle.query_detail(ix, Q[i], p)
        dV, dS = labels[i]
        assert dS <= dV <= det["C"].size
        for dv, ds, same in ((dV, dS, True), (dV - 1, min(dS, dV - 1), False)):
            if dv < 1 or ds < 1:
                continue
            P = oracle.select_by_score(det["V"], det["C"], dv)
            sl = oracle.shortlist(ix, det["qr"], P, ds, "bf16", ix.Xb)
            got = oracle.rerank(ix, det["qr"], sl, 10)[0]
            assert (set(got.tolist()) == set(plain[i].tolist())) == same or not same
        P = oracle.select_by_score(det["V"], det["C"], dV)
        sl = oracle.shortlist(ix, det["qr"], P, dS, "bf16", ix.Xb)
        assert np.array_equal(oracle.rerank(ix, det["qr"], sl, 10)[0], plain[i])
