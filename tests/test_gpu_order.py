"""The query order of the grouped scorers (crisp_query_order): a permutation
whose runs of G entries are the groups.

Which queries share a group never changes a search result (the grouped
parity suites check that), so the order is pinned here by what it must do
on batches whose answer is plain: when the batch is made of well-separated
clusters of exactly G identical queries, every group is one cluster (the
k-d splits fall at multiples of G and identical queries sort next to each
other), for groups of 64 (the k-d leaves) and of 16 (leaves split further).
Ragged and tiny batches must still give permutations, and oversize batches
are refused before any launch."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2603_05180_gb300 as crisp  # noqa: E402

DEV = torch.device("cuda:0")


def _order(Q, G):
    nq, Dp = Q.shape
    qord = torch.full((max(nq, 1),), -1, dtype=torch.int32, device=DEV)
    crisp.crisp_query_order(torch.from_numpy(np.ascontiguousarray(Q, np.float32)).to(DEV), nq, Dp, G, qord)
    return qord.cpu().numpy()[:nq]


@pytest.mark.parametrize("G,C,D", [(64, 40, 96), (16, 100, 96), (64, 200, 960), (16, 256, 33)])
def test_clusters_of_g_identical_queries_fill_one_group_each(G, C, D):
    r = np.random.default_rng(G * 1000 + C)
    centers = r.standard_normal((C, D)).astype(np.float32) * 10.0
    label = np.repeat(np.arange(C), G)
    perm = r.permutation(C * G)
    Q, label = centers[label[perm]], label[perm]
    o = _order(Q, G)
    assert np.array_equal(np.sort(o), np.arange(C * G))
    groups = label[o].reshape(C, G)
    assert np.all(groups == groups[:, :1]), "a group mixes clusters"
    assert np.array_equal(np.sort(groups[:, 0]), np.arange(C))


@pytest.mark.parametrize("nq,G", [(1, 64), (63, 64), (64, 64), (65, 64), (1000, 64), (1000, 16), (1031, 128),
                                  (16384, 64), (3000, 16)])
def test_any_batch_gives_a_permutation(nq, G):
    r = np.random.default_rng(nq + G)
    Q = r.standard_normal((nq, 40)).astype(np.float32)
    Q[: nq // 3] = Q[0]                        # many ties
    o = _order(Q, G)
    assert np.array_equal(np.sort(o), np.arange(nq))
    # deterministic
    assert np.array_equal(o, _order(Q, G))


def test_order_follows_the_leading_direction():
    """Queries on a line (one dominant direction): each group of 64 holds 64
    consecutive positions along the line."""
    nq, D = 2048, 64
    r = np.random.default_rng(3)
    t = r.permutation(nq).astype(np.float32)
    u = r.standard_normal(D).astype(np.float32)
    u /= np.linalg.norm(u)
    Q = t[:, None] * u[None, :] + 1e-3 * r.standard_normal((nq, D)).astype(np.float32)
    o = _order(Q, 64)
    g = np.sort(t[o].reshape(-1, 64), axis=1)
    assert np.all(g[:, -1] - g[:, 0] == 63)


def test_argument_errors():
    Q = torch.zeros((16385, 8), dtype=torch.float32, device=DEV)
    qord = torch.zeros((16385,), dtype=torch.int32, device=DEV)
    with pytest.raises(crisp.CrispError) as e:
        crisp.crisp_query_order(Q, 16385, 8, 64, qord)
    assert e.value.status == crisp.CRISP_EINVAL
    for nq, Dp, G in ((100, 8, 0), (100, 0, 64), (-1, 8, 64)):
        with pytest.raises(crisp.CrispError) as e:
            crisp.crisp_query_order(Q, nq, Dp, G, qord)
        assert e.value.status == crisp.CRISP_EINVAL
