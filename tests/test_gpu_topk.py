"""Stage-1 top-K (hers_topk) against the oracle's plain definition (stable
order by descending score, ties by lowest index), bit for bit."""
import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2003_12197_gb300 as H  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    H.build_library()
    c = H.Context(0)
    yield c
    c.close()


def check(ctx, s_np, k):
    idx, val = H.hers_topk(ctx, torch.from_numpy(s_np).cuda(), k)
    H.hers_check(ctx)
    oi, ov = O.topk(s_np, k)
    assert np.array_equal(idx.cpu().numpy(), oi)
    assert np.array_equal(val.cpu().numpy(), ov)


@pytest.mark.parametrize("k", [1, 7, 1000, 4096])
def test_heavy_ties_ragged_size(ctx, k):
    rng = np.random.default_rng(11)
    s = rng.integers(-5, 6, size=1_000_003).astype(np.int32)   # ~91k copies of each value
    check(ctx, s, k)


def test_full_int32_range_and_extremes(ctx):
    rng = np.random.default_rng(12)
    s = rng.integers(-2**31, 2**31, size=100_000, dtype=np.int64).astype(np.int32)
    s[[5, 77, 99_999]] = [2**31 - 1, 2**31 - 1, -2**31]
    check(ctx, s, 4096)
    check(ctx, s, 3)


def test_tiny_and_exact_k_equals_m(ctx):
    check(ctx, np.array([42], dtype=np.int32), 1)
    s = np.array([3, -1, 3, 7, 3, 0, -1], dtype=np.int32)
    for k in range(1, 8):
        check(ctx, s, k)


def test_stage1_on_decrypted_search_scores(ctx):
    """The candidates of a real search: the planted mate first, and the list
    equal to the oracle's top-K of the plaintext inner products (Eq. 1)."""
    keys = H.hers_keygen(ctx, 91)
    m, d = 3 * 4096 + 100, 32
    feats = W.gallery_features(m, d, 92)
    mate = int(W.mate_indices(m, 1, 93)[0])
    q = W.probe_for_mate(mate, d, 92, 94)
    gal, _ = H.hers_encrypt_gallery(ctx, keys, torch.from_numpy(feats).cuda(), 95)
    pr = H.hers_probe_prepare(ctx, H.hers_encrypt_probe(ctx, keys, torch.from_numpy(q).cuda(), 96))
    sc = H.hers_search(ctx, keys, gal, H.hers_blocks_for(m), d, pr)
    scores = H.hers_decrypt_scores(ctx, keys, sc, m)
    idx, val = H.hers_topk(ctx, scores, 16)
    H.hers_check(ctx)
    oi, ov = O.topk(W.plain_inner_products(feats, q).astype(np.int32), 16)
    assert np.array_equal(idx.cpu().numpy(), oi) and np.array_equal(val.cpu().numpy(), ov)
    assert int(idx[0]) == mate
    keys.close()


def test_invalid_sizes_are_rejected(ctx):
    s = torch.zeros(10, dtype=torch.int32, device="cuda")
    for k in (0, 11, 5000):
        with pytest.raises(H.HersError):
            H.hers_topk(ctx, s, k)
    H.hers_check(ctx)
