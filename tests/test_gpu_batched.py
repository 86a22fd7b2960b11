"""Batched search (many probes x uneven subsets x mixed d, one graph) against
the plain search and the oracle, bit for bit."""
import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2003_12197_gb300 as H  # noqa: E402

KEY_SEED = 2024


@pytest.fixture(scope="module")
def setup():
    H.build_library()
    ctx = H.Context(0)
    keys = H.hers_keygen(ctx, KEY_SEED)
    # three subsets: (entries, d); the middle one has a ragged last block
    specs = [(2 * 4096, 16), (4096 + 1234, 37), (3 * 4096, 24)]
    nprobes = [3, 1, 5]          # 5 -> chunks of 4 + 1 at NP = 4
    subsets, items, truth = [], [], []
    for s, ((m, d), npb) in enumerate(zip(specs, nprobes)):
        feats = W.gallery_features(m, d, 300 + s)
        gal, _ = H.hers_encrypt_gallery(ctx, keys, torch.from_numpy(feats).cuda(), 400 + s)
        nb = H.hers_blocks_for(m)
        subsets.append((feats, gal, nb, d))
        for j in range(npb):
            mate = int(W.mate_indices(m, npb, 500 + s)[j])
            q = W.probe_for_mate(mate, d, 300 + s, 600 + 10 * s + j)
            pseed = 700 + 10 * s + j
            pct = H.hers_encrypt_probe(ctx, keys, torch.from_numpy(q).cuda(), pseed)
            pr = H.hers_probe_prepare(ctx, pct)
            items.append((gal, nb, d, pr))
            truth.append((s, q, mate, H.hers_search(ctx, keys, gal, nb, d, pr), pseed))
    # interleave items of different subsets to exercise the grouping
    order = [0, 3, 4, 1, 5, 6, 2, 7, 8]
    items = [items[i] for i in order]
    truth = [truth[i] for i in order]
    torch.cuda.synchronize()
    yield dict(ctx=ctx, keys=keys, subsets=subsets, items=items, truth=truth)
    keys.close()
    ctx.close()


@pytest.mark.parametrize("variant", range(32))
def test_batched_variant_equals_plain_search(setup, variant):
    names = H.hers_batch_variants()
    if variant >= len(names):
        pytest.skip("no such variant")
    b = H.Batch(setup["ctx"], setup["keys"], setup["items"], flags=H.batch_variant_flag(variant))
    b.run()
    b.run()  # a second run of the same graph gives the same bytes
    torch.cuda.synchronize()
    t_ms, all_ms = b.trace()  # the same launches outside the graph, timed
    assert 0 < t_ms <= all_ms
    info = b.info()
    assert info["variant"] == names[variant] and info["groups"] == 3
    for i, (_, nb, _, _) in enumerate(setup["items"]):
        assert torch.equal(b.item_scores(i, nb), setup["truth"][i][3]), f"item {i} ({names[variant]})"
    b.close()


def test_batched_autotune_scores_and_oracle(setup):
    ctx, keys = setup["ctx"], setup["keys"]
    b = H.Batch(ctx, keys, setup["items"], flags=H.BATCH_AUTOTUNE)
    sc = b.run()
    torch.cuda.synchronize()
    info = b.info()
    assert len(info["tune_ms"]) == len(H.hers_batch_variants())
    for i, (gal, nb, d, pr) in enumerate(setup["items"]):
        s, q, mate, _, _ = setup["truth"][i]
        feats = setup["subsets"][s][0]
        scores = H.hers_decrypt_scores(ctx, keys, b.item_scores(i, nb), feats.shape[0])
        scores = scores.cpu().numpy().astype(np.int64)
        assert np.array_equal(scores, W.plain_inner_products(feats, q))
        assert int(np.argmax(scores)) == mate
    # the ragged subset's last block of one item against the oracle directly
    _, opk, oevk = O.keygen(KEY_SEED)
    s, q, _, _, pseed = setup["truth"][1]
    feats, _, nb, d = setup["subsets"][s]
    ogal = O.encrypt_gallery_block(opk, feats, nb - 1, 400 + s)
    oprb = O.encrypt_probe(opk, q, pseed)
    osc, _ = O.search_block(oprb, ogal, oevk)
    assert np.array_equal(H.to_u64(b.item_scores(1, nb))[nb - 1], osc)
    b.close()


@pytest.mark.parametrize("epi", [1, 2, 3, 7, 8, 12, 16, 28])
def test_batched_with_every_epilogue_form(setup, epi):
    """A batch planned on a context with another epilogue form gives the same
    bytes as the plain search (the form is captured in the batch's graph)."""
    ctx = setup["ctx"]
    keep = H.hers_get_epilogue_variant(ctx)
    H.hers_set_epilogue_variant(ctx, epi)
    try:
        b = H.Batch(ctx, setup["keys"], setup["items"], flags=H.batch_variant_flag(1))
        b.run()
        torch.cuda.synchronize()
        for i, (_, nb, _, _) in enumerate(setup["items"]):
            assert torch.equal(b.item_scores(i, nb), setup["truth"][i][3]), f"item {i}"
        b.close()
    finally:
        H.hers_set_epilogue_variant(ctx, keep)
