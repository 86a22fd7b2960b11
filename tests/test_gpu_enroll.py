"""Online single-entry enrollment (Alg 6, hers_enroll) against the oracle:
the updated block's search output bit for bit, and exact scores for the
enrolled entries."""
import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2003_12197_gb300 as H  # noqa: E402

KEY, GAL, PRB, ENR = 6101, 6102, 6103, 6104


def test_enroll_into_empty_slots_bit_exact():
    H.build_library()
    ctx = H.Context(0)
    keys = H.hers_keygen(ctx, KEY)
    _, opk, oevk = O.keygen(KEY)
    m, d = 4096 + 50, 16
    feats = W.gallery_features(m, d, 6105)
    new = W.gallery_features(3, d, 6106)                   # three entries to enroll
    slots = [(1, 50), (1, 4095), (1, 51)]                  # empty slots of block 1
    q = W.probe_for_mate(4096 + 7, d, 6105, 6107)
    gal, _ = H.hers_encrypt_gallery(ctx, keys, torch.from_numpy(feats).cuda(), GAL)
    nb = H.hers_blocks_for(m)
    for (b, v), f in zip(slots, new):
        H.hers_enroll(ctx, keys, gal, nb, d, b, v, torch.from_numpy(f).cuda(), ENR)
    pr = H.hers_probe_prepare(ctx, H.hers_encrypt_probe(ctx, keys, torch.from_numpy(q).cuda(), PRB))
    sc = H.hers_search(ctx, keys, gal, nb, d, pr)
    H.hers_check(ctx)
    got = H.to_u64(sc)
    # oracle: block 0 unchanged, block 1 with the three enrollments in order
    oprb = O.encrypt_probe(opk, q, PRB)
    blk0 = O.encrypt_gallery_block(opk, feats, 0, GAL)
    blk1 = O.encrypt_gallery_block(opk, feats, 1, GAL)
    for (b, v), f in zip(slots, new):
        blk1 = O.enroll(opk, blk1, b, v, f, ENR)
    assert np.array_equal(got[0], O.search_block(oprb, blk0, oevk)[0])
    assert np.array_equal(got[1], O.search_block(oprb, blk1, oevk)[0])
    # exact scores over all 2 N slots: enrolled entries in their slots, 0 in empty ones
    full = np.zeros((nb * 4096, d), dtype=np.int8)
    full[:m] = feats
    for (b, v), f in zip(slots, new):
        full[b * 4096 + v] = f
    scores = H.hers_decrypt_scores(ctx, keys, sc, nb * 4096).cpu().numpy().astype(np.int64)
    assert np.array_equal(scores, W.plain_inner_products(full, q))
    with pytest.raises(H.HersError):
        H.hers_enroll(ctx, keys, gal, nb, d, nb, 0, torch.from_numpy(new[0]).cuda(), ENR)
    with pytest.raises(H.HersError):
        H.hers_enroll(ctx, keys, gal, nb, d, 0, 4096, torch.from_numpy(new[0]).cuda(), ENR)
    H.hers_check(ctx)
    keys.close()
    ctx.close()
