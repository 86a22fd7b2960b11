"""The paper's plaintext modulus t = 1,032,193 (NEXT-1(a)): a context created
with it encrypts, searches and decrypts bit for bit like the oracle set to the
same t."""
import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2003_12197_gb300 as H  # noqa: E402


def test_paper_t_search_bit_exact():
    H.build_library()
    ctx = H.Context(0, t=H.T_PAPER)
    keys = H.hers_keygen(ctx, 8801)
    m, d = 4096 + 900, 32
    feats = W.gallery_features(m, d, 8802)
    mate = int(W.mate_indices(m, 1, 8803)[0])
    q = W.probe_for_mate(mate, d, 8802, 8804)
    gal, gct = H.hers_encrypt_gallery(ctx, keys, torch.from_numpy(feats).cuda(), 8805, want_ct=True)
    pct = H.hers_encrypt_probe(ctx, keys, torch.from_numpy(q).cuda(), 8806)
    pr = H.hers_probe_prepare(ctx, pct)
    nb = H.hers_blocks_for(m)
    sc = H.hers_search(ctx, keys, gal, nb, d, pr)
    scores = H.hers_decrypt_scores(ctx, keys, sc, m).cpu().numpy().astype(np.int64)
    # every epilogue form at this t (the fused scale-and-round takes its own
    # instantiation for the paper's t) gives the same bytes
    for v in range(1, len(H.hers_epilogue_variants())):
        H.hers_set_epilogue_variant(ctx, v)
        assert torch.equal(H.hers_search(ctx, keys, gal, nb, d, pr), sc), H.hers_epilogue_variants()[v]
    H.hers_set_epilogue_variant(ctx, 0)
    H.hers_check(ctx)
    O.set_plain_modulus(O.T_PAPER)
    try:
        _, opk, oevk = O.keygen(8801)
        oprb = O.encrypt_probe(opk, q, 8806)
        assert np.array_equal(H.to_u64(pct), oprb)
        for b in range(nb):
            ogal = O.encrypt_gallery_block(opk, feats, b, 8805)
            assert np.array_equal(H.to_u64(gct)[b], ogal), f"gallery block {b}"
            assert np.array_equal(H.to_u64(sc)[b], O.search_block(oprb, ogal, oevk)[0]), f"block {b}"
    finally:
        O.set_plain_modulus(O.T)
    assert np.array_equal(scores, W.plain_inner_products(feats, q))
    assert int(np.argmax(scores)) == mate
    # the default context gives different ciphertexts for the same seeds
    ctx2 = H.Context(0)
    keys2 = H.hers_keygen(ctx2, 8801)
    pct2 = H.hers_encrypt_probe(ctx2, keys2, torch.from_numpy(q).cuda(), 8806)
    assert not torch.equal(pct2, pct)
    keys2.close()
    ctx2.close()
    keys.close()
    ctx.close()
