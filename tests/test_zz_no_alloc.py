"""hers_search_noalloc, called through the C ABI, against hers_search.

hers_search_noalloc serves callers that cannot allocate device memory when
they search: its scratch is an array compiled into the library rather than
a workspace the caller allocates.  Its score ciphertexts must equal those of
hers_search bit for bit; ciphertexts are integers, so the tolerance is zero.
Two calls in a row with different probes also show that the contents a call
leaves in the shared scratch do not leak into the next result.

The file name makes pytest collect it last.
"""
import ctypes

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2003_12197_gb300 as H  # noqa: E402

HERS_E_INVAL = -1
MAX_BLOCKS = 8  # HERS_NOALLOC_MAX_BLOCKS in include/hers.h


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


def test_noalloc_search_matches_hers_search_on_two_calls():
    H.build_library()
    L = H.lib()
    ctx = H.Context(0)
    keys = H.hers_keygen(ctx, 4242)
    m, d = 6 * 4096 + 77, 48                     # 7 blocks, ragged last block
    nb = H.hers_blocks_for(m)
    assert nb <= MAX_BLOCKS
    feats = W.gallery_features(m, d, 4343)
    gal, _ = H.hers_encrypt_gallery(ctx, keys, torch.from_numpy(feats).cuda(), 4444)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call, mate in enumerate((123, m - 5)):     # two calls in a row, different probes
        q = W.probe_for_mate(mate, d, 4343, 4545 + call)
        pr = H.hers_probe_prepare(ctx, H.hers_encrypt_probe(ctx, keys, torch.from_numpy(q).cuda(),
                                                            4646 + call))
        want = H.hers_search(ctx, keys, gal, nb, d, pr)
        got = torch.full_like(want, -1)
        rc = L.hers_search_noalloc(ctx.h, keys.h, _p(gal), nb, d, _p(pr), _p(got), stream)
        assert rc == 0, L.hers_last_error(ctx.h)
        torch.cuda.synchronize()
        assert torch.equal(got, want), f"call {call}: score ciphertexts differ"
        scores = H.hers_decrypt_scores(ctx, keys, got, m).cpu().numpy().astype(np.int64)
        assert np.array_equal(scores, W.plain_inner_products(feats, q))
    # beyond the built-in scratch: rejected with a message, nothing launched
    rc = L.hers_search_noalloc(ctx.h, keys.h, _p(gal), MAX_BLOCKS + 1, d, _p(pr), _p(got), stream)
    assert rc == HERS_E_INVAL
    assert b"scratch" in L.hers_last_error(ctx.h)
    H.hers_check(ctx)
    keys.close()
    ctx.close()
