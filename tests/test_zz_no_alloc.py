"""hers_search_noalloc, called through the C ABI, against hers_search.

hers_search_noalloc serves callers that cannot allocate device memory when
they search: its scratch is an array compiled into the library rather than
a workspace the caller allocates.  Its score ciphertexts must equal those of
hers_search bit for bit; ciphertexts are integers, so the tolerance is zero.
Two calls in a row with different probes also show that the contents a call
leaves in the shared scratch do not leak into the next result.  Searches of
exactly HERS_NOALLOC_MAX_BLOCKS blocks (a full and a ragged last block) fill
the array to its end.  Both entry points run on one explicit stream.

The file name makes pytest collect it last.
"""
import ctypes
import os
import re

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2003_12197_gb300 as H  # noqa: E402

HERS_E_INVAL = -1


def _max_blocks():
    """HERS_NOALLOC_MAX_BLOCKS as include/hers.h defines it."""
    hdr = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "hers.h")
    m = re.search(r"#define\s+HERS_NOALLOC_MAX_BLOCKS\s+(\d+)u?", open(hdr).read())
    assert m, "HERS_NOALLOC_MAX_BLOCKS not found in include/hers.h"
    return int(m.group(1))


MAX_BLOCKS = _max_blocks()


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


@pytest.fixture(scope="module")
def env():
    H.build_library()
    ctx = H.Context(0)
    keys = H.hers_keygen(ctx, 4242)
    yield ctx, keys
    keys.close()
    ctx.close()


def _compare(env, m, d, mates, seed):
    """Searches of m entries (d dims) with one probe per mate, each call
    through hers_search and hers_search_noalloc on the same explicit stream."""
    ctx, keys = env
    L = H.lib()
    nb = H.hers_blocks_for(m)
    assert nb <= MAX_BLOCKS
    feats = W.gallery_features(m, d, seed)
    gal, _ = H.hers_encrypt_gallery(ctx, keys, torch.from_numpy(feats).cuda(), seed + 1)
    st = torch.cuda.Stream()
    handle = ctypes.c_void_p(st.cuda_stream)
    for call, mate in enumerate(mates):          # calls in a row, different probes
        q = W.probe_for_mate(mate, d, seed, seed + 2 + call)
        pr = H.hers_probe_prepare(ctx, H.hers_encrypt_probe(ctx, keys, torch.from_numpy(q).cuda(),
                                                            seed + 10 + call))
        st.wait_stream(torch.cuda.current_stream())   # inputs written on the default stream
        with torch.cuda.stream(st):
            want = torch.empty((nb, 2, 2, H.N), dtype=torch.int64, device="cuda")
            got = torch.full_like(want, -1)
        H.hers_search(ctx, keys, gal, nb, d, pr, out=want, stream=st)
        rc = L.hers_search_noalloc(ctx.h, keys.h, _p(gal), nb, d, _p(pr), _p(got), handle)
        assert rc == 0, L.hers_last_error(ctx.h)
        st.synchronize()
        assert torch.equal(got, want), f"m={m}, call {call}: score ciphertexts differ"
        scores = H.hers_decrypt_scores(ctx, keys, got, m).cpu().numpy().astype(np.int64)
        assert np.array_equal(scores, W.plain_inner_products(feats, q))
    H.hers_check(ctx)
    return gal, pr, got


def test_noalloc_search_matches_hers_search_on_two_calls(env):
    _compare(env, 6 * 4096 + 77, 48, (123, 6 * 4096 + 70), 4343)   # 7 blocks, ragged last block


def test_noalloc_fills_the_scratch_exactly(env):
    """nblocks == HERS_NOALLOC_MAX_BLOCKS: the last block's scratch ends at
    the array's end; a full and a ragged last block."""
    _compare(env, MAX_BLOCKS * 4096, 16, (5, MAX_BLOCKS * 4096 - 1), 5353)
    gal, pr, got = _compare(env, MAX_BLOCKS * 4096 - 100, 16, (4097,), 6363)
    ctx, keys = env
    L = H.lib()
    # beyond the built-in scratch: rejected with a message, nothing launched
    rc = L.hers_search_noalloc(ctx.h, keys.h, _p(gal), MAX_BLOCKS + 1, 16, _p(pr), _p(got),
                               ctypes.c_void_p(0))
    assert rc == HERS_E_INVAL
    assert b"scratch" in L.hers_last_error(ctx.h)
    H.hers_check(ctx)
