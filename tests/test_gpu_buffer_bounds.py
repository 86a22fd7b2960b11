"""Every caller-sized buffer is large enough for what the library writes into it.

Each buffer the library sizes for its caller (hers_gallery_bytes,
hers_probe_bytes, hers_search_workspace_bytes, hers_search_host_workspace_bytes)
is handed to the library as the first part of a larger allocation whose tail
holds a sentinel; after the calls that write the buffer, the tail must still
hold it.  A layout that outgrew its size function writes into the tail, which
is ours, so the check itself never touches memory outside the allocation.
Scores are checked against the plaintext inner products (Eq. 1) as well.
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2003_12197_gb300 as H  # noqa: E402

N = 4096
GUARD_WORDS = 1 << 20  # 8 MiB of sentinel after each buffer
SENTINEL = 0x5A5A5A5A5A5A5A5A


def guarded(nbytes, dev):
    """(view of nbytes // 8 words, whole allocation) with the tail set to SENTINEL."""
    words = nbytes // 8
    whole = torch.empty(words + GUARD_WORDS, dtype=torch.int64, device=dev)
    whole[words:] = SENTINEL
    return whole[:words], whole


def tail_intact(whole, nbytes):
    return bool((whole[nbytes // 8:] == SENTINEL).all().item())


@pytest.mark.parametrize("m,d", [(2 * N + 100, 64), (N, 17)])
def test_buffers_hold_what_the_library_writes(m, d):
    dev = torch.device("cuda", 0)
    H.build_library()
    ctx = H.Context(0)
    keys = H.hers_keygen(ctx, 77)
    nb = H.hers_blocks_for(m)
    feats = torch.from_numpy(W.gallery_features(m, d, 501)).to(dev)

    gb = H.hers_gallery_bytes(nb, d)
    gal, gal_whole = guarded(gb, dev)
    H.hers_encrypt_gallery(ctx, keys, feats, 502, out=gal)

    q = torch.from_numpy(W.quantise(np.ones((1, d)))[0]).to(dev)
    pct = H.hers_encrypt_probe(ctx, keys, q, 503)
    pb = H.hers_probe_bytes(d)
    pr, pr_whole = guarded(pb, dev)
    H.hers_probe_prepare(ctx, pct, out=pr)

    wb = H.hers_search_workspace_bytes(nb)
    ws, ws_whole = guarded(wb, dev)
    sc = H.hers_search(ctx, keys, gal, nb, d, pr, workspace=ws)

    hb = H.hers_search_host_workspace_bytes(nb, d)
    wsh, wsh_whole = guarded(hb, dev)
    sc_host = torch.empty((nb, 2, 2, N), dtype=torch.int64)
    H.hers_search_host(ctx, keys, gal, nb, d, pct.cpu(), sc_host, wsh)
    torch.cuda.synchronize()
    H.hers_check(ctx)

    assert tail_intact(gal_whole, gb), "resident gallery overran hers_gallery_bytes"
    assert tail_intact(pr_whole, pb), "prepared probe overran hers_probe_bytes"
    assert tail_intact(ws_whole, wb), "search overran hers_search_workspace_bytes"
    assert tail_intact(wsh_whole, hb), "host search overran hers_search_host_workspace_bytes"
    assert np.array_equal(sc_host.numpy(), sc.cpu().numpy())
    scores = H.hers_decrypt_scores(ctx, keys, sc, m).cpu().numpy().astype(np.int64)
    plain = feats.cpu().numpy().astype(np.int64) @ q.cpu().numpy().astype(np.int64)
    assert np.array_equal(scores, plain)
    keys.close()
    ctx.close()
