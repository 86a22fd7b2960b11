"""Streamed search over a canonical gallery (host- or device-resident), in
chunks with a ragged last chunk, against hers_search on the resident form:
bit for bit, for several probes and kernel shapes."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2003_12197_gb300 as H  # noqa: E402


@pytest.fixture(scope="module")
def env():
    H.build_library()
    ctx = H.Context(0)
    keys = H.hers_keygen(ctx, 3131)
    m, d = 5 * 4096 - 300, 16
    feats = W.gallery_features(m, d, 3232)
    f = torch.from_numpy(feats).cuda()
    _, gct = H.hers_encrypt_gallery(ctx, keys, f, 3333, resident=False)
    gal, gct2 = H.hers_encrypt_gallery(ctx, keys, f, 3333, want_ct=True)
    probes, qs = [], []
    for j in range(5):
        q = W.probe_for_mate(1000 * j + 3, d, 3232, 3434 + j)
        qs.append(q)
        probes.append(H.hers_probe_prepare(ctx, H.hers_encrypt_probe(ctx, keys, torch.from_numpy(q).cuda(), 3535 + j)))
    nb = H.hers_blocks_for(m)
    ref = [H.hers_search(ctx, keys, gal, nb, d, pr) for pr in probes]
    torch.cuda.synchronize()
    assert torch.equal(gct, gct2)   # canonical-only enrollment writes the same cts
    yield dict(ctx=ctx, keys=keys, gct=gct, probes=probes, ref=ref, nb=nb, d=d, feats=feats, qs=qs)
    keys.close()
    ctx.close()


@pytest.mark.parametrize("on_host,variant", [(False, 1), (True, 1), (False, 3), (True, 0)])
def test_streamed_equals_resident_search(env, on_host, variant):
    g = env["gct"].cpu().pin_memory() if on_host else env["gct"]
    sc = H.hers_search_stream(env["ctx"], env["keys"], g, env["nb"], env["d"], env["probes"],
                              chunk_blocks=2, variant=variant)
    torch.cuda.synchronize()
    for p in range(len(env["probes"])):
        assert torch.equal(sc[p], env["ref"][p]), f"probe {p}"
    scores = H.hers_decrypt_scores(env["ctx"], env["keys"], sc[2], env["feats"].shape[0])
    assert np.array_equal(scores.cpu().numpy().astype(np.int64),
                          W.plain_inner_products(env["feats"], env["qs"][2]))
