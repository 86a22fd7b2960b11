"""Base-w relinearisation gadget (NEXT-1(b)): device keys and the search with
the base-w key switch against the oracle, bit for bit."""
import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2003_12197_gb300 as H  # noqa: E402

KEY, WSEED = 7301, 7302


@pytest.fixture(scope="module")
def env():
    H.build_library()
    ctx = H.Context(0)
    keys = H.hers_keygen(ctx, KEY)
    sk, opk, oevk = O.keygen(KEY)
    m, d = 4096 + 777, 8
    feats = W.gallery_features(m, d, 7303)
    q = W.probe_for_mate(4096 + 5, d, 7303, 7304)
    gal, _ = H.hers_encrypt_gallery(ctx, keys, torch.from_numpy(feats).cuda(), 7305)
    pr = H.hers_probe_prepare(ctx, H.hers_encrypt_probe(ctx, keys, torch.from_numpy(q).cuda(), 7306))
    oprb = O.encrypt_probe(opk, q, 7306)
    ogal = [O.encrypt_gallery_block(opk, feats, b, 7305) for b in range(2)]
    yield dict(ctx=ctx, keys=keys, opk=opk, oevk=oevk, feats=feats, q=q, gal=gal, pr=pr, oprb=oprb,
               ogal=ogal, m=m, d=d)
    keys.close()
    ctx.close()


@pytest.mark.parametrize("logw", [27, 54, 22, 60])
def test_basew_keys_and_search_bit_exact(env, logw):
    ctx, keys = env["ctx"], env["keys"]
    assert H.lib().hers_basew_digits(logw) == O.basew_digits(logw)
    H.hers_keys_add_basew(ctx, keys, WSEED + logw, logw)
    evkw = H.hers_keys_export_basew(ctx, keys, logw)
    oevkw = O.keygen_w(KEY, WSEED + logw, logw)
    assert np.array_equal(evkw, oevkw)
    sc = H.hers_search_basew(ctx, keys, env["gal"], 2, env["d"], env["pr"])
    H.hers_check(ctx)
    got = H.to_u64(sc)
    for b in range(2):
        want = O.search_block_basew(env["oprb"], env["ogal"][b], env["oevk"], oevkw, logw)
        assert np.array_equal(got[b], want), f"block {b}"
    scores = H.hers_decrypt_scores(ctx, keys, sc, env["m"]).cpu().numpy().astype(np.int64)
    assert np.array_equal(scores, W.plain_inner_products(env["feats"], env["q"]))


def test_basew_errors(env):
    ctx = env["ctx"]
    k2 = H.hers_keygen(ctx, KEY + 1)
    with pytest.raises(H.HersError):
        H.hers_search_basew(ctx, k2, env["gal"], 2, env["d"], env["pr"])   # no base-w keys
    for bad in (21, 61, 0):
        with pytest.raises(H.HersError):
            H.hers_keys_add_basew(ctx, k2, 1, bad)
        assert H.lib().hers_basew_digits(bad) == 0
    H.hers_check(ctx)
    k2.close()
