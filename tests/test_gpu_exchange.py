"""The client/server exchange calls of the C ABI, against the existing entry
points and the oracle, bit for bit (integer work: tolerance zero).

  - server keys from pk and evk alone (Sec. 3.1: the server never holds sk):
    the same probe ciphertexts and score ciphertexts as the client's keys, and
    every call that needs sk refuses them;
  - canonical ciphertexts out of and back into the resident gallery form
    (hers_export_ct / hers_import_ct): the enrolled ciphertexts come back
    exactly (and equal the oracle's), and a re-imported gallery is the same
    resident form, searched to the same scores;
  - host-buffer forms of enrollment and decryption;
  - a block range as the search's extent.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2003_12197_gb300 as H  # noqa: E402

KEY_SEED, GAL_SEED, PRB_SEED, FEAT_SEED = 3101, 3102, 3103, 3104


@pytest.fixture(scope="module")
def env():
    H.build_library()
    ctx = H.Context(0)
    client = H.hers_keygen(ctx, KEY_SEED)
    _, pk, evk = H.hers_keys_export(ctx, client)
    server_ctx = H.Context(0)
    server = H.hers_keys_import(server_ctx, pk, evk)
    m, d = 3 * 4096 + 500, 24                      # 4 blocks, ragged last block
    feats = W.gallery_features(m, d, FEAT_SEED)
    gal, gct = H.hers_encrypt_gallery(ctx, client, torch.from_numpy(feats).cuda(), GAL_SEED, want_ct=True)
    q = W.probe_for_mate(4321, d, FEAT_SEED, FEAT_SEED + 1)
    pct = H.hers_encrypt_probe(ctx, client, torch.from_numpy(q).cuda(), PRB_SEED)
    pr = H.hers_probe_prepare(ctx, pct)
    nb = H.hers_blocks_for(m)
    sc = H.hers_search(ctx, client, gal, nb, d, pr)
    torch.cuda.synchronize()
    yield dict(ctx=ctx, client=client, server_ctx=server_ctx, server=server, pk=pk, evk=evk, feats=feats,
               gal=gal, gct=gct, q=q, pct=pct, pr=pr, sc=sc, m=m, d=d, nb=nb)
    server.close()
    client.close()
    server_ctx.close()
    ctx.close()


def test_server_keys_hold_no_secret(env):
    assert H.hers_keys_has_secret(env["client"])
    assert not H.hers_keys_has_secret(env["server"])
    sctx, server = env["server_ctx"], env["server"]
    with pytest.raises(H.HersError):
        H.hers_keys_export(sctx, server)                     # sk requested
    with pytest.raises(H.HersError):
        H.hers_decrypt_scores(sctx, server, env["sc"], env["m"])
    with pytest.raises(H.HersError):
        H.hers_decrypt_scores_host(sctx, server, env["sc"].cpu(), env["m"])
    with pytest.raises(H.HersError):
        H.hers_keys_add_basew(sctx, server, 1, 27)
    # the public parts come back as imported
    pk = np.zeros((2, 2, H.N), dtype=np.uint64)
    evk = np.zeros((2, 2, 2, H.N), dtype=np.uint64)
    sctx.check(H.lib().hers_keys_export(sctx.h, server.h, None, pk.ctypes.data, evk.ctypes.data), "export")
    assert np.array_equal(pk, env["pk"]) and np.array_equal(evk, env["evk"])


def test_server_keys_search_and_encrypt_like_the_client(env):
    sctx, server, d = env["server_ctx"], env["server"], env["d"]
    sc = H.hers_search(sctx, server, env["gal"], env["nb"], d, env["pr"])
    pct = H.hers_encrypt_probe(sctx, server, torch.from_numpy(env["q"]).cuda(), PRB_SEED)
    torch.cuda.synchronize()
    assert torch.equal(sc, env["sc"])
    assert torch.equal(pct, env["pct"])
    # and against the oracle, block 3 (the ragged one)
    _, opk, oevk = O.keygen(KEY_SEED)
    ogal = O.encrypt_gallery_block(opk, env["feats"], 3, GAL_SEED)
    oprb = O.encrypt_probe(opk, env["q"], PRB_SEED)
    osc, _ = O.search_block(oprb, ogal, oevk)
    assert np.array_equal(H.to_u64(sc)[3], osc)
    scores = H.hers_decrypt_scores(env["ctx"], env["client"], sc, env["m"]).cpu().numpy().astype(np.int64)
    assert np.array_equal(scores, W.plain_inner_products(env["feats"], env["q"]))


def test_invalid_keys_are_refused(env):
    bad = env["pk"].copy()
    bad[1, 0, 7] = np.uint64(18014398509309953)              # = q1: not a residue in [0, q1)
    with pytest.raises(H.HersError):
        H.hers_keys_import(env["server_ctx"], bad, env["evk"])


def test_export_returns_the_enrolled_ciphertexts(env):
    ctx, d, nb = env["ctx"], env["d"], env["nb"]
    out = H.hers_export_ct(ctx, env["gal"], nb, d)
    assert np.array_equal(out, H.to_u64(env["gct"]))
    _, opk, _ = O.keygen(KEY_SEED)
    assert np.array_equal(out[1], O.encrypt_gallery_block(opk, env["feats"], 1, GAL_SEED))
    part = H.hers_export_ct(ctx, env["gal"], nb, d, 2, 4)
    assert np.array_equal(part, out[2:4])
    assert H.hers_export_ct(ctx, env["gal"], nb, d, 3, 3).shape[0] == 0
    with pytest.raises(H.HersError):
        H.hers_export_ct(ctx, env["gal"], nb, d, 2, 5)


def test_import_rebuilds_the_resident_form(env):
    ctx, d, nb = env["ctx"], env["d"], env["nb"]
    cts = H.hers_export_ct(ctx, env["gal"], nb, d)
    g2 = torch.zeros_like(env["gal"])
    H.hers_import_ct(ctx, cts[:2], g2, nb, d, 0)            # in two ranges
    H.hers_import_ct(ctx, cts[2:], g2, nb, d, 2)
    torch.cuda.synchronize()
    assert torch.equal(g2, env["gal"])
    sc = H.hers_search(ctx, env["client"], g2, nb, d, env["pr"])
    torch.cuda.synchronize()
    assert torch.equal(sc, env["sc"])
    bad = cts[:1].copy()
    bad[0, 0, 1, 1, 5] = np.uint64(18014398509293569)        # = q2
    with pytest.raises(H.HersError):
        H.hers_import_ct(ctx, bad, g2, nb, d, 0)


def test_host_enrollment_equals_device_enrollment(env):
    ctx = env["ctx"]
    gal, gct = H.hers_encrypt_gallery_host(ctx, env["client"], env["feats"], GAL_SEED, want_ct=True)
    torch.cuda.synchronize()
    assert torch.equal(gal, env["gal"]) and torch.equal(gct, env["gct"])
    gal_s, _ = H.hers_encrypt_gallery_host(env["server_ctx"], env["server"], env["feats"], GAL_SEED)
    torch.cuda.synchronize()
    assert torch.equal(gal_s, env["gal"])                    # the server enrolls with pk alone


def test_host_decryption_of_host_scores(env):
    ctx, d, nb, m = env["ctx"], env["d"], env["nb"], env["m"]
    ws = torch.empty(H.hers_search_host_workspace_bytes(nb, d) // 8, dtype=torch.int64, device="cuda")
    out = torch.empty((nb, 2, 2, H.N), dtype=torch.int64).pin_memory()
    H.hers_search_host(env["server_ctx"], env["server"], env["gal"], nb, d, env["pct"].cpu(), out, ws)
    assert torch.equal(out, env["sc"].cpu())
    scores = H.hers_decrypt_scores_host(ctx, env["client"], out, m)
    assert np.array_equal(scores.astype(np.int64), W.plain_inner_products(env["feats"], env["q"]))
    dev = H.hers_decrypt_scores(ctx, env["client"], env["sc"], m).cpu().numpy()
    assert np.array_equal(scores, dev)
    assert int(np.argmax(scores)) == 4321


def test_search_range(env):
    ctx, d, nb = env["ctx"], env["d"], env["nb"]
    for b0, b1 in ((0, nb), (1, 3), (3, 4), (2, 2)):
        sc = H.hers_search_range(ctx, env["client"], env["gal"], nb, d, b0, b1, env["pr"])
        torch.cuda.synchronize()
        assert torch.equal(sc, env["sc"][b0:b1]), (b0, b1)
    for b0, b1 in ((3, 5), (2, 1)):
        with pytest.raises(H.HersError):
            H.hers_search_range(ctx, env["client"], env["gal"], nb, d, b0, b1, env["pr"])
