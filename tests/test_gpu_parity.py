"""GPU parity: the CUDA library against the CPU oracle, bit for bit.

Every input is seeded and synthetic (workloads/).  Keys, probe and gallery
ciphertexts, score ciphertexts and decrypted scores are compared element by
element with the oracle run on the same seeds; decrypted scores are also
compared with the plaintext inner products (Eq. 1), which holds at any size.
Integer work: the tolerance is zero.
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

KEY_SEED, GAL_SEED, PRB_SEED, FEAT_SEED, MATE_SEED, NOISE_SEED = 1004, 1005, 1006, 1001, 1002, 1003


@pytest.fixture(scope="module")
def ctx():
    H.build_library()
    c = H.Context(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def keys(ctx):
    k = H.hers_keygen(ctx, KEY_SEED)
    yield k
    k.close()


@pytest.fixture(scope="module")
def oracle_keys():
    return O.keygen(KEY_SEED)


def u64(t):
    return H.to_u64(t)


def run_search(ctx, keys, feats_np, q_np, gal_seed=GAL_SEED, prb_seed=PRB_SEED):
    m, d = feats_np.shape
    feats = torch.from_numpy(feats_np).cuda()
    q = torch.from_numpy(q_np).cuda()
    gal, gct = H.hers_encrypt_gallery(ctx, keys, feats, gal_seed, want_ct=True)
    pct = H.hers_encrypt_probe(ctx, keys, q, prb_seed)
    pr = H.hers_probe_prepare(ctx, pct)
    nb = H.hers_blocks_for(m)
    sc = H.hers_search(ctx, keys, gal, nb, d, pr)
    scores = H.hers_decrypt_scores(ctx, keys, sc, m)
    H.hers_check(ctx)
    torch.cuda.synchronize()
    return dict(gct=gct, pct=pct, sc=sc, scores=scores.cpu().numpy(), gal=gal, pr=pr, nb=nb)


def test_keygen_bit_exact(ctx, keys, oracle_keys):
    sk, pk, evk = H.hers_keys_export(ctx, keys)
    osk, opk, oevk = oracle_keys
    assert np.array_equal(sk, osk)
    assert np.array_equal(pk, opk)
    assert np.array_equal(evk, oevk)


def test_keygen_other_seed_differs(ctx):
    k2 = H.hers_keygen(ctx, KEY_SEED + 1)
    sk, pk, _ = H.hers_keys_export(ctx, k2)
    osk, opk, _ = O.keygen(KEY_SEED + 1)
    assert np.array_equal(sk, osk) and np.array_equal(pk, opk)
    k2.close()


def test_probe_encryption_bit_exact(ctx, keys, oracle_keys):
    d = 64
    q = W.probe_for_mate(5, d, FEAT_SEED, NOISE_SEED)
    pct = H.hers_encrypt_probe(ctx, keys, torch.from_numpy(q).cuda(), PRB_SEED)
    want = O.encrypt_probe(oracle_keys[1], q, PRB_SEED)
    assert np.array_equal(u64(pct), want)


@pytest.fixture(scope="module")
def config1(ctx, keys, oracle_keys):
    """4,096 entries (one block), d = 64, one probe with a planted mate."""
    n, d = 4096, 64
    feats = W.gallery_features(n, d, FEAT_SEED)
    mate = int(W.mate_indices(n, 1, MATE_SEED)[0])
    q = W.probe_for_mate(mate, d, FEAT_SEED, NOISE_SEED)
    res = run_search(ctx, keys, feats, q)
    ogal = O.encrypt_gallery_block(oracle_keys[1], feats, 0, GAL_SEED)
    oprb = O.encrypt_probe(oracle_keys[1], q, PRB_SEED)
    osc, st = O.search_block(oprb, ogal, oracle_keys[2])
    return dict(res=res, ogal=ogal, oprb=oprb, osc=osc, st=st, feats=feats, q=q, mate=mate)


def test_config1_gallery_cts_bit_exact(config1):
    assert np.array_equal(u64(config1["res"]["gct"])[0], config1["ogal"])


def test_config1_score_ct_bit_exact(config1):
    assert np.array_equal(u64(config1["res"]["sc"])[0], config1["osc"])


def test_config1_scores_exact_and_top1(config1, oracle_keys):
    scores = config1["res"]["scores"]
    want = W.plain_inner_products(config1["feats"], config1["q"])
    assert np.array_equal(scores.astype(np.int64), want)
    oscores, _, _ = O.decrypt(oracle_keys[0], config1["osc"])
    assert np.array_equal(scores.astype(np.int64), oscores)
    assert int(np.argmax(scores)) == config1["mate"]


@pytest.mark.parametrize("m,d", [(2 * 4096 + 1000, 16), (300, 200), (4096, 1), (1, 3)])
def test_ragged_and_edge_sizes_bit_exact(ctx, keys, oracle_keys, m, d):
    """Several blocks with a ragged tail, d > 128 (chunked accumulation), d = 1, m = 1."""
    feats = W.gallery_features(m, d, FEAT_SEED + m + d)
    q = W.probe_for_mate(m // 2, d, FEAT_SEED + m + d, NOISE_SEED)
    res = run_search(ctx, keys, feats, q)
    oprb = O.encrypt_probe(oracle_keys[1], q, PRB_SEED)
    assert np.array_equal(u64(res["pct"]), oprb)
    gct, sc = u64(res["gct"]), u64(res["sc"])
    for b in range(res["nb"]):
        ogal = O.encrypt_gallery_block(oracle_keys[1], feats, b, GAL_SEED)
        assert np.array_equal(gct[b], ogal), f"gallery block {b}"
        osc, st = O.search_block(oprb, ogal, oracle_keys[2])
        assert np.array_equal(sc[b], osc), f"score block {b}"
    assert np.array_equal(res["scores"].astype(np.int64), W.plain_inner_products(feats, q))


def test_search_host_path_matches_device_path(ctx, keys, config1):
    res = config1["res"]
    nb, d = res["nb"], 64
    ws = torch.empty(H.hers_search_host_workspace_bytes(nb, d) // 8, dtype=torch.int64,
                     device="cuda")
    pct_host = res["pct"].cpu().pin_memory()
    out = torch.empty((nb, 2, 2, 4096), dtype=torch.int64).pin_memory()
    H.hers_search_host(ctx, keys, res["gal"], nb, d, pct_host, out, ws)
    assert np.array_equal(out.numpy().view(np.uint64), u64(res["sc"]))


def test_repeat_search_is_deterministic(ctx, keys, config1):
    res = config1["res"]
    a = H.hers_search(ctx, keys, res["gal"], res["nb"], 64, res["pr"])
    b = H.hers_search(ctx, keys, res["gal"], res["nb"], 64, res["pr"])
    torch.cuda.synchronize()
    assert torch.equal(a, b) and torch.equal(a, res["sc"])


def test_invalid_arguments_are_rejected(ctx, keys):
    with pytest.raises(H.HersError):
        H.hers_encrypt_probe(ctx, keys, torch.zeros(0, dtype=torch.int8, device="cuda"), 1)
    gal = torch.zeros(16, dtype=torch.int64, device="cuda")
    with pytest.raises(H.HersError):
        H.hers_search(ctx, keys, gal, 1, 64, gal, workspace=torch.zeros(8, dtype=torch.int64,
                                                                         device="cuda"))


def test_empty_inputs(ctx, keys):
    """An empty gallery is refused at encryption; a search over zero blocks is
    accepted and writes nothing."""
    with pytest.raises(H.HersError):
        H.hers_encrypt_gallery(ctx, keys, torch.zeros((0, 16), dtype=torch.int8, device="cuda"), 1)
    out = torch.full((16,), 0x5A5A, dtype=torch.int64, device="cuda")
    dummy = torch.zeros(16, dtype=torch.int64, device="cuda")
    H.hers_search(ctx, keys, dummy, 0, 16, dummy, out=out, workspace=dummy)
    torch.cuda.synchronize()
    H.hers_check(ctx)
    assert bool((out == 0x5A5A).all())


@pytest.mark.slow
def test_config2_full_size(ctx, keys, oracle_keys):
    """1,048,576 entries (256 blocks), d = 64, one planted mate: every decrypted
    score exact; the score ciphertexts of the mate's block, the last block and
    8 seeded random blocks bit-exact against the oracle.  Then the launch
    configuration the bench times (the persistent Karatsuba tensor shape, the
    lean epilogue, three searches in flight on three streams) gives the same
    score ciphertexts for all 256 blocks."""
    m, d = 1 << 20, 64
    feats = W.gallery_features(m, d, FEAT_SEED)
    mate = int(W.mate_indices(m, 1, MATE_SEED)[0])
    q = W.probe_for_mate(mate, d, FEAT_SEED, NOISE_SEED)
    res = run_search(ctx, keys, feats, q)
    assert np.array_equal(res["scores"].astype(np.int64), W.plain_inner_products(feats, q))
    assert int(np.argmax(res["scores"])) == mate
    oprb = O.encrypt_probe(oracle_keys[1], q, PRB_SEED)
    sc = u64(res["sc"])
    rng = np.random.default_rng(20032)
    blocks = {mate // 4096, res["nb"] - 1}
    while len(blocks) < 10:
        blocks.add(int(rng.integers(0, res["nb"])))
    for b in sorted(blocks):
        ogal = O.encrypt_gallery_block(oracle_keys[1], feats, b, GAL_SEED)
        osc, _ = O.search_block(oprb, ogal, oracle_keys[2])
        assert np.array_equal(sc[b], osc), f"block {b}"
    # the bench's launch configuration
    keep_t, keep_e = H.hers_get_tensor_variant(ctx), H.hers_get_epilogue_variant(ctx)
    H.hers_set_tensor_variant(ctx, H.hers_tensor_variants().index("pnb2_s3_d4_k2_m4_ka"))
    H.hers_set_epilogue_variant(ctx, H.hers_epilogue_variants().index("split+lean"))
    try:
        nb = res["nb"]
        lanes = [(H.hers_probe_prepare(ctx, res["pct"]),
                  torch.empty(H.hers_search_workspace_bytes(nb) // 8, dtype=torch.int64, device="cuda"),
                  torch.empty((nb, 2, 2, H.N), dtype=torch.int64, device="cuda"), torch.cuda.Stream())
                 for _ in range(3)]
        torch.cuda.synchronize()
        for k in range(6):
            p_, w_, o_, st_ = lanes[k % 3]
            H.hers_probe_prepare(ctx, res["pct"], out=p_, stream=st_)
            H.hers_search(ctx, keys, res["gal"], nb, d, p_, out=o_, workspace=w_, stream=st_)
        torch.cuda.synchronize()
        H.hers_check(ctx)
        for i, (_, _, o_, _) in enumerate(lanes):
            assert np.array_equal(u64(o_), sc), f"lane {i}"
    finally:
        H.hers_set_tensor_variant(ctx, keep_t)
        H.hers_set_epilogue_variant(ctx, keep_e)


def test_inline_temporaries_on_default_stream(ctx, keys):
    """Inputs passed as temporaries: the library must run on the caller's stream
    (here the default stream), so a freed input is not overwritten while it is read."""
    m, d = 3 * 4096, 32
    feats = W.gallery_features(m, d, 77)
    q = W.probe_for_mate(5000, d, 77, 78)
    gal, _ = H.hers_encrypt_gallery(ctx, keys, torch.from_numpy(feats).cuda(), GAL_SEED)
    junk = [torch.full((m * d,), 7, dtype=torch.int8, device="cuda") for _ in range(4)]
    pct = H.hers_encrypt_probe(ctx, keys, torch.from_numpy(q).cuda(), PRB_SEED)
    junk += [torch.full((d,), -9, dtype=torch.int8, device="cuda") for _ in range(4)]
    sc = H.hers_search(ctx, keys, gal, 3, d, H.hers_probe_prepare(ctx, pct))
    scores = H.hers_decrypt_scores(ctx, keys, sc, m).cpu().numpy().astype(np.int64)
    del junk
    assert np.array_equal(scores, W.plain_inner_products(feats, q))


def test_every_tensor_shape_gives_the_same_ciphertexts(ctx, keys, oracle_keys):
    """Exact integer arithmetic makes the result independent of the kernel's
    tiling: every autotuner candidate must give the oracle's score ciphertexts,
    over 4 blocks and over the first 3 (a partial block group for the 2- and
    4-block shapes)."""
    m, d = 3 * 4096 + 17, 41   # 41: a ragged last stage at every stage depth (2, 4, 8), past 5 fold points
    feats = W.gallery_features(m, d, 99)
    q = W.probe_for_mate(4100, d, 99, 98)
    gal, _ = H.hers_encrypt_gallery(ctx, keys, torch.from_numpy(feats).cuda(), GAL_SEED)
    pr = H.hers_probe_prepare(ctx, H.hers_encrypt_probe(ctx, keys, torch.from_numpy(q).cuda(), PRB_SEED))
    names = H.hers_tensor_variants()
    assert len(names) >= 4
    keep = H.hers_get_tensor_variant(ctx)
    outs, outs3 = [], []
    for v in range(len(names)):
        H.hers_set_tensor_variant(ctx, v)
        outs.append(u64(H.hers_search(ctx, keys, gal, 4, d, pr)))
        outs3.append(u64(H.hers_search(ctx, keys, gal, 3, d, pr)))
    H.hers_set_tensor_variant(ctx, keep)
    oprb = O.encrypt_probe(oracle_keys[1], q, PRB_SEED)
    ogal = O.encrypt_gallery_block(oracle_keys[1], feats, 3, GAL_SEED)
    osc, _ = O.search_block(oprb, ogal, oracle_keys[2])
    for v, o in enumerate(outs):
        assert np.array_equal(o, outs[0]), names[v]
        assert np.array_equal(o[3], osc), names[v]
        assert np.array_equal(outs3[v], outs[0][:3]), names[v]
    chosen, ms = H.hers_autotune(ctx, keys, gal, 4, d, pr)
    assert 0 <= chosen < len(names) and len(ms) == len(names)
    H.hers_set_tensor_variant(ctx, keep)


def test_persistent_tensor_shapes_walk_many_units(ctx, keys):
    """The persistent shapes ("pnb...") run K CTAs per SM, each walking many
    (limb, tile, block group) units with one ring of stages across them.  On
    37 blocks (a partial block group for every NB > 1; about 8 units per CTA)
    at d = 41 (a ragged last stage) every one gives the score ciphertexts of
    the first, non-persistent shape, and the Karatsuba shapes ("_ka") do too."""
    m, d = 37 * 4096 - 5, 41
    feats = W.gallery_features(m, d, 4242)
    q = W.probe_for_mate(77777, d, 4242, 4343)
    gal, _ = H.hers_encrypt_gallery(ctx, keys, torch.from_numpy(feats).cuda(), GAL_SEED)
    pr = H.hers_probe_prepare(ctx, H.hers_encrypt_probe(ctx, keys, torch.from_numpy(q).cuda(), PRB_SEED))
    nb = H.hers_blocks_for(m)
    names = H.hers_tensor_variants()
    picked = [v for v, n in enumerate(names) if n.startswith("pnb") or n.endswith("_ka")]
    assert any(names[v].startswith("pnb") for v in picked)
    keep = H.hers_get_tensor_variant(ctx)
    H.hers_set_tensor_variant(ctx, 0)
    ref = u64(H.hers_search(ctx, keys, gal, nb, d, pr))
    for v in picked:
        H.hers_set_tensor_variant(ctx, v)
        assert np.array_equal(u64(H.hers_search(ctx, keys, gal, nb, d, pr)), ref), names[v]
    H.hers_set_tensor_variant(ctx, keep)
    scores = H.hers_decrypt_scores(ctx, keys, torch.from_numpy(ref.view(np.int64)).cuda(), m)
    assert np.array_equal(scores.cpu().numpy().astype(np.int64), W.plain_inner_products(feats, q))


def test_async_host_search_equals_sync(ctx, keys):
    """hers_search_host_async on two streams gives the bytes of
    hers_search_host; unpinned host buffers are refused."""
    m, d = 3 * 4096 + 17, 8
    feats = W.gallery_features(m, d, 6161)
    q = W.probe_for_mate(12, d, 6161, 6262)
    gal, _ = H.hers_encrypt_gallery(ctx, keys, torch.from_numpy(feats).cuda(), 6363)
    pct = H.hers_encrypt_probe(ctx, keys, torch.from_numpy(q).cuda(), 6464)
    nb = H.hers_blocks_for(m)
    ws = [torch.empty(H.hers_search_host_workspace_bytes(nb, d) // 8, dtype=torch.int64, device="cuda")
          for _ in range(2)]
    pct_host = pct.cpu().pin_memory()
    ref = torch.empty((nb, 2, 2, H.N), dtype=torch.int64).pin_memory()
    H.hers_search_host(ctx, keys, gal, nb, d, pct_host, ref, ws[0])
    outs = [torch.zeros((nb, 2, 2, H.N), dtype=torch.int64).pin_memory() for _ in range(2)]
    streams = [torch.cuda.Stream() for _ in range(2)]
    for k in range(4):
        H.hers_search_host_async(ctx, keys, gal, nb, d, pct_host, outs[k % 2], ws[k % 2],
                                 stream=streams[k % 2])
    torch.cuda.synchronize()
    for o in outs:
        assert torch.equal(o, ref)
    scores = H.hers_decrypt_scores(ctx, keys, ref.cuda(), m).cpu().numpy().astype(np.int64)
    assert np.array_equal(scores, W.plain_inner_products(feats, q))
    with pytest.raises(H.HersError):
        H.hers_search_host_async(ctx, keys, gal, nb, d, pct.cpu(), outs[0], ws[0], stream=streams[0])
    H.hers_check(ctx)


def test_maximum_dimension_d512_bit_exact(ctx, keys, oracle_keys):
    """d = 512, the largest supported dimension (|X| < 2^236 < QP/2): one
    ragged block, gallery, probe and score ciphertexts against the oracle, and
    the decrypted scores against Eq. 1."""
    m, d = 4000, 512
    feats = W.gallery_features(m, d, 5120)
    q = W.probe_for_mate(1234, d, 5120, 5121)
    res = run_search(ctx, keys, feats, q, gal_seed=5122, prb_seed=5123)
    ogal = O.encrypt_gallery_block(oracle_keys[1], feats, 0, 5122)
    assert np.array_equal(u64(res["gct"])[0], ogal)
    oprb = O.encrypt_probe(oracle_keys[1], q, 5123)
    assert np.array_equal(u64(res["pct"]), oprb)
    osc, st = O.search_block(oprb, ogal, oracle_keys[2])
    assert np.array_equal(u64(res["sc"])[0], osc)
    assert np.array_equal(res["scores"].astype(np.int64), W.plain_inner_products(feats, q))
    assert int(np.argmax(res["scores"])) == 1234


def test_rerandomized_search_bit_exact(ctx, keys, oracle_keys):
    """hers_search_rerand: every block's score ciphertext equals the oracle's
    search output plus its Enc(0) from the streams (seed, 0x31.., block), and
    decrypts to the plaintext inner products."""
    m, d = 2 * 4096 + 300, 16
    feats = W.gallery_features(m, d, 8181)
    q = W.probe_for_mate(4321, d, 8181, 8282)
    gal, _ = H.hers_encrypt_gallery(ctx, keys, torch.from_numpy(feats).cuda(), 8383)
    pr = H.hers_probe_prepare(ctx, H.hers_encrypt_probe(ctx, keys, torch.from_numpy(q).cuda(), 8484))
    nb = H.hers_blocks_for(m)
    plain = H.hers_search(ctx, keys, gal, nb, d, pr)
    sc = H.hers_search_rerand(ctx, keys, gal, nb, d, pr, 8585)
    H.hers_check(ctx)
    got, plain_u = u64(sc), u64(plain)
    assert not np.array_equal(got, plain_u)
    oprb = O.encrypt_probe(oracle_keys[1], q, 8484)
    for b in range(nb):
        ogal = O.encrypt_gallery_block(oracle_keys[1], feats, b, 8383)
        osc, _ = O.search_block(oprb, ogal, oracle_keys[2])
        assert np.array_equal(plain_u[b], osc), f"block {b}"
        assert np.array_equal(got[b], O.rerandomize(oracle_keys[1], osc, 8585, b)), f"block {b}"
    scores = H.hers_decrypt_scores(ctx, keys, sc, m).cpu().numpy().astype(np.int64)
    assert np.array_equal(scores, W.plain_inner_products(feats, q))


def test_searches_on_several_streams_in_flight(ctx, keys, config1):
    """Searches issued back to back on three streams of one context (their
    epilogues share the context's high-priority stream) each equal the
    sequential search; and a kernel enqueued on a caller's stream after the
    call sees the finished scores."""
    res = config1["res"]
    nb = res["nb"]
    streams = [torch.cuda.Stream() for _ in range(3)]
    outs = [torch.empty_like(res["sc"]) for _ in range(6)]
    wss = [torch.empty(H.hers_search_workspace_bytes(nb) // 8, dtype=torch.int64, device="cuda")
           for _ in range(3)]
    torch.cuda.synchronize()
    copies = []
    for k in range(6):
        st = streams[k % 3]
        H.hers_search(ctx, keys, res["gal"], nb, 64, res["pr"], out=outs[k], workspace=wss[k % 3], stream=st)
        with torch.cuda.stream(st):
            copies.append(outs[k].clone())  # ordered after the search on st
    torch.cuda.synchronize()
    for k in range(6):
        assert torch.equal(outs[k], res["sc"]), f"search {k}"
        assert torch.equal(copies[k], res["sc"]), f"copy after search {k}"


def test_every_epilogue_form_gives_the_same_ciphertexts(ctx, keys, oracle_keys):
    """The epilogue forms (split kernels, inverse NTTs fused with
    scale-and-round in clusters, the fused key switch, both; each with the
    shuffle exchange and with the lean register budget) compute the same
    exact integers: every form gives the oracle's score ciphertexts, over 3
    blocks with a ragged last block; and the epilogue autotuner keeps one."""
    m, d = 2 * 4096 + 999, 19
    feats = W.gallery_features(m, d, 4747)
    q = W.probe_for_mate(77, d, 4747, 4848)
    gal, _ = H.hers_encrypt_gallery(ctx, keys, torch.from_numpy(feats).cuda(), GAL_SEED)
    pr = H.hers_probe_prepare(ctx, H.hers_encrypt_probe(ctx, keys, torch.from_numpy(q).cuda(), PRB_SEED))
    names = H.hers_epilogue_variants()
    assert len(names) == 32 and names[8].endswith("+lean") and names[16].endswith("+ksshfl")
    keep = H.hers_get_epilogue_variant(ctx)
    outs = []
    for v in range(len(names)):
        H.hers_set_epilogue_variant(ctx, v)
        outs.append(u64(H.hers_search(ctx, keys, gal, 3, d, pr)))
    oprb = O.encrypt_probe(oracle_keys[1], q, PRB_SEED)
    for b in range(3):
        ogal = O.encrypt_gallery_block(oracle_keys[1], feats, b, GAL_SEED)
        osc, _ = O.search_block(oprb, ogal, oracle_keys[2])
        for v, o in enumerate(outs):
            assert np.array_equal(o[b], osc), (names[v], b)
    chosen, ms = H.hers_autotune_epilogue(ctx, keys, gal, 3, d, pr)
    assert 0 <= chosen < len(names) and set(ms) == set(names)
    assert H.hers_get_epilogue_variant(ctx) == chosen
    H.hers_set_epilogue_variant(ctx, keep)


def test_tensor_first_ordering_in_flight(ctx, keys, config1):
    """With the tensor kernel on the high-priority stream and the epilogue on
    the caller's (hers_set_tensor_first), searches in flight on three streams
    each equal the sequential search, and work enqueued after a search on its
    stream sees the finished scores."""
    res = config1["res"]
    nb = res["nb"]
    H.hers_set_tensor_first(ctx, True)
    try:
        assert H.hers_get_tensor_first(ctx)
        streams = [torch.cuda.Stream() for _ in range(3)]
        outs = [torch.empty_like(res["sc"]) for _ in range(6)]
        wss = [torch.empty(H.hers_search_workspace_bytes(nb) // 8, dtype=torch.int64, device="cuda")
               for _ in range(3)]
        torch.cuda.synchronize()
        copies = []
        for k in range(6):
            st = streams[k % 3]
            H.hers_search(ctx, keys, res["gal"], nb, 64, res["pr"], out=outs[k], workspace=wss[k % 3], stream=st)
            with torch.cuda.stream(st):
                copies.append(outs[k].clone())
        torch.cuda.synchronize()
        for k in range(6):
            assert torch.equal(outs[k], res["sc"]), f"search {k}"
            assert torch.equal(copies[k], res["sc"]), f"copy after search {k}"
    finally:
        H.hers_set_tensor_first(ctx, False)


def test_extension_autotune_keeps_prepared_probes_identical(ctx, keys):
    """hers_autotune_extension moves the context's cluster threshold; the
    prepared probe is the same bytes in either form (d = 16 and 64, on both
    sides of the default threshold)."""
    for d in (16, 64):
        q = W.probe_for_mate(3, d, FEAT_SEED, NOISE_SEED)
        pct = H.hers_encrypt_probe(ctx, keys, torch.from_numpy(q).cuda(), PRB_SEED)
        before = H.hers_probe_prepare(ctx, pct)
        cluster, ms = H.hers_autotune_extension(ctx, d)
        assert ms["per_polynomial"] > 0 and ms["cluster"] > 0
        after = H.hers_probe_prepare(ctx, pct)
        torch.cuda.synchronize()
        assert torch.equal(before, after), (d, cluster)
