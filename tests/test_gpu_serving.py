"""Serving loop: every request's score ciphertexts, computed in a mix of
concurrent requests with overlapping ranges, equal the same search run alone
(hers_search), bit for bit (tolerance 0).  Also: admission by the memory
pool (one request at a time when the pool is small; a request that can never
fit is refused)."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2003_12197_gb300 as H  # noqa: E402

N = 4096


def request_bytes(d, nb):
    return 8 * (14 * d * N + 29 * N * nb)


@pytest.fixture(scope="module")
def env():
    H.build_library()
    ctx = H.Context(0)
    keys = H.hers_keygen(ctx, 7007)
    gals = []
    for gi, (nb, d) in enumerate([(5, 16), (4, 24)]):
        feats = W.gallery_features(nb * N, d, 800 + gi)
        g, _ = H.hers_encrypt_gallery(ctx, keys, torch.from_numpy(feats).cuda(), 900 + gi)
        gals.append((g, nb, d, feats))
    probes = []
    for gi, (g, nb, d, feats) in enumerate(gals):
        for j in range(3):
            q = W.probe_for_mate(1000 * j + 7, d, 800 + gi, 950 + j)
            pct = H.hers_encrypt_probe(ctx, keys, torch.from_numpy(q).cuda(), 960 + 10 * gi + j)
            probes.append((gi, pct.cpu().pin_memory(), H.hers_probe_prepare(ctx, pct), q))
    torch.cuda.synchronize()
    yield dict(ctx=ctx, keys=keys, gals=gals, probes=probes)
    keys.close()
    ctx.close()


def alone(env, gi, b0, b1, probe_idx):
    g, nb, d, _ = env["gals"][gi]
    view = g[b0 * H.hers_gallery_bytes(1, d) // 8:]
    out = H.hers_search(env["ctx"], env["keys"], view, b1 - b0, d, env["probes"][probe_idx][2])
    torch.cuda.synchronize()
    return out.cpu().numpy()


def test_mix_equals_alone(env):
    rng = np.random.default_rng(5)
    srv = H.Server(env["ctx"], env["keys"], [(g, nb, d) for g, nb, d, _ in env["gals"]],
                   workspace_bytes=1 << 30, max_batch=8)
    reqs = []
    srv.pause(True)      # queue everything first, so the requests run as a mix
    for _ in range(14):
        pi = int(rng.integers(0, len(env["probes"])))
        gi = env["probes"][pi][0]
        nb = env["gals"][gi][1]
        b0 = int(rng.integers(0, nb))
        b1 = int(rng.integers(b0 + 1, nb + 1))
        out = torch.zeros((b1 - b0, 2, 2, N), dtype=torch.int64).pin_memory()
        rid = srv.submit(gi, b0, b1, env["probes"][pi][1], out)
        reqs.append((rid, gi, b0, b1, pi, out))
    srv.pause(False)
    for rid, gi, b0, b1, pi, out in reqs:
        rc, lat = srv.wait(rid)
        assert rc == 0 and lat > 0
        assert np.array_equal(out.numpy(), alone(env, gi, b0, b1, pi)), (gi, b0, b1, pi)
    st = srv.stats()
    assert st["completed"] == 14 and st["status"] == 0
    assert st["batches"] == 2 and st["max_batch_seen"] == 8   # 14 requests, max_batch 8
    # exact decrypted scores through the server for one request
    rid = srv.submit(0, 0, 5, env["probes"][0][1], out := torch.zeros((5, 2, 2, N), dtype=torch.int64).pin_memory())
    assert srv.wait(rid)[0] == 0
    g, nb, d, feats = env["gals"][0]
    sc = H.hers_decrypt_scores(env["ctx"], env["keys"], out.cuda(), feats.shape[0]).cpu().numpy()
    assert np.array_equal(sc.astype(np.int64), W.plain_inner_products(feats, env["probes"][0][3]))
    srv.close()


def test_admission_by_memory(env):
    # room for one 2-block d = 16 request (plus tables), not for the 5-block one
    pool = request_bytes(16, 2) + (1 << 16)
    srv = H.Server(env["ctx"], env["keys"], [(g, nb, d) for g, nb, d, _ in env["gals"]],
                   workspace_bytes=pool, max_batch=8)
    outs = []
    for b0 in (0, 2):
        out = torch.zeros((2, 2, 2, N), dtype=torch.int64).pin_memory()
        outs.append((srv.submit(0, b0, b0 + 2, env["probes"][1][1], out), b0, out))
    big = torch.zeros((5, 2, 2, N), dtype=torch.int64).pin_memory()
    rid_big = srv.submit(0, 0, 5, env["probes"][1][1], big)
    for rid, b0, out in outs:
        assert srv.wait(rid)[0] == 0
        assert np.array_equal(out.numpy(), alone(env, 0, b0, b0 + 2, 1))
    assert srv.wait(rid_big)[0] == -2          # HERS_E_NOMEM: can never fit this pool
    st = srv.stats()
    assert st["max_batch_seen"] == 1           # memory admitted one request at a time
    srv.close()
