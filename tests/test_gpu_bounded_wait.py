"""The bounded wait of the streaming kernels gives up, reports HERS_E_TIMEOUT
through the context's error flag, and leaves the context usable.

The failure is made on purpose without a fault: one thread waits on an
mbarrier that nothing completes, with a short budget of global time."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2003_12197_gb300 as H  # noqa: E402


@pytest.mark.parametrize("limit_ms", [5, 50])
def test_wait_runs_out_and_context_survives(limit_ms):
    H.build_library()
    ctx = H.Context(0)
    rc, ms = H.hers_selftest_wait_timeout(ctx, limit_ms * 1_000_000)
    assert rc == H.HERS_E_TIMEOUT
    # the budget is global time; the kernel ends soon after it
    assert limit_ms * 0.9 <= ms <= limit_ms + 250, ms
    assert "gave up" in H.lib().hers_last_error(ctx.h).decode()
    # the flag was cleared and the context still searches correctly
    H.hers_check(ctx)
    keys = H.hers_keygen(ctx, 31)
    m, d = 300, 8
    feats = W.gallery_features(m, d, 32)
    q = W.probe_for_mate(5, d, 32, 33)
    gal, _ = H.hers_encrypt_gallery(ctx, keys, torch.from_numpy(feats).cuda(), 34)
    pr = H.hers_probe_prepare(ctx, H.hers_encrypt_probe(ctx, keys, torch.from_numpy(q).cuda(), 35))
    sc = H.hers_search(ctx, keys, gal, 1, d, pr)
    scores = H.hers_decrypt_scores(ctx, keys, sc, m).cpu().numpy().astype(np.int64)
    assert np.array_equal(scores, W.plain_inner_products(feats, q))
    H.hers_check(ctx)
    keys.close()
    ctx.close()


def test_wait_limit_out_of_range_is_rejected():
    H.build_library()
    ctx = H.Context(0)
    for bad in (0, 999_999, 3_000_000_000):
        rc, _ = H.hers_selftest_wait_timeout(ctx, bad)
        assert rc == -1
    ctx.close()
