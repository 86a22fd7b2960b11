"""Scale-and-round at the largest tensor sums the search can form.

The exact product sums X of the search are bounded by |X| <= d N q^2 / 2 for
centred operands (|coefficient| <= (q-1)/2) and d <= 512; the library's CRT
over its search basis relies on that bound.  Ciphertexts drawn by encryption
stay far below it, so these cases feed canonical ciphertexts whose every
coefficient is +-(q-1)/2 through the public calls (hers_probe_prepare,
hers_search_stream) at d = 512:
  - all +(q-1)/2 on both sides: the middle tensor component reaches
    d N (q-1)^2 / 2 at coefficient N-1 and runs down to -(that) at 0;
  - mixed signs per polynomial;
  - seeded random signs per coefficient.
Each score ciphertext is compared with the oracle's (which sums over Z and
divides exactly) bit for bit.
"""
import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2003_12197_gb300 as H  # noqa: E402

N = 4096
D = 512
KEY_SEED = 1004
Q1, Q2 = 18014398509309953, 18014398509293569
Q = Q1 * Q2
HALF = (Q - 1) // 2


def residues(signs):
    """Canonical residues [..][2 limbs][N] of sign * (q-1)/2 for a +-1 array [..][N]."""
    out = np.empty(signs.shape[:-1] + (2, N), dtype=np.uint64)
    for j, qj in enumerate((Q1, Q2)):
        pos, neg = HALF % qj, (Q - HALF) % qj
        out[..., j, :] = np.where(signs > 0, np.uint64(pos), np.uint64(neg))
    return out


@pytest.fixture(scope="module")
def env():
    H.build_library()
    ctx = H.Context(0)
    keys = H.hers_keygen(ctx, KEY_SEED)
    _, _, oevk = O.keygen(KEY_SEED)
    yield ctx, keys, oevk
    keys.close()
    ctx.close()


def sign_patterns():
    rng = np.random.default_rng(2026)
    ones = np.ones((D, 2, N), dtype=np.int64)
    mixed_p = ones.copy()
    mixed_p[:, 1, :] = -1
    mixed_g = ones.copy()
    mixed_g[:, 0, :] = -1
    rand_p = rng.choice([-1, 1], size=(D, 2, N))
    rand_g = rng.choice([-1, 1], size=(D, 2, N))
    return {"all_positive": (ones, ones), "mixed": (mixed_p, mixed_g), "random": (rand_p, rand_g)}


@pytest.mark.parametrize("case", ["all_positive", "mixed", "random"])
def test_extreme_operands_bit_exact(env, case):
    ctx, keys, oevk = env
    sp, sg = sign_patterns()[case]
    pct = residues(sp)  # [D][2 polys][2 limbs][N]
    gct = residues(sg)
    probe = torch.from_numpy(pct.view(np.int64)).cuda()
    gallery = torch.from_numpy(gct.view(np.int64)[None]).cuda()  # [1 block][D][2][2][N]
    pr = H.hers_probe_prepare(ctx, probe)
    sc = H.hers_search_stream(ctx, keys, gallery, 1, D, [pr])
    H.hers_check(ctx)
    got = H.to_u64(sc)[0, 0]
    want, st = O.search_block(pct, gct, oevk)
    assert np.array_equal(got, want)
