"""Pins of the CPU oracle against things other than itself (CPU only).

Each test checks one oracle function against what the paper and mathematics
fix, by an independent route:

  chacha20 / samplers   the `cryptography` package's ChaCha20 keystream (RFC 8439)
                        and an independent re-implementation of the word layout;
  chi table             decimal arithmetic vs the oracle's rational-interval table;
  P1 products           Kronecker substitution with Python big integers, and
                        hand-checkable cases (x^(n-1) * x = -1, (1+x)^2 at n = 2);
  P2 encoding           brute-force psi_t, direct evaluation at psi_t^(2j+1) with
                        pow(), the slot-wise homomorphism with a big-integer product;
  keys / encryption     the RLWE relations pk0 + pk1 s = -e, evk_j = -e_j + g_j s^2,
                        ct0 + ct1 s = Delta m + small, checked with big integers;
  P3 exactness          decrypted scores equal the plaintext inner products
                        (Eq. 1), also via the paper-literal per-product form
                        (Alg 5 per product) and before relinearisation;
  scale-round           round(t X / q) by exact Fractions on a Kronecker X;
  key switch            c0' + c1' s - (c0 + c1 s + c2 s^2) = -sum_j D_j e_j;
  P4 noise              below q / (2t);
  P5 top-1              planted mate recovered at 4096 entries, d = 64;
  P6 op counts          Table 2: ceil(m/n) d products, ceil(m/n)(d-1) additions,
                        0 rotations, and one relinearisation per block;
  P7 determinism        same seed -> same bytes;
  P8 ties / bound       no rounding tie, |X| <= d 2n ((q-1)/2)^2.
"""
import decimal
import os
import re
from fractions import Fraction

import numpy as np
import pytest

import oracle as O
import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
Q1, Q2, Q, T = O.Q1, O.Q2, O.Q, O.T


# ---------------------------------------------------------------- helpers

def kron_negacyclic(a, b):
    """Negacyclic product over Z by Kronecker substitution (Python big ints)."""
    n = len(a)
    w = 2 * max(1, max(abs(int(x)) for x in list(a) + list(b)).bit_length()) + n.bit_length() + 4
    A = sum(int(x) << (w * j) for j, x in enumerate(a))
    B = sum(int(x) << (w * j) for j, x in enumerate(b))
    C = A * B
    c = []
    for _ in range(2 * n):
        dgt = C & ((1 << w) - 1)
        if dgt >> (w - 1):
            dgt -= 1 << w
        c.append(dgt)
        C = (C - dgt) >> w
    assert C == 0
    return [c[k] - c[k + n] for k in range(n)]


def ct_ints(ct):
    """[2][2][n] residues -> two lists of ints in [0, q)."""
    return O.res_to_int(ct[0]), O.res_to_int(ct[1])


def sym(x, m):
    x %= m
    return x - m if x > (m - 1) // 2 else x


def chacha_keystream_words(seed, purpose, obj, nblocks):
    crypto = pytest.importorskip("cryptography.hazmat.primitives.ciphers")
    key = int(seed).to_bytes(8, "little") + bytes(24)
    nonce12 = int(purpose).to_bytes(4, "little") + int(obj).to_bytes(8, "little")
    out = []
    for c in range(nblocks):
        ciph = crypto.Cipher(crypto.algorithms.ChaCha20(key, c.to_bytes(4, "little") + nonce12),
                             mode=None)
        out.append(np.frombuffer(ciph.encryptor().update(bytes(64)), dtype="<u4"))
    return np.concatenate(out).astype(np.uint64)


def oracle_cdt():
    txt = open(os.path.join(ROOT, "oracle", "cdt_table.h")).read()
    body = txt[txt.index("{") + 1: txt.index("}")]
    return [int(v) for v in re.findall(r"(\d+)ULL", body)]


# ---------------------------------------------------------------- PRF, samplers, chi

def test_chacha20_block_matches_rfc8439_implementation():
    crypto = pytest.importorskip("cryptography.hazmat.primitives.ciphers")
    rng = np.random.default_rng(5)
    for _ in range(8):
        key = rng.integers(0, 2**32, 8, dtype=np.uint64).astype(np.uint32)
        nonce = rng.integers(0, 2**32, 3, dtype=np.uint64).astype(np.uint32)
        ctr = int(rng.integers(0, 2**32))
        got = O.chacha20_block(key, ctr, nonce)
        c = crypto.Cipher(crypto.algorithms.ChaCha20(key.tobytes(),
                                                     ctr.to_bytes(4, "little") + nonce.tobytes()),
                          mode=None)
        want = np.frombuffer(c.encryptor().update(bytes(64)), dtype="<u4")
        assert np.array_equal(got, want)


def test_samplers_follow_the_stream_layout():
    n, seed, purpose, obj = 64, 0x1234_5678_9ABC, 0x21, 77
    words = chacha_keystream_words(seed, purpose, obj, nblocks=8)
    # ternary: 32-bit word k (attempt 0), value (w mod 3) - 1
    tern = O.sample(seed, purpose, obj, n, kind=0)
    assert all(w < 0xFFFFFFFF for w in words[:n])
    assert np.array_equal(tern, (words[:n] % 3).astype(np.int64) - 1)
    # 64-bit word k = words (2k, 2k+1)
    w64 = [int(words[2 * k]) | (int(words[2 * k + 1]) << 32) for k in range(n)]
    uni = O.sample(seed, purpose, obj, n, kind=2, qj=Q1)
    assert [int(v) for v in uni] == [w & ((1 << 54) - 1) for w in w64]  # no rejection here
    cdt = oracle_cdt()
    gau = O.sample(seed, purpose, obj, n, kind=1)
    want = [int(np.searchsorted(np.array(cdt, dtype=object), w, side="right")) - 19 for w in w64]
    assert [int(v) for v in gau] == want


def test_chi_table_two_ways():
    """The oracle's rational-interval table equals a 80-digit decimal evaluation."""
    decimal.getcontext().prec = 80
    D = decimal.Decimal
    two_s2 = 2 * D("3.2") ** 2
    rho = [(-D(k * k) / two_s2).exp() for k in range(-19, 20)]
    tot = sum(rho)
    want, acc = [], D(0)
    for i in range(38):
        acc += rho[i]
        want.append(int((acc / tot * D(2) ** 64).to_integral_value(rounding=decimal.ROUND_FLOOR)))
    assert oracle_cdt() == want


def test_chi_statistics():
    """Mean ~ 0 and variance ~ the truncated sigma^2 within sampling error."""
    xs = np.concatenate([O.sample(99, 0x03, o, 4096, kind=1) for o in range(16)])
    n = len(xs)
    w = np.exp(-np.arange(-19, 20) ** 2 / (2 * 3.2 ** 2))
    var = float((np.arange(-19, 20) ** 2 * w).sum() / w.sum())
    assert abs(xs.mean()) < 5 * np.sqrt(var / n)
    assert abs(xs.var() - var) < 5 * var * np.sqrt(2.0 / n)
    assert xs.min() >= -19 and xs.max() <= 19
    tern = np.concatenate([O.sample(99, 0x01, o, 4096, kind=0) for o in range(8)])
    for v in (-1, 0, 1):
        frac = (tern == v).mean()
        assert abs(frac - 1 / 3) < 5 * np.sqrt(2 / 9 / len(tern))


def test_uniform_sampler_range():
    for qj in (Q1, Q2):
        u = O.sample(7, 0x02, 0, 4096, kind=2, qj=qj).astype(np.uint64)
        assert int(u.max()) < qj
        assert abs(float(u.astype(np.float64).mean()) / qj - 0.5) < 0.03


# ---------------------------------------------------------------- P1 products

@pytest.mark.parametrize("n", [8, 64, 4096])
def test_negacyclic_product_vs_kronecker(n):
    rng = np.random.default_rng(n)
    lim = 1 << 107
    a = [int.from_bytes(rng.bytes(14), "little") % (2 * lim - 1) - (lim - 1) for _ in range(n)]
    b = [int.from_bytes(rng.bytes(14), "little") % (2 * lim - 1) - (lim - 1) for _ in range(n)]
    assert O.negacyclic_z(a, b) == kron_negacyclic(a, b)


def test_negacyclic_hand_cases():
    n = 16
    xn1 = [0] * n
    xn1[n - 1] = 1
    x = [0] * n
    x[1] = 1
    assert O.negacyclic_z(xn1, x) == [-1] + [0] * (n - 1)          # x^(n-1) * x = -1
    assert O.negacyclic_z([1, 1], [1, 1]) == [0, 2]               # (1+x)^2 = 2x at n = 2
    big = (1 << 106) + 12345
    assert O.negacyclic_z([big, 0], [-big, 0]) == [-big * big, 0]


# ---------------------------------------------------------------- P2 encoding

@pytest.mark.parametrize("n", [8, 64, 4096])
def test_psi_t_is_smallest_primitive_root(n):
    psi = O.psi_t(n)
    assert pow(psi, n, T) == T - 1
    if n <= 64:
        assert all(pow(x, n, T) != T - 1 for x in range(2, psi))


def test_decode_is_evaluation_at_odd_powers():
    n = 64
    rng = np.random.default_rng(3)
    m = rng.integers(0, T, n).astype(np.uint32)
    psi = O.psi_t(n)
    slots = O.decode(m, n)
    for j in (0, 1, 17, 63):
        r = pow(psi, 2 * j + 1, T)
        v = sum(int(m[k]) * pow(r, k, T) for k in range(n)) % T
        assert slots[j] == sym(v, T)


@pytest.mark.parametrize("n", [64, 4096])
def test_encode_decode_round_trip(n):
    rng = np.random.default_rng(n + 1)
    slots = rng.integers(-(T - 1) // 2, (T - 1) // 2 + 1, n)
    assert np.array_equal(O.decode(O.encode(slots, n), n), slots)


def test_slotwise_homomorphism_and_constant_encoding():
    n = 64
    rng = np.random.default_rng(11)
    a = rng.integers(-127, 128, n)
    b = rng.integers(-127, 128, n)
    ma, mb = O.encode(a, n), O.encode(b, n)
    prod = [v % T for v in kron_negacyclic([int(x) for x in ma], [int(x) for x in mb])]
    assert np.array_equal(O.decode(np.array(prod, dtype=np.uint32), n), a * b)
    c = O.encode(np.full(n, -42), n)
    assert int(c[0]) == T - 42 and not c[1:].any()


# ---------------------------------------------------------------- keys and encryption

def _poly_mul_q(a, s):
    return [v % Q for v in kron_negacyclic(a, s)]


def test_keygen_rlwe_relations():
    n = 64
    sk, pk, evk = O.keygen(2024, n)
    s = [int(v) for v in sk]
    assert set(s) <= {-1, 0, 1}
    pk0, pk1 = ct_ints(pk)
    e = [sym(x + y, Q) for x, y in zip(pk0, _poly_mul_q(pk1, s))]
    assert max(abs(v) for v in e) <= 19 and any(e)
    s2 = kron_negacyclic(s, s)
    g = [Q2 * pow(Q2, -1, Q1), Q1 * pow(Q1, -1, Q2)]
    assert g[0] % Q1 == 1 and g[0] % Q2 == 0 and (g[0] + g[1]) % Q == 1
    for j in range(2):
        e0, e1 = ct_ints(evk[j])
        ej = [sym(x + y - g[j] * z, Q) for x, y, z in zip(e0, _poly_mul_q(e1, s), s2)]
        assert max(abs(v) for v in ej) <= 19 and any(ej)


def test_encrypt_relation_and_decrypt():
    n = 64
    sk, pk, _ = O.keygen(1, n)
    s = [int(v) for v in sk]
    rng = np.random.default_rng(2)
    slots = rng.integers(-1000, 1000, n)
    m = O.encode(slots, n)
    ct = O.encrypt(pk, m, seed=5, purpose_base=O.PURPOSE_GALLERY, obj=3, n=n)
    c0, c1 = ct_ints(ct)
    delta = Q // T
    noise = [sym(x + y - delta * int(mm), Q) for x, y, mm in zip(c0, _poly_mul_q(c1, s), m)]
    assert max(abs(v) for v in noise) <= 2 * 19 * n + 19
    got, pt, nz = O.decrypt(sk, ct, n)
    assert np.array_equal(got, slots) and np.array_equal(pt, m)
    assert nz == max(abs(v) for v in noise)


@pytest.mark.parametrize("n", [64, 4096])
def test_decrypt_of_encrypt(n):
    sk, pk, _ = O.keygen(77, n)
    rng = np.random.default_rng(n)
    slots = rng.integers(-(T - 1) // 2, (T - 1) // 2 + 1, n)
    ct = O.encrypt(pk, O.encode(slots, n), seed=9, purpose_base=O.PURPOSE_PROBE, obj=0, n=n)
    got, _, nz = O.decrypt(sk, ct, n)
    assert np.array_equal(got, slots)
    assert nz < Q // (2 * T)


# ---------------------------------------------------------------- search, tiny brute force

@pytest.fixture(scope="module")
def tiny():
    n, d = 8, 3
    sk, pk, evk = O.keygen(31337, n)
    rng = np.random.default_rng(8)
    feats = rng.integers(-127, 128, (n, d)).astype(np.int8)
    q = rng.integers(-127, 128, d).astype(np.int8)
    g = O.encrypt_gallery_block(pk, feats, 0, seed=4, n=n)
    p = O.encrypt_probe(pk, q, seed=6, n=n)
    out, pre, st = O.search_block(p, g, evk, n, want_pre=True)
    return dict(n=n, d=d, sk=sk, pk=pk, evk=evk, feats=feats, q=q, g=g, p=p, out=out, pre=pre,
                st=st)


def test_scale_round_brute_force(tiny):
    """c_k = [round(t X_k / q)]_q with X from Kronecker products of the lifted ciphertexts."""
    n, d = tiny["n"], tiny["d"]
    X = [[0] * n for _ in range(3)]
    for i in range(d):
        a0, a1 = [[sym(v, Q) for v in pol] for pol in ct_ints(tiny["p"][i])]
        b0, b1 = [[sym(v, Q) for v in pol] for pol in ct_ints(tiny["g"][i])]
        for k, (u, v) in enumerate(zip(kron_negacyclic(a0, b0), kron_negacyclic(a1, b1))):
            X[0][k] += u
            X[2][k] += v
        for k, (u, v) in enumerate(zip(kron_negacyclic(a0, b1), kron_negacyclic(a1, b0))):
            X[1][k] += u + v
    for c in range(3):
        want = []
        for x in X[c]:
            f = Fraction(T * x, Q)
            assert f - f.__floor__() != Fraction(1, 2)
            want.append(round(f) % Q)
        assert O.res_to_int(tiny["pre"][c]) == want


def test_key_switch_relation(tiny):
    n = tiny["n"]
    s = [int(v) for v in tiny["sk"]]
    c0, c1, c2 = (O.res_to_int(tiny["pre"][c]) for c in range(3))
    o0, o1 = ct_ints(tiny["out"])
    s2 = kron_negacyclic(s, s)
    g = [Q2 * pow(Q2, -1, Q1), Q1 * pow(Q1, -1, Q2)]
    lhs = [(x + y) % Q for x, y in zip(o0, _poly_mul_q(o1, s))]
    rhs = [(a + b + c) % Q for a, b, c in zip(c0, _poly_mul_q(c1, s), _poly_mul_q(c2, s2))]
    corr = [0] * n  # sum_j D_j e_j, with e_j = -(evk_j0 + evk_j1 s - g_j s^2)
    for j, qj in enumerate((Q1, Q2)):
        e0, e1 = ct_ints(tiny["evk"][j])
        ej = [-sym(x + y - g[j] * z, Q) for x, y, z in zip(e0, _poly_mul_q(e1, s), s2)]
        assert max(abs(v) for v in ej) <= 19
        Dj = [v % qj for v in c2]
        for k, v in enumerate(kron_negacyclic(Dj, ej)):
            corr[k] += v
    assert lhs == [(r - c) % Q for r, c in zip(rhs, corr)]


def test_tiny_scores_and_counters(tiny):
    want = W.plain_inner_products(tiny["feats"], tiny["q"])
    got, _, nz = O.decrypt(tiny["sk"], tiny["out"], tiny["n"])
    assert np.array_equal(got, want)
    got3, _, _ = O.decrypt(tiny["sk"], tiny["pre"], tiny["n"])
    assert np.array_equal(got3, want)
    st = tiny["st"]
    assert st["tensor_products"] == tiny["d"] and st["tensor_adds"] == tiny["d"] - 1
    assert st["key_switches"] == 1 and st["rotations"] == 0 and st["ties"] == 0


@pytest.mark.parametrize("with_init", [False, True])
def test_per_product_form_decrypts_the_same(with_init):
    n, d = 64, 8
    sk, pk, evk = O.keygen(555, n)
    rng = np.random.default_rng(12)
    feats = rng.integers(-127, 128, (n, d)).astype(np.int8)
    q = rng.integers(-127, 128, d).astype(np.int8)
    g = O.encrypt_gallery_block(pk, feats, 0, seed=1, n=n)
    p = O.encrypt_probe(pk, q, seed=2, n=n)
    init = O.encrypt(pk, np.zeros(n, np.uint32), 3, O.PURPOSE_PROBE, 999, n) if with_init else None
    out_pp, st = O.search_block_per_product(p, g, evk, init, n)
    out, _ = O.search_block(p, g, evk, n)
    want = W.plain_inner_products(feats, q)
    assert np.array_equal(O.decrypt(sk, out_pp, n)[0], want)
    assert np.array_equal(O.decrypt(sk, out, n)[0], want)
    assert not np.array_equal(out_pp, out)
    assert st["key_switches"] == d and st["scale_rounds"] == d


def test_op_counts_table2_multi_block():
    """Table 2: ceil(m/n) d products, ceil(m/n) (d-1) additions, no rotations."""
    n, d, m = 16, 5, 40
    sk, pk, evk = O.keygen(8, n)
    feats = np.random.default_rng(1).integers(-127, 128, (m, d)).astype(np.int8)
    q = feats[17].copy()
    nb = -(-m // n)
    blocks = [O.encrypt_gallery_block(pk, feats, b, seed=3, n=n) for b in range(nb)]
    p = O.encrypt_probe(pk, q, seed=4, n=n)
    outs, st = O.search_gallery(p, blocks, evk, n)
    assert st["tensor_products"] == nb * d and st["tensor_adds"] == nb * (d - 1)
    assert st["rotations"] == 0 and st["key_switches"] == nb
    scores = np.concatenate([O.decrypt(sk, o, n)[0] for o in outs])[:m]
    assert np.array_equal(scores, W.plain_inner_products(feats, q))


def test_determinism():
    n = 32
    a = O.keygen(5, n)
    b = O.keygen(5, n)
    c = O.keygen(6, n)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    assert not np.array_equal(a[1], c[1])
    m = O.encode(np.arange(n), n)
    e1 = O.encrypt(a[1], m, 1, O.PURPOSE_GALLERY, 0, n)
    assert np.array_equal(e1, O.encrypt(a[1], m, 1, O.PURPOSE_GALLERY, 0, n))
    assert not np.array_equal(e1, O.encrypt(a[1], m, 1, O.PURPOSE_GALLERY, 1, n))
    assert not np.array_equal(e1, O.encrypt(a[1], m, 1, O.PURPOSE_PROBE, 0, n))


# ---------------------------------------------------------------- full size (n = 4096, d = 64)

@pytest.fixture(scope="module")
def full_block():
    """4,096 gallery entries at d = 64 (one block), one probe with a planted mate."""
    n, d = 4096, 64
    feats = W.gallery_features(n, d, seed=1001)
    mate = int(W.mate_indices(n, 1, seed=1002)[0])
    q = W.probe_for_mate(mate, d, gallery_seed=1001, probe_seed=1003)
    sk, pk, evk = O.keygen(1004, n)
    g = O.encrypt_gallery_block(pk, feats, 0, seed=1005, n=n)
    p = O.encrypt_probe(pk, q, seed=1006, n=n)
    out, st = O.search_block(p, g, evk, n)
    return dict(feats=feats, q=q, mate=mate, sk=sk, out=out, st=st, d=d)


def test_full_block_exact_scores_noise_and_top1(full_block):
    fb = full_block
    scores, _, noise = O.decrypt(fb["sk"], fb["out"])
    want = W.plain_inner_products(fb["feats"], fb["q"])
    assert np.array_equal(scores, want)                       # P3
    assert noise < Q // (2 * T)                                # P4
    margin_bits = (Q // (2 * T)).bit_length() - noise.bit_length()
    assert margin_bits >= 16
    assert int(np.argmax(scores)) == fb["mate"]               # P5
    st = fb["st"]
    assert st["ties"] == 0 and st["bound_violations"] == 0    # P8
    bound = fb["d"] * 2 * 4096 * ((Q - 1) // 2) ** 2
    assert st["max_x_bits"] <= bound.bit_length()


# ---------------------------------------------------------------- paper facts

def test_paper_parameter_facts():
    """Sec. 4.1: the paper's t = 1,032,193 is prime and = 1 mod 2n (so it batches)."""
    import json
    facts = json.load(open(os.path.join(ROOT, "tests", "golden", "paper_facts.json")))
    tp = facts["paper_t"]["value"]
    assert tp % (2 * facts["paper_n"]["value"]) == 1
    assert all(tp % p for p in range(2, int(tp ** 0.5) + 1))
    # the paper's t cannot hold every score of arbitrary int8 vectors (2 d 127^2 > t
    # for d >= 32), only those of L2-normalised features (|score| < 131^2 < t/2)
    assert 2 * 32 * 127 ** 2 > tp and 131 ** 2 < tp // 2
    # the default t holds |score| <= d 127^2 < t/2 for any int8 vectors, d <= 128
    assert 128 * 127 ** 2 < T // 2
    # gallery sizes: 100M entries, d = 64, two 64-bit limbs per coefficient
    blocks = -(-100_000_000 // 4096)
    assert blocks == facts["table3_blocks_100M"]["value"]
    assert round(blocks * 64 * 2 * 2 * 4096 * 8 / 1e9, 1) == 204.8


def test_block_rows_encryption_matches_full_array_form():
    n, d = 16, 3
    sk, pk, _ = O.keygen(9, n)
    feats = np.random.default_rng(4).integers(-127, 128, (3 * n - 5, d)).astype(np.int8)
    for b in range(3):
        a = O.encrypt_gallery_block(pk, feats, b, seed=12, n=n)
        r = O.encrypt_gallery_block_rows(pk, feats[b * n:(b + 1) * n], b, seed=12, n=n)
        assert np.array_equal(a, r)


def test_topk_matches_sorted_with_index_ties():
    """Stage-1 top-K: against Python's sorted() with key (-score, index), on
    small-range scores full of ties, for every k from 1 to m."""
    rng = np.random.default_rng(7)
    for m in (1, 2, 7, 50):
        s = rng.integers(-3, 4, size=m).astype(np.int32)
        want_all = sorted(range(m), key=lambda i: (-int(s[i]), i))
        for k in range(1, m + 1):
            idx, val = O.topk(s, k)
            assert list(idx) == want_all[:k]
            assert list(val) == [int(s[i]) for i in want_all[:k]]
    # k larger than m is clipped; the planted maximum comes first
    s = rng.integers(-1000, 1000, size=1000).astype(np.int32)
    s[617] = 5000
    idx, val = O.topk(s, 5000)
    assert len(idx) == 1000 and idx[0] == 617 and val[0] == 5000
    assert np.all(np.diff(val.astype(np.int64)) <= 0)


def test_rerandomization_adds_a_fresh_zero():
    """Output re-randomisation: the added ciphertext decrypts to 0 with small
    noise, the sum decrypts to the same message, and different blocks or
    seeds give different randomness."""
    n = 4096
    sk, pk, evk = O.keygen(2222)
    m = np.arange(n, dtype=np.uint32) % O.T
    ct = O.encrypt(pk, m, 3333, O.PURPOSE_PROBE, 0)
    r = O.rerandomize(pk, ct, 4444, 7)
    zero = O.encrypt(pk, np.zeros(n, dtype=np.uint32), 4444, O.PURPOSE_RERAND, 7)
    # residue-wise sum, checked against Python integers limb by limb
    for poly in range(2):
        for l, q in enumerate((O.Q1, O.Q2)):
            want = [(int(a) + int(b)) % q for a, b in zip(ct[poly, l], zero[poly, l])]
            assert list(map(int, r[poly, l])) == want
    _, pt0, noise0 = O.decrypt(sk, zero)
    assert not np.any(pt0) and noise0 < O.Q // (2 * O.T) >> 40
    _, pt, _ = O.decrypt(sk, r)
    assert np.array_equal(pt, m)
    assert not np.array_equal(O.rerandomize(pk, ct, 4444, 8), r)
    assert not np.array_equal(O.rerandomize(pk, ct, 4445, 7), r)


def test_enrollment_changes_only_its_slot():
    """Alg 6: after enrolling an entry into an empty slot v, every dimension's
    ciphertext decrypts to the old slots with slot v replaced by the entry's
    feature; the added ciphertext uses its own randomness stream."""
    n, d = 4096, 3
    sk, pk, evk = O.keygen(5151)
    feats = np.array([[7, -3, 100], [1, 2, 3]], dtype=np.int8)      # two entries, slots 0 and 1
    blk = O.encrypt_gallery_block(pk, feats, 0, 5252)
    new = np.array([-127, 55, 0], dtype=np.int8)
    v = 4000
    upd = O.enroll(pk, blk, 0, v, new, 5353)
    for i in range(d):
        slots, _, noise = O.decrypt(sk, upd[i])
        want = np.zeros(n, dtype=np.int64)
        want[:2] = feats[:, i]
        want[v] = new[i]
        assert np.array_equal(slots, want)
        assert noise < O.Q // (2 * O.T) >> 30
    again = O.enroll(pk, blk, 0, v, new, 5353)
    assert np.array_equal(again, upd)
    assert not np.array_equal(O.enroll(pk, blk, 0, v, new, 5354), upd)


def test_basew_keys_and_key_switch_identity():
    """Base-w gadget (w = 2^27, l = 4): each key satisfies
    evkw_j0 + evkw_j1 s = w^j s^2 - e_j over Z mod q with small e_j; the key
    switch satisfies c0' + c1' s - (c0 + c1 s + c2 s^2) = -sum_j D_j e_j, with
    c2 = sum_j D_j w^j, checked with Python integers."""
    n, logw = 4096, 27
    assert O.basew_digits(logw) == 4 and O.basew_digits(54) == 2 and O.basew_digits(16) == 7
    sk, pk, evk = O.keygen(7171)
    evkw = O.keygen_w(7171, 7272, logw)
    assert evkw.shape == (4, 2, 2, n)
    q = O.Q
    s = [int(x) for x in sk]
    def val(poly):        # CRT of the two limbs, centred in (-q/2, q/2)
        return [x - q if x > q // 2 else x for x in O.res_to_int(poly)]

    def mul(a, b):        # negacyclic product over Z (the pinned oracle routine; |a|, |b| < 2^107)
        return [int(x) for x in O.negacyclic_z(list(a), list(b))]
    s2 = mul(s, s)
    errs = []
    for j in range(4):
        e0, e1 = val(evkw[j, 0]), val(evkw[j, 1])
        lhs = [(x + y) % q for x, y in zip(e0, mul(e1, s))]
        e = [((pow(2, logw * j, q) * z - x) % q) for z, x in zip(s2, lhs)]
        e = [x - q if x > q // 2 else x for x in e]
        assert max(abs(x) for x in e) <= 19
        errs.append(e)
    # key switch of a random 3-component ciphertext
    rng = np.random.default_rng(5)
    ct3 = np.zeros((3, 2, n), dtype=np.uint64)
    for p in range(3):
        ct3[p, 0] = rng.integers(0, O.Q1, n, dtype=np.uint64)
        ct3[p, 1] = rng.integers(0, O.Q2, n, dtype=np.uint64)
    out = O.keyswitch_w(ct3, evkw, logw)
    c0, c1, c2 = val(ct3[0]), val(ct3[1]), val(ct3[2])
    o0, o1 = val(out[0]), val(out[1])
    lhs = [(a + b) % q for a, b in zip(o0, mul(o1, s))]
    rhs0 = [(a + b + c) % q for a, b, c in zip(c0, mul(c1, s), mul(c2, s2))]
    diff = [(x - y) % q for x, y in zip(lhs, rhs0)]
    diff = [x - q if x > q // 2 else x for x in diff]
    # exactly -sum_j D_j (*) e_j, with D_j the base-2^27 digits of c2 in [0, q)
    c2u = O.res_to_int(ct3[2])
    want = [0] * n
    for j in range(4):
        Dj = [(c >> (logw * j)) & ((1 << logw) - 1) for c in c2u]
        assert sum(Dj) > 0
        for k, v in enumerate(mul(Dj, errs[j])):
            want[k] -= v
    assert diff == want


def test_paper_plain_modulus_t1032193():
    """The paper's t = 1,032,193 (Sec. 4.1), selected at run time: psi_t by
    brute force, the encode/decode round trip and the slot-wise product, and a
    full block whose decrypted scores equal the plaintext inner products
    (L2-normalised int8 features keep |score| < 131^2 < t/2)."""
    tp = O.T_PAPER
    assert tp % (2 * 4096) == 1 and all(tp % p for p in range(2, 1016))
    O.set_plain_modulus(tp)
    try:
        assert O.plain_modulus() == tp
        psi = O.psi_t()
        assert pow(psi, 4096, tp) == tp - 1
        assert all(pow(x, 4096, tp) != tp - 1 for x in range(2, psi))
        rng = np.random.default_rng(9)
        slots = rng.integers(-(tp - 1) // 2, (tp - 1) // 2 + 1, 4096)
        assert np.array_equal(O.decode(O.encode(slots)), slots)
        sk, pk, evk = O.keygen(4242)
        m, d = 4096, 64
        feats = W.gallery_features(m, d, 4343)
        mate = int(W.mate_indices(m, 1, 4444)[0])
        q = W.probe_for_mate(mate, d, 4343, 4545)
        plain = W.plain_inner_products(feats, q)
        assert np.abs(plain).max() < 131 ** 2 < tp // 2
        osc, st = O.search_block(O.encrypt_probe(pk, q, 4646), O.encrypt_gallery_block(pk, feats, 0, 4747), evk)
        slots_out, _, noise = O.decrypt(sk, osc)
        assert np.array_equal(slots_out, plain)
        assert int(np.argmax(slots_out)) == mate
        assert noise < O.Q // (2 * tp) >> 16
    finally:
        O.set_plain_modulus(O.T)
    assert O.plain_modulus() == O.T
