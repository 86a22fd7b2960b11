"""Host check of the search basis: the generated constants and the exact
scale-and-round / CRT they drive (CPU, exact Python integers).

The library computes the tensor sums X of a search (Alg 5's exact product
before rounding, summed over the dimensions) mod eight primes below 2^30 and
reconstructs X + q 2^129 by the CRT.  This test reads hers_consts.h, re-derives
every search-basis constant from its definition, and runs the kernels'
arithmetic step by step (the 32-bit Shoup products, the fixed-point overflow
count alpha, the 27-bit digit columns, the quotient estimate and its
correction) against exact rounding round(t X / q) for both plaintext moduli,
at the bound |X| = d N q^2 / 2 of d <= 512, on rounding boundaries, and on
random values; the return of centred lifts to mod q (enrollment); and the
extension's reduction of a centred lift mod each r_i.
"""
import os
import random
import re

import pytest

HDR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                   "paper_2003_12197_gb300", "csrc", "hers_consts.h")
N = 4096


@pytest.fixture(scope="module", name="c")
def consts():
    src = open(HDR).read()

    def arr(name):
        m = re.search(r"#define HERS_%s_INIT \{ (.*) \}\n" % name, src)
        return [int(x.rstrip("ULu")) for x in m.group(1).split(", ")]

    def scal(name):
        return int(re.search(r"constexpr uint64_t %s = (\d+)ULL" % name, src).group(1))

    pl = re.search(r"#define HERS_PLAIN_INIT \{ (.*) \}\n", src).group(1)
    ents = re.findall(r"\{ (\d+)ULL, (\d+), (\d+)ULL, (\d+)ULL, (\d+)ULL, " + r", ".join([r"\{ (.*?) \}"] * 9) + r" \}", pl)

    def nums(s):
        return [int(x.rstrip("ULu")) for x in s.split(", ")]

    plains = [dict(t=int(e[0]), b_cols=nums(e[9]), bm_cols=nums(e[10]), a_cols=nums(e[11]),
                   am_cols=nums(e[12]), dshift=nums(e[13])) for e in ents]
    mods = arr("MOD")
    return dict(q1=mods[0], q2=mods[1], R=arr("SMOD"), MINV=arr("MINV"), MINV_S=arr("MINV_S"), HM=arr("HM"),
                PHI=arr("PHI"), MIQ=arr("MI_Q_COLS"), MQ=arr("M_Q_COLS"), SR32=arr("SR32"), SMU=arr("SMU"),
                SOFF63=arr("SOFF63"), MU=scal("MU_Q144"), K=(scal("KROUND_HI") << 64) | scal("KROUND_LO"),
                Q=(scal("Q_HI") << 64) | scal("Q_LO"), plains=plains, Q1R=arr("Q1_MOD_R"),
                LB=arr("LIFT_B"), LNQ=arr("LIFT_NQ"), MU59=arr("MU59"), Q1INV=scal("Q1INV_Q2"),
                HQLO=scal("HALFQ_LO"), HQHI=scal("HALFQ_HI"))


def is_prime(n):
    if n < 2:
        return False
    for p in (2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37):
        if n % p == 0:
            return n == p
    d, s = n - 1, 0
    while d % 2 == 0:
        d //= 2
        s += 1
    for a in (2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37):
        x = pow(a, d, n)
        if x in (1, n - 1):
            continue
        for _ in range(s - 1):
            x = x * x % n
            if x == n - 1:
                break
        else:
            return False
    return True


def cols(x, n):
    return [(x >> (27 * i)) & ((1 << 27) - 1) for i in range(n)]


def test_constants_follow_their_definitions(c):
    R, q1, q2 = c["R"], c["q1"], c["q2"]
    q = q1 * q2
    assert c["Q"] == q and q.bit_length() == 108
    assert len(set(R)) == 8 and all(is_prime(r) and r % (2 * N) == 1 and r < 1 << 30 for r in R)
    M = 1
    for r in R:
        M *= r
    H = q << 129
    for i, r in enumerate(R):
        Mi = M // r
        assert c["MINV"][i] == pow(Mi, -1, r) and c["MINV_S"][i] == (c["MINV"][i] << 32) // r
        assert c["HM"][i] == (H % r) * c["MINV"][i] % r
        assert c["PHI"][i] == (1 << 60) // r
        assert c["SR32"][i] == (1 << 32) % r and c["SMU"][i] == (1 << 64) // r
        assert c["SOFF63"][i] % r == 0 and (1 << 63) - r < c["SOFF63"][i] <= 1 << 63
        for j, qj in enumerate((q1, q2)):
            assert c["MIQ"][(i * 2 + j) * 2:(i * 2 + j) * 2 + 2] == cols(Mi % qj, 2)
    for j, qj in enumerate((q1, q2)):
        assert c["MQ"][j * 2:j * 2 + 2] == cols(M % qj, 2)
    assert c["MU"] == (1 << 144) // q and c["K"] == (q - 1) // 2 + 8 * q
    for P in c["plains"]:
        t = P["t"]
        for i, r in enumerate(R):
            A, B = divmod(t * (M // r), q)
            assert P["b_cols"][i * 4:i * 4 + 4] == cols(B, 4)
            for j, qj in enumerate((q1, q2)):
                assert P["a_cols"][(i * 2 + j) * 2:(i * 2 + j) * 2 + 2] == cols(A % qj, 2)
        AM, BM = divmod(t * M, q)
        assert P["bm_cols"] == cols(BM, 4)
        assert P["am_cols"] == sum((cols(AM % qj, 2) for qj in (q1, q2)), [])
        assert P["dshift"] == [(8 + (t << 129)) % qj for qj in (q1, q2)]
    # the ranges the kernels rely on
    xmax = 512 * N * q * q // 2
    assert M // 16 < H - xmax and H + xmax < M // 5


def shoup32(x, w, ws, r):
    return (x * w - ((x * ws) >> 32) * r) & 0xFFFFFFFF


def crt_y(c, x):
    """The kernels' crt_y: y_i and the overflow count alpha of X' = X + q 2^129."""
    y, acc = [], 0
    for i, r in enumerate(c["R"]):
        v = shoup32(x[i], c["MINV"][i], c["MINV_S"][i], r) + c["HM"][i]
        assert v < 3 * r
        v = v - 2 * r if v >= 2 * r else v
        v = v - r if v >= r else v
        y.append(v)
        acc += v * c["PHI"][i]
    assert acc < 1 << 64
    return y, acc >> 60


def combine_q(c, y, alpha, cols_, mcols, j, extra):
    qj = (c["q1"], c["q2"])[j]
    c0 = sum(y[i] * cols_[(i * 2 + j) * 2] for i in range(8))
    c1 = sum(y[i] * cols_[(i * 2 + j) * 2 + 1] for i in range(8))
    assert c0 < 1 << 63 and c1 < 1 << 63
    s0 = c0 - alpha * mcols[j * 2] + extra + 16 * qj
    s1 = c1 - alpha * mcols[j * 2 + 1]
    assert 0 < s0 < 1 << 63 and s1 > -(1 << 30)
    v = (s1 << 27) + s0
    assert 0 < v < 1 << 108
    return v % qj


def scale_round(c, X, P):
    q = c["Q"]
    y, alpha = crt_y(c, [X % r for r in c["R"]])
    col = []
    for w in range(4):
        s = sum(y[i] * P["b_cols"][i * 4 + w] for i in range(8))
        assert s < 1 << 64
        col.append(s - alpha * P["bm_cols"][w])
    Rm = (col[0] + (col[1] << 27) + (col[2] << 54) + (col[3] << 81) + c["K"]) % (1 << 128)
    Rs = col[3] * 2 + (col[2] >> 26) + (col[1] >> 53) + ((c["K"] >> 64) >> 16)
    assert 0 < Rs < 1 << 63
    Q = (Rs * c["MU"]) >> 64
    rem = (Rm - Q * q) % (1 << 128)
    if rem >> 127:
        rem -= 1 << 128
    if rem < 0:
        Q -= 1
    elif rem >= q:
        Q += 1
    return [combine_q(c, y, alpha, P["a_cols"], P["am_cols"], j, Q - P["dshift"][j]) for j in range(2)]


def test_scale_and_round_is_exact(c):
    q, q1, q2 = c["Q"], c["q1"], c["q2"]
    xmax = 512 * N * q * q // 2
    rng = random.Random(31337)
    base = [0, 1, -1, xmax, -xmax, xmax - 1, -xmax + 1, q // 2, -(q // 2), q, -q]
    base += [rng.randint(-xmax, xmax) for _ in range(400)]
    for P in c["plains"]:
        t = P["t"]
        cases = list(base)
        for _ in range(100):  # one unit either side of a rounding boundary t X / q = k + 1/2
            k = rng.randint(-(xmax * t // q), xmax * t // q)
            X = (k * q + q // 2) // t
            cases += [X - 1, X, X + 1]
        for X in cases:
            want = (t * X + (q - 1) // 2) // q
            assert scale_round(c, X, P) == [want % q1, want % q2], X


def test_centred_lift_returns_to_mod_q(c):
    q, q1, q2 = c["Q"], c["q1"], c["q2"]
    rng = random.Random(7)
    for v in [0, 1, -1, (q - 1) // 2, -((q - 1) // 2)] + [rng.randint(-(q // 2), q // 2) for _ in range(300)]:
        y, alpha = crt_y(c, [v % r for r in c["R"]])
        assert [combine_q(c, y, alpha, c["MIQ"], c["MQ"], j, 0) for j in range(2)] == [v % q1, v % q2]


def test_partial_fold_keeps_the_residue(c):
    rng = random.Random(11)
    for i, r in enumerate(c["R"]):
        for _ in range(200):
            s = rng.randint(-(1 << 63) + 1, (1 << 63) - 1)
            hi, lo = s >> 32, s & 0xFFFFFFFF
            f = hi * c["SR32"][i] + lo  # the kernels' pfold
            assert f % r == s % r and abs(f) < (1 << 61) + (1 << 32)
            # 8 dimensions of the middle sum (2 products, below 2^59) and 16 of
            # the outer ones (1 product, below 2^58) stay below 2^63
            assert abs(f) + 8 * (1 << 59) < 1 << 63 and abs(f) + 16 * (1 << 58) < 1 << 63
            # the batched kernel's Karatsuba sums: 4 products of (a0 + a1)(b0 + b1)
            assert abs(f) + 4 * (r - 1) ** 2 < (1 << 63) - r
            u = (f + c["SOFF63"][i]) & ((1 << 64) - 1)
            qe = (u * c["SMU"][i]) >> 64
            rr = (u - qe * r) & 0xFFFFFFFF
            assert rr < 2 * r and (rr if rr < r else rr - r) == s % r


def test_extension_reduces_the_centred_lift(c):
    """The extension kernel's steps: Garner digit h of the residue pair, the sign
    of x = x1 + q1 h against (q-1)/2 from the stored (q-1)/2 = HI q1 + LO, and
    x - [neg] q mod r_i from x1 and the 27-bit digits of h (sum below 2^59,
    Barrett estimate short by at most 2), against v mod r_i for the centred v."""
    q, q1, q2 = c["Q"], c["q1"], c["q2"]
    assert c["Q1INV"] == pow(q1, -1, q2) and c["HQHI"] * q1 + c["HQLO"] == (q - 1) // 2
    rng = random.Random(5)
    half = (q - 1) // 2
    vals = [0, 1, -1, half, -half, half - 1, -half + 1, q1, -q1, q2, -q2, q1 - 1, 1 << 100, -(1 << 100)]
    vals += [rng.randint(-half, half) for _ in range(2000)]
    for v in vals:
        x1, x2 = v % q1, v % q2
        h = (x2 - x1 % q2) * c["Q1INV"] % q2
        neg = h > c["HQHI"] or (h == c["HQHI"] and x1 > c["HQLO"])
        assert x1 + q1 * h - neg * q == v
        hl, hh = h & ((1 << 27) - 1), h >> 27
        for i, r in enumerate(c["R"]):
            s = x1 + hl * c["Q1R"][i] + hh * c["LB"][i] + (c["LNQ"][i] if neg else 0)
            assert s < 1 << 59
            est = ((s >> 27) * c["MU59"][i]) >> 32
            rem = s - est * r
            assert 0 <= rem < 3 * r
            assert rem % r == v % r, (v, i)


def test_karatsuba_middle_term(c):
    """The batched kernel's middle tensor component: with T0 = sum a0 b0,
    T2 = sum a1 b1 and S = sum (a0 + a1)(b0 + b1) reduced to [0, r) (x0, x2,
    xs), x1 = ((xs + 2r - x0 - x2) - 2r if >= 2r) - r if >= r equals
    sum (a0 b1 + a1 b0) mod r, at the extreme centred residues and at random."""
    rng = random.Random(13)
    for r in c["R"]:
        h = (r - 1) // 2
        for _ in range(300):
            d = rng.randint(1, 16)
            pick = lambda: rng.choice([h, -h, 0, 1, -1, rng.randint(-h, h)])
            a = [(pick(), pick()) for _ in range(d)]
            b = [(pick(), pick()) for _ in range(d)]
            t0 = sum(x[0] * y[0] for x, y in zip(a, b))
            t2 = sum(x[1] * y[1] for x, y in zip(a, b))
            s = sum((x[0] + x[1]) * (y[0] + y[1]) for x, y in zip(a, b))
            x0, x2, xs = t0 % r, t2 % r, s % r
            v = xs + 2 * r - x0 - x2
            assert 0 < v < 3 * r and v < 1 << 32
            v = v - 2 * r if v >= 2 * r else v
            v = v - r if v >= r else v
            assert v == sum(x[0] * y[1] + x[1] * y[0] for x, y in zip(a, b)) % r
