"""Generates hers_consts.h: every compile-time constant of the CUDA library.

Moduli.  The ciphertext modulus q = q1 q2 uses the two largest primes below
2^54 with p = 1 (mod 2N), N = 4096.  The plaintext modulus t = 4169729 is the
smallest prime = 1 (mod 2N) above 2 * 128 * 127^2, so that every score
|<q, p_j>| <= d 127^2 of a d <= 128 int8 search stays below t/2 (Sec. 3.2: the
plaintext ring must hold the result of the computation).  The paper's own
t = 1032193 (Sec. 4.1), also = 1 (mod 2N), is the second plaintext modulus: it
holds the scores of L2-normalised features quantised at scale 127
(|score| < 131^2 for d <= 64), which is the regime the paper uses it in.

Search basis.  The exact ciphertext product of Alg 5, summed over the d
dimensions, is computed in a basis private to the library: the eight largest
primes r_0 > ... > r_7 below 2^30 with r = 1 (mod 2N), M = r_0 ... r_7
(about 2^240).  Both operands are centred lifts, |x| <= q/2, so the sum X of
d <= 512 negacyclic products has |X| <= d N q^2 / 2 < 2^236.  Scale-and-round
and the return to mod q use X' = X + H with H = q 2^129 (a multiple of q),
which lies in [0.06 M, 0.19 M]: the CRT sum of X' then wraps M a number of
times alpha that a 60-bit fixed-point sum of y_i / r_i decides exactly.
Residues of the basis are below 2^30, so a resident value is one centred
int32 and a product of two is below 2^58.

Roots.  For t the 2N-th root psi_t is the smallest x >= 2 with x^N = -1: it
fixes which evaluation point psi_t^(2j+1) each plaintext slot j is.  For the
other primes any primitive 2N-th root serves (their NTT domain never leaves
the library); psi = x^((p-1)/2N) for the first x that gives one.

The chi table (truncated discrete Gaussian, sigma 3.2, |e| <= 19) is computed
with 80-digit decimal arithmetic.  Run `python gen_consts.py` to rewrite the
header and `python gen_consts.py --check` to confirm it is current.
"""
import decimal
import os
import sys

N = 4096
LOGN = 12
T = 4169729
T_PAPER = 1032193
SIGMA = decimal.Decimal("3.2")
CHI_BOUND = 19


def is_prime(n):
    if n < 2:
        return False
    small = (2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37)
    for p in small:
        if n % p == 0:
            return n == p
    d, s = n - 1, 0
    while d % 2 == 0:
        d //= 2
        s += 1
    for a in small:  # deterministic for n < 3.3e24
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


def ntt_primes(count, bits=54):
    out = []
    k = ((1 << bits) - 2) // (2 * N)
    while len(out) < count:
        p = k * 2 * N + 1
        if p < (1 << bits) and is_prime(p):
            out.append(p)
        k -= 1
    return out


def smallest_psi(p):
    """Smallest x >= 2 with x^N = -1 (mod p): used for t, where it fixes the slot order."""
    x = 2
    while pow(x, N, p) != p - 1:
        x += 1
    return x


def first_psi(p):
    """x^((p-1)/2N) for the smallest x >= 2 that makes it a 2N-th root with psi^N = -1.

    Used for the RNS primes, whose NTT domain is private to the library: any
    primitive 2N-th root serves, and this one is found in a few steps.
    """
    x = 2
    while True:
        y = pow(x, (p - 1) // (2 * N), p)
        if pow(y, N, p) == p - 1:
            return y
        x += 1


def shoup(w, p):
    return (w << 64) // p


def chi_cdt():
    decimal.getcontext().prec = 80
    D = decimal.Decimal
    rho = [(-D(k * k) / (2 * SIGMA * SIGMA)).exp() for k in range(-CHI_BOUND, CHI_BOUND + 1)]
    total = sum(rho)
    out, acc = [], D(0)
    for r in rho[:-1]:
        acc += r
        v = acc / total * D(2) ** 64
        fl = int(v.to_integral_value(rounding=decimal.ROUND_FLOOR))
        # refuse an entry that 80 digits could not decide
        assert abs(v - fl) > D(10) ** -30 and abs(v - fl - 1) > D(10) ** -30
        out.append(fl)
    return out


def mixed_radix(x, radices):
    digs = []
    for r in radices:
        digs.append(x % r)
        x //= r
    return digs


def columns(x, n, bits=27):
    """x as n digits of `bits` bits, least significant first (x < 2^(n bits))."""
    assert 0 <= x < 1 << (n * bits)
    return [(x >> (bits * i)) & ((1 << bits) - 1) for i in range(n)]


def shoup32(w, p):
    return (w << 32) // p


def build():
    q1, q2 = ntt_primes(2)
    q = q1 * q2
    R = ntt_primes(8, bits=30)
    M = 1
    for r in R:
        M *= r
    H = q << 129
    mods = [q1, q2, T, T_PAPER]
    assert is_prime(T) and T % (2 * N) == 1 and T > 2 * 128 * 127 ** 2
    assert is_prime(T_PAPER) and T_PAPER % (2 * N) == 1
    C = []  # (name, value) scalar uint64 constants
    arrays = []  # (name, list)

    arrays.append(("MOD", mods))
    psis = [first_psi(p) for p in (q1, q2)] + [smallest_psi(T), smallest_psi(T_PAPER)]
    arrays.append(("PSI", psis))
    arrays.append(("NINV", [pow(N, -1, p) for p in mods]))
    arrays.append(("NINV_S", [shoup(pow(N, -1, p), p) for p in mods]))
    arrays.append(("ONE_S", [shoup(1, p) for p in mods]))              # floor(2^64 / p)
    arrays.append(("BARRETT", [(1 << 108) // p for p in (q1, q2)]))   # floor(2^108 / p)

    # lift of a residue pair (mod q1, q2) to x = x1 + q1 h in [0, q) (Garner)
    C.append(("Q1INV_Q2", pow(q1, -1, q2)))
    C.append(("Q1INV_Q2_S", shoup(pow(q1, -1, q2), q2)))
    half_q = (q - 1) // 2
    C.append(("HALFQ_LO", half_q % q1))
    C.append(("HALFQ_HI", half_q // q1))
    C.append(("Q_LO", q & ((1 << 64) - 1)))
    C.append(("Q_HI", q >> 64))

    # search basis r_0..r_7: NTT and reduction constants
    arrays.append(("SMOD", R))
    arrays.append(("SPSI", [first_psi(r) for r in R]))
    arrays.append(("SNINV", [pow(N, -1, r) for r in R]))
    arrays.append(("SNINV_S", [shoup32(pow(N, -1, r), r) for r in R]))   # floor(w 2^32 / r)
    arrays.append(("SMU", [(1 << 64) // r for r in R]))                  # Barrett, 64-bit inputs
    arrays.append(("SR32", [(1 << 32) % r for r in R]))                  # partial folds
    arrays.append(("SOFF63", [r * ((1 << 63) // r) for r in R]))         # multiple of r just below 2^63
    # extension: the centred lift x = x1 + q1 h - [neg] q mod r from x1 and the
    # 27-bit digits of h: [q1]_r, [q1 2^27]_r, [-q]_r, and the Barrett factor
    # floor(2^59 / r) of the sum
    arrays.append(("Q1_MOD_R", [q1 % r for r in R]))
    arrays.append(("LIFT_B", [(q1 << 27) % r for r in R]))
    arrays.append(("LIFT_NQ", [(-q) % r for r in R]))
    arrays.append(("MU59", [(1 << 59) // r for r in R]))
    # CRT of X' = X + H: y_i = x_i Minv_i + HM_i (mod r_i), alpha = floor(sum y_i phi_i / 2^60)
    minv = [pow(M // r, -1, r) for r in R]
    arrays.append(("MINV", minv))
    arrays.append(("MINV_S", [shoup32(m, r) for m, r in zip(minv, R)]))
    arrays.append(("HM", [(H % r) * m % r for m, r in zip(minv, R)]))
    arrays.append(("PHI", [(1 << 60) // r for r in R]))
    # X' mod q_j = sum y_i [M_i]_qj - alpha [M]_qj (return of a resident value to mod q)
    mi_cols = []
    for r in R:
        for qj in (q1, q2):
            mi_cols += columns((M // r) % qj, 2)
    arrays.append(("MI_Q_COLS", mi_cols))          # [i][j][2] 27-bit digits
    m_cols = []
    for qj in (q1, q2):
        m_cols += columns(M % qj, 2)
    arrays.append(("M_Q_COLS", m_cols))            # [j][2]
    C.append(("MU_Q144", (1 << 144) // q))
    K = (q - 1) // 2 + 8 * q
    C.append(("KROUND_LO", K & ((1 << 64) - 1)))
    C.append(("KROUND_HI", K >> 64))

    # per plaintext modulus: {t, modulus index, q1 mod t, q mod t, q^-1 mod t
    # (decryption: pt = [-r q^-1]_t with r = [t v]_q centred), t mod q_l and
    # its Shoup companion (decryption), Delta = floor(q / t) mod q_l and
    # companions (encryption), and the scale-and-round tables: with
    # t M_i = A_i q + B_i and t M = A_M q + B_M, the 27-bit digits of B_i, B_M
    # and of A_i, A_M mod q_j, and D_j = [8 + t 2^129]_qj}
    plains = []
    for idx, t in ((2, T), (3, T_PAPER)):
        delta = q // t
        b_cols, a_cols = [], []
        for r in R:
            A, B = divmod(t * (M // r), q)
            b_cols += columns(B, 4)
            for qj in (q1, q2):
                a_cols += columns(A % qj, 2)
        AM, BM = divmod(t * M, q)
        am_cols = []
        for qj in (q1, q2):
            am_cols += columns(AM % qj, 2)
        dj = [(8 + (t << 129)) % qj for qj in (q1, q2)]
        u32 = lambda xs: ", ".join(f"{x}u" for x in xs)
        plains.append(
            "{ %dULL, %d, %dULL, %dULL, %dULL, { %s }, { %s }, { %s }, { %s }, { %s }, { %s }, { %s }, { %s }, { %s } }" % (
                t, idx, q1 % t, q % t, pow(q % t, -1, t),
                ", ".join(f"{t % x}ULL" for x in (q1, q2)),
                ", ".join(f"{shoup(t % x, x)}ULL" for x in (q1, q2)),
                ", ".join(f"{delta % x}ULL" for x in (q1, q2)),
                ", ".join(f"{shoup(delta % x, x)}ULL" for x in (q1, q2)),
                u32(b_cols), u32(columns(BM, 4)), u32(a_cols), u32(am_cols),
                ", ".join(f"{x}ULL" for x in dj)))
    arrays.append(("PLAIN", plains))

    # sanity of the ranges the kernels rely on
    assert q1 > q2 and q.bit_length() == 108 and q > 1 << 107
    assert all(r < 1 << 30 and r > 1 << 29 for r in R) and len(set(R)) == 8
    assert max(R) < 2 * min(R)  # a residue mod r_i is reduced mod r_k by one subtraction
    xmax = 512 * N * q * q // 2  # |X| for d <= 512
    assert H - xmax > M // 16 and H + xmax < M // 5  # X'/M in [1/16, 1/5]
    # alpha from 60-bit fixed point: error below 2^-27, far inside the margins above
    assert sum(((1 << 60) // r) * (r - 1) for r in R) < 1 << 64
    # scale-and-round magnitudes: column sums below 2^61, R below 2^142
    assert 8 * (1 << 30) * (1 << 27) < 1 << 61
    assert 8 * (1 << 30) * q + K < 1 << 142
    assert (1 << 144) // q < 1 << 37
    # tensor: centred residues below 2^29, products below 2^58; a partial fold
    # leaves |s| < 2^61 + 2^32, then 8 dimensions add below 2^62 (middle term)
    assert all((r - 1) // 2 < 1 << 29 for r in R)
    assert (1 << 61) + (1 << 32) + 8 * (1 << 59) < 1 << 63
    # batched tensor (Karatsuba): S sums products of two sums of centred
    # residues, |(a0 + a1)(b0 + b1)| <= (r - 1)^2 < 2^60; 4 dimensions after a
    # partial fold, or 7 from zero, stay below 2^63 - r (fold_full's range)
    assert all((1 << 61) + (1 << 32) + 4 * (r - 1) ** 2 < (1 << 63) - r for r in R)
    assert all(7 * (r - 1) ** 2 < (1 << 63) - r for r in R)
    # extension: the sum S = x1 + hl [q1]_r + hh [q1 2^27]_r (+ [-q]_r) of
    # x1, h < 2^54 stays below 2^59, so S >> 27 and floor(2^59 / r) fit 32
    # bits, and S - est r lies in [0, 3r) with 3r < 2^32
    assert q1 < 1 << 54 and q2 < 1 << 54
    assert all((1 << 54) + r + 2 * ((1 << 27) - 1) * (r - 1) < 1 << 59 for r in R)
    assert all((1 << 59) // r < 1 << 32 and 3 * r < 1 << 32 for r in R)

    cdt = chi_cdt()
    return mods, psis, C, arrays, cdt


def header():
    mods, psis, C, arrays, cdt = build()
    o = ["/* Generated by gen_consts.py -- do not edit. */",
         "#pragma once",
         "#include <stdint.h>",
         "",
         "namespace hers {",
         f"constexpr int N = {N};",
         f"constexpr int LOGN = {LOGN};",
         "constexpr int NUM_Q = 2;       /* q1, q2 */",
         "constexpr int MOD_T = 2;       /* index of the default t in the modulus arrays */",
         "constexpr int MOD_T_PAPER = 3; /* index of the paper's t */",
         "constexpr int NUM_MODS = 4;",
         "constexpr int NUM_S = 8;       /* search basis r_0 .. r_7 */",
         "constexpr int CHI_MIN = -19;",
         "constexpr int CHI_LEN = 38;",
         ""]
    for name, v in C:
        o.append(f"constexpr uint64_t {name} = {v}ULL;")
    o.append("")
    for name, vals in arrays:
        body = ", ".join(v if isinstance(v, str) else f"{v}ULL" for v in vals)
        o.append(f"#define HERS_{name}_INIT {{ {body} }}")
    o.append("#define HERS_CHI_CDT_INIT { " + ", ".join(f"{v}ULL" for v in cdt) + " }")
    o += ["}  // namespace hers", ""]
    return "\n".join(o)


def main(argv):
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "hers_consts.h")
    text = header()
    if len(argv) > 1 and argv[1] == "--check":
        cur = open(out).read() if os.path.exists(out) else ""
        if cur != text:
            print("hers_consts.h is stale")
            return 1
        return 0
    with open(out, "w") as f:
        f.write(text)
    return 0


if __name__ == "__main__":
    sys.exit(main(sys.argv))
