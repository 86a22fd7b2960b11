"""Generates hers_consts.h: every compile-time constant of the CUDA library.

Moduli.  The ciphertext modulus q = q1 q2 uses the two largest primes below
2^54 with p = 1 (mod 2N), N = 4096; the auxiliary basis P = p1 p2 p3 (private
to the library, used for the exact ciphertext product and rounding of Alg 5)
uses the next three.  The plaintext modulus t = 4169729 is the smallest prime
= 1 (mod 2N) above 2 * 128 * 127^2, so that every score |<q, p_j>| <= d 127^2
of a d <= 128 int8 search stays below t/2 (Sec. 3.2: the plaintext ring must
hold the result of the computation).  The paper's own t = 1032193 (Sec. 4.1),
also = 1 (mod 2N), is the second plaintext modulus: it holds the scores of
L2-normalised features quantised at scale 127 (|score| < 131^2 for d <= 64),
which is the regime the paper uses it in.

Roots.  For t the 2N-th root psi_t is the smallest x >= 2 with x^N = -1: it
fixes which evaluation point psi_t^(2j+1) each plaintext slot j is.  For the
RNS primes any primitive 2N-th root serves (their NTT domain never leaves the
library); psi = x^((p-1)/2N) for the first x that gives one.

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


def build():
    primes = ntt_primes(5)
    q1, q2, p1, p2, p3 = primes
    q = q1 * q2
    P = p1 * p2 * p3
    mods = primes + [T, T_PAPER]
    assert is_prime(T) and T % (2 * N) == 1 and T > 2 * 128 * 127 ** 2
    assert is_prime(T_PAPER) and T_PAPER % (2 * N) == 1
    C = []  # (name, value) scalar uint64 constants
    arrays = []  # (name, list)

    arrays.append(("MOD", mods))
    psis = [first_psi(p) for p in primes] + [smallest_psi(T), smallest_psi(T_PAPER)]
    arrays.append(("PSI", psis))
    arrays.append(("NINV", [pow(N, -1, p) for p in mods]))
    arrays.append(("NINV_S", [shoup(pow(N, -1, p), p) for p in mods]))
    arrays.append(("ONE_S", [shoup(1, p) for p in mods]))              # floor(2^64 / p)
    arrays.append(("BARRETT", [(1 << 108) // p for p in primes]))     # floor(2^108 / p)
    arrays.append(("OFF63", [p * ((1 << 63) // p) for p in primes]))  # multiple of p just below 2^63
    arrays.append(("R27", [(1 << 27) % p for p in mods]))
    arrays.append(("R27_S", [shoup((1 << 27) % p, p) for p in mods]))
    arrays.append(("R54", [(1 << 54) % p for p in mods]))
    arrays.append(("R54_S", [shoup((1 << 54) % p, p) for p in mods]))

    # base extension Q -> {q1, q2, p1, p2, p3} of a centred x in (-q/2, q/2)
    C.append(("Q1INV_Q2", pow(q1, -1, q2)))
    C.append(("Q1INV_Q2_S", shoup(pow(q1, -1, q2), q2)))
    half_q = (q - 1) // 2
    C.append(("HALFQ_LO", half_q % q1))
    C.append(("HALFQ_HI", half_q // q1))
    arrays.append(("Q1_MOD", [q1 % p for p in primes]))
    arrays.append(("Q1_MOD_S", [shoup(q1 % p, p) for p in primes]))
    arrays.append(("Q_MOD", [q % p for p in primes]))

    # exact scale-and-round round(t X / q), with P
    arrays.append(("QINV_P", [pow(q, -1, p) for p in (p1, p2, p3)]))
    arrays.append(("QINV_P_S", [shoup(pow(q, -1, p), p) for p in (p1, p2, p3)]))
    C.append(("P1INV_P2", pow(p1, -1, p2)))
    C.append(("P1INV_P2_S", shoup(pow(p1, -1, p2), p2)))
    C.append(("P1INV_P3", pow(p1, -1, p3)))
    C.append(("P1INV_P3_S", shoup(pow(p1, -1, p3), p3)))
    C.append(("P2INV_P3", pow(p2, -1, p3)))
    C.append(("P2INV_P3_S", shoup(pow(p2, -1, p3), p3)))
    half_P = (P - 1) // 2
    z = mixed_radix(half_P, (p1, p2, p3))
    assert z[0] + p1 * z[1] + p1 * p2 * z[2] == half_P
    C.append(("HALFP_D1", z[0]))
    C.append(("HALFP_D2", z[1]))
    C.append(("HALFP_D3", z[2]))
    arrays.append(("P1_MOD_Q", [p1 % x for x in (q1, q2)]))
    arrays.append(("P1_MOD_Q_S", [shoup(p1 % x, x) for x in (q1, q2)]))
    arrays.append(("P1P2_MOD_Q", [(p1 * p2) % x for x in (q1, q2)]))
    arrays.append(("P1P2_MOD_Q_S", [shoup((p1 * p2) % x, x) for x in (q1, q2)]))
    arrays.append(("P_MOD_Q", [P % x for x in (q1, q2)]))

    # per plaintext modulus: {t, modulus index, q1 mod t, q mod t, q^-1 mod t
    # (decryption: pt = [-r q^-1]_t with r = [t v]_q centred), t mod p and its
    # Shoup companion for the five RNS primes (t x in scale-and-round and
    # decryption), Delta = floor(q / t) mod q_l and companions (encryption)}
    plains = []
    for idx, t in ((5, T), (6, T_PAPER)):
        delta = q // t
        plains.append("{ %dULL, %d, %dULL, %dULL, %dULL, { %s }, { %s }, { %s }, { %s } }" % (
            t, idx, q1 % t, q % t, pow(q % t, -1, t),
            ", ".join(f"{t % p}ULL" for p in primes),
            ", ".join(f"{shoup(t % p, p)}ULL" for p in primes),
            ", ".join(f"{delta % x}ULL" for x in (q1, q2)),
            ", ".join(f"{shoup(delta % x, x)}ULL" for x in (q1, q2))))
    arrays.append(("PLAIN", plains))

    # sanity of the ranges the kernels rely on
    assert q1 > q2 > p1 > p2 > p3 and q1 < 2 * p3
    assert q.bit_length() == 108 and P.bit_length() == 162
    assert (q * P).bit_length() == 270

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
         "constexpr int NUM_RNS = 5;     /* q1, q2, p1, p2, p3 */",
         "constexpr int MOD_T = 5;       /* index of the default t in the modulus arrays */",
         "constexpr int MOD_T_PAPER = 6; /* index of the paper's t */",
         "constexpr int NUM_MODS = 7;",
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
