"""Writes oracle/cdt_table.h: the cumulative table of the error distribution chi.

TEST INFRASTRUCTURE (oracle side).  App. A of the paper samples the FV error
terms e, e1, e2 from "a discrete truncated Gaussian" chi without fixing its
width or truncation.  The reading used here: width sigma = 3.2 (the usual FV
choice), support |e| <= 19 = floor(6 sigma), weights rho(k) = exp(-k^2 / (2 sigma^2))
normalised over the support.  The sampler draws a uniform 64-bit word U and
returns the smallest k with U < T[k], where T[k] = floor(2^64 * F(k)) and
F(k) = sum_{j <= k} rho(j) / sum_j rho(j), k = -19..18 (U beyond T[18] gives 19).

This generator is exact: every exp() value is enclosed in a rational interval
from a Taylor series with an explicit remainder bound (Python Fractions only),
and the script refuses to write a table entry whose floor is not decided by the
interval.  The CUDA library derives its own copy of the table by a different
route (decimal arithmetic); the tests check that both give identical integers.
"""
from fractions import Fraction
import os
import sys

SIGMA = Fraction(16, 5)          # 3.2
BOUND = 19                       # floor(6 * sigma)
TERMS = 160                      # Taylor terms for exp(x), x <= 17.7


def exp_interval(x: Fraction):
    """Rational interval [lo, hi] containing exp(x) for 0 <= x < TERMS/2."""
    s = Fraction(0)
    term = Fraction(1)
    for n in range(TERMS):
        s += term
        term = term * x / (n + 1)
    # remainder sum_{n >= TERMS} x^n/n! <= term * 1/(1 - x/(TERMS+1))
    rem = term / (1 - x / (TERMS + 1))
    return s, s + rem


def cdt_table():
    two_s2 = 2 * SIGMA * SIGMA
    lo_w, hi_w = [], []
    for k in range(-BOUND, BOUND + 1):
        elo, ehi = exp_interval(Fraction(k * k) / two_s2)
        # rho(k) = 1 / exp(k^2 / 2 sigma^2)
        lo_w.append(1 / ehi)
        hi_w.append(1 / elo)
    tot_lo, tot_hi = sum(lo_w), sum(hi_w)
    table = []
    cum_lo = Fraction(0)
    cum_hi = Fraction(0)
    for idx in range(2 * BOUND):          # k = -19 .. 18
        cum_lo += lo_w[idx]
        cum_hi += hi_w[idx]
        # F = C / (C + R) with C the weights up to k and R the rest: F grows
        # with C and falls with R, so the interval ends pair C_lo with R_hi.
        f_lo = cum_lo / (cum_lo + sum(hi_w[idx + 1:]))
        f_hi = cum_hi / (cum_hi + sum(lo_w[idx + 1:]))
        v_lo = (f_lo * (1 << 64)).__floor__()
        v_hi = (f_hi * (1 << 64)).__floor__()
        if v_lo != v_hi:
            raise RuntimeError(f"CDT entry {idx} not decided by the interval")
        table.append(v_lo)
    assert tot_hi >= tot_lo
    return table


def header_text(table):
    lines = [
        "/* Generated by oracle/gen_cdt.py -- do not edit.",
        " * Cumulative table of the truncated discrete Gaussian chi (sigma = 3.2,",
        " * |e| <= 19): ORC_CDT[i] = floor(2^64 * P(e <= i - 19)), i = 0..37. */",
        "#ifndef ORC_CDT_TABLE_H",
        "#define ORC_CDT_TABLE_H",
        "#define ORC_CDT_LEN 38",
        "#define ORC_CDT_MIN (-19)",
        "static const unsigned long long ORC_CDT[ORC_CDT_LEN] = {",
    ]
    for v in table:
        lines.append(f"    {v}ULL,")
    lines += ["};", "#endif", ""]
    return "\n".join(lines)


def main(argv):
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "cdt_table.h")
    text = header_text(cdt_table())
    if len(argv) > 1 and argv[1] == "--check":
        with open(out) as f:
            if f.read() != text:
                print("cdt_table.h is stale")
                return 1
        return 0
    with open(out, "w") as f:
        f.write(text)
    return 0


if __name__ == "__main__":
    sys.exit(main(sys.argv))
