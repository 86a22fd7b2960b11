/*
 * HERS oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, exact CPU implementation of the HERS encrypted search
 * (Engelsma, Jain, Boddeti, "HERS: Homomorphically Encrypted Representation
 * Search"): FV key generation, encryption and decryption (App. A, Algs 1-3),
 * the SIMD row encoding of probe and gallery (Sec. 3.2, Eqs 2-3), and the
 * server's search loop (Alg 7) with the degree-2 tensor accumulated over the
 * d dimensions, scaled by t/q once and relinearised once per gallery block
 * (the ciphertext multiply of Alg 5 with its per-product rounding moved after
 * the sum of Eq. 4; the paper-literal per-product form is also here, as a
 * cross-check that decrypts to the same scores).
 *
 * Arithmetic: polynomials over Z with schoolbook negacyclic products
 * (x^n = -1), integers up to 320 bits in a small fixed-width two's-complement
 * type, rounding by exact long division.  No NTT, no RNS beyond reading and
 * writing the two-residue exchange format of a ciphertext.
 *
 * Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline / reference
 * legs may load this library.  It shares no code, header, table or helper with
 * the CUDA library, and the CUDA library never calls it.
 *
 * Parameters (readings of App. A and Sec. 4.1, where the paper leaves them open):
 *   q = q1*q2, q1 = 18014398509309953, q2 = 18014398509293569 (108 bits);
 *   t = 4169729 (prime, t = 1 mod 8192); secret and u ternary; chi = discrete
 *   Gaussian, sigma 3.2, |e| <= 19; relinearisation gadget g_j = (q/q_j) *
 *   [(q/q_j)^-1]_{q_j}, j = 1, 2.
 * Every random draw comes from ChaCha20 (RFC 8439) addressed by
 * (seed, purpose, object, coefficient, attempt): see prf_* below.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include "cdt_table.h"

typedef unsigned __int128 u128;
typedef __int128 i128;

#define ORC_Q1 18014398509309953ULL
#define ORC_Q2 18014398509293569ULL
/* The plaintext modulus t: 4169729 by default, or the paper's 1032193 (Sec.
 * 4.1) after orc_set_t; both are primes = 1 (mod 2n).  Set it before any
 * other call, not while one runs. */
static uint64_t g_orc_t = 4169729ULL;
#define ORC_T g_orc_t
#define ORC_MAXN 4096

/* status codes shared with the Python wrapper */
#define ORC_OK 0
#define ORC_E_ARG (-1)
#define ORC_E_SAMPLER (-2)
#define ORC_E_BOUND (-3)
#define ORC_E_TIE (-4)
#define ORC_E_MEM (-5)

/* ------------------------------------------------------------------------ */
/* Small exact integer helpers                                              */
/* ------------------------------------------------------------------------ */

static u128 orc_q(void) { return (u128)ORC_Q1 * ORC_Q2; }

static uint64_t mulmod64(uint64_t a, uint64_t b, uint64_t m) {
    return (uint64_t)(((u128)a * b) % m);
}

/* a * b mod t for a, b < t < 2^23 (the product fits in 64 bits) */
static uint64_t mulmod_t(uint64_t a, uint64_t b) { return (a * b) % ORC_T; }

int orc_set_t(uint64_t t) {
    if (t != 4169729ULL && t != 1032193ULL) return ORC_E_ARG;
    g_orc_t = t;
    return ORC_OK;
}

static uint64_t powmod64(uint64_t b, uint64_t e, uint64_t m) {
    uint64_t r = 1 % m;
    b %= m;
    while (e) {
        if (e & 1) r = mulmod64(r, b, m);
        b = mulmod64(b, b, m);
        e >>= 1;
    }
    return r;
}

/* inverse modulo a prime m by Fermat's little theorem */
static uint64_t invmod64(uint64_t a, uint64_t m) { return powmod64(a, m - 2, m); }

/* [q1^-1]_{q2}, computed once by init_consts() before any parallel region */
static uint64_t Q1INV_MOD_Q2;
static void init_consts(void) { Q1INV_MOD_Q2 = invmod64(ORC_Q1 % ORC_Q2, ORC_Q2); }

/* x mod q from its residues (x1 mod q1, x2 mod q2), x in [0, q) (CRT) */
static u128 crt2(uint64_t x1, uint64_t x2) {
    uint64_t q1inv = Q1INV_MOD_Q2;
    uint64_t x1r = x1 % ORC_Q2;
    uint64_t diff = (x2 >= x1r) ? x2 - x1r : x2 + ORC_Q2 - x1r;
    uint64_t h = mulmod64(diff, q1inv, ORC_Q2);
    return (u128)x1 + (u128)ORC_Q1 * h;
}

/* symmetric representative of x in [0, q): (-(q-1)/2 .. (q-1)/2] (App. A) */
static i128 lift_sym(u128 x) {
    u128 q = orc_q();
    return (x > (q - 1) / 2) ? (i128)x - (i128)q : (i128)x;
}

/* canonical x mod q in [0, q) for any i128 */
static u128 mod_q_i128(i128 x) {
    i128 q = (i128)orc_q();
    i128 r = x % q;
    if (r < 0) r += q;
    return (u128)r;
}

/* ---------------------- fixed-width 320-bit integers --------------------- */

#define BW 5
typedef struct { uint64_t w[BW]; } bi; /* two's complement, little-endian words */

static bi bi_zero(void) { bi r; memset(&r, 0, sizeof r); return r; }

static bi bi_from_i128(i128 v) {
    bi r;
    u128 u = (u128)v;
    uint64_t ext = (v < 0) ? ~0ULL : 0ULL;
    r.w[0] = (uint64_t)u;
    r.w[1] = (uint64_t)(u >> 64);
    for (int i = 2; i < BW; i++) r.w[i] = ext;
    return r;
}

static bi bi_from_u128(u128 v) {
    bi r = bi_zero();
    r.w[0] = (uint64_t)v;
    r.w[1] = (uint64_t)(v >> 64);
    return r;
}

static int bi_is_neg(const bi *a) { return (int)(a->w[BW - 1] >> 63); }

static void bi_add(bi *a, const bi *b) {
    u128 c = 0;
    for (int i = 0; i < BW; i++) {
        c += (u128)a->w[i] + b->w[i];
        a->w[i] = (uint64_t)c;
        c >>= 64;
    }
}

static bi bi_neg(bi a) {
    for (int i = 0; i < BW; i++) a.w[i] = ~a.w[i];
    bi one = bi_zero();
    one.w[0] = 1;
    bi_add(&a, &one);
    return a;
}

/* a << s for 0 <= s < 64*BW (arithmetic on the two's-complement pattern) */
static bi bi_shl(bi a, int s) {
    bi r = bi_zero();
    int ws = s / 64, bs = s % 64;
    for (int i = BW - 1; i >= ws; i--) {
        uint64_t v = a.w[i - ws] << bs;
        if (bs && i - ws - 1 >= 0) v |= a.w[i - ws - 1] >> (64 - bs);
        r.w[i] = v;
    }
    return r;
}

/* unsigned magnitude multiply by a 64-bit value, in place (no overflow check) */
static void bi_mag_mul_u64(bi *a, uint64_t m) {
    u128 c = 0;
    for (int i = 0; i < BW; i++) {
        c += (u128)a->w[i] * m;
        a->w[i] = (uint64_t)c;
        c >>= 64;
    }
}

/* signed a * m for a 64-bit unsigned m */
static bi bi_mul_u64(bi a, uint64_t m) {
    int neg = bi_is_neg(&a);
    if (neg) a = bi_neg(a);
    bi_mag_mul_u64(&a, m);
    return neg ? bi_neg(a) : a;
}

/* exact product of two unsigned 128-bit values as a 320-bit integer */
static bi bi_mul_u128(u128 x, u128 y) {
    uint64_t x0 = (uint64_t)x, x1 = (uint64_t)(x >> 64);
    uint64_t y0 = (uint64_t)y, y1 = (uint64_t)(y >> 64);
    bi r = bi_zero(), t;
    r = bi_from_u128((u128)x0 * y0);
    t = bi_shl(bi_from_u128((u128)x0 * y1), 64); bi_add(&r, &t);
    t = bi_shl(bi_from_u128((u128)x1 * y0), 64); bi_add(&r, &t);
    t = bi_shl(bi_from_u128((u128)x1 * y1), 128); bi_add(&r, &t);
    return r;
}

/* compare magnitudes |a| <= b (b non-negative) */
static int bi_cmp_u(const bi *a, const bi *b) {
    for (int i = BW - 1; i >= 0; i--) {
        if (a->w[i] != b->w[i]) return a->w[i] < b->w[i] ? -1 : 1;
    }
    return 0;
}

/* unsigned long division of a non-negative bi by 0 < D < 2^126 */
static void bi_udivmod(const bi *n, u128 D, bi *quo, u128 *rem) {
    bi qv = bi_zero();
    u128 r = 0;
    for (int bit = 64 * BW - 1; bit >= 0; bit--) {
        r = (r << 1) | ((n->w[bit / 64] >> (bit % 64)) & 1);
        if (r >= D) {
            r -= D;
            qv.w[bit / 64] |= 1ULL << (bit % 64);
        }
    }
    *quo = qv;
    *rem = r;
}

/* floor division n = D*quo + rem with 0 <= rem < D, for any signed n */
static void bi_floordiv(const bi *n, u128 D, bi *quo, u128 *rem) {
    if (!bi_is_neg(n)) {
        bi_udivmod(n, D, quo, rem);
        return;
    }
    bi m = bi_neg(*n);
    bi qq;
    u128 rr;
    bi_udivmod(&m, D, &qq, &rr);
    if (rr == 0) {
        *quo = bi_neg(qq);
        *rem = 0;
    } else {
        bi one = bi_zero();
        one.w[0] = 1;
        bi_add(&qq, &one);
        *quo = bi_neg(qq);
        *rem = D - rr;
    }
}

/* n mod q in [0, q) for any signed n */
static u128 bi_mod_q(const bi *n) {
    bi quo;
    u128 r;
    bi_floordiv(n, orc_q(), &quo, &r);
    return r;
}

/*
 * round(t * X / q) = floor((2 t X + q) / (2 q)).  Because q is odd, 2tX + q is
 * odd and 2q is even, so the quotient is never exactly k + 1/2: a tie cannot
 * happen (the remainder is never 0).  *tie is set if it happened anyway.
 */
static bi round_t_over_q(const bi *X, int *tie) {
    u128 q = orc_q();
    bi n = bi_mul_u64(*X, 2 * ORC_T);
    bi qb = bi_from_u128(q);
    bi_add(&n, &qb);
    bi quo;
    u128 rem;
    bi_floordiv(&n, 2 * q, &quo, &rem);
    if (tie) *tie = (rem == 0);
    return quo;
}

/* ------------------------------------------------------------------------ */
/* ChaCha20 (RFC 8439, Sec. 2.3) and the samplers                           */
/* ------------------------------------------------------------------------ */

static uint32_t rotl32(uint32_t x, int r) { return (x << r) | (x >> (32 - r)); }

static void quarter(uint32_t *s, int a, int b, int c, int d) {
    s[a] += s[b]; s[d] ^= s[a]; s[d] = rotl32(s[d], 16);
    s[c] += s[d]; s[b] ^= s[c]; s[b] = rotl32(s[b], 12);
    s[a] += s[b]; s[d] ^= s[a]; s[d] = rotl32(s[d], 8);
    s[c] += s[d]; s[b] ^= s[c]; s[b] = rotl32(s[b], 7);
}

/* one 64-byte ChaCha20 block: 16 little-endian 32-bit words */
void orc_chacha20_block(const uint32_t key[8], uint32_t counter, const uint32_t nonce[3],
                        uint32_t out[16]) {
    uint32_t init[16], x[16];
    /* the four constant words spell "expand 32-byte k" in little endian */
    init[0] = 0x61707865u; init[1] = 0x3320646eu; init[2] = 0x79622d32u; init[3] = 0x6b206574u;
    for (int i = 0; i < 8; i++) init[4 + i] = key[i];
    init[12] = counter;
    init[13] = nonce[0]; init[14] = nonce[1]; init[15] = nonce[2];
    memcpy(x, init, sizeof x);
    for (int r = 0; r < 10; r++) {
        quarter(x, 0, 4, 8, 12); quarter(x, 1, 5, 9, 13);
        quarter(x, 2, 6, 10, 14); quarter(x, 3, 7, 11, 15);
        quarter(x, 0, 5, 10, 15); quarter(x, 1, 6, 11, 12);
        quarter(x, 2, 7, 8, 13); quarter(x, 3, 4, 9, 14);
    }
    for (int i = 0; i < 16; i++) out[i] = x[i] + init[i];
}

/*
 * A stream is ChaCha20 keyed by (seed_lo, seed_hi, 0, 0, 0, 0, 0, 0) with nonce
 * (purpose, obj_lo, obj_hi).  Its 32-bit word number W sits in block W / 16 at
 * position W % 16; its 64-bit word number w is the pair of 32-bit words
 * (2w = low half, 2w+1 = high half).
 */
typedef struct {
    uint32_t key[8], nonce[3];
    uint32_t blk[16];
    int64_t ctr; /* counter of the cached block, -1 = none */
} prf_t;

static void prf_init(prf_t *p, uint64_t seed, uint32_t purpose, uint64_t obj) {
    memset(p, 0, sizeof *p);
    p->key[0] = (uint32_t)seed;
    p->key[1] = (uint32_t)(seed >> 32);
    p->nonce[0] = purpose;
    p->nonce[1] = (uint32_t)obj;
    p->nonce[2] = (uint32_t)(obj >> 32);
    p->ctr = -1;
}

static uint32_t prf_w32(prf_t *p, uint64_t W) {
    int64_t c = (int64_t)(W >> 4);
    if (c != p->ctr) {
        orc_chacha20_block(p->key, (uint32_t)c, p->nonce, p->blk);
        p->ctr = c;
    }
    return p->blk[W & 15];
}

static uint64_t prf_w64(prf_t *p, uint64_t w) {
    uint64_t lo = prf_w32(p, 2 * w), hi = prf_w32(p, 2 * w + 1);
    return lo | (hi << 32);
}

#define ORC_MAX_ATTEMPTS 16

/* ternary in {-1,0,1}: 32-bit word W = a*n + k for attempt a; accept w < 3*floor(2^32/3) */
static int sample_ternary(uint64_t seed, uint32_t purpose, uint64_t obj, int n, int8_t *out) {
    prf_t p;
    prf_init(&p, seed, purpose, obj);
    const uint32_t lim = 3u * (0xFFFFFFFFu / 3u);
    for (int k = 0; k < n; k++) {
        int a;
        for (a = 0; a < ORC_MAX_ATTEMPTS; a++) {
            uint32_t w = prf_w32(&p, (uint64_t)a * n + k);
            if (w < lim) {
                out[k] = (int8_t)((int)(w % 3u) - 1);
                break;
            }
        }
        if (a == ORC_MAX_ATTEMPTS) return ORC_E_SAMPLER;
    }
    return ORC_OK;
}

/* uniform mod qj: 64-bit word w = a*n + k masked to 54 bits, accept if < qj */
static int sample_uniform(uint64_t seed, uint32_t purpose, uint64_t obj, int n, uint64_t qj,
                          uint64_t *out) {
    prf_t p;
    prf_init(&p, seed, purpose, obj);
    const uint64_t mask = (1ULL << 54) - 1;
    for (int k = 0; k < n; k++) {
        int a;
        for (a = 0; a < ORC_MAX_ATTEMPTS; a++) {
            uint64_t v = prf_w64(&p, (uint64_t)a * n + k) & mask;
            if (v < qj) {
                out[k] = v;
                break;
            }
        }
        if (a == ORC_MAX_ATTEMPTS) return ORC_E_SAMPLER;
    }
    return ORC_OK;
}

/* chi: 64-bit word U = word k; e = smallest value v in -19..18 with U < CDT(v), else 19 */
static void sample_gauss(uint64_t seed, uint32_t purpose, uint64_t obj, int n, int8_t *out) {
    prf_t p;
    prf_init(&p, seed, purpose, obj);
    for (int k = 0; k < n; k++) {
        uint64_t U = prf_w64(&p, (uint64_t)k);
        int i = 0;
        while (i < ORC_CDT_LEN && !(U < ORC_CDT[i])) i++;
        out[k] = (int8_t)(ORC_CDT_MIN + i);
    }
}

/* stream purposes (nonce word 0) */
#define PRF_KG_SK 0x01u
#define PRF_KG_PK_A 0x02u  /* obj = limb */
#define PRF_KG_PK_E 0x03u
#define PRF_KG_EVK_A 0x04u /* obj = 2*j + limb */
#define PRF_KG_EVK_E 0x05u /* obj = j */
#define PRF_KG_EVKW_A 0x06u /* base-w evaluation keys: obj = 2*j + limb */
#define PRF_KG_EVKW_E 0x07u /* obj = j */
/* encryption: base + 0 -> u, base + 1 -> e1, base + 2 -> e2 */

int orc_sample(uint64_t seed, uint32_t purpose, uint64_t obj, int n, int kind, uint64_t qj,
               int64_t *out) {
    if (n <= 0 || n > 1 << 20) return ORC_E_ARG;
    int rc = ORC_OK;
    if (kind == 0) {
        int8_t *tmp = malloc(n);
        rc = sample_ternary(seed, purpose, obj, n, tmp);
        for (int k = 0; k < n; k++) out[k] = tmp[k];
        free(tmp);
    } else if (kind == 1) {
        int8_t *tmp = malloc(n);
        sample_gauss(seed, purpose, obj, n, tmp);
        for (int k = 0; k < n; k++) out[k] = tmp[k];
        free(tmp);
    } else {
        uint64_t *tmp = malloc(n * sizeof(uint64_t));
        rc = sample_uniform(seed, purpose, obj, n, qj, tmp);
        for (int k = 0; k < n; k++) out[k] = (int64_t)tmp[k];
        free(tmp);
    }
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Polynomial arithmetic in Z[x]/(x^n + 1)                                  */
/* ------------------------------------------------------------------------ */

static int valid_n(int n) { return n >= 2 && n <= ORC_MAXN && (n & (n - 1)) == 0; }

/* out[k] = [ (a (*) s)[k] ]_q for a in [0,q)^n and a small signed polynomial s */
static void negacyclic_small_mod_q(int n, const u128 *a, const int32_t *s, u128 *out) {
#pragma omp parallel for schedule(static)
    for (int k = 0; k < n; k++) {
        i128 acc = 0; /* |acc| <= n * max|s| * q < 2^127 for the sizes used */
        for (int j = 0; j < n; j++) {
            int l = k - j;
            i128 term = (i128)a[j] * s[l >= 0 ? l : l + n];
            acc += (l >= 0) ? term : -term;
        }
        out[k] = mod_q_i128(acc);
    }
}

/* (s (*) s) over Z for a small s */
static void negacyclic_small_z(int n, const int32_t *a, const int32_t *b, int32_t *out) {
    for (int k = 0; k < n; k++) {
        int64_t acc = 0;
        for (int j = 0; j < n; j++) {
            int l = k - j;
            int64_t term = (int64_t)a[j] * b[l >= 0 ? l : l + n];
            acc += (l >= 0) ? term : -term;
        }
        out[k] = (int32_t)acc;
    }
}

/*
 * Exact sums of products of integers |x| < 2^107, written in two digits
 * x = hi * 2^54 + lo with 0 <= lo < 2^54.  Three partial sums, each an i128:
 * x*y = hh*2^108 + (hl+lh)*2^54 + ll.  n <= 4096 terms of each partial
 * product fit in an i128 with room to spare (|term| < 2^107).
 */
typedef struct { int64_t hi; uint64_t lo; } dig;
typedef struct { i128 hh, mid, ll; } part;

static dig to_dig(i128 x) {
    dig d;
    i128 lo = x & (((i128)1 << 54) - 1); /* x mod 2^54, in [0, 2^54) */
    d.lo = (uint64_t)lo;
    d.hi = (int64_t)((x - lo) >> 54);
    return d;
}

static void part_mac(part *p, dig x, dig y) {
    p->hh += (i128)x.hi * y.hi;
    p->mid += (i128)x.hi * (i128)y.lo + (i128)x.lo * (i128)y.hi;
    p->ll += (i128)((u128)x.lo * y.lo);
}

static void part_msub(part *p, dig x, dig y) {
    p->hh -= (i128)x.hi * y.hi;
    p->mid -= (i128)x.hi * (i128)y.lo + (i128)x.lo * (i128)y.hi;
    p->ll -= (i128)((u128)x.lo * y.lo);
}

/* acc += hh*2^108 + mid*2^54 + ll */
static void part_flush(const part *p, bi *acc) {
    bi t;
    t = bi_shl(bi_from_i128(p->hh), 108); bi_add(acc, &t);
    t = bi_shl(bi_from_i128(p->mid), 54); bi_add(acc, &t);
    t = bi_from_i128(p->ll); bi_add(acc, &t);
}

/* coefficient k of the negacyclic product a (*) b over Z, added into *p */
static void negacyclic_coeff(int n, int k, const dig *a, const dig *b, part *p) {
    for (int j = 0; j <= k; j++) part_mac(p, a[j], b[k - j]);
    for (int j = k + 1; j < n; j++) part_msub(p, a[j], b[k - j + n]); /* x^n = -1 */
}

/*
 * Exported for the product pin: out[k] (5 little-endian words, two's
 * complement) = (a (*) b)[k] over Z for |a[j]|, |b[j]| < 2^107 given as
 * (lo, hi) 64-bit word pairs of their i128 values.
 */
int orc_negacyclic_z(int n, const int64_t *a_words, const int64_t *b_words, uint64_t *out) {
    if (!valid_n(n)) return ORC_E_ARG;
    dig *a = malloc(n * sizeof(dig)), *b = malloc(n * sizeof(dig));
    for (int j = 0; j < n; j++) {
        i128 av = (i128)(((u128)(uint64_t)a_words[2 * j + 1] << 64) | (uint64_t)a_words[2 * j]);
        i128 bv = (i128)(((u128)(uint64_t)b_words[2 * j + 1] << 64) | (uint64_t)b_words[2 * j]);
        a[j] = to_dig(av);
        b[j] = to_dig(bv);
    }
#pragma omp parallel for schedule(static)
    for (int k = 0; k < n; k++) {
        part p = {0, 0, 0};
        bi acc = bi_zero();
        negacyclic_coeff(n, k, a, b, &p);
        part_flush(&p, &acc);
        memcpy(out + (size_t)BW * k, acc.w, sizeof acc.w);
    }
    free(a);
    free(b);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Batch encoding mod t (Sec. 3.2; "BatchEncode" of Algs 6-7)                */
/* ------------------------------------------------------------------------ */

/* psi_t: the smallest x >= 2 with x^n = -1 (mod t), a primitive 2n-th root of unity */
uint64_t orc_psi_t(int n) {
    for (uint64_t x = 2; x < ORC_T; x++)
        if (powmod64(x, (uint64_t)n, ORC_T) == ORC_T - 1) return x;
    return 0;
}

/*
 * Slot j of a plaintext m(x) in R_t is m(psi_t^(2j+1)), j = 0..n-1.
 * Encode: m_k = n^-1 * sum_j slot_j * psi_t^-((2j+1)k) (mod t), the inverse of
 * evaluation at the n distinct roots of x^n + 1 mod t.  O(n^2).
 */
int orc_encode(int n, const int64_t *slots, uint32_t *m) {
    if (!valid_n(n)) return ORC_E_ARG;
    uint64_t psi = orc_psi_t(n), two_n = 2 * (uint64_t)n;
    uint64_t *pw = malloc(two_n * sizeof(uint64_t));
    pw[0] = 1;
    for (uint64_t e = 1; e < two_n; e++) pw[e] = mulmod64(pw[e - 1], psi, ORC_T);
    uint64_t ninv = invmod64((uint64_t)n, ORC_T);
    uint64_t *sl = malloc(n * sizeof(uint64_t));
    for (int j = 0; j < n; j++) {
        int64_t v = slots[j] % (int64_t)ORC_T;
        sl[j] = (uint64_t)(v < 0 ? v + (int64_t)ORC_T : v);
    }
#pragma omp parallel for schedule(static)
    for (int k = 0; k < n; k++) {
        uint64_t acc = 0;
        for (int j = 0; j < n; j++) {
            uint64_t e = ((uint64_t)(2 * j + 1) * (uint64_t)k) % two_n;
            uint64_t inv_pow = pw[(two_n - e) % two_n]; /* psi^-e */
            acc = (acc + mulmod_t(sl[j], inv_pow)) % ORC_T;
        }
        m[k] = (uint32_t)mulmod64(acc, ninv, ORC_T);
    }
    free(pw);
    free(sl);
    return ORC_OK;
}

/* Decode: slot_j = m(psi_t^(2j+1)) mod t, centred in [-(t-1)/2, (t-1)/2] */
int orc_decode(int n, const uint32_t *m, int64_t *slots) {
    if (!valid_n(n)) return ORC_E_ARG;
    uint64_t psi = orc_psi_t(n), two_n = 2 * (uint64_t)n;
    uint64_t *pw = malloc(two_n * sizeof(uint64_t));
    pw[0] = 1;
    for (uint64_t e = 1; e < two_n; e++) pw[e] = mulmod64(pw[e - 1], psi, ORC_T);
#pragma omp parallel for schedule(static)
    for (int j = 0; j < n; j++) {
        uint64_t acc = 0;
        for (int k = 0; k < n; k++) {
            uint64_t e = ((uint64_t)(2 * j + 1) * (uint64_t)k) % two_n;
            acc = (acc + mulmod_t(m[k] % ORC_T, pw[e])) % ORC_T;
        }
        slots[j] = (acc > (ORC_T - 1) / 2) ? (int64_t)acc - (int64_t)ORC_T : (int64_t)acc;
    }
    free(pw);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Exchange format: a polynomial mod q as residues [limb][n]                 */
/* ------------------------------------------------------------------------ */

/* poly mod q from residues r[0..n) mod q1 and r[n..2n) mod q2 */
static void poly_from_res(int n, const uint64_t *r, u128 *x) {
    for (int k = 0; k < n; k++) x[k] = crt2(r[k], r[n + k]);
}

static void poly_to_res(int n, const u128 *x, uint64_t *r) {
    for (int k = 0; k < n; k++) {
        r[k] = (uint64_t)(x[k] % ORC_Q1);
        r[n + k] = (uint64_t)(x[k] % ORC_Q2);
    }
}

/* ------------------------------------------------------------------------ */
/* Alg 1: key generation                                                    */
/* ------------------------------------------------------------------------ */

/*
 * sk: n int8 in {-1,0,1}.  pk: [2 polys][2 limbs][n].  evk: [2 digits][2 polys][2 limbs][n].
 * pk = ([-(a s + e)]_q, a); evk_j = ([-(a_j s + e_j) + g_j s^2]_q, a_j),
 * with g_1 = q2 * [q2^-1]_{q1}, g_2 = q1 * [q1^-1]_{q2} (so g_1 + g_2 = 1 mod q and
 * g_j = 1 mod q_j, 0 mod the other prime).
 */
int orc_keygen(int n, uint64_t seed, int8_t *sk, uint64_t *pk, uint64_t *evk) {
    init_consts();
    if (!valid_n(n)) return ORC_E_ARG;
    int rc = ORC_OK;
    u128 q = orc_q();
    int32_t *s = malloc(n * sizeof(int32_t)), *s2 = malloc(n * sizeof(int32_t));
    int8_t *e8 = malloc(n);
    uint64_t *r = malloc(2 * n * sizeof(uint64_t));
    u128 *a = malloc(n * sizeof(u128)), *as = malloc(n * sizeof(u128)), *c0 = malloc(n * sizeof(u128));

    if ((rc = sample_ternary(seed, PRF_KG_SK, 0, n, sk)) != ORC_OK) goto done;
    for (int k = 0; k < n; k++) s[k] = sk[k];

    /* public key */
    if ((rc = sample_uniform(seed, PRF_KG_PK_A, 0, n, ORC_Q1, r)) != ORC_OK) goto done;
    if ((rc = sample_uniform(seed, PRF_KG_PK_A, 1, n, ORC_Q2, r + n)) != ORC_OK) goto done;
    poly_from_res(n, r, a);
    sample_gauss(seed, PRF_KG_PK_E, 0, n, e8);
    negacyclic_small_mod_q(n, a, s, as);
    for (int k = 0; k < n; k++) c0[k] = mod_q_i128(-((i128)as[k] + e8[k]));
    poly_to_res(n, c0, pk);
    poly_to_res(n, a, pk + 2 * n);

    /* evaluation keys (RNS gadget, two digits) */
    negacyclic_small_z(n, s, s, s2);
    u128 g[2];
    g[0] = (u128)ORC_Q2 * invmod64(ORC_Q2 % ORC_Q1, ORC_Q1);
    g[1] = (u128)ORC_Q1 * invmod64(ORC_Q1 % ORC_Q2, ORC_Q2);
    for (int j = 0; j < 2; j++) {
        if ((rc = sample_uniform(seed, PRF_KG_EVK_A, 2 * j, n, ORC_Q1, r)) != ORC_OK) goto done;
        if ((rc = sample_uniform(seed, PRF_KG_EVK_A, 2 * j + 1, n, ORC_Q2, r + n)) != ORC_OK) goto done;
        poly_from_res(n, r, a);
        sample_gauss(seed, PRF_KG_EVK_E, (uint64_t)j, n, e8);
        negacyclic_small_mod_q(n, a, s, as);
        for (int k = 0; k < n; k++) {
            u128 gs2 = mod_q_i128((i128)(g[j] % q) * s2[k]); /* |g s2| < 2^108 * 2^12 */
            i128 v = -((i128)as[k] + e8[k]) + (i128)gs2;
            c0[k] = mod_q_i128(v);
        }
        poly_to_res(n, c0, evk + (size_t)j * 4 * n);
        poly_to_res(n, a, evk + (size_t)j * 4 * n + 2 * n);
    }
done:
    free(s); free(s2); free(e8); free(r); free(a); free(as); free(c0);
    return rc;
}

/*
 * Number of digits of the base-w gadget with w = 2^logw: l = ceil(bits(q) / logw),
 * so that c = sum_{j<l} D_j w^j with D_j in [0, w) for every c in [0, q).
 */
int orc_basew_digits(int logw) {
    init_consts();
    int bits = 0;
    for (u128 q = orc_q(); q; q >>= 1) bits++;
    return (bits + logw - 1) / logw;
}

/*
 * Base-w evaluation keys (Alg 1 with the power-of-two gadget g_j = w^j,
 * w = 2^logw, 16 <= logw <= 60): evkw_j = ([-(a_j s + e_j) + w^j s^2]_q, a_j)
 * for j = 0 .. l-1.  s is the secret key of sk_seed (its stream 0x01);
 * a_j (uniform mod q, limb by limb) and e_j come from w_seed's streams 0x06
 * (obj 2j + limb) and 0x07 (obj j).  evkw: [l][2 polys][2 limbs][n].
 */
int orc_keygen_w(int n, uint64_t sk_seed, uint64_t w_seed, int logw, uint64_t *evkw) {
    init_consts();
    if (!valid_n(n) || logw < 16 || logw > 60) return ORC_E_ARG;
    int rc = ORC_OK, l = orc_basew_digits(logw);
    u128 q = orc_q();
    int8_t *sk = malloc(n), *e8 = malloc(n);
    int32_t *s = malloc(n * sizeof(int32_t)), *s2 = malloc(n * sizeof(int32_t));
    uint64_t *r = malloc(2 * n * sizeof(uint64_t));
    u128 *a = malloc(n * sizeof(u128)), *as = malloc(n * sizeof(u128)), *c0 = malloc(n * sizeof(u128));
    if ((rc = sample_ternary(sk_seed, PRF_KG_SK, 0, n, sk)) != ORC_OK) goto done;
    for (int k = 0; k < n; k++) s[k] = sk[k];
    negacyclic_small_z(n, s, s, s2);
    for (int j = 0; j < l; j++) {
        if ((rc = sample_uniform(w_seed, PRF_KG_EVKW_A, 2 * j, n, ORC_Q1, r)) != ORC_OK) goto done;
        if ((rc = sample_uniform(w_seed, PRF_KG_EVKW_A, 2 * j + 1, n, ORC_Q2, r + n)) != ORC_OK) goto done;
        poly_from_res(n, r, a);
        sample_gauss(w_seed, PRF_KG_EVKW_E, (uint64_t)j, n, e8);
        negacyclic_small_mod_q(n, a, s, as);
        const u128 g = ((u128)1 << (logw * j)) % q; /* w^j < 2^108 */
        for (int k = 0; k < n; k++) {
            u128 gs2 = mod_q_i128((i128)g * s2[k]); /* |g s2| < 2^108 * 2^12 */
            c0[k] = mod_q_i128(-((i128)as[k] + e8[k]) + (i128)gs2);
        }
        poly_to_res(n, c0, evkw + (size_t)j * 4 * n);
        poly_to_res(n, a, evkw + (size_t)j * 4 * n + 2 * n);
    }
done:
    free(sk); free(e8); free(s); free(s2); free(r); free(a); free(as); free(c0);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Alg 2: encryption                                                        */
/* ------------------------------------------------------------------------ */

/*
 * ct = ([Delta m + pk0 u + e1]_q, [pk1 u + e2]_q), Delta = floor(q/t), m in [0,t)^n.
 * u, e1, e2 come from the streams (seed, purpose_base + 0/1/2, obj).
 * pk, ct: [2 polys][2 limbs][n] residues.
 */
int orc_encrypt(int n, const uint64_t *pk, const uint32_t *m, uint64_t seed,
                uint32_t purpose_base, uint64_t obj, uint64_t *ct) {
    init_consts();
    if (!valid_n(n)) return ORC_E_ARG;
    u128 q = orc_q(), delta = q / ORC_T;
    int rc;
    int8_t *u8 = malloc(n), *e1 = malloc(n), *e2 = malloc(n);
    int32_t *u = malloc(n * sizeof(int32_t));
    u128 *p0 = malloc(n * sizeof(u128)), *p1 = malloc(n * sizeof(u128));
    u128 *t0 = malloc(n * sizeof(u128)), *t1 = malloc(n * sizeof(u128));
    if ((rc = sample_ternary(seed, purpose_base + 0, obj, n, u8)) != ORC_OK) goto done;
    sample_gauss(seed, purpose_base + 1, obj, n, e1);
    sample_gauss(seed, purpose_base + 2, obj, n, e2);
    for (int k = 0; k < n; k++) u[k] = u8[k];
    poly_from_res(n, pk, p0);
    poly_from_res(n, pk + 2 * n, p1);
    negacyclic_small_mod_q(n, p0, u, t0);
    negacyclic_small_mod_q(n, p1, u, t1);
    for (int k = 0; k < n; k++) {
        u128 dm = (delta * (m[k] % ORC_T)) % q; /* Delta < 2^86, m < 2^22 */
        t0[k] = mod_q_i128((i128)dm + (i128)t0[k] + e1[k]);
        t1[k] = mod_q_i128((i128)t1[k] + e2[k]);
    }
    poly_to_res(n, t0, ct);
    poly_to_res(n, t1, ct + 2 * n);
done:
    free(u8); free(e1); free(e2); free(u); free(p0); free(p1); free(t0); free(t1);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Search: Eq. 4 over one gallery block, Alg 7's inner loop                  */
/* ------------------------------------------------------------------------ */

typedef struct {
    uint64_t tensor_products; /* ct x ct tensor products (Table 2 "Multiplication") */
    uint64_t tensor_adds;     /* additions of tensors / ciphertexts (Table 2 "Addition") */
    uint64_t scale_rounds;    /* c_k = [round(t X_k / q)]_q, per ciphertext */
    uint64_t key_switches;    /* relinearisations */
    uint64_t rotations;       /* always 0 for this encoding (Table 2) */
    uint64_t ties;            /* rounding ties met (provably 0) */
    uint64_t bound_violations;/* |X| above d * 2n * ((q-1)/2)^2 (provably 0) */
    uint64_t max_x_bits;      /* largest bit length of |X_k| seen */
} orc_stats;

static int bi_bitlen_abs(const bi *x) {
    bi a = bi_is_neg(x) ? bi_neg(*x) : *x;
    for (int i = BW - 1; i >= 0; i--)
        if (a.w[i]) return 64 * i + 64 - __builtin_clzll(a.w[i]);
    return 0;
}

/* load a ciphertext [2][2][n] as lifted digit polynomials */
static void load_ct_dig(int n, const uint64_t *ct, dig *c0, dig *c1) {
    for (int k = 0; k < n; k++) {
        c0[k] = to_dig(lift_sym(crt2(ct[k], ct[n + k])));
        c1[k] = to_dig(lift_sym(crt2(ct[2 * n + k], ct[3 * n + k])));
    }
}

/*
 * Relinearisation with the RNS gadget (Alg 5, last three steps):
 * D_j = c2 mod q_j as integers in [0, q_j);
 * (c0', c1') = ([c0 + sum_j D_j evk_j[0]]_q, [c1 + sum_j D_j evk_j[1]]_q).
 */
static void key_switch(int n, const u128 *c0, const u128 *c1, const u128 *c2,
                       const uint64_t *evk, u128 *o0, u128 *o1) {
    dig *D[2], *E[2][2];
    for (int j = 0; j < 2; j++) {
        D[j] = malloc(n * sizeof(dig));
        uint64_t qj = j == 0 ? ORC_Q1 : ORC_Q2;
        for (int k = 0; k < n; k++) D[j][k] = to_dig((i128)(uint64_t)(c2[k] % qj));
        for (int c = 0; c < 2; c++) {
            E[j][c] = malloc(n * sizeof(dig));
            const uint64_t *e = evk + (size_t)j * 4 * n + (size_t)c * 2 * n;
            for (int k = 0; k < n; k++) E[j][c][k] = to_dig((i128)crt2(e[k], e[n + k]));
        }
    }
#pragma omp parallel for schedule(static)
    for (int k = 0; k < n; k++) {
        bi a0 = bi_from_u128(c0[k]), a1 = bi_from_u128(c1[k]);
        for (int j = 0; j < 2; j++) {
            part p0 = {0, 0, 0}, p1 = {0, 0, 0};
            negacyclic_coeff(n, k, D[j], E[j][0], &p0);
            negacyclic_coeff(n, k, D[j], E[j][1], &p1);
            part_flush(&p0, &a0);
            part_flush(&p1, &a1);
        }
        o0[k] = bi_mod_q(&a0);
        o1[k] = bi_mod_q(&a1);
    }
    for (int j = 0; j < 2; j++) {
        free(D[j]);
        free(E[j][0]);
        free(E[j][1]);
    }
}

/*
 * Relinearisation with the base-w gadget (Alg 5 with g_j = w^j): the
 * coefficients of c2, as integers in [0, q), are cut into l digits D_j in
 * [0, w), c2 = sum_j D_j w^j; (c0', c1') = ([c0 + sum_j D_j evkw_j[0]]_q,
 * [c1 + sum_j D_j evkw_j[1]]_q), products exact over Z.
 */
static void key_switch_w(int n, const u128 *c0, const u128 *c1, const u128 *c2, const uint64_t *evkw,
                         int logw, u128 *o0, u128 *o1) {
    const int l = orc_basew_digits(logw);
    const u128 mask = ((u128)1 << logw) - 1;
    dig *D = malloc((size_t)l * n * sizeof(dig));
    dig *E0 = malloc((size_t)l * n * sizeof(dig)), *E1 = malloc((size_t)l * n * sizeof(dig));
    for (int j = 0; j < l; j++) {
        const uint64_t *e0 = evkw + (size_t)j * 4 * n, *e1 = e0 + 2 * n;
        for (int k = 0; k < n; k++) {
            D[(size_t)j * n + k] = to_dig((i128)((c2[k] >> (logw * j)) & mask));
            E0[(size_t)j * n + k] = to_dig((i128)crt2(e0[k], e0[n + k]));
            E1[(size_t)j * n + k] = to_dig((i128)crt2(e1[k], e1[n + k]));
        }
    }
#pragma omp parallel for schedule(static)
    for (int k = 0; k < n; k++) {
        bi a0 = bi_from_u128(c0[k]), a1 = bi_from_u128(c1[k]);
        for (int j = 0; j < l; j++) {
            part p0 = {0, 0, 0}, p1 = {0, 0, 0};
            negacyclic_coeff(n, k, D + (size_t)j * n, E0 + (size_t)j * n, &p0);
            negacyclic_coeff(n, k, D + (size_t)j * n, E1 + (size_t)j * n, &p1);
            part_flush(&p0, &a0);
            part_flush(&p1, &a1);
        }
        o0[k] = bi_mod_q(&a0);
        o1[k] = bi_mod_q(&a1);
    }
    free(D); free(E0); free(E1);
}

/* ct3 [3][2][n] canonical (c0, c1, c2) -> out [2][2][n] with the base-w gadget */
int orc_keyswitch_w(int n, const uint64_t *ct3, const uint64_t *evkw, int logw, uint64_t *out) {
    init_consts();
    if (!valid_n(n) || logw < 16 || logw > 60) return ORC_E_ARG;
    u128 *c = malloc((size_t)3 * n * sizeof(u128)), *o0 = malloc(n * sizeof(u128)), *o1 = malloc(n * sizeof(u128));
    for (int p = 0; p < 3; p++) poly_from_res(n, ct3 + (size_t)p * 2 * n, c + (size_t)p * n);
    key_switch_w(n, c, c + n, c + 2 * n, evkw, logw, o0, o1);
    poly_to_res(n, o0, out);
    poly_to_res(n, o1, out + 2 * n);
    free(c); free(o0); free(o1);
    return ORC_OK;
}

/* bound B = d * 2n * ((q-1)/2)^2 on |X_k| */
static bi x_bound(int n, int d) {
    u128 h = (orc_q() - 1) / 2;
    bi b = bi_mul_u128(h, h);
    bi_mag_mul_u64(&b, (uint64_t)d * 2 * (uint64_t)n);
    return b;
}

/* c_k = [round(t X_k / q)]_q for the three tensor polynomials X[0..3n) */
static void scale_round(int n, const bi *X, u128 *c, orc_stats *st) {
    uint64_t ties = 0;
#pragma omp parallel for schedule(static) reduction(+ : ties)
    for (int k = 0; k < 3 * n; k++) {
        int tie = 0;
        bi y = round_t_over_q(&X[k], &tie);
        ties += (uint64_t)tie;
        c[k] = bi_mod_q(&y);
    }
    st->ties += ties;
    st->scale_rounds += 1;
}

/*
 * Score ciphertext of one gallery block.
 * probe, gal: d ciphertexts [d][2][2][n]; evk [2][2][2][n]; out [2][2][n].
 * pre_ks (optional) receives (c0, c1, c2) before relinearisation, [3][2][n].
 *
 *   1. lift every ciphertext coefficient to (-(q-1)/2, (q-1)/2];
 *   2. over Z: X0 = sum_i a0 (*) b0, X1 = sum_i (a0 (*) b1 + a1 (*) b0), X2 = sum_i a1 (*) b1;
 *   3. c_k = [round(t X_k / q)]_q;
 *   4. relinearise (c0, c1, c2) -> (c0', c1').
 */
int orc_search_block(int n, int d, const uint64_t *probe, const uint64_t *gal,
                     const uint64_t *evk, uint64_t *out, uint64_t *pre_ks, orc_stats *st) {
    init_consts();
    if (!valid_n(n) || d <= 0 || d > 4096) return ORC_E_ARG;
    size_t ctw = (size_t)4 * n; /* words per ciphertext */
    dig *A0 = malloc((size_t)d * n * sizeof(dig)), *A1 = malloc((size_t)d * n * sizeof(dig));
    dig *B0 = malloc((size_t)d * n * sizeof(dig)), *B1 = malloc((size_t)d * n * sizeof(dig));
    bi *X = malloc((size_t)3 * n * sizeof(bi));
    u128 *c = malloc((size_t)3 * n * sizeof(u128));
    u128 *o0 = malloc(n * sizeof(u128)), *o1 = malloc(n * sizeof(u128));
    if (!A0 || !A1 || !B0 || !B1 || !X || !c || !o0 || !o1) return ORC_E_MEM;
    for (int i = 0; i < d; i++) {
        load_ct_dig(n, probe + i * ctw, A0 + (size_t)i * n, A1 + (size_t)i * n);
        load_ct_dig(n, gal + i * ctw, B0 + (size_t)i * n, B1 + (size_t)i * n);
    }
#pragma omp parallel for schedule(dynamic, 4)
    for (int k = 0; k < n; k++) {
        bi x0 = bi_zero(), x1 = bi_zero(), x2 = bi_zero();
        for (int i = 0; i < d; i++) {
            const dig *a0 = A0 + (size_t)i * n, *a1 = A1 + (size_t)i * n;
            const dig *b0 = B0 + (size_t)i * n, *b1 = B1 + (size_t)i * n;
            part p0 = {0, 0, 0}, p1 = {0, 0, 0}, p2 = {0, 0, 0};
            negacyclic_coeff(n, k, a0, b0, &p0);
            negacyclic_coeff(n, k, a0, b1, &p1);
            negacyclic_coeff(n, k, a1, b0, &p1);
            negacyclic_coeff(n, k, a1, b1, &p2);
            part_flush(&p0, &x0);
            part_flush(&p1, &x1);
            part_flush(&p2, &x2);
        }
        X[k] = x0;
        X[n + k] = x1;
        X[2 * n + k] = x2;
    }
    st->tensor_products += (uint64_t)d;
    st->tensor_adds += (uint64_t)(d - 1);

    bi bound = x_bound(n, d);
    for (int k = 0; k < 3 * n; k++) {
        bi a = bi_is_neg(&X[k]) ? bi_neg(X[k]) : X[k];
        if (bi_cmp_u(&a, &bound) > 0) st->bound_violations++;
        uint64_t bl = (uint64_t)bi_bitlen_abs(&X[k]);
        if (bl > st->max_x_bits) st->max_x_bits = bl;
    }
    scale_round(n, X, c, st);
    if (pre_ks)
        for (int p = 0; p < 3; p++) poly_to_res(n, c + (size_t)p * n, pre_ks + (size_t)p * 2 * n);
    key_switch(n, c, c + n, c + 2 * n, evk, o0, o1);
    st->key_switches += 1;
    poly_to_res(n, o0, out);
    poly_to_res(n, o1, out + 2 * n);
    int rc = (st->ties || st->bound_violations) ? ORC_E_BOUND : ORC_OK;
    free(A0); free(A1); free(B0); free(B1); free(X); free(c); free(o0); free(o1);
    return rc;
}

/*
 * Paper-literal form of Alg 7's inner loop with Alg 5 applied to every
 * product: s <- init (zero if init == NULL); for each i: s <- CipherAdd(s,
 * CipherMultiply(ct_i, D_i)), where CipherMultiply scales and rounds each of
 * its three tensor polynomials and relinearises before the addition.  Used
 * only as a cross-check: it decrypts to the same scores as orc_search_block
 * but gives a different ciphertext.
 */
int orc_search_block_per_product(int n, int d, const uint64_t *probe, const uint64_t *gal,
                                 const uint64_t *evk, const uint64_t *init, uint64_t *out,
                                 orc_stats *st) {
    init_consts();
    if (!valid_n(n) || d <= 0 || d > 4096) return ORC_E_ARG;
    size_t ctw = (size_t)4 * n;
    u128 q = orc_q();
    dig *a0 = malloc(n * sizeof(dig)), *a1 = malloc(n * sizeof(dig));
    dig *b0 = malloc(n * sizeof(dig)), *b1 = malloc(n * sizeof(dig));
    bi *X = malloc((size_t)3 * n * sizeof(bi));
    u128 *c = malloc((size_t)3 * n * sizeof(u128));
    u128 *o0 = malloc(n * sizeof(u128)), *o1 = malloc(n * sizeof(u128));
    u128 *s0 = malloc(n * sizeof(u128)), *s1 = malloc(n * sizeof(u128));
    if (init) {
        poly_from_res(n, init, s0);
        poly_from_res(n, init + 2 * n, s1);
    } else {
        memset(s0, 0, n * sizeof(u128));
        memset(s1, 0, n * sizeof(u128));
    }
    bi bound = x_bound(n, 1);
    for (int i = 0; i < d; i++) {
        load_ct_dig(n, probe + i * ctw, a0, a1);
        load_ct_dig(n, gal + i * ctw, b0, b1);
#pragma omp parallel for schedule(static)
        for (int k = 0; k < n; k++) {
            part p0 = {0, 0, 0}, p1 = {0, 0, 0}, p2 = {0, 0, 0};
            bi x0 = bi_zero(), x1 = bi_zero(), x2 = bi_zero();
            negacyclic_coeff(n, k, a0, b0, &p0);
            negacyclic_coeff(n, k, a0, b1, &p1);
            negacyclic_coeff(n, k, a1, b0, &p1);
            negacyclic_coeff(n, k, a1, b1, &p2);
            part_flush(&p0, &x0);
            part_flush(&p1, &x1);
            part_flush(&p2, &x2);
            X[k] = x0;
            X[n + k] = x1;
            X[2 * n + k] = x2;
        }
        st->tensor_products += 1;
        for (int k = 0; k < 3 * n; k++) {
            bi a = bi_is_neg(&X[k]) ? bi_neg(X[k]) : X[k];
            if (bi_cmp_u(&a, &bound) > 0) st->bound_violations++;
        }
        scale_round(n, X, c, st);
        key_switch(n, c, c + n, c + 2 * n, evk, o0, o1);
        st->key_switches += 1;
        for (int k = 0; k < n; k++) { /* CipherAdd (Alg 4) */
            s0[k] = (s0[k] + o0[k]) % q;
            s1[k] = (s1[k] + o1[k]) % q;
        }
        if (i > 0 || init) st->tensor_adds += 1;
    }
    poly_to_res(n, s0, out);
    poly_to_res(n, s1, out + 2 * n);
    int rc = (st->ties || st->bound_violations) ? ORC_E_BOUND : ORC_OK;
    free(a0); free(a1); free(b0); free(b1); free(X); free(c); free(o0); free(o1);
    free(s0); free(s1);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Alg 3: decryption                                                        */
/* ------------------------------------------------------------------------ */

/*
 * pt = [round(t/q [c0 + c1 s (+ c2 s^2)]_q)]_t, then slots = decode(pt).
 * ct: [ncomp][2 limbs][n] with ncomp = 2, or 3 for an unrelinearised (c0, c1, c2).
 * pt_out (optional): [n] in [0, t).  noise_out (optional, 2 words): max over k of
 * |[v_k - Delta pt_k]_q| as a 128-bit value, v = [c0 + c1 s (+ c2 s^2)]_q.
 */
int orc_decrypt(int n, const int8_t *sk, const uint64_t *ct, int ncomp, int64_t *slots,
                uint32_t *pt_out, uint64_t *noise_out) {
    init_consts();
    if (!valid_n(n) || (ncomp != 2 && ncomp != 3)) return ORC_E_ARG;
    u128 q = orc_q(), delta = q / ORC_T;
    int32_t *s = malloc(n * sizeof(int32_t));
    u128 *c0 = malloc(n * sizeof(u128)), *c1 = malloc(n * sizeof(u128)), *tmp = malloc(n * sizeof(u128));
    u128 *c1s = malloc(n * sizeof(u128));
    uint32_t *pt = malloc(n * sizeof(uint32_t));
    for (int k = 0; k < n; k++) s[k] = sk[k];
    poly_from_res(n, ct, c0);
    poly_from_res(n, ct + 2 * n, c1);
    negacyclic_small_mod_q(n, c1, s, c1s);
    if (ncomp == 3) { /* c2 s^2 = (c2 s) s */
        u128 *c2 = malloc(n * sizeof(u128)), *c2s = malloc(n * sizeof(u128));
        poly_from_res(n, ct + 4 * n, c2);
        negacyclic_small_mod_q(n, c2, s, c2s);
        negacyclic_small_mod_q(n, c2s, s, tmp);
        for (int k = 0; k < n; k++) c1s[k] = (c1s[k] + tmp[k]) % q;
        free(c2);
        free(c2s);
    }
    u128 maxnoise = 0;
    int tie_seen = 0;
    for (int k = 0; k < n; k++) {
        u128 v = (c0[k] + c1s[k]) % q;
        i128 vs = lift_sym(v);
        bi X = bi_from_i128(vs);
        int tie = 0;
        bi y = round_t_over_q(&X, &tie);
        tie_seen |= tie;
        bi yq;
        u128 r;
        bi_floordiv(&y, ORC_T, &yq, &r); /* [y]_t in [0, t) */
        pt[k] = (uint32_t)r;
        i128 e = lift_sym(mod_q_i128(vs - (i128)(delta * r)));
        u128 ae = (u128)(e < 0 ? -e : e);
        if (ae > maxnoise) maxnoise = ae;
    }
    if (pt_out) memcpy(pt_out, pt, n * sizeof(uint32_t));
    if (noise_out) {
        noise_out[0] = (uint64_t)maxnoise;
        noise_out[1] = (uint64_t)(maxnoise >> 64);
    }
    int rc = slots ? orc_decode(n, pt, slots) : ORC_OK;
    free(s); free(c0); free(c1); free(tmp); free(c1s); free(pt);
    return tie_seen ? ORC_E_TIE : rc;
}

/* constants for the wrapper's self-description */
void orc_params(uint64_t *out) {
    out[0] = ORC_Q1;
    out[1] = ORC_Q2;
    out[2] = ORC_T;
    out[3] = ORC_MAXN;
}
