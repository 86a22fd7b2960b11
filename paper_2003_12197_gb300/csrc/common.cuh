// Device-side building blocks of the HERS library: compile-time moduli and
// constants, 64-bit modular arithmetic on the integer pipes, the ChaCha20
// stream and samplers every random draw comes from, and the negacyclic NTT
// over one polynomial held in shared memory.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "hers_consts.h"

namespace hers {

// ---------------------------------------------------------------- constants
// Modulus index i: 0 = q1, 1 = q2, 2 = the default t, 3 = the paper's t.
static __constant__ uint64_t c_mod[NUM_MODS] = HERS_MOD_INIT;
static __constant__ uint64_t c_ninv[NUM_MODS] = HERS_NINV_INIT;
static __constant__ uint64_t c_ninv_s[NUM_MODS] = HERS_NINV_S_INIT;
static __constant__ uint64_t c_one_s[NUM_MODS] = HERS_ONE_S_INIT;
static __constant__ uint64_t c_barrett[NUM_Q] = HERS_BARRETT_INIT;
static __constant__ uint64_t c_chi_cdt[CHI_LEN] = HERS_CHI_CDT_INIT;

// Search basis r_0 .. r_7 (primes below 2^30, = 1 mod 2N; M = their product):
// the basis of the resident form and of the exact tensor sums.
static __constant__ uint32_t c_smod[NUM_S] = HERS_SMOD_INIT;
static __constant__ uint32_t c_sninv[NUM_S] = HERS_SNINV_INIT;      // N^-1 mod r
static __constant__ uint32_t c_sninv_s[NUM_S] = HERS_SNINV_S_INIT;  // its Shoup companion (2^32)
static __constant__ uint64_t c_smu[NUM_S] = HERS_SMU_INIT;          // floor(2^64 / r)
static __constant__ uint32_t c_sr32[NUM_S] = HERS_SR32_INIT;        // 2^32 mod r
static __constant__ uint64_t c_soff63[NUM_S] = HERS_SOFF63_INIT;    // multiple of r just below 2^63
// Extension: [q1]_r, [q1 2^27]_r, [-q]_r and floor(2^59 / r) (see lift_mod_r).
static __constant__ uint32_t c_q1_mod_r[NUM_S] = HERS_Q1_MOD_R_INIT;
static __constant__ uint32_t c_lift_b[NUM_S] = HERS_LIFT_B_INIT;
static __constant__ uint32_t c_lift_nq[NUM_S] = HERS_LIFT_NQ_INIT;
static __constant__ uint32_t c_mu59[NUM_S] = HERS_MU59_INIT;
// CRT of X' = X + q 2^129: y_i = x_i Minv_i + HM_i mod r_i, Minv_i = (M / r_i)^-1
// mod r_i, HM_i = (q 2^129 mod r_i) Minv_i; alpha = floor(sum y_i PHI_i / 2^60).
static __constant__ uint32_t c_minv[NUM_S] = HERS_MINV_INIT;
static __constant__ uint32_t c_minv_s[NUM_S] = HERS_MINV_S_INIT;
static __constant__ uint32_t c_hm[NUM_S] = HERS_HM_INIT;
static __constant__ uint32_t c_phi[NUM_S] = HERS_PHI_INIT;  // floor(2^60 / r) < 2^31
// 27-bit digits of (M / r_i) mod q_j, [i][j][2], and of M mod q_j, [j][2].
static __constant__ uint32_t c_mi_q_cols[NUM_S * 4] = HERS_MI_Q_COLS_INIT;
static __constant__ uint32_t c_m_q_cols[4] = HERS_M_Q_COLS_INIT;

// Plaintext modulus t and what depends on it; a context uses entry 0 (the
// default t = 4169729) or entry 1 (the paper's t = 1032193), and its keys
// carry the index (DevKeys::pm).
struct PlainMod {
    uint64_t t;
    int mod;                                 // index of t in the modulus arrays
    uint64_t q1_mod_t, q_mod_t, qinv_t;      // decryption: pt = [-r q^-1]_t
    uint64_t t_mod[NUM_Q], t_s[NUM_Q];       // t mod q_l and its Shoup companion
    uint64_t delta[2], delta_s[2];           // Delta = floor(q / t) mod q_l
    // scale-and-round (t M_i = A_i q + B_i, t M = A_M q + B_M), 27-bit digits:
    uint32_t b_cols[NUM_S * 4];              // B_i, [i][4]
    uint32_t bm_cols[4];                     // B_M
    uint32_t a_cols[NUM_S * 4];              // A_i mod q_j, [i][j][2]
    uint32_t am_cols[4];                     // A_M mod q_j, [j][2]
    uint64_t dshift[2];                      // [8 + t 2^129] mod q_j
};
static __constant__ PlainMod c_plain[2] = HERS_PLAIN_INIT;

// Resident (search) form of ciphertexts: NTT domain over the search basis,
// each residue as its centred value (one int32, |v| < 2^29), tiled so that
// everything one search CTA streams is contiguous, with the two polynomials
// of a ciphertext interleaved per coefficient (one 8-byte load gives both):
//   [block][limb r_l][tile][dim][TILE coefficients][poly]
// A gallery block occupies 16 d N int32 (8 d N 64-bit words); a prepared
// probe is block 0 of it.  Offsets below count int32 elements.
constexpr int TILE = 256;
constexpr int NTILES = N / TILE;
__host__ __device__ __forceinline__ uint64_t resident_offset(uint64_t b, int limb, int k, uint32_t d,
                                                             uint32_t i, int poly) {
    return ((((b * NUM_S + (uint64_t)limb) * NTILES + (uint64_t)(k / TILE)) * d + i) * TILE +
            (uint64_t)(k % TILE)) * 2 + (uint64_t)poly;
}

// Twiddle table of modulus i inside the table buffer the context owns:
// [i][forward, inverse][N] pairs (w, w'), w' = floor(w 2^64 / p) (Shoup), so
// one 16-byte load fetches a twiddle with its companion.  Entry 0 of the
// inverse table (never used as a butterfly twiddle) holds the last inverse
// stage's twiddle times N^-1.  After the NUM_MODS tables come those of the
// search basis in the same form with 32-bit words: pairs (w, floor(w 2^32 / r)).
__device__ __forceinline__ const ulonglong2* tw_fwd(const uint64_t* tw, int i) {
    return (const ulonglong2*)(tw + (size_t)4 * N * i);
}
__device__ __forceinline__ const ulonglong2* tw_inv(const uint64_t* tw, int i) {
    return (const ulonglong2*)(tw + (size_t)4 * N * i + 2 * N);
}
__device__ __forceinline__ const uint2* tw32_fwd(const uint64_t* tw, int i) {
    return (const uint2*)(tw + (size_t)4 * N * NUM_MODS) + (size_t)2 * N * i;
}
__device__ __forceinline__ const uint2* tw32_inv(const uint64_t* tw, int i) {
    return (const uint2*)(tw + (size_t)4 * N * NUM_MODS) + (size_t)2 * N * i + N;
}

// ---------------------------------------------------------------- arithmetic

__device__ __forceinline__ uint64_t csub(uint64_t x, uint64_t p) { return x >= p ? x - p : x; }

__device__ __forceinline__ uint64_t add_mod(uint64_t a, uint64_t b, uint64_t p) { return csub(a + b, p); }

__device__ __forceinline__ uint64_t sub_mod(uint64_t a, uint64_t b, uint64_t p) {
    return a >= b ? a - b : a + p - b;
}

// Shoup multiplication by a fixed w < p with ws = floor(w 2^64 / p):
// x w mod p, lazily in [0, 2p), for any x < 2^64 and p < 2^63.
__device__ __forceinline__ uint64_t shoup_lazy(uint64_t x, uint64_t w, uint64_t ws, uint64_t p) {
    return x * w - __umul64hi(x, ws) * p;
}

__device__ __forceinline__ uint64_t shoup(uint64_t x, uint64_t w, uint64_t ws, uint64_t p) {
    return csub(shoup_lazy(x, w, ws, p), p);
}

// Shoup multiplication with a truncated quotient, for the NTT butterflies.
// The high half of x ws is taken from three of the four 32x32 partial
// products (xh wsh exactly, the high words of xh wsl and xl wsh); the dropped
// fractions sum to less than 3, so the quotient is short of Shoup's by 0, 1 or
// 2 and x w - q p lies in [0, 4p) (Shoup's own lies in [0, 2p)).  Needs p <
// 2^61 so that 4p fits; costs one 32x32->64 and two 32x32-high products in
// place of a 64x64-high product.
__device__ __forceinline__ uint64_t shoup4(uint64_t x, uint64_t w, uint64_t ws, uint64_t p) {
    const uint32_t xl = (uint32_t)x, xh = (uint32_t)(x >> 32);
    const uint32_t sl = (uint32_t)ws, sh = (uint32_t)(ws >> 32);
    const uint64_t q = (uint64_t)xh * sh + __umulhi(xh, sl) + __umulhi(xl, sh);
    return x * w - q * p;
}
// shoup4 reduced to [0, p).
__device__ __forceinline__ uint64_t shoup4_full(uint64_t x, uint64_t w, uint64_t ws, uint64_t p) {
    return csub(csub(shoup4(x, w, ws, p), 2 * p), p);
}

// x mod p_i for any 64-bit x (Shoup with w = 1).
__device__ __forceinline__ uint64_t reduce64(uint64_t x, int i) {
    return csub(shoup_lazy(x, 1, c_one_s[i], c_mod[i]), c_mod[i]);
}

// mod-t arithmetic (t < 2^23): products fit in 64 bits
__device__ __forceinline__ uint64_t mul_mod_t(uint64_t a, uint64_t b, uint64_t t) { return (a * b) % t; }

// ---------------------------------------------------------------- search-basis arithmetic (r < 2^30)
__device__ __forceinline__ uint32_t csub32(uint32_t x, uint32_t p) { return min(x, x - p); }
// Shoup with 32-bit words: x w mod r in [0, 2r) for any x < 2^32, w < r, ws = floor(w 2^32 / r).
__device__ __forceinline__ uint32_t shoup32(uint32_t x, uint32_t w, uint32_t ws, uint32_t r) {
    return x * w - __umulhi(x, ws) * r;
}
// x mod r_i for any 64-bit x (Barrett with mu = floor(2^64 / r): the quotient
// estimate is at most one short).
__device__ __forceinline__ uint32_t reduce_r(uint64_t x, int i) {
    const uint32_t r = c_smod[i];
    return csub32((uint32_t)x - (uint32_t)__umul64hi(x, c_smu[i]) * r, r);
}
// Partial fold of a signed 64-bit sum s: s' = hi(s) (2^32 mod r) + lo(s) = s (mod r)
// with |s'| < 2^61 + 2^32 (one 32x32->64 multiply-add).
__device__ __forceinline__ int64_t pfold(int64_t s, int32_t r32) {
    int64_t out = (int64_t)(uint64_t)(uint32_t)s;
    asm("mad.wide.s32 %0, %1, %2, %0;" : "+l"(out) : "r"((int32_t)(s >> 32)), "r"(r32));
    return out;
}
// Residue in [0, r_i) of a signed 64-bit sum with |s| < 2^63 - r_i.
__device__ __forceinline__ uint32_t fold_full(int64_t s, int i) { return reduce_r((uint64_t)s + c_soff63[i], i); }
// Centred value of a residue v in [0, r) (the resident storage), and back.
__device__ __forceinline__ int32_t centre32(uint32_t v, uint32_t r) {
    return v > (r - 1) / 2 ? (int32_t)(v - r) : (int32_t)v;
}
__device__ __forceinline__ uint32_t uncentre32(int32_t c, uint32_t r) {
    return c < 0 ? (uint32_t)(c + (int32_t)r) : (uint32_t)c;
}

// x mod q_i (i = 0, 1) for x = hi 2^64 + lo < 2^108: Barrett with
// mu = floor(2^108 / q), quotient estimate floor(floor(x / 2^53) mu / 2^55),
// at most 2 below the true one.
__device__ __forceinline__ uint64_t reduce128(uint64_t lo, uint64_t hi, int i) {
    const uint64_t p = c_mod[i];
    const uint64_t z = (hi << 11) | (lo >> 53);
    const uint64_t mu = c_barrett[i];
    const uint64_t qh = (__umul64hi(z, mu) << 9) | ((z * mu) >> 55);
    uint64_t r = lo - qh * p;
    r = csub(r, p);
    return csub(r, p);
}

// a b mod q_i for a, b < q_i (i = 0, 1).
__device__ __forceinline__ uint64_t mul_mod(uint64_t a, uint64_t b, int i) {
    return reduce128(a * b, __umul64hi(a, b), i);
}

__device__ __forceinline__ int brev12(int x) { return (int)(__brev((unsigned)x) >> (32 - LOGN)); }

// Word of coefficient x of a polynomial held in shared memory (swizzled order,
// see the NTT section below).
__device__ __forceinline__ int swz(int x) { return x ^ ((x >> 4) & 15); }

// ---------------------------------------------------------------- ChaCha20 (RFC 8439, Sec. 2.3)

__device__ __forceinline__ uint32_t rotl32(uint32_t x, int r) { return __funnelshift_l(x, x, r); }

#define HERS_QR(a, b, c, d)                                  \
    a += b; d ^= a; d = rotl32(d, 16);                      \
    c += d; b ^= c; b = rotl32(b, 12);                      \
    a += b; d ^= a; d = rotl32(d, 8);                       \
    c += d; b ^= c; b = rotl32(b, 7);

// Block `counter` of the stream keyed by (seed_lo, seed_hi, 0 x 6) with nonce
// (purpose, obj_lo, obj_hi): 16 little-endian words.
__device__ __forceinline__ void chacha20(uint64_t seed, uint32_t purpose, uint64_t obj,
                                         uint32_t counter, uint32_t out[16]) {
    uint32_t s[16];
    s[0] = 0x61707865u; s[1] = 0x3320646eu; s[2] = 0x79622d32u; s[3] = 0x6b206574u;
    s[4] = (uint32_t)seed; s[5] = (uint32_t)(seed >> 32);
    s[6] = s[7] = s[8] = s[9] = s[10] = s[11] = 0u;
    s[12] = counter;
    s[13] = purpose; s[14] = (uint32_t)obj; s[15] = (uint32_t)(obj >> 32);
    uint32_t x0 = s[0], x1 = s[1], x2 = s[2], x3 = s[3], x4 = s[4], x5 = s[5], x6 = s[6], x7 = s[7];
    uint32_t x8 = s[8], x9 = s[9], x10 = s[10], x11 = s[11], x12 = s[12], x13 = s[13], x14 = s[14], x15 = s[15];
#pragma unroll
    for (int r = 0; r < 10; r++) {
        HERS_QR(x0, x4, x8, x12) HERS_QR(x1, x5, x9, x13) HERS_QR(x2, x6, x10, x14) HERS_QR(x3, x7, x11, x15)
        HERS_QR(x0, x5, x10, x15) HERS_QR(x1, x6, x11, x12) HERS_QR(x2, x7, x8, x13) HERS_QR(x3, x4, x9, x14)
    }
    out[0] = x0 + s[0]; out[1] = x1 + s[1]; out[2] = x2 + s[2]; out[3] = x3 + s[3];
    out[4] = x4 + s[4]; out[5] = x5 + s[5]; out[6] = x6 + s[6]; out[7] = x7 + s[7];
    out[8] = x8 + s[8]; out[9] = x9 + s[9]; out[10] = x10 + s[10]; out[11] = x11 + s[11];
    out[12] = x12 + s[12]; out[13] = x13 + s[13]; out[14] = x14 + s[14]; out[15] = x15 + s[15];
}
#undef HERS_QR

// Stream purposes (nonce word 0).  Encryption streams: base + 0 = u, + 1 = e1, + 2 = e2.
constexpr uint32_t PRF_KG_SK = 0x01u;
constexpr uint32_t PRF_KG_PK_A = 0x02u;   // obj = limb
constexpr uint32_t PRF_KG_PK_E = 0x03u;
constexpr uint32_t PRF_KG_EVK_A = 0x04u;  // obj = 2 j + limb
constexpr uint32_t PRF_KG_EVK_E = 0x05u;  // obj = j
constexpr uint32_t PRF_KG_EVKW_A = 0x06u; // base-w evaluation keys: obj = 2 j + limb
constexpr uint32_t PRF_KG_EVKW_E = 0x07u; // obj = j
constexpr uint32_t PRF_GALLERY = 0x11u;   // obj = block * d + dim
constexpr uint32_t PRF_PROBE = 0x21u;     // obj = dim
constexpr uint32_t PRF_RERAND = 0x31u;    // output re-randomisation Enc(0); obj = block
constexpr uint32_t PRF_ENROLL = 0x41u;    // online enrollment (Alg 6); obj = (b N + v) d + dim
constexpr int MAX_ATTEMPTS = 16;

// One coefficient k of a ternary stream, walking attempts a = 0, 1, ...
// (32-bit word a N + k; accept w < 3 floor(2^32 / 3)).  Returns -2 when all
// attempts were rejected.
static __device__ __noinline__ int ternary_slow(uint64_t seed, uint32_t purpose, uint64_t obj, int k) {
    for (int a = 0; a < MAX_ATTEMPTS; a++) {
        uint32_t W = (uint32_t)(a * N + k);
        uint32_t blk[16];
        chacha20(seed, purpose, obj, W >> 4, blk);
        uint32_t w = blk[W & 15];
        if (w < 0xFFFFFFFFu) return (int)(w % 3u) - 1;
    }
    return -2;
}

// One coefficient k of a uniform stream mod p (64-bit word a N + k masked to
// 54 bits, accept below p).  Returns ~0 when all attempts were rejected.
static __device__ __noinline__ uint64_t uniform_slow(uint64_t seed, uint32_t purpose, uint64_t obj, int k,
                                              uint64_t p) {
    for (int a = 0; a < MAX_ATTEMPTS; a++) {
        uint32_t w = (uint32_t)(a * N + k);
        uint32_t blk[16];
        chacha20(seed, purpose, obj, w >> 3, blk);
        uint64_t v = ((uint64_t)blk[(2 * w + 1) & 15] << 32 | blk[(2 * w) & 15]) & ((1ull << 54) - 1);
        if (v < p) return v;
    }
    return ~0ull;
}

__device__ __forceinline__ int chi_from_word(uint64_t U) {
    int c = 0;
#pragma unroll
    for (int j = 0; j < CHI_LEN; j++) c += (c_chi_cdt[j] <= U) ? 1 : 0;
    return CHI_MIN + c;
}

// Fill the shared-memory polynomial out (swizzled order) with a ternary
// polynomial as residues mod p (-1 -> p - 1).
// All threads of the CTA call this; the block stream is split over threads.
__device__ __forceinline__ void sample_ternary_mod(uint64_t seed, uint32_t purpose, uint64_t obj,
                                                   uint64_t p, uint64_t* out, int* err) {
    for (int c = threadIdx.x; c < N / 16; c += blockDim.x) {
        uint32_t blk[16];
        chacha20(seed, purpose, obj, (uint32_t)c, blk);
#pragma unroll
        for (int j = 0; j < 16; j++) {
            int k = 16 * c + j;
            int v;
            if (blk[j] < 0xFFFFFFFFu) v = (int)(blk[j] % 3u) - 1;
            else v = ternary_slow(seed, purpose, obj, k);
            if (v == -2) { atomicOr(err, 1); v = 0; }
            out[swz(k)] = v < 0 ? p - 1 : (uint64_t)v;
        }
    }
}

// Fill the shared-memory polynomial out (swizzled order) with a uniform
// polynomial mod p.
__device__ __forceinline__ void sample_uniform(uint64_t seed, uint32_t purpose, uint64_t obj,
                                               uint64_t p, uint64_t* out, int* err) {
    for (int c = threadIdx.x; c < N / 8; c += blockDim.x) {
        uint32_t blk[16];
        chacha20(seed, purpose, obj, (uint32_t)c, blk);
#pragma unroll
        for (int j = 0; j < 8; j++) {
            int k = 8 * c + j;
            uint64_t v = (((uint64_t)blk[2 * j + 1] << 32) | blk[2 * j]) & ((1ull << 54) - 1);
            if (v >= p) {
                v = uniform_slow(seed, purpose, obj, k, p);
                if (v == ~0ull) { atomicOr(err, 1); v = 0; }
            }
            out[swz(k)] = v;
        }
    }
}

// ---------------------------------------------------------------- NTT (one polynomial in smem)
//
// Negacyclic NTT of one N = 4096 polynomial held in shared memory by a CTA of
// NTT_THREADS = 256 threads, 16 coefficients per thread.  The twelve radix-2
// stages run as three phases of four stages on registers:
//   phase A: thread t holds x = t + 256 a        (stages with distance 2048 .. 256)
//   phase B: thread t holds x = 256 (t/16) + (t%16) + 16 a   (distance 128 .. 16)
//   phase C: thread t holds x = 16 t + a         (distance 8 .. 1),   a = 0..15.
// Between A and B the CTA synchronises; B and C exchange data only inside
// groups of 16 threads (half a warp), so a __syncwarp suffices.
//
// Polynomials live in shared memory in swizzled order: coefficient x is at
// word swz(x) = x ^ ((x >> 4) & 15).  Every access pattern used here and in
// the kernels (t + 256 a, t + 512 a, the three phases) then touches each bank
// at most twice per warp, the minimum for 32 8-byte words.
//
// Forward: Cooley-Tukey with psi-powers in bit-reversed order; input residues
// < 2p, output fully reduced in bit-reversed order: index j holds the
// evaluation at psi^(2 brev(j) + 1).
// Inverse: Gentleman-Sande with inverse psi-powers; bit-reversed input < 2p,
// natural-order output times N^-1 (folded into the last stage), fully reduced.
// All NTT_THREADS threads must call these; they begin and end with a barrier.
constexpr int NTT_THREADS = 256;

// Twiddle index of a butterfly.  In every phase, the pairs (a, a + h) of
// stage h with a = 2h j + r, r < h, share one twiddle: for the three base
// patterns, base + STRIDE r < 2 STRIDE h whenever base is taken modulo
// 2 STRIDE h, so i = floor(base / (2 STRIDE h)) + j.  Each stage therefore
// loads 8 / h twiddles (15 per phase) rather than 8.
template <int STRIDE>
__device__ __forceinline__ void ct_phase(uint64_t v[16], int base, const ulonglong2* __restrict__ w,
                                         uint64_t p) {
    const uint64_t four_p = 4 * p;
#pragma unroll
    for (int h = 8; h >= 1; h >>= 1) {
        const int t = STRIDE * h;       // butterfly distance
        const int m = N / (2 * t);      // groups in this stage
        const int i0 = base / (2 * t);
#pragma unroll
        for (int j = 0; j < 8 / h; j++) {
            const ulonglong2 W = __ldg(w + m + i0 + j);
#pragma unroll
            for (int r = 0; r < h; r++) {
                const int a = 2 * h * j + r;
                // no reduction of U: inputs < 2p grow by < 4p per stage, so
                // every value stays below 50p < 2^60 over the twelve stages
                const uint64_t U = v[a];
                const uint64_t V = shoup4(v[a + h], W.x, W.y, p);
                v[a] = U + V;
                v[a + h] = U - V + four_p;
            }
        }
    }
}

// LAST: this phase holds the final stage (distance 2048), whose outputs are
// multiplied by N^-1 on the way (twiddle entry 0 carries W N^-1).  Values stay
// below 4p between stages; the last stage reduces fully.
template <int STRIDE, bool LAST>
__device__ __forceinline__ void gs_phase(uint64_t v[16], int base, const ulonglong2* __restrict__ w,
                                         uint64_t p, uint64_t ninv, uint64_t ninv_s) {
    const uint64_t four_p = 4 * p;
#pragma unroll
    for (int h = 1; h <= 8; h <<= 1) {
        const int t = STRIDE * h;
        const int m = N / (2 * t);
        const int i0 = base / (2 * t);
#pragma unroll
        for (int j = 0; j < 8 / h; j++) {
            const ulonglong2 W = __ldg(LAST && h == 8 ? w : w + m + i0 + j);
#pragma unroll
            for (int r = 0; r < h; r++) {
                const int a = 2 * h * j + r;
                const uint64_t U = v[a], V = v[a + h];
                if (LAST && h == 8) {
                    v[a] = shoup4_full(U + V, ninv, ninv_s, p);
                    v[a + h] = shoup4_full(U - V + four_p, W.x, W.y, p);
                } else {
                    const uint64_t S = U + V;
                    v[a] = S >= four_p ? S - four_p : S;
                    v[a + h] = shoup4(U - V + four_p, W.x, W.y, p);
                }
            }
        }
    }
}

// Transposes the 16 x 16 matrix of 64-bit words held by the 16 lanes of each
// half-warp (lane i holds row i in v; afterwards it holds column i): four
// rounds of 64-bit __shfl_xor_sync (distances 8, 4, 2, 1), each swapping the
// off-diagonal halves of the blocks of that size.  Every lane of the warp
// must call it.
__device__ __forceinline__ void transpose16_shfl64(uint64_t v[16], int i) {
#pragma unroll
    for (int m = 8; m >= 1; m >>= 1) {
        const bool hi = (i & m) != 0;
#pragma unroll
        for (int a = 0; a < 16; a++) {
            if (a & m) continue;
            const uint64_t send = hi ? v[a] : v[a | m];
            const uint64_t recv = __shfl_xor_sync(0xffffffffu, send, m);
            if (hi) v[a] = recv;
            else v[a | m] = recv;
        }
    }
}

// t: the calling thread's index among the NTT_THREADS threads that run the
// transform (as for the 32-bit transforms below).  SHFL: the exchange
// between the two phases that stay inside a half-warp (coefficients
// 256 (t / 16) + (t % 16) + 16 a and 16 t + a, a 16 x 16 transpose) goes
// through warp shuffles instead of shared memory.
template <bool SHFL = false>
__device__ __forceinline__ void ntt_fwd_smem(uint64_t* sm, const ulonglong2* __restrict__ w, uint64_t p,
                                             uint64_t one_s, int t = threadIdx.x) {
    uint64_t v[16];
    __syncthreads();
    {   // phase A
        const int base = t;
#pragma unroll
        for (int a = 0; a < 16; a++) v[a] = sm[swz(base + 256 * a)];
        ct_phase<256>(v, base, w, p);
#pragma unroll
        for (int a = 0; a < 16; a++) sm[swz(base + 256 * a)] = v[a];
    }
    __syncthreads();
    {   // phase B
        const int base = 256 * (t >> 4) + (t & 15);
#pragma unroll
        for (int a = 0; a < 16; a++) v[a] = sm[swz(base + 16 * a)];
        ct_phase<16>(v, base, w, p);
        if (SHFL) {
            transpose16_shfl64(v, t & 15);
        } else {
#pragma unroll
            for (int a = 0; a < 16; a++) sm[swz(base + 16 * a)] = v[a];
        }
    }
    if (!SHFL) __syncwarp();
    {   // phase C, then full reduction (values < 50p)
        const int base = 16 * t;
        if (!SHFL) {
#pragma unroll
            for (int a = 0; a < 16; a++) v[a] = sm[swz(base + a)];
        }
        ct_phase<1>(v, base, w, p);
#pragma unroll
        for (int a = 0; a < 16; a++) sm[swz(base + a)] = csub(shoup_lazy(v[a], 1, one_s, p), p);
    }
    __syncthreads();
}

template <bool SHFL = false>
__device__ __forceinline__ void ntt_inv_smem(uint64_t* sm, const ulonglong2* __restrict__ w, uint64_t p,
                                             uint64_t ninv, uint64_t ninv_s, int t = threadIdx.x) {
    uint64_t v[16];
    __syncthreads();
    {   // phase C pattern first (distances 1 .. 8)
        const int base = 16 * t;
#pragma unroll
        for (int a = 0; a < 16; a++) v[a] = sm[swz(base + a)];
        gs_phase<1, false>(v, base, w, p, ninv, ninv_s);
        if (SHFL) {
            transpose16_shfl64(v, t & 15);
        } else {
#pragma unroll
            for (int a = 0; a < 16; a++) sm[swz(base + a)] = v[a];
        }
    }
    if (!SHFL) __syncwarp();
    {   // distances 16 .. 128
        const int base = 256 * (t >> 4) + (t & 15);
        if (!SHFL) {
#pragma unroll
            for (int a = 0; a < 16; a++) v[a] = sm[swz(base + 16 * a)];
        }
        gs_phase<16, false>(v, base, w, p, ninv, ninv_s);
#pragma unroll
        for (int a = 0; a < 16; a++) sm[swz(base + 16 * a)] = v[a];
    }
    __syncthreads();
    {   // distances 256 .. 2048, the last stage times N^-1: fully reduced
        const int base = t;
#pragma unroll
        for (int a = 0; a < 16; a++) v[a] = sm[swz(base + 256 * a)];
        gs_phase<256, true>(v, base, w, p, ninv, ninv_s);
#pragma unroll
        for (int a = 0; a < 16; a++) sm[swz(base + 256 * a)] = v[a];
    }
    __syncthreads();
}

template <bool SHFL = false>
__device__ __forceinline__ void ntt_fwd_mod(uint64_t* a, const uint64_t* tw, int i) {
    ntt_fwd_smem<SHFL>(a, tw_fwd(tw, i), c_mod[i], c_one_s[i]);
}
template <bool SHFL = false>
__device__ __forceinline__ void ntt_inv_mod(uint64_t* a, const uint64_t* tw, int i) {
    ntt_inv_smem<SHFL>(a, tw_inv(tw, i), c_mod[i], c_ninv[i], c_ninv_s[i]);
}
// Out-of-line versions for kernels that run several NTTs among other work:
// each call then gets its own register allocation.
static __device__ __noinline__ void ntt_fwd_call(uint64_t* a, const uint64_t* tw, int i) {
    ntt_fwd_mod(a, tw, i);
}
static __device__ __noinline__ void ntt_inv_call(uint64_t* a, const uint64_t* tw, int i) {
    ntt_inv_mod(a, tw, i);
}

// ---------------------------------------------------------------- NTT over the search basis (32-bit words)
//
// The same transform, schedule and twiddle order as above on residues mod
// r < 2^30 held in 32-bit words.  Butterflies keep values below 4r < 2^32
// (Harvey): forward, U is brought below 2r before U + V and U - V + 2r with
// V = x w mod r in [0, 2r); inverse, U + V is brought below 2r and
// (U - V + 2r) w lands in [0, 2r).  Forward input < 4r, output fully reduced
// in bit-reversed order; inverse input < 2r, output natural order times N^-1,
// fully reduced.
//
// Swizzle for 4-byte words: coefficient x at word swz32(x) = x ^ ((x >> 4) & 15)
// ^ (((x >> 8) & 1) << 4).  In every access pattern used (t + 256 a, the three
// phases) each half-warp's 16 words fall in 16 distinct banks and the two
// halves in opposite halves of the 32 banks: one wavefront per access.
__device__ __forceinline__ int swz32(int x) { return x ^ ((x >> 4) & 15) ^ (((x >> 8) & 1) << 4); }

template <int STRIDE>
__device__ __forceinline__ void ct_phase32(uint32_t v[16], int base, const uint2* __restrict__ w, uint32_t r) {
    const uint32_t two_r = 2 * r;
#pragma unroll
    for (int h = 8; h >= 1; h >>= 1) {
        const int t = STRIDE * h;
        const int m = N / (2 * t);
        const int i0 = base / (2 * t);
#pragma unroll
        for (int j = 0; j < 8 / h; j++) {
            const uint2 W = __ldg(w + m + i0 + j);
#pragma unroll
            for (int q = 0; q < h; q++) {
                const int a = 2 * h * j + q;
                const uint32_t U = csub32(v[a], two_r);
                const uint32_t V = shoup32(v[a + h], W.x, W.y, r);
                v[a] = U + V;
                v[a + h] = U - V + two_r;
            }
        }
    }
}

template <int STRIDE, bool LAST>
__device__ __forceinline__ void gs_phase32(uint32_t v[16], int base, const uint2* __restrict__ w, uint32_t r,
                                           uint32_t ninv, uint32_t ninv_s) {
    const uint32_t two_r = 2 * r;
#pragma unroll
    for (int h = 1; h <= 8; h <<= 1) {
        const int t = STRIDE * h;
        const int m = N / (2 * t);
        const int i0 = base / (2 * t);
#pragma unroll
        for (int j = 0; j < 8 / h; j++) {
            const uint2 W = __ldg(LAST && h == 8 ? w : w + m + i0 + j);
#pragma unroll
            for (int q = 0; q < h; q++) {
                const int a = 2 * h * j + q;
                const uint32_t U = v[a], V = v[a + h];
                if (LAST && h == 8) {
                    v[a] = csub32(shoup32(U + V, ninv, ninv_s, r), r);
                    v[a + h] = csub32(shoup32(U - V + two_r, W.x, W.y, r), r);
                } else {
                    v[a] = csub32(U + V, two_r);
                    v[a + h] = shoup32(U - V + two_r, W.x, W.y, r);
                }
            }
        }
    }
}

// t: the calling thread's index among the NTT_THREADS threads that run the
// transform (a CTA may run several transforms side by side, one per group of
// NTT_THREADS threads; every group takes the same path through the barriers).
__device__ __forceinline__ void ntt32_fwd_smem(uint32_t* sm, const uint2* __restrict__ w, uint32_t r,
                                               int t = threadIdx.x) {
    uint32_t v[16];
    __syncthreads();
    {
        const int base = t;
#pragma unroll
        for (int a = 0; a < 16; a++) v[a] = sm[swz32(base + 256 * a)];
        ct_phase32<256>(v, base, w, r);
#pragma unroll
        for (int a = 0; a < 16; a++) sm[swz32(base + 256 * a)] = v[a];
    }
    __syncthreads();
    {
        const int base = 256 * (t >> 4) + (t & 15);
#pragma unroll
        for (int a = 0; a < 16; a++) v[a] = sm[swz32(base + 16 * a)];
        ct_phase32<16>(v, base, w, r);
#pragma unroll
        for (int a = 0; a < 16; a++) sm[swz32(base + 16 * a)] = v[a];
    }
    __syncwarp();
    {
        const int base = 16 * t;
#pragma unroll
        for (int a = 0; a < 16; a++) v[a] = sm[swz32(base + a)];
        ct_phase32<1>(v, base, w, r);
#pragma unroll
        for (int a = 0; a < 16; a++) sm[swz32(base + a)] = csub32(csub32(v[a], 2 * r), r);
    }
    __syncthreads();
}

__device__ __forceinline__ void ntt32_inv_smem(uint32_t* sm, const uint2* __restrict__ w, uint32_t r,
                                               uint32_t ninv, uint32_t ninv_s, int t = threadIdx.x) {
    uint32_t v[16];
    __syncthreads();
    {
        const int base = 16 * t;
#pragma unroll
        for (int a = 0; a < 16; a++) v[a] = sm[swz32(base + a)];
        gs_phase32<1, false>(v, base, w, r, ninv, ninv_s);
#pragma unroll
        for (int a = 0; a < 16; a++) sm[swz32(base + a)] = v[a];
    }
    __syncwarp();
    {
        const int base = 256 * (t >> 4) + (t & 15);
#pragma unroll
        for (int a = 0; a < 16; a++) v[a] = sm[swz32(base + 16 * a)];
        gs_phase32<16, false>(v, base, w, r, ninv, ninv_s);
#pragma unroll
        for (int a = 0; a < 16; a++) sm[swz32(base + 16 * a)] = v[a];
    }
    __syncthreads();
    {
        const int base = t;
#pragma unroll
        for (int a = 0; a < 16; a++) v[a] = sm[swz32(base + 256 * a)];
        gs_phase32<256, true>(v, base, w, r, ninv, ninv_s);
#pragma unroll
        for (int a = 0; a < 16; a++) sm[swz32(base + 256 * a)] = v[a];
    }
    __syncthreads();
}

// Transposes the 16 x 16 matrix held by the 16 lanes of each half-warp (lane
// i of the half-warp holds row i in v) so that lane i holds column i: four
// rounds of __shfl_xor_sync (distances 8, 4, 2, 1), each swapping the
// off-diagonal halves of the blocks of that size.  Every lane of the warp
// must call it.
__device__ __forceinline__ void transpose16_shfl(uint32_t v[16], int i) {
#pragma unroll
    for (int m = 8; m >= 1; m >>= 1) {
        const bool hi = (i & m) != 0;
#pragma unroll
        for (int a = 0; a < 16; a++) {
            if (a & m) continue;
            const uint32_t send = hi ? v[a] : v[a | m];
            const uint32_t recv = __shfl_xor_sync(0xffffffffu, send, m);
            if (hi) v[a] = recv;
            else v[a | m] = recv;
        }
    }
}

// The inverse transform with its first and last phases on registers: v holds
// the bit-reversed inputs at coefficients 16 t + a on entry and the outputs
// (natural order, times N^-1, fully reduced) at coefficients t + 256 a on
// exit, so the caller loads and stores them directly; sm (N words) carries
// only the middle phase.  Ends with no barrier after its last shared-memory
// read; a caller that reuses sm synchronises first.
// SHFL: the first exchange (a transpose within each half-warp: coefficients
// 16 t + a to 256 (t / 16) + (t % 16) + 16 a) goes through warp shuffles
// instead of shared memory.
template <bool SHFL = false>
__device__ __forceinline__ void ntt32_inv_regs(uint32_t v[16], uint32_t* sm, const uint2* __restrict__ w,
                                               uint32_t r, uint32_t ninv, uint32_t ninv_s, int t) {
    gs_phase32<1, false>(v, 16 * t, w, r, ninv, ninv_s);
    if (SHFL) {
        transpose16_shfl(v, t & 15);
    } else {
#pragma unroll
        for (int a = 0; a < 16; a++) sm[swz32(16 * t + a)] = v[a];
        __syncwarp();
    }
    {
        const int base = 256 * (t >> 4) + (t & 15);
        if (!SHFL) {
#pragma unroll
            for (int a = 0; a < 16; a++) v[a] = sm[swz32(base + 16 * a)];
        }
        gs_phase32<16, false>(v, base, w, r, ninv, ninv_s);
#pragma unroll
        for (int a = 0; a < 16; a++) sm[swz32(base + 16 * a)] = v[a];
    }
    __syncthreads();
#pragma unroll
    for (int a = 0; a < 16; a++) v[a] = sm[swz32(t + 256 * a)];
    gs_phase32<256, true>(v, t, w, r, ninv, ninv_s);
}

// The forward transform with its first phase on registers: v holds the
// inputs (below 2r) at coefficients t + 256 a on entry; the outputs
// (bit-reversed order, fully reduced) are in sm at swz32(k) on exit, after a
// CTA barrier.  The barrier before the first shared-memory store lets a
// caller still reading sm's previous contents (in other threads) finish.
__device__ __forceinline__ void ntt32_fwd_regs(uint32_t v[16], uint32_t* sm, const uint2* __restrict__ w,
                                               uint32_t r, int t) {
    ct_phase32<256>(v, t, w, r);
    __syncthreads();
#pragma unroll
    for (int a = 0; a < 16; a++) sm[swz32(t + 256 * a)] = v[a];
    __syncthreads();
    {
        const int base = 256 * (t >> 4) + (t & 15);
#pragma unroll
        for (int a = 0; a < 16; a++) v[a] = sm[swz32(base + 16 * a)];
        ct_phase32<16>(v, base, w, r);
#pragma unroll
        for (int a = 0; a < 16; a++) sm[swz32(base + 16 * a)] = v[a];
    }
    __syncwarp();
    {
        const int base = 16 * t;
#pragma unroll
        for (int a = 0; a < 16; a++) v[a] = sm[swz32(base + a)];
        ct_phase32<1>(v, base, w, r);
#pragma unroll
        for (int a = 0; a < 16; a++) sm[swz32(base + a)] = csub32(csub32(v[a], 2 * r), r);
    }
    __syncthreads();
}

__device__ __forceinline__ void ntt32_fwd_mod(uint32_t* a, const uint64_t* tw, int i, int t = threadIdx.x) {
    ntt32_fwd_smem(a, tw32_fwd(tw, i), c_smod[i], t);
}
__device__ __forceinline__ void ntt32_inv_mod(uint32_t* a, const uint64_t* tw, int i, int t = threadIdx.x) {
    ntt32_inv_smem(a, tw32_inv(tw, i), c_smod[i], c_sninv[i], c_sninv_s[i], t);
}

// ---------------------------------------------------------------- mbarrier + bulk async copy (TMA engine)
// Used by the streaming kernels: a producer lane issues cp.async.bulk copies
// global -> shared that complete on an mbarrier; consumers wait on it.  Every
// wait is bounded: after WAIT_NS of global time (or WAIT_LIMIT polls) the
// caller gives up and reports.
constexpr uint32_t WAIT_LIMIT = 1u << 24;

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Bounded wait for the phase of parity `parity`; false if it gave up, after
// limit_ns of global time or WAIT_LIMIT polls, whichever comes first.
constexpr uint64_t WAIT_NS = 2000000000ull;
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint64_t limit_ns = WAIT_NS) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = globaltimer_ns();
    for (uint32_t it = 0; it < WAIT_LIMIT; it++) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 15) == 15 && globaltimer_ns() - t0 > limit_ns) return false;
    }
    return false;
}
__device__ __forceinline__ uint64_t policy_evict_first() {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}
__device__ __forceinline__ uint64_t policy_evict_normal() {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_normal.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}
__device__ __forceinline__ uint64_t policy_evict_last() {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}
// Bulk copy of `bytes` (multiple of 16, both addresses 16-byte aligned) from
// global to this CTA's shared memory, completing on `bar`.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar,
                                         uint64_t policy) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint "
        "[%0], [%1], %2, [%3], %4;" ::"r"(smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar)), "l"(policy)
        : "memory");
}

// Prefetch of `bytes` (multiple of 16, 16-byte aligned) from global memory
// into L2, with no destination in shared memory and no completion to wait for.
__device__ __forceinline__ void bulk_prefetch_l2(const void* src, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}

// ---------------------------------------------------------------- base extension Q -> r_i
// x given by its residues (x1 mod q1, x2 mod q2), read as the centred integer
// in (-q/2, q/2] (App. A's symmetric representative), and reduced mod each
// prime r_i of the search basis, exactly.
struct Lifted {
    uint64_t x1;   // x1 in [0, q1)
    uint64_t h;    // Garner digit in [0, q2): x = x1 + q1 h in [0, q)
    bool neg;      // x > (q-1)/2, i.e. the centred value is x - q
};

__device__ __forceinline__ Lifted lift_q(uint64_t x1, uint64_t x2) {
    const uint64_t q2 = c_mod[1];
    uint64_t x1r = csub(x1, q2);  // q1 < 2 q2
    uint64_t h = shoup(sub_mod(x2, x1r, q2), Q1INV_Q2, Q1INV_Q2_S, q2);
    Lifted L;
    L.x1 = x1;
    L.h = h;
    L.neg = (h > HALFQ_HI) || (h == HALFQ_HI && x1 > HALFQ_LO);
    return L;
}

// A lift packed for reduction mod many r_i: {x1 low word, x1 high word,
// h mod 2^27, floor(h / 2^27) | neg << 31} (h < 2^54, so the top digit
// leaves bit 31 free).
__device__ __forceinline__ uint4 lift_pack(uint64_t x1, uint64_t x2) {
    const Lifted L = lift_q(x1, x2);
    return make_uint4((uint32_t)L.x1, (uint32_t)(L.x1 >> 32), (uint32_t)L.h & ((1u << 27) - 1),
                      (uint32_t)(L.h >> 27) | ((uint32_t)L.neg << 31));
}

// The centred lift mod r_i from its packed form: with h = hl + 2^27 hh,
//   x - [neg] q = x1 + hl [q1]_r + hh [q1 2^27]_r + [neg] [-q]_r  (mod r),
// a sum S below 2^59 (x1 < 2^54, each product below 2^57).  Barrett with
// mu = floor(2^59 / r): est = floor(floor(S / 2^27) mu / 2^32) is short of
// floor(S / r) by at most 2, so S - est r lies in [0, 3r) and is computed in
// 32 bits.
__device__ __forceinline__ uint32_t lift_mod_r(uint4 g, int i) {
    const uint32_t r = c_smod[i];
    uint64_t s = ((uint64_t)g.y << 32 | g.x) + ((g.w >> 31) ? c_lift_nq[i] : 0u);
    s += (uint64_t)g.z * c_q1_mod_r[i];
    s += (uint64_t)(g.w & ((1u << 27) - 1)) * c_lift_b[i];
    const uint32_t est = __umulhi((uint32_t)(s >> 27), c_mu59[i]);
    return csub32(csub32((uint32_t)s - est * r, 2 * r), r);
}

// ---------------------------------------------------------------- CRT over the search basis
//
// For residues x_i = X mod r_i of an integer X with X' = X + q 2^129 in
// [M/16, M/5] (every value this library reconstructs: the tensor sums,
// |X| < 2^236, and centred lifts, |X| < q/2), the CRT gives
//   X' = sum_i y_i M_i - alpha M,   y_i = [x'_i M_i^-1]_{r_i},  M_i = M / r_i,
// with alpha = floor(sum_i y_i / r_i) (as 0 <= X' < M).  That sum is alpha +
// X'/M with X'/M in [1/16, 1/5]; PHI_i = floor(2^60 / r_i) computes it short by
// less than 2^-27, so the floor of the fixed-point sum is alpha exactly.
__device__ __forceinline__ uint32_t crt_y(const uint32_t x[NUM_S], uint32_t y[NUM_S]) {
    uint64_t acc = 0;
#pragma unroll
    for (int i = 0; i < NUM_S; i++) {
        const uint32_t r = c_smod[i];
        const uint32_t v = shoup32(x[i], c_minv[i], c_minv_s[i], r) + c_hm[i];  // < 3r
        y[i] = csub32(csub32(v, 2 * r), r);
        acc += (uint64_t)y[i] * c_phi[i];
    }
    return (uint32_t)(acc >> 60);
}

// (sum_i y_i A_ij - alpha A_Mj + extra) mod q_j, with A_ij and A_Mj < q_j given as
// two 27-bit digits (cols [i][j][2], mcols [j][2]) and |extra| < 2^56: column
// sums of y (< 2^30) times a digit stay below 2^60.
__device__ __forceinline__ uint64_t crt_combine_q(const uint32_t y[NUM_S], uint32_t alpha, const uint32_t* cols,
                                                  const uint32_t* mcols, int j, int64_t extra) {
    uint64_t c0 = 0, c1 = 0;
#pragma unroll
    for (int i = 0; i < NUM_S; i++) {
        c0 += (uint64_t)y[i] * cols[(i * 2 + j) * 2];
        c1 += (uint64_t)y[i] * cols[(i * 2 + j) * 2 + 1];
    }
    const int64_t s0 = (int64_t)c0 - (int64_t)alpha * mcols[j * 2] + extra + (int64_t)(16 * c_mod[j]);
    const int64_t s1 = (int64_t)c1 - (int64_t)alpha * mcols[j * 2 + 1];
    // s0 > 0 (16 q_j > 2^58 covers the negative terms), s1 > -2^30
    const __int128 v = ((__int128)s1 << 27) + s0;  // in (0, 2^88)
    return reduce128((uint64_t)v, (uint64_t)(v >> 64), j);
}

}  // namespace hers
