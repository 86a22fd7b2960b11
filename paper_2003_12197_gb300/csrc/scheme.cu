// FV scheme kernels of the HERS library: key generation (App. A, Alg 1),
// SIMD encoding + encryption of gallery rows and probe dimensions (Sec. 3.2
// Eqs 2-3; Alg 2), extension of canonical ciphertexts to the resident NTT
// form over the search basis, and decryption + decoding of score ciphertexts (Alg 3).
#include <cooperative_groups.h>

#include "common.cuh"
#include "internal.h"

namespace hers {

__device__ __forceinline__ uint64_t shoup_companion(uint64_t w, uint64_t p) {
    return (uint64_t)(((unsigned __int128)w << 64) / p);
}

// ---------------------------------------------------------------- key generation
//
// Grid (2 limbs, 3 components): component 0 is pk, 1 and 2 are evk_1, evk_2.
// Each CTA works on one limb q_l of one component:
//   c0 = [-(a s + e) + g_j s^2]_{q_l},  c1 = a,
// with g_j = 1 mod q_j and 0 mod the other prime, so the s^2 term appears only
// in the limb l = j.  Products use the NTT mod q_l (exact ring arithmetic mod q_l).
__global__ void __launch_bounds__(NTT_THREADS, 2) k_keygen(const uint64_t* __restrict__ tw,
                                                        uint64_t seed, DevKeys K, int* err) {
    extern __shared__ uint64_t sm[];
    uint64_t* S = sm;
    uint64_t* A = sm + N;
    uint64_t* X = sm + 2 * N;
    const int limb = blockIdx.x, comp = blockIdx.y;
    const uint64_t p = c_mod[limb];

    sample_ternary_mod(seed, PRF_KG_SK, 0, p, S, err);
    __syncthreads();
    if (limb == 0 && comp == 0)
        for (int k = threadIdx.x; k < N; k += blockDim.x)
            K.sk[k] = S[swz(k)] == 0 ? 0 : (S[swz(k)] == 1 ? 1 : -1);
    ntt_fwd_call(S, tw, limb);
    if (comp == 0)
        for (int k = threadIdx.x; k < N; k += blockDim.x) {
            K.s_ntt[(limb * 2 + 0) * N + k] = S[swz(k)];
            K.s_ntt[(limb * 2 + 1) * N + k] = shoup_companion(S[swz(k)], p);
        }

    const uint32_t pa = comp == 0 ? PRF_KG_PK_A : PRF_KG_EVK_A;
    const uint64_t oa = comp == 0 ? (uint64_t)limb : (uint64_t)(2 * (comp - 1) + limb);
    sample_uniform(seed, pa, oa, p, A, err);
    __syncthreads();
    // canonical output: [2 polys][2 limbs][N] for pk, [j][2][2][N] for evk_j
    uint64_t* outc = comp == 0 ? K.pk : K.evk + (size_t)(comp - 1) * 4 * N;
    for (int k = threadIdx.x; k < N; k += blockDim.x) outc[(2 + limb) * N + k] = A[swz(k)];
    ntt_fwd_call(A, tw, limb);
    const bool gadget = comp >= 1 && (comp - 1) == limb;
    for (int k = threadIdx.x; k < N; k += blockDim.x) {
        const int x = swz(k);
        A[x] = mul_mod(A[x], S[x], limb);
        if (gadget) X[x] = mul_mod(S[x], S[x], limb);
    }
    ntt_inv_call(A, tw, limb);
    if (gadget) ntt_inv_call(X, tw, limb);  // uniform per CTA

    // e from its stream; 8 coefficients per ChaCha block
    const uint32_t pe = comp == 0 ? PRF_KG_PK_E : PRF_KG_EVK_E;
    const uint64_t oe = comp == 0 ? 0 : (uint64_t)(comp - 1);
    for (int c = threadIdx.x; c < N / 8; c += blockDim.x) {
        uint32_t blk[16];
        chacha20(seed, pe, oe, (uint32_t)c, blk);
#pragma unroll
        for (int j = 0; j < 8; j++) {
            const int k = 8 * c + j;
            const int e = chi_from_word(((uint64_t)blk[2 * j + 1] << 32) | blk[2 * j]);
            uint64_t v = add_mod(A[swz(k)], e < 0 ? p - (uint64_t)(-e) : (uint64_t)e, p);
            v = v == 0 ? 0 : p - v;  // -(a s + e)
            if (gadget) v = add_mod(v, X[swz(k)], p);
            outc[limb * N + k] = v;
        }
    }
}

// Forward NTT of canonical key polynomials, stored with Shoup companions.
// Poly index P of a [..][2 limbs][N] array has limb P % 2; out is [..][2][N].
__global__ void __launch_bounds__(NTT_THREADS) k_key_ntt(const uint64_t* __restrict__ tw,
                                                         const uint64_t* __restrict__ in,
                                                         uint64_t* __restrict__ out) {
    extern __shared__ uint64_t sm[];
    const int P = blockIdx.x, limb = P & 1;
    const uint64_t p = c_mod[limb];
    for (int k = threadIdx.x; k < N; k += blockDim.x) sm[swz(k)] = in[(size_t)P * N + k];
    ntt_fwd_call(sm, tw, limb);
    for (int k = threadIdx.x; k < N; k += blockDim.x) {
        out[((size_t)P * 2 + 0) * N + k] = sm[swz(k)];
        out[((size_t)P * 2 + 1) * N + k] = shoup_companion(sm[swz(k)], p);
    }
}

cudaError_t launch_keygen(const uint64_t* tw, uint64_t seed, DevKeys k, int* err, cudaStream_t st) {
    const int smem = 3 * N * 8;
    cudaError_t e = cudaFuncSetAttribute(k_keygen, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    k_keygen<<<dim3(2, 3), NTT_THREADS, smem, st>>>(tw, seed, k, err);
    count_launches(1);
    e = cudaGetLastError();
    return e != cudaSuccess ? e : launch_key_ntt(tw, k, st);
}

cudaError_t launch_key_ntt(const uint64_t* tw, const DevKeys& k, cudaStream_t st) {
    k_key_ntt<<<4, NTT_THREADS, N * 8, st>>>(tw, k.pk, k.pk_ntt);
    k_key_ntt<<<8, NTT_THREADS, N * 8, st>>>(tw, k.evk, k.evk_ntt);
    count_launches(2);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- base-w evaluation keys
//
// Grid (2 limbs, ndig digits).  CTA (l, j) writes limb l of
//   evkw_j = ([-(a_j s + e_j) + w^j s^2]_q, a_j),  w = 2^logw,
// with a_j uniform mod q_l from the stream (seed, 0x06, 2 j + l) and e_j
// from (seed, 0x07, j); s from the keys' NTT form.  Products in the NTT
// domain mod q_l; w^j mod q_l by repeated doubling.
uint32_t basew_digits(uint32_t logw) {
    // bits(q1 q2) = 108
    return (108 + logw - 1) / logw;
}

__global__ void __launch_bounds__(NTT_THREADS, 2) k_keygen_w(const uint64_t* __restrict__ tw, uint64_t seed,
                                                          uint32_t logw, DevKeys K, uint64_t* __restrict__ evkw,
                                                          int* err) {
    extern __shared__ uint64_t sm[];
    uint64_t* A = sm;
    uint64_t* X = sm + N;
    const int limb = blockIdx.x;
    const uint32_t j = blockIdx.y;
    const uint64_t p = c_mod[limb];
    const uint64_t* s = K.s_ntt + (size_t)limb * 2 * N;  // NTT(s) mod q_l, then companions

    sample_uniform(seed, PRF_KG_EVKW_A, (uint64_t)(2 * j + limb), p, A, err);
    __syncthreads();
    uint64_t* out = evkw + (size_t)j * 4 * N;
    for (int k = threadIdx.x; k < N; k += blockDim.x) out[(2 + limb) * N + k] = A[swz(k)];
    ntt_fwd_call(A, tw, limb);
    for (int k = threadIdx.x; k < N; k += blockDim.x) {
        const int x = swz(k);
        A[x] = mul_mod(A[x], s[k], limb);
        X[x] = mul_mod(s[k], s[k], limb);
    }
    ntt_inv_call(A, tw, limb);
    ntt_inv_call(X, tw, limb);
    uint64_t g = 1;  // w^j mod q_l
    for (uint32_t i = 0; i < logw * j; i++) g = add_mod(g, g, p);
    for (int c = threadIdx.x; c < N / 8; c += blockDim.x) {
        uint32_t blk[16];
        chacha20(seed, PRF_KG_EVKW_E, (uint64_t)j, (uint32_t)c, blk);
#pragma unroll
        for (int i = 0; i < 8; i++) {
            const int k = 8 * c + i;
            const int e = chi_from_word(((uint64_t)blk[2 * i + 1] << 32) | blk[2 * i]);
            uint64_t v = add_mod(A[swz(k)], e < 0 ? p - (uint64_t)(-e) : (uint64_t)e, p);
            v = v == 0 ? 0 : p - v;  // -(a s + e)
            out[limb * N + k] = add_mod(v, mul_mod(g, X[swz(k)], limb), p);
        }
    }
}

cudaError_t launch_keygen_w(const uint64_t* tw, uint64_t seed, uint32_t logw, uint32_t ndig, const DevKeys& k,
                            uint64_t* evkw, uint64_t* evkw_ntt, int* err, cudaStream_t st) {
    const int smem = 2 * N * 8;
    cudaError_t e = cudaFuncSetAttribute(k_keygen_w, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    k_keygen_w<<<dim3(2, ndig), NTT_THREADS, smem, st>>>(tw, seed, logw, k, evkw, err);
    k_key_ntt<<<4 * ndig, NTT_THREADS, N * 8, st>>>(tw, evkw, evkw_ntt);
    count_launches(2);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- encryption
//
// Grid (nct, 2 limbs).  CTA (c, l) writes limb l of ciphertext ct_begin + c:
//   ct0 = [Delta m + pk0 u + e1]_q,  ct1 = [pk1 u + e2]_q   (Alg 2)
// The plaintext m is computed in the CTA:
//   probe (Eq. 2): dimension i in every slot, i.e. the constant polynomial q[i];
//   gallery (Eq. 3): ct c = b d + i has slot j = feats[b N + j][i] (0 past m);
//     slot j is the evaluation at psi_t^(2j+1), which the forward NTT mod t
//     puts at index brev(j), so m = INTT_t of the slots placed at brev(j).
//   zero (mode ENC_ZERO): m = 0, an encryption of zero for output
//     re-randomisation (Alg 7's Encrypt(0)); ciphertext c is block c;
//   slot (mode ENC_SLOT, Alg 6): ciphertext c is dimension c of one entry at
//     global slot m = b N + v: slot v holds feats[c], every other slot 0.
// Randomness: u, e1, e2 are the streams (seed, base + 0/1/2, obj) with
// obj = b d + i (gallery), i (probe) or the block (zero).
__global__ void __launch_bounds__(NTT_THREADS, 2) k_encrypt(const uint64_t* __restrict__ tw,
                                                         const uint64_t* __restrict__ pk_ntt,
                                                         const int8_t* __restrict__ feats,
                                                         uint64_t m, uint32_t d, uint64_t ct_begin,
                                                         int mode, uint64_t seed, int pm,
                                                         uint64_t* __restrict__ out, int* err) {
    const PlainMod& P = c_plain[pm];
    extern __shared__ uint64_t sm[];
    uint64_t* U = sm;
    uint64_t* B = sm + N;
    uint64_t* M = sm + 2 * N;
    const uint64_t c = ct_begin + blockIdx.x;
    const int limb = blockIdx.y;
    const uint64_t p = c_mod[limb];
    const uint32_t base = mode == ENC_PROBE  ? PRF_PROBE
                          : mode == ENC_ZERO ? PRF_RERAND
                          : mode == ENC_SLOT ? PRF_ENROLL
                                             : PRF_GALLERY;
    // gallery: b d + i; probe: i; zero: block; slot: (b N + v) d + i
    const uint64_t obj = mode == ENC_SLOT ? m * d + c : c;

    // plaintext
    if (mode == ENC_ZERO) {
        for (int k = threadIdx.x; k < N; k += blockDim.x) M[swz(k)] = 0;
    } else if (mode == ENC_SLOT) {
        const int v = feats[c];
        const uint32_t slot = (uint32_t)(m % N);
        for (int s = threadIdx.x; s < N; s += blockDim.x)
            M[swz(brev12(s))] = s == (int)slot ? (v < 0 ? P.t - (uint64_t)(-v) : (uint64_t)v) : 0;
        ntt_inv_call(M, tw, P.mod);
    } else if (mode == ENC_PROBE) {
        const int v = feats[c];
        const uint64_t mv = v < 0 ? P.t - (uint64_t)(-v) : (uint64_t)v;
        for (int k = threadIdx.x; k < N; k += blockDim.x) M[swz(k)] = k == 0 ? mv : 0;
    } else {
        const uint64_t b = c / d, i = c % d;
        for (int s = threadIdx.x; s < N; s += blockDim.x) {
            const uint64_t e = b * N + (uint64_t)s;
            const int v = e < m ? feats[e * d + i] : 0;
            M[swz(brev12(s))] = v < 0 ? P.t - (uint64_t)(-v) : (uint64_t)v;
        }
        ntt_inv_call(M, tw, P.mod);
    }

    // u, NTT, products with the public key
    sample_ternary_mod(seed, base + 0, obj, p, U, err);
    ntt_fwd_call(U, tw, limb);
    const uint64_t* pk0 = pk_ntt + (size_t)((0 * 2 + limb) * 2) * N;
    const uint64_t* pk1 = pk_ntt + (size_t)((1 * 2 + limb) * 2) * N;
    for (int k = threadIdx.x; k < N; k += blockDim.x) {
        const int x = swz(k);
        const uint64_t u = U[x];
        B[x] = shoup(u, pk1[k], pk1[N + k], p);
        U[x] = shoup(u, pk0[k], pk0[N + k], p);
    }
    ntt_inv_call(U, tw, limb);
    ntt_inv_call(B, tw, limb);

    // add Delta m + e1 and e2, write the canonical ciphertext limb
    uint64_t* o0 = out + ((size_t)blockIdx.x * 4 + 0 * 2 + limb) * N;
    uint64_t* o1 = out + ((size_t)blockIdx.x * 4 + 1 * 2 + limb) * N;
    for (int cb = threadIdx.x; cb < N / 8; cb += blockDim.x) {
        uint32_t blk[16];
        chacha20(seed, base + 1, obj, (uint32_t)cb, blk);
#pragma unroll
        for (int j = 0; j < 8; j++) {
            const int k = 8 * cb + j;
            const int e1 = chi_from_word(((uint64_t)blk[2 * j + 1] << 32) | blk[2 * j]);
            const int x = swz(k);
            uint64_t v0 = add_mod(U[x], shoup(M[x], P.delta[limb], P.delta_s[limb], p), p);
            o0[k] = e1 < 0 ? sub_mod(v0, (uint64_t)(-e1), p) : add_mod(v0, (uint64_t)e1, p);
        }
        chacha20(seed, base + 2, obj, (uint32_t)cb, blk);
#pragma unroll
        for (int j = 0; j < 8; j++) {
            const int k = 8 * cb + j;
            const int e2 = chi_from_word(((uint64_t)blk[2 * j + 1] << 32) | blk[2 * j]);
            const uint64_t x1 = B[swz(k)];
            o1[k] = e2 < 0 ? sub_mod(x1, (uint64_t)(-e2), p) : add_mod(x1, (uint64_t)e2, p);
        }
    }
}

cudaError_t launch_encrypt(const uint64_t* tw, const DevKeys& k, const int8_t* feats, uint64_t m,
                           uint32_t d, uint64_t ct_begin, uint64_t nct, int mode, uint64_t seed,
                           uint64_t* out_ct, int* err, cudaStream_t st) {
    const int smem = 3 * N * 8;
    cudaError_t e = cudaFuncSetAttribute(k_encrypt, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    const uint64_t chunk = 1u << 30;  // grid.x limit is 2^31 - 1
    for (uint64_t off = 0; off < nct; off += chunk) {
        const uint64_t n = nct - off < chunk ? nct - off : chunk;
        k_encrypt<<<dim3((unsigned)n, 2), NTT_THREADS, smem, st>>>(
            tw, k.pk_ntt, feats, m, d, ct_begin + off, mode, seed, k.pm, out_ct + off * 4 * N, err);
        count_launches(1);
    }
    return cudaGetLastError();
}

// out[c] = out[c] + add[c] (mod q_l, per polynomial and limb) for nct
// canonical ciphertexts: homomorphic addition (App. A), used to add Enc(0).
__global__ void __launch_bounds__(256) k_ct_add(uint64_t* __restrict__ out, const uint64_t* __restrict__ add) {
    const uint64_t c = blockIdx.y;
    const int row = blockIdx.z;  // poly * 2 + limb
    const int k = blockIdx.x * 256 + threadIdx.x;
    const uint64_t q = c_mod[row & 1];
    const size_t at = (c * 4 + row) * N + k;
    out[at] = add_mod(out[at], add[at], q);
}

cudaError_t launch_ct_add(uint64_t* out, const uint64_t* add, uint64_t nct, cudaStream_t st) {
    for (uint64_t off = 0; off < nct; off += 65535) {
        const uint64_t n = nct - off < 65535 ? nct - off : 65535;
        k_ct_add<<<dim3(N / 256, (unsigned)n, 4), 256, 0, st>>>(out + off * 4 * N, add + off * 4 * N);
        count_launches(1);
    }
    return cudaGetLastError();
}

// One CTA per polynomial P = 2 i + poly of block b = b0 + blockIdx.y: reads
// its eight limbs from the resident form (centred values, NTT domain over the
// search basis), undoes the NTTs (R2C_GROUPS groups of NTT_THREADS threads,
// each for NUM_S / R2C_GROUPS limbs), recovers the canonical residues mod q1,
// q2 by the CRT of the search basis (the resident value is the centred lift x,
// |x| < q/2, so x' = x + q 2^129 is in range and x' = x mod q), adds
// add[i][poly][l] (when add is non-null) and writes out[i][poly][l]; add and
// out advance by d ciphertexts per block.
constexpr int R2C_GROUPS = 4;
constexpr int R2C_SMEM = NUM_S * N * 4;
__global__ void __launch_bounds__(NTT_THREADS * R2C_GROUPS, 1) k_resident_to_canonical_add(
    const uint64_t* __restrict__ tw, const uint64_t* __restrict__ resident, uint64_t b0, uint32_t d,
    const uint64_t* __restrict__ add, uint64_t* __restrict__ out) {
    extern __shared__ uint32_t sm32[];
    const uint64_t b = b0 + blockIdx.y;
    const uint32_t i = blockIdx.x >> 1;
    const int poly = (int)(blockIdx.x & 1);
    const int32_t* res = (const int32_t*)resident;
    const int grp = threadIdx.x / NTT_THREADS, t = threadIdx.x % NTT_THREADS;
    for (int lg = 0; lg < NUM_S / R2C_GROUPS; lg++) {
        const int l = grp * (NUM_S / R2C_GROUPS) + lg;
        uint32_t* s = sm32 + l * N;
        const uint32_t r = c_smod[l];
        for (int k = t; k < N; k += NTT_THREADS) s[swz32(k)] = uncentre32(res[resident_offset(b, l, k, d, i, poly)], r);
        ntt32_inv_mod(s, tw, l, t);
    }
    const size_t row = ((size_t)blockIdx.y * d * 4 + ((size_t)i * 2 + poly) * 2) * N;
    for (int k = threadIdx.x; k < N; k += blockDim.x) {
        uint32_t x[NUM_S], y[NUM_S];
#pragma unroll
        for (int l = 0; l < NUM_S; l++) x[l] = sm32[l * N + swz32(k)];
        const uint32_t alpha = crt_y(x, y);
#pragma unroll
        for (int j = 0; j < 2; j++) {
            const uint64_t v = crt_combine_q(y, alpha, c_mi_q_cols, c_m_q_cols, j, 0);
            out[row + j * N + k] = add ? add_mod(v, add[row + j * N + k], c_mod[j]) : v;
        }
    }
}

cudaError_t launch_resident_to_canonical_add(const uint64_t* tw, const uint64_t* resident, uint64_t b,
                                             uint32_t d, const uint64_t* add, uint64_t* out, cudaStream_t st,
                                             uint32_t nb) {
    cudaError_t e = cudaFuncSetAttribute(k_resident_to_canonical_add, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         R2C_SMEM);
    if (e != cudaSuccess) return e;
    k_resident_to_canonical_add<<<dim3(2 * d, nb), NTT_THREADS * R2C_GROUPS, R2C_SMEM, st>>>(tw, resident, b, d,
                                                                                            add, out);
    count_launches(1);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- extension to the search form
//
// Takes each coefficient of a canonical ciphertext polynomial P (residues mod
// q1, q2) to its centred representative x in (-q/2, q/2] (App. A), reduces it
// mod the primes of the search basis, and writes NTT_{r_l}(x mod r_l), as
// centred int32, at the resident (tiled) position of ciphertext
// ct_begin + P/2 = b d + i.  Exactness of the later tensor product needs the
// centred lift: the product of two such polynomials over Z, summed over
// d <= 512 dimensions, stays below 2^236 < M / 2^4.
//
// A CTA covers all NUM_S primes of one polynomial.  It lifts every
// coefficient once, into shared memory in the packed form of lift_pack (16
// bytes per coefficient); then EXT_GROUPS groups of NTT_THREADS threads run
// NUM_S / EXT_GROUPS transforms each.  A thread reduces its 16 first-phase
// coefficients (t + 256 a) mod r_l straight into registers, the other two
// phases pass through the group's own N words of shared memory, and the
// outputs go from there to the resident form: coefficient t + 256 a lies in
// tile a at position t, so a thread's 16 outputs of one prime are one base
// address and a fixed stride apart.  96 KiB of shared memory and 64
// registers give two CTAs per SM.
constexpr int EXT_GROUPS = 2;
constexpr int EXT_THREADS = NTT_THREADS * EXT_GROUPS;
constexpr int EXT_SMEM = N * 16 + EXT_GROUPS * N * 4;
__global__ void __launch_bounds__(EXT_THREADS, 2) k_extend_ntt(const uint64_t* __restrict__ tw,
                                                              const uint64_t* __restrict__ ct, uint64_t ct_begin,
                                                              uint32_t d, uint64_t* __restrict__ out) {
    extern __shared__ uint4 smx[];  // [N] packed lifts, then [EXT_GROUPS][N] transform words
    const uint64_t P = blockIdx.x;
    {
        const uint64_t* x1 = ct + (P * 2 + 0) * N;
        const uint64_t* x2 = ct + (P * 2 + 1) * N;
        uint64_t a[N / EXT_THREADS], b[N / EXT_THREADS];
#pragma unroll
        for (int j = 0; j < N / EXT_THREADS; j++) {
            a[j] = x1[threadIdx.x + j * EXT_THREADS];
            b[j] = x2[threadIdx.x + j * EXT_THREADS];
        }
#pragma unroll
        for (int j = 0; j < N / EXT_THREADS; j++) smx[threadIdx.x + j * EXT_THREADS] = lift_pack(a[j], b[j]);
    }
    __syncthreads();
    const uint64_t c = ct_begin + P / 2;
    const uint64_t blk = c / d;
    const uint32_t i = (uint32_t)(c % d);
    const int poly = (int)(P & 1);
    const int grp = threadIdx.x / NTT_THREADS, t = threadIdx.x % NTT_THREADS;
    uint32_t* buf = (uint32_t*)(smx + N) + grp * N;
    const uint64_t tile_stride = (uint64_t)d * TILE * 2;  // int32 words from tile a to a + 1
#pragma unroll 1
    for (int lg = 0; lg < NUM_S / EXT_GROUPS; lg++) {
        const int l = lg * EXT_GROUPS + grp;
        const uint32_t r = c_smod[l];
        uint32_t v[16];
#pragma unroll
        for (int a = 0; a < 16; a++) v[a] = lift_mod_r(smx[t + 256 * a], l);
        ntt32_fwd_regs(v, buf, tw32_fwd(tw, l), r, t);  // ends with a CTA barrier
        int32_t* o = (int32_t*)out + resident_offset(blk, l, t, d, i, poly);
#pragma unroll
        for (int a = 0; a < 16; a++) o[a * tile_stride] = centre32(buf[swz32(t + 256 * a)], r);
    }
}

// The same extension for a few polynomials (a probe, an enrollment), where
// one CTA per polynomial leaves most SMs idle and each CTA runs its eight
// transforms at the pace of its own latency.  A cluster of NUM_S CTAs takes
// one polynomial, CTA rank l the transform mod r_l.  Rank l lifts
// coefficients [l N/NUM_S, (l+1) N/NUM_S) into its own shared memory; after a
// cluster barrier each CTA reads the packed lifts of its 16 first-phase
// coefficients from their owners' shared memory (distributed shared memory),
// so every coefficient is still lifted once.  A CTA arrives on a second
// cluster barrier when its remote reads are done and waits on it before it
// exits, so no CTA's shared memory goes away while a peer reads it.
constexpr int EXTC_SLICE = N / NUM_S;  // coefficients lifted per CTA
static_assert(EXTC_SLICE == 2 * NTT_THREADS, "two lifts per thread; owner of t + 256 a is a / 2");
__global__ void __cluster_dims__(NUM_S, 1, 1) __launch_bounds__(NTT_THREADS, 4)
    k_extend_ntt_cluster(const uint64_t* __restrict__ tw, const uint64_t* __restrict__ ct, uint64_t ct_begin,
                         uint32_t d, uint64_t* __restrict__ out) {
    namespace cg = cooperative_groups;
    __shared__ uint4 lifts[EXTC_SLICE];
    __shared__ uint32_t buf[N];
    const cg::cluster_group cluster = cg::this_cluster();
    const int l = (int)cluster.block_rank();
    const uint64_t P = blockIdx.x / NUM_S;
    const int t = threadIdx.x;
    {
        const uint64_t* x1 = ct + (P * 2 + 0) * N + l * EXTC_SLICE;
        const uint64_t* x2 = ct + (P * 2 + 1) * N + l * EXTC_SLICE;
        const uint64_t a0 = x1[t], b0 = x2[t], a1 = x1[t + NTT_THREADS], b1 = x2[t + NTT_THREADS];
        lifts[t] = lift_pack(a0, b0);
        lifts[t + NTT_THREADS] = lift_pack(a1, b1);
    }
    cluster.sync();
    const uint32_t r = c_smod[l];
    uint32_t v[16];
#pragma unroll
    for (int a = 0; a < 16; a++)  // coefficient t + 256 a: rank a / 2, slot t + 256 (a % 2)
        v[a] = lift_mod_r(*cluster.map_shared_rank(lifts + t + NTT_THREADS * (a & 1), a >> 1), l);
    cluster.barrier_arrive();
    ntt32_fwd_regs(v, buf, tw32_fwd(tw, l), r, t);
    const uint64_t c = ct_begin + P / 2;
    const uint64_t blk = c / d;
    const uint32_t i = (uint32_t)(c % d);
    const uint64_t tile_stride = (uint64_t)d * TILE * 2;
    int32_t* o = (int32_t*)out + resident_offset(blk, l, t, d, i, (int)(P & 1));
#pragma unroll
    for (int a = 0; a < 16; a++) o[a * tile_stride] = centre32(buf[swz32(t + 256 * a)], r);
    cluster.barrier_wait();
}

// By default up to EXT_CLUSTER_MAX_POLYS polynomials per call take the cluster
// form: probes of d <= 32.  Measured (probe preparation in a CUDA graph,
// cluster form against one CTA per polynomial): d = 16, 14.2 against 27.3 us;
// d = 32, 23.2 against 27.6 us; d = 48, equal; d = 64, 38.9 against 28.3 us,
// as 8 CTAs per polynomial no longer fit one wave.  A context's probe
// preparation uses its own threshold (hers_autotune_extension).
cudaError_t launch_extend_ntt(const uint64_t* tw, const uint64_t* ct, uint64_t nct, uint64_t ct_begin,
                              uint32_t d, uint64_t* out, cudaStream_t st, uint64_t cluster_max_polys) {
    if (2 * nct <= cluster_max_polys) {
        k_extend_ntt_cluster<<<(unsigned)(2 * nct * NUM_S), NTT_THREADS, 0, st>>>(tw, ct, ct_begin, d, out);
        count_launches(1);
        return cudaGetLastError();
    }
    cudaError_t e = cudaFuncSetAttribute(k_extend_ntt, cudaFuncAttributeMaxDynamicSharedMemorySize, EXT_SMEM);
    if (e != cudaSuccess) return e;
    const uint64_t chunk = 1u << 30;  // polynomials per launch
    for (uint64_t off = 0; off < 2 * nct; off += chunk) {
        const uint64_t n = 2 * nct - off < chunk ? 2 * nct - off : chunk;
        k_extend_ntt<<<(unsigned)n, EXT_THREADS, EXT_SMEM, st>>>(tw, ct + off * 2 * N, ct_begin + off / 2, d, out);
        count_launches(1);
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------- decryption + decoding
//
// One CTA per block b.  v = [c0 + c1 s]_q per limb (NTT product with s);
// pt = round(t v / q) mod t computed exactly as pt = [-r q^-1]_t with
// r = [t v]_q centred (t v = q pt' + r, |r| < q/2, so pt' = (t v - r)/q);
// slots = NTT_t(pt), slot j at index brev(j), centred mod t.
__global__ void __launch_bounds__(NTT_THREADS, 2) k_decrypt(const uint64_t* __restrict__ tw,
                                                         const uint64_t* __restrict__ s_ntt,
                                                         const uint64_t* __restrict__ cts,
                                                         int32_t* __restrict__ scores, uint64_t m, int pm) {
    extern __shared__ uint64_t sm[];
    const PlainMod& P = c_plain[pm];
    const uint64_t t = P.t;
    uint64_t* V0 = sm;
    uint64_t* V1 = sm + N;
    uint64_t* PT = sm + 2 * N;
    const uint64_t b = blockIdx.x;
    const uint64_t* ct = cts + b * 4 * N;
    for (int l = 0; l < 2; l++) {
        uint64_t* V = l ? V1 : V0;
        const uint64_t p = c_mod[l];
        for (int k = threadIdx.x; k < N; k += blockDim.x) V[swz(k)] = ct[(2 + l) * N + k];
        ntt_fwd_call(V, tw, l);
        const uint64_t* s = s_ntt + (size_t)l * 2 * N;
        for (int k = threadIdx.x; k < N; k += blockDim.x) V[swz(k)] = shoup(V[swz(k)], s[k], s[N + k], p);
        ntt_inv_call(V, tw, l);
        for (int k = threadIdx.x; k < N; k += blockDim.x) V[swz(k)] = add_mod(V[swz(k)], ct[l * N + k], p);
    }
    __syncthreads();
    for (int k = threadIdx.x; k < N; k += blockDim.x) {
        const uint64_t a1 = shoup(V0[swz(k)], P.t_mod[0], P.t_s[0], c_mod[0]);
        const uint64_t a2 = shoup(V1[swz(k)], P.t_mod[1], P.t_s[1], c_mod[1]);
        const Lifted L = lift_q(a1, a2);
        uint64_t r = (a1 % t + mul_mod_t(P.q1_mod_t, L.h % t, t)) % t;
        if (L.neg) r = (r + t - P.q_mod_t) % t;
        PT[swz(k)] = mul_mod_t((t - r) % t, P.qinv_t, t);
    }
    ntt_fwd_call(PT, tw, P.mod);
    for (int j = threadIdx.x; j < N; j += blockDim.x) {
        const uint64_t e = b * N + (uint64_t)brev12(j);
        if (e < m) {
            const uint64_t v = PT[swz(j)];
            scores[e] = v > (t - 1) / 2 ? (int32_t)((int64_t)v - (int64_t)t) : (int32_t)v;
        }
    }
}

cudaError_t launch_decrypt(const uint64_t* tw, const DevKeys& k, const uint64_t* scores_ct,
                           uint64_t nblocks, int32_t* scores, uint64_t m, cudaStream_t st) {
    const int smem = 3 * N * 8;
    cudaError_t e = cudaFuncSetAttribute(k_decrypt, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    const uint64_t chunk = 1u << 30;
    for (uint64_t off = 0; off < nblocks; off += chunk) {
        const uint64_t n = nblocks - off < chunk ? nblocks - off : chunk;
        k_decrypt<<<(unsigned)n, NTT_THREADS, smem, st>>>(tw, k.s_ntt, scores_ct + off * 4 * N,
                                                          scores + off * N, m > off * N ? m - off * N : 0, k.pm);
        count_launches(1);
    }
    return cudaGetLastError();
}

}  // namespace hers
