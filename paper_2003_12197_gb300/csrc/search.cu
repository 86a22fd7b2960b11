// Encrypted search kernels of the HERS library (Alg 7 server loop; Eq. 4;
// the ciphertext multiply of Alg 5 with its rounding and relinearisation
// moved after the sum over the d dimensions):
//
//   tensor   X_k = sum_i tensor_k(probe_i, gallery_i^b), k = 0, 1, 2, exactly,
//            as residues mod q1 q2 p1 p2 p3 in the NTT domain (pointwise);
//   intt     X_k back to the coefficient domain (15 polynomials per block);
//   scale    c_k = [round(t X_k / q)]_q, exact (RNS, no floating point);
//   keyswitch (c0, c1, c2) -> (c0 + sum_j D_j evk_j0, c1 + sum_j D_j evk_j1),
//            D_j = c2 mod q_j, once per gallery block.
#include "common.cuh"
#include "internal.h"

namespace hers {

// ---------------------------------------------------------------- tensor accumulate
//
// X_k = sum_i tensor_k(probe_i, gallery_i^b) for k = 0, 1, 2, per (block,
// limb, coefficient), in the NTT domain (pointwise), exactly mod p_l:
//   T0 = sum a0 b0,  T1 = sum (a0 b1 + a1 b0),  T2 = sum a1 b1.
//
// Organisation (sm_103a): CTA (tile, l, group) has TILE consumer threads, one
// coefficient each, for NB gallery blocks, plus one producer warp.  In the
// resident layout everything a CTA reads is contiguous: the probe's
// [dim][poly][TILE] run and one such run per block.  The producer's elected
// lane streams DPS dimensions per stage with one cp.async.bulk per run into a
// STAGES-deep shared-memory ring; "full" mbarriers track the copies and
// "empty" mbarriers (one arrival per consumer warp) hand stages back.
//
// Arithmetic: operands are split-stored signed 27-bit digits of the centred
// residue, x = xh 2^27 + xl with |xh|, |xl| <= 2^26 (split_store), and
//   x y = xh yh 2^54 + ((xh+xl)(yh+yl) - xh yh - xl yl) 2^27 + xl yl,
//   T1 = (a0+a1)(b0+b1) - T0 - T2,
// so each (dimension, coefficient, limb, block) costs 9 32x32->64 signed
// multiply-adds (mad.wide.s32) into 64-bit sums without reduction.  The
// largest partial product is (2^28)^2 = 2^56, so 64 dimensions sum to at most
// 2^62 and the sums are folded mod p every KCHUNK = 64 dimensions.  A wait
// that runs out (WAIT_NS, 2 s) sets bit 2 of *err.
constexpr int KCHUNK = 64;

__device__ __forceinline__ void madw(int64_t& acc, int32_t a, int32_t b) {
    asm("mad.wide.s32 %0, %1, %2, %0;" : "+l"(acc) : "r"(a), "r"(b));
}

// Residue mod p_l of the digit sums of one component:
// value = LL + (MM - HH - LL) 2^27 + HH 2^54, each term a signed 64-bit sum.
__device__ __forceinline__ uint64_t fold_signed(int64_t LL, int64_t HH, int64_t MM, int l, uint64_t p) {
    return reduce64(shoup_lazy(signed_to_unsigned(LL, l), 1, c_one_s[l], p) +
                        shoup_lazy(signed_to_unsigned(MM - HH - LL, l), c_r27[l], c_r27_s[l], p) +
                        shoup_lazy(signed_to_unsigned(HH, l), c_r54[l], c_r54_s[l], p),
                    l);
}

// GORDER: block groups vary fastest over the grid (x = group, y = (limb,
// tile)), so the CTAs in flight share one (limb, tile) run of the probe and
// it stays in L2 when the whole probe (d x 320 KiB) does not fit; otherwise
// tiles vary fastest (x = tile, y = limb, z = group) and the CTAs in flight
// read neighbouring runs of one block.
template <int NB, int STAGES, int DPS, int MINB, bool GORDER>
__global__ void __launch_bounds__(TILE + 32, MINB)
    k_tensor(const uint64_t* __restrict__ gal, const uint64_t* __restrict__ probe,
             uint64_t* __restrict__ acc, uint64_t nblocks, uint32_t d, int* err) {
    static_assert(KCHUNK % DPS == 0, "stages must not straddle a fold");
    extern __shared__ __align__(128) uint64_t sm[];
    __shared__ __align__(8) uint64_t full[STAGES], empty[STAGES];
    constexpr int RUN = DPS * 2 * TILE;         // words of one run per stage
    constexpr int STAGE_WORDS = (1 + NB) * RUN;
    const int tile = GORDER ? (int)(blockIdx.y % NTILES) : (int)blockIdx.x;
    const int l = GORDER ? (int)(blockIdx.y / NTILES) : (int)blockIdx.y;
    const uint64_t b0 = (uint64_t)(GORDER ? blockIdx.x : blockIdx.z) * NB;
    const int nb = (int)((nblocks - b0) < (uint64_t)NB ? (nblocks - b0) : NB);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t nst = (d + DPS - 1) / DPS;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; s++) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], TILE / 32);
        }
        mbar_fence_init();
    }
    __syncthreads();

    if (warp == TILE / 32) {  // producer warp
        if (lane == 0) {
            const uint64_t pol_g = policy_evict_first(), pol_p = policy_evict_last();
            const uint64_t* pr = probe + resident_offset(0, l, tile * TILE, d, 0, 0);
            const uint64_t* gr = gal + resident_offset(b0, l, tile * TILE, d, 0, 0);
            const size_t gstride = (size_t)10 * d * N;  // words per gallery block
            uint32_t issued = 0;
            for (uint32_t si = 0; si < nst; si++) {
                const int st = (int)(si % STAGES);
                if (si >= STAGES && !mbar_wait(&empty[st], ((si / STAGES) + 1) & 1)) {
                    atomicOr(err, 2);
                    break;
                }
                issued = si + 1;
                const uint32_t nd = min((uint32_t)DPS, d - si * DPS);
                const uint32_t bytes = nd * 2 * TILE * 8;
                uint64_t* dst = sm + (size_t)st * STAGE_WORDS;
                mbar_expect_tx(&full[st], bytes * (uint32_t)(1 + nb));
                bulk_g2s(dst, pr + (size_t)si * RUN, bytes, &full[st], pol_p);
                for (int j = 0; j < nb; j++)
                    bulk_g2s(dst + (1 + j) * RUN, gr + j * gstride + (size_t)si * RUN, bytes, &full[st],
                             pol_g);
            }
            // drain: the last stages' copies land before this thread leaves
            for (uint32_t si = issued > STAGES ? issued - STAGES : 0; si < issued; si++)
                if (!mbar_wait(&full[si % STAGES], (si / STAGES) & 1)) atomicOr(err, 2);
        }
        return;
    }

    // consumers
    const int t = threadIdx.x;
    const uint64_t p = c_mod[l];
    uint64_t fold[NB][3];
#pragma unroll
    for (int j = 0; j < NB; j++) fold[j][0] = fold[j][1] = fold[j][2] = 0;
    int64_t s[NB][9];  // per block: LL0 HH0 MM0 | LL2 HH2 MM2 | LLk HHk MMk
#pragma unroll
    for (int j = 0; j < NB; j++)
#pragma unroll
        for (int r = 0; r < 9; r++) s[j][r] = 0;
    for (uint32_t si = 0; si < nst; si++) {
        const int st = (int)(si % STAGES);
        if (!mbar_wait(&full[st], (si / STAGES) & 1)) {
            atomicOr(err, 2);
            return;
        }
        const uint32_t nd = min((uint32_t)DPS, d - si * DPS);
        const uint64_t* base = sm + (size_t)st * STAGE_WORDS + t;
#pragma unroll
        for (int dd = 0; dd < DPS; dd++) {
            if ((uint32_t)dd < nd) {
                const uint64_t A0 = base[dd * 2 * TILE], A1 = base[dd * 2 * TILE + TILE];
                const int32_t a0l = (int32_t)(uint32_t)A0, a0h = (int32_t)(uint32_t)(A0 >> 32);
                const int32_t a1l = (int32_t)(uint32_t)A1, a1h = (int32_t)(uint32_t)(A1 >> 32);
                const int32_t a0s = a0l + a0h, a1s = a1l + a1h;
                const int32_t sal = a0l + a1l, sah = a0h + a1h, sas = sal + sah;
#pragma unroll
                for (int j = 0; j < NB; j++) {
                    if (j < nb) {
                        const uint64_t* g = base + (1 + j) * RUN + dd * 2 * TILE;
                        const uint64_t B0 = g[0], B1 = g[TILE];
                        const int32_t b0l = (int32_t)(uint32_t)B0, b0h = (int32_t)(uint32_t)(B0 >> 32);
                        const int32_t b1l = (int32_t)(uint32_t)B1, b1h = (int32_t)(uint32_t)(B1 >> 32);
                        const int32_t b0s = b0l + b0h, b1s = b1l + b1h;
                        const int32_t sbl = b0l + b1l, sbh = b0h + b1h, sbs = sbl + sbh;
                        madw(s[j][0], a0l, b0l);
                        madw(s[j][1], a0h, b0h);
                        madw(s[j][2], a0s, b0s);
                        madw(s[j][3], a1l, b1l);
                        madw(s[j][4], a1h, b1h);
                        madw(s[j][5], a1s, b1s);
                        madw(s[j][6], sal, sbl);
                        madw(s[j][7], sah, sbh);
                        madw(s[j][8], sas, sbs);
                    }
                }
            }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[st]);
        const uint32_t done = si * DPS + nd;
        if (done % KCHUNK == 0 || done == d) {
            // fold: value = LL + (MM - HH - LL) 2^27 + HH 2^54 (mod p)
#pragma unroll
            for (int j = 0; j < NB; j++) {
                uint64_t v[3];
#pragma unroll
                for (int c = 0; c < 3; c++) {
                    v[c] = fold_signed(s[j][3 * c], s[j][3 * c + 1], s[j][3 * c + 2], l, p);
                    s[j][3 * c] = s[j][3 * c + 1] = s[j][3 * c + 2] = 0;
                }
                // T0 = v0, T2 = v1, T1 = K - T0 - T2 with K = v2
                fold[j][0] = add_mod(fold[j][0], v[0], p);
                fold[j][2] = add_mod(fold[j][2], v[1], p);
                fold[j][1] = add_mod(fold[j][1], sub_mod(sub_mod(v[2], v[0], p), v[1], p), p);
            }
        }
    }
    const int k = tile * TILE + t;
#pragma unroll
    for (int j = 0; j < NB; j++)
        if (j < nb)
#pragma unroll
            for (int c = 0; c < 3; c++) acc[(((b0 + j) * 3 + c) * 5 + l) * N + k] = fold[j][c];
}

// The variants the autotuner chooses from: (blocks per CTA, pipeline stages,
// dimensions per stage, minimum CTAs per SM for the register budget).
using TensorFn = void (*)(const uint64_t*, const uint64_t*, uint64_t*, uint64_t, uint32_t, int*);
struct TensorVariant {
    const char* name;
    TensorFn fn;
    int nb, stages, dps;
    bool gorder;
};
// name: nb<blocks per CTA>_s<stages>_d<dimensions per stage>_m<CTAs/SM>, and
// a leading "g" for the group-fastest grid order
#define HERS_TV(NB, S, D, M) {"nb" #NB "_s" #S "_d" #D "_m" #M, k_tensor<NB, S, D, M, false>, NB, S, D, false}
#define HERS_TVG(NB, S, D, M) {"gnb" #NB "_s" #S "_d" #D "_m" #M, k_tensor<NB, S, D, M, true>, NB, S, D, true}
static const TensorVariant kTensorVariants[] = {
    HERS_TV(2, 6, 1, 1),  HERS_TV(2, 4, 2, 2),  HERS_TV(2, 3, 2, 3),  HERS_TV(1, 4, 2, 3),
    HERS_TV(1, 6, 2, 2),  HERS_TV(2, 2, 4, 2),  HERS_TV(4, 3, 2, 1),  HERS_TV(1, 3, 4, 3),
    HERS_TVG(2, 2, 4, 2), HERS_TVG(2, 4, 2, 2), HERS_TVG(1, 3, 4, 3), HERS_TVG(2, 3, 2, 3),
};
#undef HERS_TV
#undef HERS_TVG
constexpr int NUM_TENSOR_VARIANTS = sizeof(kTensorVariants) / sizeof(kTensorVariants[0]);

int tensor_variant_count() { return NUM_TENSOR_VARIANTS; }
const char* tensor_variant_name(int v) {
    return (v >= 0 && v < NUM_TENSOR_VARIANTS) ? kTensorVariants[v].name : nullptr;
}

cudaError_t launch_tensor(int variant, const uint64_t* gallery, uint64_t nblocks, uint32_t d,
                          const uint64_t* probe, uint64_t* X, int* err, cudaStream_t st) {
    if (variant < 0 || variant >= NUM_TENSOR_VARIANTS) return cudaErrorInvalidValue;
    const TensorVariant& v = kTensorVariants[variant];
    const int smem = v.stages * (1 + v.nb) * v.dps * 2 * TILE * 8;
    cudaError_t e = cudaFuncSetAttribute(v.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    const uint64_t max_groups = v.gorder ? 0x7FFFFFFFull : 65535ull;  // grid x or z limit
    const uint64_t max_z = max_groups * v.nb;
    for (uint64_t g0 = 0; g0 < nblocks; g0 += max_z) {
        const uint64_t nb = nblocks - g0 < max_z ? nblocks - g0 : max_z;
        const unsigned groups = (unsigned)((nb + v.nb - 1) / v.nb);
        const dim3 grid = v.gorder ? dim3(groups, NTILES * 5, 1) : dim3(NTILES, 5, groups);
        v.fn<<<grid, TILE + 32, smem, st>>>(gallery + g0 * 10ull * d * N, probe, X + g0 * 15 * N, nb,
                                            d, err);
        count_launches(1);
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------- batched NTTs
// CTA per polynomial of a contiguous [npolys][N] array; modulus index
// mod_off + (P % mod_period).
template <bool INV>
__global__ void __launch_bounds__(NTT_THREADS, 3) k_ntt_batch(const uint64_t* __restrict__ tw,
                                                           uint64_t* __restrict__ data,
                                                           int mod_period, int mod_off) {
    extern __shared__ uint64_t sm[];
    const uint64_t P = blockIdx.x;
    const int mi = mod_off + (int)(P % (uint64_t)mod_period);
    uint64_t* g = data + P * N;
    for (int k = threadIdx.x; k < N; k += blockDim.x) sm[swz(k)] = g[k];
    if (INV) ntt_inv_mod(sm, tw, mi);
    else ntt_fwd_mod(sm, tw, mi);
    for (int k = threadIdx.x; k < N; k += blockDim.x) g[k] = sm[swz(k)];
}

// ---------------------------------------------------------------- exact scale-and-round
//
// Thread per (b, poly c, k).  X has residues x_0..x_4 mod (q1, q2, p1, p2, p3),
// |X| < q P / 2.  With r = [t X]_q centred, Y = (t X - r) / q is an integer
// and equals round(t X / q) (|r| < q/2, q odd: no tie), |Y| < 2^150 < P/2:
//   Y mod p_i = (t x_i - r) q^-1 mod p_i,   i = p1, p2, p3;
//   Y from its three residues by mixed radix (Garner), centred by comparing
//   the digits with those of (P-1)/2;   c = Y mod q_l, l = 1, 2.
// Writes c to C[b][c][l][N] and, for c = 2, the relinearisation digits
// D_1 = c2 mod q1, D_2 = c2 mod q2 reduced into both limbs:
// KS[b][0] = D_1 mod q1, [1] = D_1 mod q2, [2] = D_2 mod q1, [3] = D_2 mod q2.
__global__ void __launch_bounds__(256) k_scale_round(const uint64_t* __restrict__ X,
                                                     uint64_t* __restrict__ C,
                                                     uint64_t* __restrict__ KS, int pm) {
    const PlainMod& P = c_plain[pm];
    const int k = blockIdx.x * 256 + threadIdx.x;
    const int c = blockIdx.y;
    const uint64_t b = blockIdx.z;
    const uint64_t* x = X + ((b * 3 + c) * 5) * N + k;
    const uint64_t x0 = x[0], x1 = x[N], x2 = x[2 * N], x3 = x[3 * N], x4 = x[4 * N];
    const uint64_t q1 = c_mod[0], q2 = c_mod[1];

    // r = [t X]_q
    const uint64_t a1 = shoup(x0, P.t_mod[0], P.t_s[0], q1);
    const uint64_t a2 = shoup(x1, P.t_mod[1], P.t_s[1], q2);
    const Lifted R = lift_q(a1, a2);
    uint64_t y[3];
#pragma unroll
    for (int i = 0; i < 3; i++) {
        const int mi = 2 + i;
        const uint64_t p = c_mod[mi];
        const uint64_t xi = i == 0 ? x2 : (i == 1 ? x3 : x4);
        const uint64_t rm = lifted_mod(R, mi, a2);
        const uint64_t tx = shoup(xi, P.t_mod[mi], P.t_s[mi], p);
        y[i] = shoup(sub_mod(tx, rm, p), c_qinv_p[i], c_qinv_p_s[i], p);
    }
    // mixed radix Y = y1 + p1 z2 + p1 p2 z3
    const uint64_t p2 = c_mod[3], p3 = c_mod[4];
    const uint64_t z1 = y[0];
    const uint64_t z2 = shoup(sub_mod(y[1], csub(z1, p2), p2), P1INV_P2, P1INV_P2_S, p2);
    uint64_t t3 = shoup(sub_mod(y[2], csub(z1, p3), p3), P1INV_P3, P1INV_P3_S, p3);
    const uint64_t z3 = shoup(sub_mod(t3, csub(z2, p3), p3), P2INV_P3, P2INV_P3_S, p3);
    const bool neg = (z3 > HALFP_D3) || (z3 == HALFP_D3 && (z2 > HALFP_D2 || (z2 == HALFP_D2 && z1 > HALFP_D1)));
    uint64_t out[2];
#pragma unroll
    for (int l = 0; l < 2; l++) {
        const uint64_t q = c_mod[l];
        uint64_t v = add_mod(z1, shoup(z2, c_p1_mod_q[l], c_p1_mod_q_s[l], q), q);
        v = add_mod(v, shoup(z3, c_p1p2_mod_q[l], c_p1p2_mod_q_s[l], q), q);
        if (neg) v = sub_mod(v, c_p_mod_q[l], q);
        out[l] = v;
        C[((b * 3 + c) * 2 + l) * N + k] = v;
    }
    if (c == 2) {
        uint64_t* ks = KS + b * 4 * N + k;
        ks[0] = out[0];
        ks[N] = csub(out[0], q2);
        ks[2 * N] = out[1];
        ks[3 * N] = out[1];
    }
}

// ---------------------------------------------------------------- key switch
// KS (NTT domain) x evk_j (NTT, Shoup): O[b][c][l] = sum_j D_j evk_j[c][l].
__global__ void __launch_bounds__(256) k_ks_mul(const uint64_t* __restrict__ KS,
                                                const uint64_t* __restrict__ evk_ntt,
                                                uint64_t* __restrict__ O) {
    const int k = blockIdx.x * 256 + threadIdx.x;
    const int l = blockIdx.y;
    const uint64_t b = blockIdx.z;
    const uint64_t q = c_mod[l];
    const uint64_t D1 = KS[(b * 4 + l) * N + k], D2 = KS[(b * 4 + 2 + l) * N + k];
#pragma unroll
    for (int c = 0; c < 2; c++) {
        const uint64_t* e1 = evk_ntt + (size_t)(((0 * 2 + c) * 2 + l) * 2) * N;
        const uint64_t* e2 = evk_ntt + (size_t)(((1 * 2 + c) * 2 + l) * 2) * N;
        const uint64_t v = shoup_lazy(D1, e1[k], e1[N + k], q) + shoup_lazy(D2, e2[k], e2[N + k], q);
        O[((b * 2 + c) * 2 + l) * N + k] = reduce64(v, l);
    }
}

// out[b][c][l] = C[b][c][l] + O[b][c][l] mod q_l (O in the coefficient domain)
__global__ void __launch_bounds__(256) k_ks_finish(const uint64_t* __restrict__ C,
                                                   const uint64_t* __restrict__ O,
                                                   uint64_t* __restrict__ out) {
    const int k = blockIdx.x * 256 + threadIdx.x;
    const int l = blockIdx.y & 1, c = blockIdx.y >> 1;
    const uint64_t b = blockIdx.z;
    const uint64_t q = c_mod[l];
    out[((b * 2 + c) * 2 + l) * N + k] =
        add_mod(C[((b * 3 + c) * 2 + l) * N + k], O[((b * 2 + c) * 2 + l) * N + k], q);
}

// ---------------------------------------------------------------- pipeline
// Epilogue over npairs (probe, block) pairs whose accumulators are in
// X [npairs][3][5][N] (NTT domain): inverse NTTs, exact scale-and-round into
// C [npairs][3][2][N] and KS [npairs][4][N], key switch (the output O reuses X),
// ---------------------------------------------------------------- base-w key switch
// Digits of c2 (C[b][2], canonical) in base w = 2^logw: the coefficient as an
// integer c = x1 + q1 h in [0, q) (Garner), D_j = floor(c / w^j) mod w, each
// stored as a residue in both limbs: W[b][j][l][N] = D_j mod q_l.
__global__ void __launch_bounds__(256) k_digits_w(const uint64_t* __restrict__ C, uint32_t logw, uint32_t ndig,
                                                  uint64_t* __restrict__ W) {
    const int k = blockIdx.x * 256 + threadIdx.x;
    const uint64_t b = blockIdx.z;
    const uint64_t* c2 = C + ((b * 3 + 2) * 2) * N;
    const uint64_t x1 = c2[k], x2 = c2[N + k];
    const Lifted L = lift_q(x1, x2);
    const unsigned __int128 c = (unsigned __int128)x1 + (unsigned __int128)c_mod[0] * L.h;
    const unsigned __int128 mask = ((unsigned __int128)1 << logw) - 1;
    uint64_t* w = W + b * ndig * 2 * N + k;
    for (uint32_t j = 0; j < ndig; j++) {
        const uint64_t dj = (uint64_t)((c >> (logw * j)) & mask);  // < 2^60
        w[(j * 2 + 0) * N] = dj % c_mod[0];
        w[(j * 2 + 1) * N] = dj % c_mod[1];
    }
}

// O[b][c][l] = sum_j D_j evkw_j[c][l] (NTT domain, Shoup with the keys' companions).
__global__ void __launch_bounds__(256) k_ks_mul_w(const uint64_t* __restrict__ W,
                                                  const uint64_t* __restrict__ evkw_ntt, uint32_t ndig,
                                                  uint64_t* __restrict__ O) {
    const int k = blockIdx.x * 256 + threadIdx.x;
    const int l = blockIdx.y;
    const uint64_t b = blockIdx.z;
    const uint64_t q = c_mod[l];
#pragma unroll
    for (int c = 0; c < 2; c++) {
        uint64_t v = 0;  // each term < 2q, at most 5 terms: < 10q < 2^58
        for (uint32_t j = 0; j < ndig; j++) {
            const uint64_t* e = evkw_ntt + (size_t)(((j * 2 + c) * 2 + l) * 2) * N;
            v += shoup_lazy(W[((b * ndig + j) * 2 + l) * N + k], e[k], e[N + k], q);
        }
        O[((b * 2 + c) * 2 + l) * N + k] = reduce64(v, l);
    }
}

// canonical score ciphertexts into out [npairs][2][2][N].
cudaError_t launch_epilogue(const uint64_t* tw, const DevKeys& k, uint64_t npairs, uint64_t* X,
                            uint64_t* C, uint64_t* KS, uint64_t* out, cudaStream_t st,
                            cudaEvent_t* ev, const KeySwitchW* ksw) {
    uint64_t nl = 0;
    uint64_t* O = X;
    const uint64_t max_z = 65535;
    const uint64_t chunk = 1u << 30;
    for (uint64_t off = 0; off < npairs * 15; off += chunk) {
        const uint64_t n = npairs * 15 - off < chunk ? npairs * 15 - off : chunk;
        k_ntt_batch<true><<<(unsigned)n, NTT_THREADS, N * 8, st>>>(tw, X + off * N, 5, 0);
        nl++;
    }
    if (ev) cudaEventRecord(ev[0], st);
    for (uint64_t b0 = 0; b0 < npairs; b0 += max_z) {
        const uint64_t nb = npairs - b0 < max_z ? npairs - b0 : max_z;
        k_scale_round<<<dim3(N / 256, 3, (unsigned)nb), 256, 0, st>>>(X + b0 * 15 * N, C + b0 * 6 * N,
                                                                     KS + b0 * 4 * N, k.pm);
        nl++;
    }
    if (ev) cudaEventRecord(ev[1], st);
    if (ksw) {
        // base-w gadget: digits after O in X, NTT, multiply-accumulate with evkw
        uint64_t* W = X + npairs * 4 * N;
        const uint64_t per = (uint64_t)ksw->ndig * 2;
        for (uint64_t b0 = 0; b0 < npairs; b0 += max_z) {
            const uint64_t nb = npairs - b0 < max_z ? npairs - b0 : max_z;
            k_digits_w<<<dim3(N / 256, 1, (unsigned)nb), 256, 0, st>>>(C + b0 * 6 * N, ksw->logw, ksw->ndig,
                                                                       W + b0 * per * N);
            nl++;
        }
        for (uint64_t off = 0; off < npairs * per; off += chunk) {
            const uint64_t n = npairs * per - off < chunk ? npairs * per - off : chunk;
            k_ntt_batch<false><<<(unsigned)n, NTT_THREADS, N * 8, st>>>(tw, W + off * N, 2, 0);
            nl++;
        }
        for (uint64_t b0 = 0; b0 < npairs; b0 += max_z) {
            const uint64_t nb = npairs - b0 < max_z ? npairs - b0 : max_z;
            k_ks_mul_w<<<dim3(N / 256, 2, (unsigned)nb), 256, 0, st>>>(W + b0 * per * N, ksw->evkw_ntt,
                                                                       ksw->ndig, O + b0 * 4 * N);
            nl++;
        }
    } else {
        for (uint64_t off = 0; off < npairs * 4; off += chunk) {
            const uint64_t n = npairs * 4 - off < chunk ? npairs * 4 - off : chunk;
            k_ntt_batch<false><<<(unsigned)n, NTT_THREADS, N * 8, st>>>(tw, KS + off * N, 2, 0);
            nl++;
        }
        for (uint64_t b0 = 0; b0 < npairs; b0 += max_z) {
            const uint64_t nb = npairs - b0 < max_z ? npairs - b0 : max_z;
            k_ks_mul<<<dim3(N / 256, 2, (unsigned)nb), 256, 0, st>>>(KS + b0 * 4 * N, k.evk_ntt,
                                                                     O + b0 * 4 * N);
            nl++;
        }
    }
    for (uint64_t off = 0; off < npairs * 4; off += chunk) {
        const uint64_t n = npairs * 4 - off < chunk ? npairs * 4 - off : chunk;
        k_ntt_batch<true><<<(unsigned)n, NTT_THREADS, N * 8, st>>>(tw, O + off * N, 2, 0);
        nl++;
    }
    for (uint64_t b0 = 0; b0 < npairs; b0 += max_z) {
        const uint64_t nb = npairs - b0 < max_z ? npairs - b0 : max_z;
        k_ks_finish<<<dim3(N / 256, 4, (unsigned)nb), 256, 0, st>>>(C + b0 * 6 * N, O + b0 * 4 * N,
                                                                    out + b0 * 4 * N);
        nl++;
    }
    count_launches(nl);
    return cudaGetLastError();
}

// Workspace per block: X [3][5][N] (reused for O [2][2][N]), C [3][2][N], KS [4][N].
cudaError_t launch_search(const uint64_t* tw, const DevKeys& k, const uint64_t* gallery,
                          uint64_t nblocks, uint32_t d, const uint64_t* probe, uint64_t* scores_ct,
                          uint64_t* ws, int* err, cudaStream_t st, cudaEvent_t* ev, int variant,
                          const KeySwitchW* ksw) {
    if (nblocks == 0) return cudaSuccess;
    uint64_t* X = ws;
    uint64_t* C = X + nblocks * 15 * N;
    uint64_t* KS = C + nblocks * 6 * N;
    if (ev) cudaEventRecord(ev[0], st);
    cudaError_t e = launch_tensor(variant, gallery, nblocks, d, probe, X, err, st);
    if (e != cudaSuccess) return e;
    if (ev) cudaEventRecord(ev[1], st);
    e = launch_epilogue(tw, k, nblocks, X, C, KS, scores_ct, st, ev ? ev + 2 : nullptr, ksw);
    if (ev) cudaEventRecord(ev[4], st);
    return e;
}

}  // namespace hers
