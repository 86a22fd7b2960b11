// Encrypted search kernels of the HERS library (Alg 7 server loop; Eq. 4;
// the ciphertext multiply of Alg 5 with its rounding and relinearisation
// moved after the sum over the d dimensions):
//
//   tensor   X_k = sum_i tensor_k(probe_i, gallery_i^b), k = 0, 1, 2, exactly,
//            as residues mod r_0 .. r_7 (the search basis) in the NTT domain;
//   intt     X_k back to the coefficient domain (24 polynomials per block);
//   scale    c_k = [round(t X_k / q)]_q, exact (CRT, no floating point);
//   keyswitch (c0, c1, c2) -> (c0 + sum_j D_j evk_j0, c1 + sum_j D_j evk_j1),
//            D_j = c2 mod q_j, once per gallery block.
#include <cooperative_groups.h>

#include <string>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace hers {

// ---------------------------------------------------------------- tensor accumulate
//
// X_k = sum_i tensor_k(probe_i, gallery_i^b) for k = 0, 1, 2, per (block,
// limb, coefficient), in the NTT domain (pointwise), exactly mod r_l:
//   T0 = sum a0 b0,  T1 = sum (a0 b1 + a1 b0),  T2 = sum a1 b1.
//
// Organisation (sm_103a): CTA (tile, l, group) has TILE consumer threads, one
// coefficient each, for NB gallery blocks, plus one producer warp.  The
// consumers walk the ring a lap (STAGES stages) per iteration, with constant
// stage indices, and take an unpredicated path for full stages.  In the
// resident layout everything a CTA reads is contiguous: the probe's
// [dim][TILE][poly] run and one such run per block.  The producer's elected
// lane streams DPS dimensions per stage with one cp.async.bulk per run into a
// STAGES-deep shared-memory ring; "full" mbarriers track the copies and
// "empty" mbarriers (one arrival per consumer thread, no lane test) hand
// stages back.
//
// Arithmetic: operands are the centred residues (|a|, |b| < 2^29), so each
// (dimension, coefficient, limb, block) costs four 32x32->64 signed
// multiply-adds (mad.wide.s32) into 64-bit sums: T1 grows by less than 2^59
// per dimension, T0 and T2 by less than 2^58.  A partial fold (pfold) brings a
// sum back below 2^61 + 2^32 in magnitude: T1 every PFOLD = 8 dimensions and
// T0, T2 every 2 PFOLD, so every sum stays below 2^63 (2^61 + 2^32 + 8 2^59
// and 2^61 + 2^32 + 16 2^58); the last dimension ends with a full reduction
// mod r_l.  A wait that runs out (WAIT_NS, 2 s) sets bit 2 of *err.
//
// KA (Karatsuba's middle term): three products per (dimension, coefficient,
// limb, block) instead of four, T0 += a0 b0, T2 += a1 b1 and
// S += (a0 + a1)(b0 + b1), with T1 = S - T0 - T2 formed mod r_l at the end.
// The sums a0 + a1 and b0 + b1 are below 2^30, their product below 2^60, so S
// is folded every KFOLD_S = 4 dimensions (2^61 + 2^32 + 4 2^60 < 2^63) and
// T0, T2 every KFOLD_02 = 16.  The kernel stays bound by HBM either way; the
// multiply pipe it leaves free is what an epilogue running beside it uses.
constexpr int PFOLD = 8;
constexpr int KFOLD_S = 4, KFOLD_02 = 16;

__device__ __forceinline__ void madw(int64_t& acc, int32_t a, int32_t b) {
    asm("mad.wide.s32 %0, %1, %2, %0;" : "+l"(acc) : "r"(a), "r"(b));
}

// One stage's products: for dd < nd and block j < nb, the four products of
// the probe row and gallery row j.  With FULL (nd = DPS, nb = NB) the loops
// carry no predicates.
// With KA, s[j][1] holds S and the three products above replace the four.
template <int NB, int DPS, int RUN, bool FULL, bool KA>
__device__ __forceinline__ void tensor_stage(int64_t (&s)[NB][3], const int2* base, uint32_t nd, int nb) {
#pragma unroll
    for (int dd = 0; dd < DPS; dd++) {
        if (FULL || (uint32_t)dd < nd) {
            const int2 A = base[dd * TILE];
            const int32_t as = A.x + A.y;
#pragma unroll
            for (int j = 0; j < NB; j++) {
                if (FULL || j < nb) {
                    const int2 G = base[(1 + j) * (RUN / 2) + dd * TILE];
                    madw(s[j][0], A.x, G.x);
                    if (KA) {
                        madw(s[j][1], as, G.x + G.y);
                    } else {
                        madw(s[j][1], A.x, G.y);
                        madw(s[j][1], A.y, G.x);
                    }
                    madw(s[j][2], A.y, G.y);
                }
            }
        }
    }
}

// GORDER: block groups vary fastest over the grid (x = group, y = (limb,
// tile)), so the CTAs in flight share one (limb, tile) run of the probe and
// it stays in L2 when the whole probe (d x 256 KiB) does not fit; otherwise
// tiles vary fastest (x = tile, y = limb, z = group) and the CTAs in flight
// read neighbouring runs of one block.
template <int NB, int STAGES, int DPS, int MINB, bool GORDER, bool KA = false>
__global__ void __launch_bounds__(TILE + 32, MINB)
    k_tensor(const int32_t* __restrict__ gal, const int32_t* __restrict__ probe,
             uint32_t* __restrict__ acc, uint64_t nblocks, uint32_t d, int* err) {
    static_assert((KA ? KFOLD_S : PFOLD) % DPS == 0, "stages must not straddle a partial fold");
    extern __shared__ __align__(128) int32_t smr[];
    __shared__ __align__(8) uint64_t full[STAGES], empty[STAGES];
    constexpr int RUN = DPS * 2 * TILE;         // elements of one run per stage
    constexpr int STAGE_ELEMS = (1 + NB) * RUN;
    const int tile = GORDER ? (int)(blockIdx.y % NTILES) : (int)blockIdx.x;
    const int l = GORDER ? (int)(blockIdx.y / NTILES) : (int)blockIdx.y;
    const uint64_t b0 = (uint64_t)(GORDER ? blockIdx.x : blockIdx.z) * NB;
    const int nb = (int)((nblocks - b0) < (uint64_t)NB ? (nblocks - b0) : NB);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t nst = (d + DPS - 1) / DPS;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; s++) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], TILE);  // every consumer thread arrives
        }
        mbar_fence_init();
    }
    __syncthreads();

    if (warp == TILE / 32) {  // producer warp
        if (lane == 0) {
            const uint64_t pol_g = policy_evict_first(), pol_p = policy_evict_last();
            const int32_t* pr = probe + resident_offset(0, l, tile * TILE, d, 0, 0);
            const int32_t* gr = gal + resident_offset(b0, l, tile * TILE, d, 0, 0);
            const size_t gstride = (size_t)NUM_S * 2 * d * N;  // elements per gallery block
            uint32_t issued = 0;
            for (uint32_t si = 0; si < nst; si++) {
                const int st = (int)(si % STAGES);
                if (si >= STAGES && !mbar_wait(&empty[st], ((si / STAGES) + 1) & 1)) {
                    atomicOr(err, 2);
                    break;
                }
                issued = si + 1;
                const uint32_t nd = min((uint32_t)DPS, d - si * DPS);
                const uint32_t bytes = nd * 2 * TILE * 4;
                int32_t* dst = smr + (size_t)st * STAGE_ELEMS;
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

    // consumers: the ring is walked STAGES stages per lap, so stage indices are
    // constants and the phase parity flips once per lap
    const int t = threadIdx.x;
    const int32_t r32 = (int32_t)c_sr32[l];
    int64_t s[NB][3];
#pragma unroll
    for (int j = 0; j < NB; j++) s[j][0] = s[j][1] = s[j][2] = 0;
    for (uint32_t s0 = 0; s0 < nst; s0 += STAGES) {
        const uint32_t parity = (s0 / STAGES) & 1;
#pragma unroll
        for (int st = 0; st < STAGES; st++) {
            const uint32_t si = s0 + st;
            if (si >= nst) break;
            if (!mbar_wait(&full[st], parity)) {
                atomicOr(err, 2);
                return;
            }
            const uint32_t nd = min((uint32_t)DPS, d - si * DPS);
            const int2* base = (const int2*)(smr + st * STAGE_ELEMS) + t;  // (poly 0, poly 1) pairs
            if (nd == DPS && nb == NB) tensor_stage<NB, DPS, RUN, true, KA>(s, base, nd, nb);
            else tensor_stage<NB, DPS, RUN, false, KA>(s, base, nd, nb);
            mbar_arrive(&empty[st]);
            const uint32_t done = si * DPS + nd;
            constexpr uint32_t F1 = KA ? KFOLD_S : PFOLD, F02 = KA ? KFOLD_02 : 2 * PFOLD;
            if (done % F1 == 0 && done < d) {
                const bool all = done % F02 == 0;
#pragma unroll
                for (int j = 0; j < NB; j++) {
                    s[j][1] = pfold(s[j][1], r32);
                    if (all) {
                        s[j][0] = pfold(s[j][0], r32);
                        s[j][2] = pfold(s[j][2], r32);
                    }
                }
            }
        }
    }
    const int k = tile * TILE + t;
#pragma unroll
    for (int j = 0; j < NB; j++)
        if (j < nb) {
            if (KA) {
                const uint32_t r = c_smod[l];
                const uint32_t x0 = fold_full(s[j][0], l), x2 = fold_full(s[j][2], l);
                const uint32_t x1 = csub32(csub32(fold_full(s[j][1], l) + 2 * r - x0 - x2, 2 * r), r);
                acc[(((b0 + j) * 3 + 0) * NUM_S + l) * N + k] = x0;
                acc[(((b0 + j) * 3 + 1) * NUM_S + l) * N + k] = x1;
                acc[(((b0 + j) * 3 + 2) * NUM_S + l) * N + k] = x2;
            } else {
#pragma unroll
                for (int c = 0; c < 3; c++) acc[(((b0 + j) * 3 + c) * NUM_S + l) * N + k] = fold_full(s[j][c], l);
            }
        }
}

// The same products as a persistent kernel: a grid of K CTAs per SM, CTA b
// taking units b, b + grid, b + 2 grid, ... of the (limb, tile, block group)
// units, block groups fastest (the CTAs in flight share a (limb, tile) run of
// the probe).  Producer and consumers derive the same unit sequence from the
// CTA index, so no tables or descriptors are exchanged, and the ring of
// stages runs on across units (stage counter G: slot G % STAGES, phase
// (G / STAGES) & 1).  The CTAs stay resident for the whole launch, so a
// kernel of another stream (the epilogue of the search in flight beside it)
// gets the registers and shared memory the K CTAs leave on each SM, and
// never displaces the streaming CTAs.
template <int NB, int STAGES, int DPS, int MINB, bool KA>
__global__ void __launch_bounds__(TILE + 32, MINB)
    k_tensor_persist(const int32_t* __restrict__ gal, const int32_t* __restrict__ probe,
                     uint32_t* __restrict__ acc, uint64_t nblocks, uint32_t d, int* err) {
    static_assert((KA ? KFOLD_S : PFOLD) % DPS == 0, "stages must not straddle a partial fold");
    extern __shared__ __align__(128) int32_t smr[];
    __shared__ __align__(8) uint64_t full[STAGES], empty[STAGES];
    constexpr int RUN = DPS * 2 * TILE;
    constexpr int STAGE_ELEMS = (1 + NB) * RUN;
    const uint64_t ngroups = (nblocks + NB - 1) / NB;
    const uint64_t nunits = ngroups * NUM_S * NTILES;
    const uint32_t nst = (d + DPS - 1) / DPS;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; s++) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], TILE);
        }
        mbar_fence_init();
    }
    __syncthreads();

    if (warp == TILE / 32) {  // producer warp
        if (lane == 0) {
            const uint64_t pol_g = policy_evict_first(), pol_p = policy_evict_last();
            const size_t gstride = (size_t)NUM_S * 2 * d * N;
            uint32_t G = 0;
            bool failed = false;
            for (uint64_t u = blockIdx.x; u < nunits && !failed; u += gridDim.x) {
                const uint64_t b0 = (u % ngroups) * NB;
                const uint32_t lt = (uint32_t)(u / ngroups);
                const int tile = (int)(lt % NTILES), l = (int)(lt / NTILES);
                const int nb = (int)((nblocks - b0) < (uint64_t)NB ? (nblocks - b0) : NB);
                const int32_t* pr = probe + resident_offset(0, l, tile * TILE, d, 0, 0);
                const int32_t* gr = gal + resident_offset(b0, l, tile * TILE, d, 0, 0);
                for (uint32_t si = 0; si < nst; si++, G++) {
                    const int st = (int)(G % STAGES);
                    if (G >= STAGES && !mbar_wait(&empty[st], ((G / STAGES) + 1) & 1)) {
                        atomicOr(err, 2);
                        failed = true;
                        break;
                    }
                    const uint32_t nd = min((uint32_t)DPS, d - si * DPS);
                    const uint32_t bytes = nd * 2 * TILE * 4;
                    int32_t* dst = smr + (size_t)st * STAGE_ELEMS;
                    mbar_expect_tx(&full[st], bytes * (uint32_t)(1 + nb));
                    bulk_g2s(dst, pr + (size_t)si * RUN, bytes, &full[st], pol_p);
                    for (int j = 0; j < nb; j++)
                        bulk_g2s(dst + (1 + j) * RUN, gr + j * gstride + (size_t)si * RUN, bytes, &full[st],
                                 pol_g);
                }
            }
            // drain: the last stages' copies land before this thread leaves
            for (uint32_t i = G > STAGES ? G - STAGES : 0; i < G; i++)
                if (!mbar_wait(&full[i % STAGES], (i / STAGES) & 1)) atomicOr(err, 2);
        }
        return;
    }

    const int t = threadIdx.x;
    uint32_t G = 0;
    for (uint64_t u = blockIdx.x; u < nunits; u += gridDim.x) {
        const uint64_t b0 = (u % ngroups) * NB;
        const uint32_t lt = (uint32_t)(u / ngroups);
        const int tile = (int)(lt % NTILES), l = (int)(lt / NTILES);
        const int nb = (int)((nblocks - b0) < (uint64_t)NB ? (nblocks - b0) : NB);
        const int32_t r32 = (int32_t)c_sr32[l];
        int64_t s[NB][3];
#pragma unroll
        for (int j = 0; j < NB; j++) s[j][0] = s[j][1] = s[j][2] = 0;
        for (uint32_t si = 0; si < nst; si++, G++) {
            const int st = (int)(G % STAGES);
            if (!mbar_wait(&full[st], (G / STAGES) & 1)) {
                atomicOr(err, 2);
                return;
            }
            const uint32_t nd = min((uint32_t)DPS, d - si * DPS);
            const int2* base = (const int2*)(smr + st * STAGE_ELEMS) + t;
            if (nd == DPS && nb == NB) tensor_stage<NB, DPS, RUN, true, KA>(s, base, nd, nb);
            else tensor_stage<NB, DPS, RUN, false, KA>(s, base, nd, nb);
            mbar_arrive(&empty[st]);
            const uint32_t done = si * DPS + nd;
            constexpr uint32_t F1 = KA ? KFOLD_S : PFOLD, F02 = KA ? KFOLD_02 : 2 * PFOLD;
            if (done % F1 == 0 && done < d) {
                const bool all = done % F02 == 0;
#pragma unroll
                for (int j = 0; j < NB; j++) {
                    s[j][1] = pfold(s[j][1], r32);
                    if (all) {
                        s[j][0] = pfold(s[j][0], r32);
                        s[j][2] = pfold(s[j][2], r32);
                    }
                }
            }
        }
        const int k = tile * TILE + t;
#pragma unroll
        for (int j = 0; j < NB; j++)
            if (j < nb) {
                uint32_t x0 = fold_full(s[j][0], l), x1 = fold_full(s[j][1], l), x2 = fold_full(s[j][2], l);
                if (KA) {
                    const uint32_t r = c_smod[l];
                    x1 = csub32(csub32(x1 + 2 * r - x0 - x2, 2 * r), r);
                }
                acc[(((b0 + j) * 3 + 0) * NUM_S + l) * N + k] = x0;
                acc[(((b0 + j) * 3 + 1) * NUM_S + l) * N + k] = x1;
                acc[(((b0 + j) * 3 + 2) * NUM_S + l) * N + k] = x2;
            }
    }
}

// The variants the autotuner chooses from: (blocks per CTA, pipeline stages,
// dimensions per stage, minimum CTAs per SM for the register budget).
using TensorFn = void (*)(const int32_t*, const int32_t*, uint32_t*, uint64_t, uint32_t, int*);
struct TensorVariant {
    const char* name;
    TensorFn fn;
    int nb, stages, dps;
    bool gorder;
    int persist;  // > 0: k_tensor_persist with this many CTAs per SM
};
// name: nb<blocks per CTA>_s<stages>_d<dimensions per stage>_m<CTAs/SM>, and
// a leading "g" for the group-fastest grid order
#define HERS_TV(NB, S, D, M) {"nb" #NB "_s" #S "_d" #D "_m" #M, k_tensor<NB, S, D, M, false>, NB, S, D, false}
#define HERS_TVG(NB, S, D, M) {"gnb" #NB "_s" #S "_d" #D "_m" #M, k_tensor<NB, S, D, M, true>, NB, S, D, true}
// the Karatsuba form (KA) of the same shapes: a trailing "_ka"
#define HERS_TVK(NB, S, D, M, GO, PFX) \
    {PFX "nb" #NB "_s" #S "_d" #D "_m" #M "_ka", k_tensor<NB, S, D, M, GO, true>, NB, S, D, GO}
// persistent Karatsuba form, K CTAs per SM: "pnb<NB>_s<S>_d<D>_k<K>_ka"
#define HERS_TVP(NB, S, D, K) \
    {"pnb" #NB "_s" #S "_d" #D "_k" #K "_ka", k_tensor_persist<NB, S, D, K, true>, NB, S, D, false, K}
// and with the four products: "pnb<NB>_s<S>_d<D>_k<K>"
#define HERS_TVQ(NB, S, D, K) \
    {"pnb" #NB "_s" #S "_d" #D "_k" #K, k_tensor_persist<NB, S, D, K, false>, NB, S, D, false, K}
// persistent Karatsuba form, K CTAs per SM, registers budgeted for M CTAs per
// SM (M > K: fewer registers, more left to another kernel beside it)
#define HERS_TVR(NB, S, D, K, M) \
    {"pnb" #NB "_s" #S "_d" #D "_k" #K "_m" #M "_ka", k_tensor_persist<NB, S, D, M, true>, NB, S, D, false, K}
static const TensorVariant kTensorVariants[] = {
    HERS_TV(2, 4, 4, 2),  HERS_TV(2, 3, 4, 3),  HERS_TV(2, 2, 8, 2),  HERS_TV(1, 4, 4, 3),
    HERS_TV(4, 2, 4, 2),  HERS_TV(2, 4, 2, 3),  HERS_TV(2, 2, 4, 4),  HERS_TV(1, 2, 8, 3),
    HERS_TV(4, 2, 2, 3),  HERS_TVG(2, 3, 4, 3), HERS_TVG(2, 4, 4, 2), HERS_TVG(1, 4, 4, 3),
    // one CTA per SM with a deep ring: an SM keeps registers and shared memory
    // for CTAs of another search's epilogue running beside it
    HERS_TV(2, 6, 4, 1),  HERS_TV(2, 8, 4, 1),  HERS_TV(4, 4, 4, 1),
    HERS_TVK(2, 3, 4, 3, true, "g"), HERS_TVK(2, 4, 4, 2, true, "g"), HERS_TVK(1, 4, 4, 3, true, "g"),
    HERS_TVK(2, 3, 4, 3, false, ""), HERS_TVK(2, 4, 4, 2, false, ""), HERS_TVK(2, 4, 2, 3, false, ""),
    HERS_TVP(2, 3, 4, 2), HERS_TVP(2, 4, 4, 2), HERS_TVP(2, 2, 4, 2), HERS_TVP(2, 2, 4, 3),
    HERS_TVP(1, 4, 4, 2), HERS_TVP(4, 2, 4, 2), HERS_TVP(2, 6, 4, 1),
    HERS_TVP(2, 3, 2, 2), HERS_TVP(2, 4, 2, 2), HERS_TVP(2, 5, 2, 2), HERS_TVP(1, 3, 4, 3),
    HERS_TVQ(2, 3, 4, 2), HERS_TVR(2, 3, 4, 2, 4), HERS_TVR(2, 3, 4, 2, 3),
};
#undef HERS_TV
#undef HERS_TVG
#undef HERS_TVK
#undef HERS_TVP
#undef HERS_TVQ
#undef HERS_TVR
constexpr int NUM_TENSOR_VARIANTS = sizeof(kTensorVariants) / sizeof(kTensorVariants[0]);

int tensor_variant_count() { return NUM_TENSOR_VARIANTS; }
const char* tensor_variant_name(int v) {
    return (v >= 0 && v < NUM_TENSOR_VARIANTS) ? kTensorVariants[v].name : nullptr;
}

// X: accumulators [nblocks][3][NUM_S][N] (uint32, residues in [0, r_l)).
cudaError_t launch_tensor(int variant, const uint64_t* gallery, uint64_t nblocks, uint32_t d,
                          const uint64_t* probe, uint32_t* X, int* err, cudaStream_t st) {
    if (variant < 0 || variant >= NUM_TENSOR_VARIANTS) return cudaErrorInvalidValue;
    const TensorVariant& v = kTensorVariants[variant];
    const int smem = v.stages * (1 + v.nb) * v.dps * 2 * TILE * 4;
    cudaError_t e = cudaFuncSetAttribute(v.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    if (v.persist > 0) {
        int dev = 0, sms = 0, occ = 0;
        e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, v.fn, TILE + 32, smem);
        if (e != cudaSuccess) return e;
        if (occ < 1) return cudaErrorInvalidConfiguration;
        const uint64_t nunits = (nblocks + v.nb - 1) / v.nb * NUM_S * NTILES;
        const uint64_t want = (uint64_t)sms * (uint64_t)(v.persist < occ ? v.persist : occ);
        const unsigned grid = (unsigned)(nunits < want ? nunits : want);
        v.fn<<<grid, TILE + 32, smem, st>>>((const int32_t*)gallery, (const int32_t*)probe, X, nblocks, d, err);
        count_launches(1);
        return cudaGetLastError();
    }
    const uint64_t max_groups = v.gorder ? 0x7FFFFFFFull : 65535ull;  // grid x or z limit
    const uint64_t max_z = max_groups * v.nb;
    for (uint64_t g0 = 0; g0 < nblocks; g0 += max_z) {
        const uint64_t nb = nblocks - g0 < max_z ? nblocks - g0 : max_z;
        const unsigned groups = (unsigned)((nb + v.nb - 1) / v.nb);
        const dim3 grid = v.gorder ? dim3(groups, NTILES * NUM_S, 1) : dim3(NTILES, NUM_S, groups);
        v.fn<<<grid, TILE + 32, smem, st>>>((const int32_t*)(gallery + g0 * RES_WORDS_PER_DIM * d),
                                            (const int32_t*)probe, X + g0 * 3 * NUM_S * N, nb, d, err);
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

// Inverse NTTs over the search basis: polynomial P of [npolys][N] uint32 is
// mod r_(P % NUM_S).  Each thread loads its 16 phase-one coefficients (16 t ..
// 16 t + 15, four 16-byte loads) and stores its 16 outputs (t + 256 a,
// coalesced) directly; shared memory carries only the middle phase.
// LEAN: a register budget for 5 CTAs per SM (48 registers) instead of 4, so
// that more CTAs fit beside the persistent tensor kernel of a search in flight.
template <bool SHFL, bool LEAN = false>
__global__ void __launch_bounds__(NTT_THREADS, LEAN ? 5 : 4) k_intt32_batch(const uint64_t* __restrict__ tw,
                                                              uint32_t* __restrict__ data) {
    __shared__ uint32_t sm32[N];
    const uint64_t P = blockIdx.x;
    const int mi = (int)(P % NUM_S);
    const int t = threadIdx.x;
    uint32_t* g = data + P * N;
    uint32_t v[16];
    const uint4* g4 = (const uint4*)(g + 16 * t);
#pragma unroll
    for (int i = 0; i < 4; i++) {
        const uint4 u = g4[i];
        v[4 * i] = u.x;
        v[4 * i + 1] = u.y;
        v[4 * i + 2] = u.z;
        v[4 * i + 3] = u.w;
    }
    ntt32_inv_regs<SHFL>(v, sm32, tw32_inv(tw, mi), c_smod[mi], c_sninv[mi], c_sninv_s[mi], t);
#pragma unroll
    for (int a = 0; a < 16; a++) g[t + 256 * a] = v[a];
}

// ---------------------------------------------------------------- exact scale-and-round
//
// Thread per (b, poly c, k).  X has residues x_l = X mod r_l, |X| < 2^236.
// With X' = X + q 2^129 = sum_i y_i M_i - alpha M (crt_y) and, per plaintext
// modulus, t M_i = A_i q + B_i and t M = A_M q + B_M:
//   round(t X / q) = floor((t X + (q-1)/2) / q)            (q odd: no tie)
//                  = sum_i y_i A_i - alpha A_M - 8 + floor(R / q) - t 2^129,
//   R = sum_i y_i B_i - alpha B_M + (q-1)/2 + 8 q   (0 < R < 2^142).
// R is formed from 27-bit digit columns (column sums below 2^61); floor(R / q)
// is estimated from floor(R / 2^80) times floor(2^144 / q) to within one and
// corrected with the exact remainder R - Q q, computed mod 2^128 (it lies in
// (-q, 2q)).  The result mod q_l then follows from the digits of A_i mod q_l.
// Writes c to C[b][c][l][N] and, for c = 2, the relinearisation digits
// D_1 = c2 mod q1, D_2 = c2 mod q2 reduced into both limbs:
// KS[b][0] = D_1 mod q1, [1] = D_1 mod q2, [2] = D_2 mod q1, [3] = D_2 mod q2.
// PM: the context's plaintext modulus entry, a template argument so that the
// digit tables are read as constant operands at fixed offsets.
template <int PM>
__device__ __forceinline__ void scale_round_coeff(const uint32_t xv[NUM_S], uint64_t out[2]) {
    const PlainMod& P = c_plain[PM];
    uint32_t y[NUM_S];
    const uint32_t alpha = crt_y(xv, y);

    int64_t col[4];
#pragma unroll
    for (int w = 0; w < 4; w++) {
        uint64_t s = 0;
#pragma unroll
        for (int i = 0; i < NUM_S; i++) s += (uint64_t)y[i] * P.b_cols[i * 4 + w];
        col[w] = (int64_t)s - (int64_t)alpha * P.bm_cols[w];
    }
    typedef unsigned __int128 u128;
    const u128 K = ((u128)KROUND_HI << 64) | KROUND_LO;
    const u128 Rm = (u128)(__int128)col[0] + ((u128)(__int128)col[1] << 27) + ((u128)(__int128)col[2] << 54) +
                    ((u128)(__int128)col[3] << 81) + K;  // R mod 2^128
    const int64_t Rs = col[3] * 2 + (col[2] >> 26) + (col[1] >> 53) + (int64_t)(KROUND_HI >> 16);
    uint64_t Q = __umul64hi((uint64_t)Rs, MU_Q144);
    const u128 qq = ((u128)Q_HI << 64) | Q_LO;
    const __int128 rem = (__int128)(Rm - (u128)Q * qq);
    if (rem < 0) Q--;
    else if (rem >= (__int128)qq) Q++;
#pragma unroll
    for (int l = 0; l < 2; l++) out[l] = crt_combine_q(y, alpha, P.a_cols, P.am_cols, l, (int64_t)Q - (int64_t)P.dshift[l]);
}

// Writes c's two limbs to C[b][c][l][N] at k and, for c = 2, the
// relinearisation digits KS[b][0..3] (see k_scale_round).
__device__ __forceinline__ void store_scaled(uint64_t* __restrict__ C, uint64_t* __restrict__ KS, uint64_t b, int c,
                                             int k, const uint64_t out[2]) {
#pragma unroll
    for (int l = 0; l < 2; l++) C[((b * 3 + c) * 2 + l) * N + k] = out[l];
    if (c == 2) {
        uint64_t* ks = KS + b * 4 * N + k;
        ks[0] = out[0];
        ks[N] = csub(out[0], c_mod[1]);
        ks[2 * N] = out[1];
        ks[3 * N] = out[1];
    }
}

template <int PM>
__global__ void __launch_bounds__(256) k_scale_round(const uint32_t* __restrict__ X,
                                                     uint64_t* __restrict__ C,
                                                     uint64_t* __restrict__ KS) {
    const int k = blockIdx.x * 256 + threadIdx.x;
    const int c = blockIdx.y;
    const uint64_t b = blockIdx.z;
    const uint32_t* x = X + ((b * 3 + c) * NUM_S) * N + k;
    uint32_t xv[NUM_S];
#pragma unroll
    for (int l = 0; l < NUM_S; l++) xv[l] = x[(size_t)l * N];
    uint64_t out[2];
    scale_round_coeff<PM>(xv, out);
    store_scaled(C, KS, b, c, k, out);
}

// The inverse NTTs and the scale-and-round in one kernel.  A cluster of NUM_S
// CTAs takes one accumulator polynomial (block b, component c): CTA rank l
// undoes the NTT mod r_l (k_intt32_batch's schedule) and keeps the
// coefficients in its shared memory; after a cluster barrier each CTA
// rounds N / NUM_S coefficients, reading their eight residues from the eight
// CTAs' shared memory (distributed shared memory).  The X accumulators are
// read once and not written back.  A second cluster barrier keeps every CTA's
// shared memory alive until its peers' reads are done.
constexpr int ISC_SLICE = N / NUM_S;  // coefficients rounded per CTA
static_assert(ISC_SLICE == 2 * NTT_THREADS, "two coefficients per thread");
template <int PM, bool SHFL>
__global__ void __cluster_dims__(NUM_S, 1, 1) __launch_bounds__(NTT_THREADS, 4)
    k_intt_scale_cluster(const uint64_t* __restrict__ tw, const uint32_t* __restrict__ X,
                         uint64_t* __restrict__ C, uint64_t* __restrict__ KS) {
    namespace cg = cooperative_groups;
    __shared__ uint32_t sm32[N];
    const cg::cluster_group cluster = cg::this_cluster();
    const int l = (int)cluster.block_rank();
    const int c = blockIdx.y;
    const uint64_t b = blockIdx.z;
    const int t = threadIdx.x;
    const uint32_t* g = X + ((b * 3 + c) * NUM_S + l) * N;
    uint32_t v[16];
    const uint4* g4 = (const uint4*)(g + 16 * t);
#pragma unroll
    for (int i = 0; i < 4; i++) {
        const uint4 u = g4[i];
        v[4 * i] = u.x;
        v[4 * i + 1] = u.y;
        v[4 * i + 2] = u.z;
        v[4 * i + 3] = u.w;
    }
    ntt32_inv_regs<SHFL>(v, sm32, tw32_inv(tw, l), c_smod[l], c_sninv[l], c_sninv_s[l], t);
    __syncthreads();  // the transform's last shared-memory reads are done
#pragma unroll
    for (int a = 0; a < 16; a++) sm32[t + 256 * a] = v[a];  // natural order, fully reduced
    cluster.sync();
#pragma unroll
    for (int h = 0; h < 2; h++) {
        const int k = l * ISC_SLICE + h * NTT_THREADS + t;
        uint32_t xv[NUM_S];
#pragma unroll
        for (int i = 0; i < NUM_S; i++) xv[i] = *cluster.map_shared_rank(sm32 + k, i);
        uint64_t out[2];
        scale_round_coeff<PM>(xv, out);
        store_scaled(C, KS, b, c, k, out);
    }
    cluster.sync();
}

// ---------------------------------------------------------------- key switch
// RNS gadget (Alg 5's relinearisation with one digit per prime): for output
// c = 0, 1 and limb l, O_cl = sum_j D_j evk_j[c][l], D_j = c2 mod q_j.
// k_ks_fwd_mul: CTA per (b, j, l) = row of KS: D_j mod q_l to the NTT domain,
// times evk_j[c][l] (NTT values with Shoup companions) for both c, into
// P[b][j][c][l] (reduced).  k_ks_inv_finish: CTA per (b, c, l):
// P[b][0][c][l] + P[b][1][c][l] back to coefficients, plus C[b][c][l], into
// out[b][c][l].  LEAN: a register budget for 4 CTAs per SM instead of 3 (as
// for k_intt32_batch).  SHFL: the NTTs' in-warp exchange by shuffles.
template <bool LEAN, bool SHFL = false>
__global__ void __launch_bounds__(NTT_THREADS, LEAN ? 4 : 3) k_ks_fwd_mul(const uint64_t* __restrict__ tw,
                                                            const uint64_t* __restrict__ KS,
                                                            const uint64_t* __restrict__ evk_ntt,
                                                            uint64_t* __restrict__ P) {
    extern __shared__ uint64_t sm[];
    const uint64_t x = blockIdx.x;  // (b * 2 + j) * 2 + l
    const uint64_t b = x >> 2;
    const int j = (int)((x >> 1) & 1), l = (int)(x & 1);
    const uint64_t q = c_mod[l];
    const uint64_t* src = KS + x * N;
    for (int k = threadIdx.x; k < N; k += blockDim.x) sm[swz(k)] = src[k];
    ntt_fwd_mod<SHFL>(sm, tw, l);
#pragma unroll
    for (int c = 0; c < 2; c++) {
        const uint64_t* e = evk_ntt + (size_t)(((j * 2 + c) * 2 + l) * 2) * N;
        uint64_t* dst = P + (((b * 2 + j) * 2 + c) * 2 + l) * N;
        for (int k = threadIdx.x; k < N; k += blockDim.x) dst[k] = shoup(sm[swz(k)], e[k], e[N + k], q);
    }
}

template <bool LEAN, bool SHFL = false>
__global__ void __launch_bounds__(NTT_THREADS, LEAN ? 4 : 3) k_ks_inv_finish(const uint64_t* __restrict__ tw,
                                                               const uint64_t* __restrict__ P,
                                                               const uint64_t* __restrict__ C,
                                                               uint64_t* __restrict__ out) {
    extern __shared__ uint64_t sm[];
    const uint64_t x = blockIdx.x;  // (b * 2 + c) * 2 + l
    const uint64_t b = x >> 2;
    const int c = (int)((x >> 1) & 1), l = (int)(x & 1);
    const uint64_t q = c_mod[l];
    const uint64_t* p0 = P + (((b * 2 + 0) * 2 + c) * 2 + l) * N;
    const uint64_t* p1 = P + (((b * 2 + 1) * 2 + c) * 2 + l) * N;
    for (int k = threadIdx.x; k < N; k += blockDim.x) sm[swz(k)] = add_mod(p0[k], p1[k], q);
    ntt_inv_mod<SHFL>(sm, tw, l);
    const uint64_t* cc = C + ((b * 3 + c) * 2 + l) * N;
    for (int k = threadIdx.x; k < N; k += blockDim.x) out[x * N + k] = add_mod(cc[k], sm[swz(k)], q);
}

// The key switch in one kernel: CTA per (b, l), two groups of NTT_THREADS
// threads.  Group j takes D_j mod q_l (row (b, j, l) of KS) to the NTT
// domain; then group c forms O_cl = D_0 evk_0[c][l] + D_1 evk_1[c][l] from
// both transformed digits, undoes its NTT and adds C[b][c][l] into
// out[b][c][l].  No intermediate leaves shared memory.
__global__ void __launch_bounds__(2 * NTT_THREADS, 1) k_ks_fused(const uint64_t* __restrict__ tw,
                                                             const uint64_t* __restrict__ KS,
                                                             const uint64_t* __restrict__ evk_ntt,
                                                             const uint64_t* __restrict__ C,
                                                             uint64_t* __restrict__ out) {
    extern __shared__ uint64_t sm[];
    const uint64_t b = blockIdx.x >> 1;
    const int l = (int)(blockIdx.x & 1);
    const int grp = threadIdx.x / NTT_THREADS, t = threadIdx.x % NTT_THREADS;
    const uint64_t q = c_mod[l];
    uint64_t* s = sm + grp * N;
    const uint64_t* src = KS + ((b * 2 + grp) * 2 + l) * N;
    for (int k = t; k < N; k += NTT_THREADS) s[swz(k)] = src[k];
    ntt_fwd_smem(s, tw_fwd(tw, l), q, c_one_s[l], t);
    const uint64_t* e0 = evk_ntt + (size_t)(((0 * 2 + grp) * 2 + l) * 2) * N;
    const uint64_t* e1 = evk_ntt + (size_t)(((1 * 2 + grp) * 2 + l) * 2) * N;
    uint64_t o[16];
#pragma unroll
    for (int a = 0; a < 16; a++) {
        const int k = t + NTT_THREADS * a, x = swz(k);
        o[a] = add_mod(shoup(sm[x], e0[k], e0[N + k], q), shoup(sm[N + x], e1[k], e1[N + k], q), q);
    }
    __syncthreads();  // both groups are done reading both digits
#pragma unroll
    for (int a = 0; a < 16; a++) s[swz(t + NTT_THREADS * a)] = o[a];
    ntt_inv_smem(s, tw_inv(tw, l), q, c_ninv[l], c_ninv_s[l], t);
    const uint64_t* cc = C + ((b * 3 + grp) * 2 + l) * N;
    uint64_t* dst = out + ((b * 2 + grp) * 2 + l) * N;
    for (int k = t; k < N; k += NTT_THREADS) dst[k] = add_mod(cc[k], s[swz(k)], q);
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

// ---------------------------------------------------------------- pipeline
// Epilogue over npairs (probe, block) pairs whose accumulators are in X as
// uint32 [npairs][3][NUM_S][N] (NTT domain): inverse NTTs, exact
// scale-and-round into C [npairs][3][2][N] and KS [npairs][4][N], key switch
// (its intermediates reuse the X area: the partial products P [npairs][8][N],
// or with the base-w gadget O [npairs][2][2][N] and the digits), canonical
// score ciphertexts into out [npairs][2][2][N].
const char* epilogue_variant_name(int v) {
    // the base form (flags 1, 2), then "+shfl", "+lean", "+ksshfl" for flags 4, 8, 16
    static const std::vector<std::string> names = [] {
        static const char* base[4] = {"split", "intt_scale_cluster", "ks_fused", "intt_scale_cluster+ks_fused"};
        std::vector<std::string> n;
        for (int f = 0; f < EPI_VARIANTS; f++)
            n.push_back(std::string(base[f & 3]) + ((f & EPI_INTT_SHFL) ? "+shfl" : "") +
                        ((f & EPI_LEAN) ? "+lean" : "") + ((f & EPI_KS_SHFL) ? "+ksshfl" : ""));
        return n;
    }();
    return (v >= 0 && v < EPI_VARIANTS) ? names[v].c_str() : nullptr;
}

cudaError_t launch_epilogue(const uint64_t* tw, const DevKeys& k, uint64_t npairs, uint64_t* X,
                            uint64_t* C, uint64_t* KS, uint64_t* out, cudaStream_t st,
                            cudaEvent_t* ev, const KeySwitchW* ksw, int epi) {
    uint64_t nl = 0;
    uint64_t* O = X;
    uint32_t* X32 = (uint32_t*)X;  // accumulators [npairs][3][NUM_S][N]
    const uint64_t max_z = 65535;
    const uint64_t chunk = 1u << 30;
    if (epi & EPI_INTT_SCALE_CLUSTER) {
        // inverse NTTs and scale-and-round in one kernel (clusters of NUM_S CTAs)
        for (uint64_t b0 = 0; b0 < npairs; b0 += max_z) {
            const uint64_t nb = npairs - b0 < max_z ? npairs - b0 : max_z;
            const dim3 grid(NUM_S, 3, (unsigned)nb);
            const uint32_t* x = X32 + b0 * 3 * NUM_S * N;
            uint64_t* c = C + b0 * 6 * N;
            uint64_t* ks = KS + b0 * 4 * N;
            const bool sh = (epi & EPI_INTT_SHFL) != 0;
            if (k.pm == 0 && !sh) k_intt_scale_cluster<0, false><<<grid, NTT_THREADS, 0, st>>>(tw, x, c, ks);
            else if (k.pm == 0) k_intt_scale_cluster<0, true><<<grid, NTT_THREADS, 0, st>>>(tw, x, c, ks);
            else if (!sh) k_intt_scale_cluster<1, false><<<grid, NTT_THREADS, 0, st>>>(tw, x, c, ks);
            else k_intt_scale_cluster<1, true><<<grid, NTT_THREADS, 0, st>>>(tw, x, c, ks);
            nl++;
        }
        if (ev) {
            cudaEventRecord(ev[0], st);
            cudaEventRecord(ev[1], st);
        }
    } else {
        const uint64_t npolys = npairs * 3 * NUM_S;  // chunks are multiples of NUM_S
        for (uint64_t off = 0; off < npolys; off += chunk) {
            const uint64_t n = npolys - off < chunk ? npolys - off : chunk;
            const bool sh = (epi & EPI_INTT_SHFL) != 0, lean = (epi & EPI_LEAN) != 0;
            if (sh && lean) k_intt32_batch<true, true><<<(unsigned)n, NTT_THREADS, 0, st>>>(tw, X32 + off * N);
            else if (sh) k_intt32_batch<true><<<(unsigned)n, NTT_THREADS, 0, st>>>(tw, X32 + off * N);
            else if (lean) k_intt32_batch<false, true><<<(unsigned)n, NTT_THREADS, 0, st>>>(tw, X32 + off * N);
            else k_intt32_batch<false><<<(unsigned)n, NTT_THREADS, 0, st>>>(tw, X32 + off * N);
            nl++;
        }
        if (ev) cudaEventRecord(ev[0], st);
        for (uint64_t b0 = 0; b0 < npairs; b0 += max_z) {
            const uint64_t nb = npairs - b0 < max_z ? npairs - b0 : max_z;
            const dim3 grid(N / 256, 3, (unsigned)nb);
            if (k.pm == 0)
                k_scale_round<0><<<grid, 256, 0, st>>>(X32 + b0 * 3 * NUM_S * N, C + b0 * 6 * N, KS + b0 * 4 * N);
            else
                k_scale_round<1><<<grid, 256, 0, st>>>(X32 + b0 * 3 * NUM_S * N, C + b0 * 6 * N, KS + b0 * 4 * N);
            nl++;
        }
        if (ev) cudaEventRecord(ev[1], st);
    }
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
    } else if (epi & EPI_KS_FUSED) {
        // RNS gadget, one kernel per (pair, limb)
        cudaFuncSetAttribute(k_ks_fused, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * N * 8);
        for (uint64_t off = 0; off < npairs * 2; off += chunk) {  // chunk: an even number of rows
            const uint64_t n = npairs * 2 - off < chunk ? npairs * 2 - off : chunk;
            k_ks_fused<<<(unsigned)n, 2 * NTT_THREADS, 2 * N * 8, st>>>(tw, KS + off * 2 * N, k.evk_ntt,
                                                                       C + off / 2 * 6 * N, out + off * 2 * N);
            nl++;
        }
    } else {
        // RNS gadget: partial products P [npairs][2 j][2 c][2 l][N] in the X area
        uint64_t* P = X;
        for (uint64_t off = 0; off < npairs * 4; off += chunk) {  // chunk: a multiple of 4 rows
            const uint64_t n = npairs * 4 - off < chunk ? npairs * 4 - off : chunk;
            const uint64_t* ks = KS + off * N;
            uint64_t* pp = P + off * 2 * N;
            const bool lean = (epi & EPI_LEAN) != 0, sh = (epi & EPI_KS_SHFL) != 0;
            if (lean && sh) k_ks_fwd_mul<true, true><<<(unsigned)n, NTT_THREADS, N * 8, st>>>(tw, ks, k.evk_ntt, pp);
            else if (lean) k_ks_fwd_mul<true><<<(unsigned)n, NTT_THREADS, N * 8, st>>>(tw, ks, k.evk_ntt, pp);
            else if (sh) k_ks_fwd_mul<false, true><<<(unsigned)n, NTT_THREADS, N * 8, st>>>(tw, ks, k.evk_ntt, pp);
            else k_ks_fwd_mul<false><<<(unsigned)n, NTT_THREADS, N * 8, st>>>(tw, ks, k.evk_ntt, pp);
            nl++;
        }
        for (uint64_t off = 0; off < npairs * 4; off += chunk) {
            const uint64_t n = npairs * 4 - off < chunk ? npairs * 4 - off : chunk;
            const uint64_t* pp = P + off * 2 * N;
            const uint64_t* cc = C + off / 4 * 6 * N;
            uint64_t* o = out + off * N;
            const bool lean = (epi & EPI_LEAN) != 0, sh = (epi & EPI_KS_SHFL) != 0;
            if (lean && sh) k_ks_inv_finish<true, true><<<(unsigned)n, NTT_THREADS, N * 8, st>>>(tw, pp, cc, o);
            else if (lean) k_ks_inv_finish<true><<<(unsigned)n, NTT_THREADS, N * 8, st>>>(tw, pp, cc, o);
            else if (sh) k_ks_inv_finish<false, true><<<(unsigned)n, NTT_THREADS, N * 8, st>>>(tw, pp, cc, o);
            else k_ks_inv_finish<false><<<(unsigned)n, NTT_THREADS, N * 8, st>>>(tw, pp, cc, o);
            nl++;
        }
    }
    count_launches(nl);
    return cudaGetLastError();
}

// Workspace per block (64-bit words): X, 15 N, holding the accumulators
// [3][NUM_S][N] as uint32 (12 N words), later the key switch's intermediates
// (8 N words); C [3][2][N]; KS [4][N].
cudaError_t launch_search(const uint64_t* tw, const DevKeys& k, const uint64_t* gallery,
                          uint64_t nblocks, uint32_t d, const uint64_t* probe, uint64_t* scores_ct,
                          uint64_t* ws, int* err, cudaStream_t st, cudaEvent_t* ev, int variant,
                          const KeySwitchW* ksw, const EpilogueStream* ep, int epi) {
    if (nblocks == 0) return cudaSuccess;
    uint64_t* X = ws;
    uint64_t* C = X + nblocks * 15 * N;
    uint64_t* KS = C + nblocks * 6 * N;
    if (ev) cudaEventRecord(ev[0], st);
    if (ep && ep->tensor_first) {
        // the tensor kernel on the high-priority stream, the epilogue on st
        cudaError_t e = cudaEventRecord(ep->ev[0], st);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(ep->stream, ep->ev[0], 0);
        if (e == cudaSuccess) e = launch_tensor(variant, gallery, nblocks, d, probe, (uint32_t*)X, err, ep->stream);
        if (e == cudaSuccess && ev) e = cudaEventRecord(ev[1], ep->stream);
        if (e == cudaSuccess) e = cudaEventRecord(ep->ev[1], ep->stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(st, ep->ev[1], 0);
        if (e != cudaSuccess) return e;
        e = launch_epilogue(tw, k, nblocks, X, C, KS, scores_ct, st, ev ? ev + 2 : nullptr, ksw, epi);
        if (ev) cudaEventRecord(ev[4], st);
        return e;
    }
    cudaError_t e = launch_tensor(variant, gallery, nblocks, d, probe, (uint32_t*)X, err, st);
    if (e != cudaSuccess) return e;
    if (ev) cudaEventRecord(ev[1], st);
    cudaStream_t es = st;
    if (ep) {
        e = cudaEventRecord(ep->ev[0], st);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(ep->stream, ep->ev[0], 0);
        if (e != cudaSuccess) return e;
        es = ep->stream;
    }
    e = launch_epilogue(tw, k, nblocks, X, C, KS, scores_ct, es, ev ? ev + 2 : nullptr, ksw, epi);
    if (ev) cudaEventRecord(ev[4], es);
    if (ep) {
        cudaError_t ej = cudaEventRecord(ep->ev[1], es);
        if (ej == cudaSuccess) ej = cudaStreamWaitEvent(st, ep->ev[1], 0);
        if (e == cudaSuccess) e = ej;
    }
    return e;
}

}  // namespace hers
