// Batched encrypted search: many probes against uneven gallery subsets of
// mixed dimensionality in one persistent launch, captured with the rest of
// the pipeline as a single CUDA graph (Alg 7's server loop for many probes at
// once; the result for every (probe, block) pair is the one hers_search gives).
//
// Items (probe, subset) that share a resident gallery form a group.  A group's
// probes are cut into chunks of G NP; a work unit is (chunk, block, limb,
// tile).  The persistent tensor kernel's producer warp claims units from an
// atomic counter and streams, per stage, the chunk's probe rows and the
// block's gallery rows into a shared-memory ring (cp.async.bulk + mbarriers,
// as in k_tensor).  The CTA's G groups of consumers each take NP of the
// chunk's probes against the one copy of the gallery rows, so each gallery
// byte read from HBM serves up to G NP probes.  The epilogue (inverse NTTs,
// exact scale-and-round, key switch) then runs over all pairs.
#include <stdio.h>

#include <algorithm>
#include <map>
#include <new>
#include <utility>
#include <vector>

#include "common.cuh"
#include "hers.h"
#include "internal.h"

namespace hers {

constexpr uint32_t UNIT_STOP = 0xFFFFFFFFu;
// Partial-fold periods in dimensions: the Karatsuba sums S (products below
// 2^60) every BPFOLD_S, T0 and T2 (below 2^58) every BPFOLD_02.  A folded sum
// is below 2^61 + 2^32, so 4 more S products stay below 7 2^60 + 2^32 and 16
// more T0/T2 products below 2^62 + 2^61 + 2^32, both inside a signed 64-bit.
constexpr int BPFOLD_S = 4;
constexpr int BPFOLD_02 = 16;

// Stage descriptor word: dimensions (8 bits), probes (5), blocks (4), limb
// (4), flags (5).
constexpr int HD_NP = 8, HD_NB = 13, HD_LIMB = 17, HD_FLAGS = 21;
// Stage descriptor flags (written by the producer with each stage).
constexpr uint32_t F_FIRST = 1;  // first stage of a unit: sums start at zero
constexpr uint32_t F_FOLD = 2;   // partial fold of the S sums after this stage
constexpr uint32_t F_LAST = 4;   // last stage of a unit: store the unit's results
constexpr uint32_t F_STOP = 8;   // no more units: the consumers leave
constexpr uint32_t F_FOLD02 = 16;  // partial fold of the T0 and T2 sums after this stage

__device__ __forceinline__ void madw_b(int64_t& acc, int32_t a, int32_t b) {
    asm("mad.wide.s32 %0, %1, %2, %0;" : "+l"(acc) : "r"(a), "r"(b));
}

// The same signed 64-bit multiply-accumulate as a carry chain: the low words
// of the product and the sum with carry out, then the signed high word of the
// product plus the carry, so no separate 64-bit add follows the multiply.
__device__ __forceinline__ void madc_b(int64_t& acc, int32_t a, int32_t b) {
    uint32_t lo = (uint32_t)acc, hi = (uint32_t)((uint64_t)acc >> 32);
    asm("mad.lo.cc.u32 %0, %2, %3, %0;\n\t"
        "madc.hi.s32 %1, %2, %3, %1;"
        : "+r"(lo), "+r"(hi)
        : "r"(a), "r"(b));
    acc = (int64_t)(((uint64_t)hi << 32) | lo);
}

template <bool CC>
__device__ __forceinline__ void mac_b(int64_t& acc, int32_t a, int32_t b) {
    if (CC) madc_b(acc, a, b);
    else madw_b(acc, a, b);
}

// A unit's table entries.  The scalars stay in the producer's registers; the
// probe pointers and output pairs (NPC = G NP of each) go to a shared-memory
// slot, so the producer's register count does not grow with the chunk size.
struct UnitRegs {
    const uint64_t* gallery;
    uint32_t d, np, nb, block, limb, tile;
    bool last;  // the last chunk to read these gallery rows
};

// Unit u's table entries: the segment holding u (binary search over the
// segments' first units), then u's chunk, block group, limb and tile within it.
template <int NPC, int NB>
__device__ __forceinline__ void load_unit(UnitRegs& r, const uint64_t** probe_slot, uint64_t* pair_slot,
                                          const BatchChunk* __restrict__ chunks,
                                          const BatchSeg* __restrict__ segs, uint32_t nsegs, uint32_t u) {
    uint32_t lo = 0, hi = nsegs - 1;
    while (lo < hi) {
        const uint32_t mid = (lo + hi + 1) >> 1;
        if (segs[mid].first_unit <= u) lo = mid;
        else hi = mid - 1;
    }
    const BatchSeg S = segs[lo];
    uint32_t x = u - S.first_unit;
    const uint32_t c = x % S.nch;
    x /= S.nch;
    const uint32_t bg = x % S.nbg;
    x /= S.nbg;
    const BatchChunk* C = chunks + S.first_chunk + c;
    r.gallery = C->gallery;
    r.d = C->d;
    r.np = C->np;
    r.block = S.s0 + bg * NB;
    r.nb = min((uint32_t)NB, S.s1 - r.block);
    r.last = c + 1 == S.nch;
    r.tile = x % NTILES;
    r.limb = x / NTILES;
#pragma unroll
    for (int q = 0; q < NPC; q++) {  // entries past np are zero in the table
        probe_slot[q] = C->probe[q];
        pair_slot[q] = C->pair[q] + r.block;
    }
}

// One stage's products into the 64-bit sums: for dd < nd, probe q < np,
// block j < nb, the tensor of (probe row q) x (gallery row j) (centred int32
// residues, see k_tensor) by Karatsuba's three products: T0 += a0 g0,
// T2 += a1 g1 and S += (a0 + a1)(g0 + g1), so that the middle component
// a0 g1 + a1 g0 of Alg 5's tensor is S - T0 - T2 (formed mod r_l at the end).
// The sums a0 + a1 and g0 + g1 are below r < 2^30 in magnitude, their
// product below 2^60.  With FULL (nd = DPS, np = NP, nb = NB) the loops carry
// no predicates.
// pb: this group's first probe run; gb: the first gallery run (both already
// offset to the thread's coefficient).
template <int NP, int NB, int DPS, bool FULL, bool CC>
__device__ __forceinline__ void stage_products(int64_t (&s)[NP][NB][3], const int2* pb, const int2* gb,
                                               uint32_t nd, uint32_t np, uint32_t nbu) {
    constexpr int RUN2 = DPS * TILE;  // (poly 0, poly 1) pairs of one run
#pragma unroll
    for (int dd = 0; dd < DPS; dd++) {
        if (FULL || (uint32_t)dd < nd) {
            int32_t a0[NP], a1[NP], as[NP];
#pragma unroll
            for (int q = 0; q < NP; q++) {
                const int2 A = pb[q * RUN2 + dd * TILE];
                a0[q] = A.x;
                a1[q] = A.y;
                as[q] = A.x + A.y;
            }
#pragma unroll
            for (int j = 0; j < NB; j++) {
                if (FULL || (uint32_t)j < nbu) {
                    const int2 G = gb[j * RUN2 + dd * TILE];
                    const int32_t g0 = G.x, g1 = G.y, gs = G.x + G.y;
#pragma unroll
                    for (int q = 0; q < NP; q++) {
                        if (FULL || (uint32_t)q < np) {
                            mac_b<CC>(s[q][j][0], a0[q], g0);
                            mac_b<CC>(s[q][j][1], as[q], gs);
                            mac_b<CC>(s[q][j][2], a1[q], g1);
                        }
                    }
                }
            }
        }
    }
}

// Persistent batched tensor kernel.  A CTA has G groups of TILE consumer
// threads (one coefficient each) and one producer warp.  The producer's
// elected lane claims units from the atomic counter one unit ahead (the claim
// and the unit's table reads overlap the current unit's stages), and for each
// stage writes a descriptor (dimensions, probes, blocks, limb, flags; on the
// last stage the output pairs) into shared memory before the stage's copies,
// so the consumers read no tables from global memory.  A stage holds the
// chunk's G NP probe runs, then NB gallery runs; group g takes probes
// g NP .. g NP + NP - 1 against every gallery run and keeps their NP x NB x 3
// sums of its coefficient in registers.

// POL selects the L2 policies of the copies: false, probe rows evict-last
// and gallery rows evict-first; true, probe rows evict-normal and gallery rows
// evict-normal except on the last chunk to read them (evict-first), so that
// the chunks of one block that follow the first find its rows in L2 and
// probe rows of finished (limb, tile) slices do not crowd them out.
// PF > 0: the producer also prefetches into L2 the gallery rows of the stage
// PF stages ahead (in this unit, or the first stages of the next one), so a
// stage's copy into shared memory finds them in L2 and the ring only has to
// cover L2 latency.
// CC: the multiply-accumulates as carry chains (madc_b) instead of mad.wide.
template <int NP, int NB, int STAGES, int DPS, int MINB, int G, bool POL, int PF = 0, bool CC = false>
__global__ void __launch_bounds__(G * TILE + 32, MINB)
    k_tensor_batched(const BatchChunk* __restrict__ chunks, const BatchSeg* __restrict__ segs, uint32_t nsegs,
                     uint32_t nunits, uint32_t* counter, uint32_t* __restrict__ X, int* err) {
    constexpr int NPC = G * NP;  // probes of a chunk
    static_assert(BPFOLD_S % DPS == 0 && BPFOLD_02 % BPFOLD_S == 0, "stages must not straddle a partial fold");
    static_assert(NPC <= BATCH_NPMAX && NPC < 32 && NB <= 15 && DPS <= 255 && NUM_S <= 16, "descriptor fields");
    static_assert(G * TILE + 32 <= 1024, "threads per CTA");
    extern __shared__ __align__(128) int32_t smr[];
    __shared__ __align__(8) uint64_t full[STAGES], empty[STAGES];
    __shared__ uint32_t hdr_info[STAGES], hdr_k0[STAGES];
    __shared__ uint64_t hdr_pair[STAGES][NPC];
    __shared__ const uint64_t* unit_probe[2][NPC];  // the producer's current and next unit
    __shared__ uint64_t unit_pair[2][NPC];
    constexpr int RUN = DPS * 2 * TILE;
    constexpr int STAGE_ELEMS = (NPC + NB) * RUN;  // NPC probe runs, then NB gallery runs
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; s++) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], G * TILE);  // every consumer thread arrives
        }
        mbar_fence_init();
    }
    __syncthreads();

    if (warp == G * TILE / 32) {  // producer warp
        if (lane == 0) {
            const uint64_t pol_first = policy_evict_first();
            const uint64_t pol_p = POL ? policy_evict_normal() : policy_evict_last();
            const uint64_t pol_keep = POL ? policy_evict_normal() : pol_first;
            uint32_t g = 0;  // stages issued by this CTA
            bool failed = false;
            uint32_t u = atomicAdd(counter, 1u);
            UnitRegs cur = {}, nxt = {};
            int cs = 0;  // shared-memory slot of the current unit's probes and pairs
            if (u < nunits) load_unit<NPC, NB>(cur, unit_probe[0], unit_pair[0], chunks, segs, nsegs, u);
            while (!failed) {
                const bool stop = u >= nunits;
                const uint32_t un = stop ? UNIT_STOP : atomicAdd(counter, 1u);  // next unit, claimed now
                const uint32_t nst = stop ? 1 : (cur.d + DPS - 1) / DPS;
                for (uint32_t si = 0; si < nst; si++, g++) {
                    const int st = (int)(g % STAGES);
                    if (g >= STAGES && !mbar_wait(&empty[st], ((g / STAGES) + 1) & 1)) {
                        atomicOr(err, 2);
                        failed = true;
                        break;
                    }
                    if (stop) {
                        hdr_info[st] = F_STOP << HD_FLAGS;
                        mbar_arrive(&full[st]);
                        continue;
                    }
                    const uint32_t nd = min((uint32_t)DPS, cur.d - si * DPS), done = si * DPS + nd;
                    const uint32_t flags = (si == 0 ? F_FIRST : 0u) |
                                           ((done % BPFOLD_S == 0 && done < cur.d) ? F_FOLD : 0u) |
                                           ((done % BPFOLD_02 == 0 && done < cur.d) ? F_FOLD02 : 0u) |
                                           (done == cur.d ? F_LAST : 0u);
                    hdr_info[st] = nd | (cur.np << HD_NP) | (cur.nb << HD_NB) | (cur.limb << HD_LIMB) |
                                   (flags << HD_FLAGS);
                    if (flags & F_LAST) {
                        hdr_k0[st] = cur.tile * TILE;
                        for (uint32_t q = 0; q < cur.np; q++) hdr_pair[st][q] = unit_pair[cs][q];
                    }
                    const uint32_t bytes = nd * 2 * TILE * 4;
                    int32_t* dst = smr + (size_t)st * STAGE_ELEMS;
                    const uint64_t pol_g = cur.last ? pol_first : pol_keep;
                    mbar_expect_tx(&full[st], bytes * (cur.np + cur.nb));
                    const uint64_t off = resident_offset(0, cur.limb, cur.tile * TILE, cur.d, 0, 0) +
                                         (uint64_t)si * RUN;
                    for (uint32_t q = 0; q < cur.np; q++)
                        bulk_g2s(dst + q * RUN, (const int32_t*)unit_probe[cs][q] + off, bytes, &full[st], pol_p);
#pragma unroll
                    for (int j = 0; j < NB; j++)
                        if ((uint32_t)j < cur.nb)
                            bulk_g2s(dst + (NPC + j) * RUN,
                                     (const int32_t*)cur.gallery +
                                         resident_offset(cur.block + j, cur.limb, cur.tile * TILE, cur.d, 0, 0) +
                                         (uint64_t)si * RUN,
                                     bytes, &full[st], pol_g);
                    // the next unit's tables, once this unit's first stage is on its way
                    if (si == 0 && un < nunits)
                        load_unit<NPC, NB>(nxt, unit_probe[cs ^ 1], unit_pair[cs ^ 1], chunks, segs, nsegs, un);
                    if (PF > 0) {
                        // gallery rows PF stages ahead into L2
                        const uint32_t ahead = si + PF;
                        const UnitRegs* pu = ahead < nst ? &cur : &nxt;
                        const uint32_t pst = ahead < nst ? ahead : ahead - nst;
                        if ((ahead < nst || un < nunits) && pst * DPS < pu->d) {
                            const uint32_t pnd = min((uint32_t)DPS, pu->d - pst * DPS);
#pragma unroll
                            for (int j = 0; j < NB; j++)
                                if ((uint32_t)j < pu->nb)
                                    bulk_prefetch_l2((const int32_t*)pu->gallery +
                                                         resident_offset(pu->block + j, pu->limb, pu->tile * TILE,
                                                                         pu->d, 0, 0) +
                                                         (uint64_t)pst * RUN,
                                                     pnd * 2 * TILE * 4);
                        }
                    }
                }
                if (stop) break;
                u = un;
                cur = nxt;
                cs ^= 1;
            }
            // drain: the copies of the last stages issued land before this thread leaves
            for (uint32_t i = g > STAGES ? g - STAGES : 0; i < g; i++)
                if (!mbar_wait(&full[i % STAGES], (i / STAGES) & 1)) atomicOr(err, 2);
        }
        return;
    }

    // consumers: group grp, coefficient t of the tile
    const int grp = G == 1 ? 0 : threadIdx.x / TILE;
    const int t = G == 1 ? threadIdx.x : threadIdx.x % TILE;
    int64_t s[NP][NB][3];
    for (uint32_t g = 0;; g++) {
        const int st = (int)(g % STAGES);
        if (!mbar_wait(&full[st], (g / STAGES) & 1)) {
            atomicOr(err, 2);
            return;
        }
        const uint32_t info = hdr_info[st];
        const uint32_t flags = info >> HD_FLAGS;
        if (flags & F_STOP) break;
        const uint32_t nd = info & 0xFF, npc = (info >> HD_NP) & 31, nbu = (info >> HD_NB) & 15;
        const int l = (int)((info >> HD_LIMB) & 15);
        // this group's probes of the chunk
        const uint32_t np = npc > (uint32_t)(grp * NP) ? min((uint32_t)NP, npc - grp * NP) : 0u;
        // what the last stage stores, read before the stage is handed back
        uint64_t opair[NP];
        uint32_t k0 = 0;
        if (flags & F_LAST) {
            k0 = hdr_k0[st];
#pragma unroll
            for (int q = 0; q < NP; q++) opair[q] = (uint32_t)q < np ? hdr_pair[st][grp * NP + q] : 0;
        }
        if (flags & F_FIRST) {
#pragma unroll
            for (int q = 0; q < NP; q++)
#pragma unroll
                for (int j = 0; j < NB; j++) s[q][j][0] = s[q][j][1] = s[q][j][2] = 0;
        }
        const int2* sbase = (const int2*)(smr + (size_t)st * STAGE_ELEMS) + t;  // (poly 0, poly 1) pairs
        const int2* pb = sbase + grp * NP * (RUN / 2);
        const int2* gb = sbase + NPC * (RUN / 2);
        if (nd == DPS && np == NP && nbu == NB)
            stage_products<NP, NB, DPS, true, CC>(s, pb, gb, nd, np, nbu);
        else if (np > 0)
            stage_products<NP, NB, DPS, false, CC>(s, pb, gb, nd, np, nbu);
        mbar_arrive(&empty[st]);
        if (flags & F_FOLD) {
            const int32_t r32 = (int32_t)c_sr32[l];
            const bool all = (flags & F_FOLD02) != 0;
#pragma unroll
            for (int q = 0; q < NP; q++)
#pragma unroll
                for (int j = 0; j < NB; j++) {
                    s[q][j][1] = pfold(s[q][j][1], r32);
                    if (all) {
                        s[q][j][0] = pfold(s[q][j][0], r32);
                        s[q][j][2] = pfold(s[q][j][2], r32);
                    }
                }
        }
        if (flags & F_LAST) {
            const uint32_t k = k0 + t;
#pragma unroll
            for (int q = 0; q < NP; q++)
                if ((uint32_t)q < np)
#pragma unroll
                    for (int j = 0; j < NB; j++)
                        if ((uint32_t)j < nbu) {
                            const uint64_t pair = opair[q] + j;
                            const uint32_t r = c_smod[l];
                            const uint32_t x0 = fold_full(s[q][j][0], l), x2 = fold_full(s[q][j][2], l);
                            const uint32_t x1 = csub32(csub32(fold_full(s[q][j][1], l) + 2 * r - x0 - x2, 2 * r), r);
                            X[((pair * 3 + 0) * NUM_S + l) * N + k] = x0;
                            X[((pair * 3 + 1) * NUM_S + l) * N + k] = x1;
                            X[((pair * 3 + 2) * NUM_S + l) * N + k] = x2;
                        }
        }
    }
}

using BatchFn = void (*)(const BatchChunk*, const BatchSeg*, uint32_t, uint32_t, uint32_t*, uint32_t*, int*);
struct BatchVariant {
    const char* name;
    BatchFn fn;
    int np, nb, stages, dps, minb, groups;
};
// name: np<probes per group>_nb<blocks>_s<stages>_d<dims per stage>_m<CTAs/SM>,
// with a trailing _g<groups> when a CTA has more than one group of consumers
#define HERS_BV(NP, NB, S, D, M) \
    {"np" #NP "_nb" #NB "_s" #S "_d" #D "_m" #M, k_tensor_batched<NP, NB, S, D, M, 1, false>, NP, NB, S, D, M, 1}
#define HERS_BVG(NP, NB, S, D, M, G)                                                                             \
    {"np" #NP "_nb" #NB "_s" #S "_d" #D "_m" #M "_g" #G, k_tensor_batched<NP, NB, S, D, M, G, false>, NP, NB, S, D, \
     M, G}
// the same shapes with the L2 policies of POL = true ("_l2" names)
#define HERS_BVP(NP, NB, S, D, M, G)                                                                             \
    {"np" #NP "_nb" #NB "_s" #S "_d" #D "_m" #M "_g" #G "_l2", k_tensor_batched<NP, NB, S, D, M, G, true>, NP, NB, \
     S, D, M, G}
// the L2-policy shapes with gallery rows prefetched into L2 PF stages ahead ("_pf<PF>")
#define HERS_BVF(NP, NB, S, D, M, G, PF)                                                                 \
    {"np" #NP "_nb" #NB "_s" #S "_d" #D "_m" #M "_g" #G "_l2_pf" #PF,                                     \
     k_tensor_batched<NP, NB, S, D, M, G, true, PF>, NP, NB, S, D, M, G}
// the L2-policy shapes with carry-chain multiply-accumulates ("_cc")
#define HERS_BVC(NP, NB, S, D, M, G)                                                                     \
    {"np" #NP "_nb" #NB "_s" #S "_d" #D "_m" #M "_g" #G "_l2_cc",                                         \
     k_tensor_batched<NP, NB, S, D, M, G, true, 0, true>, NP, NB, S, D, M, G}
static const BatchVariant kBatchVariants[] = {
    HERS_BV(1, 2, 4, 4, 2), HERS_BV(2, 2, 2, 4, 3), HERS_BV(2, 2, 3, 4, 2), HERS_BV(2, 2, 4, 2, 2),
    HERS_BV(4, 1, 2, 4, 2), HERS_BV(4, 2, 2, 4, 2), HERS_BV(4, 2, 3, 2, 2), HERS_BV(2, 1, 3, 4, 3),
    HERS_BV(1, 1, 4, 4, 3), HERS_BV(2, 1, 4, 4, 2), HERS_BV(4, 1, 4, 2, 2), HERS_BV(1, 2, 3, 4, 3),
    HERS_BVG(2, 2, 2, 4, 2, 2), HERS_BVG(2, 2, 3, 2, 2, 2), HERS_BVG(2, 2, 4, 4, 1, 2),
    HERS_BVG(4, 2, 2, 4, 1, 2), HERS_BVG(2, 1, 3, 4, 2, 2), HERS_BVG(4, 1, 2, 4, 2, 2),
    HERS_BVP(2, 2, 2, 4, 3, 1), HERS_BVP(4, 2, 2, 4, 2, 1), HERS_BVP(2, 2, 3, 4, 2, 1),
    HERS_BVP(2, 2, 2, 4, 2, 2),
    HERS_BVF(2, 2, 2, 4, 3, 1, 4), HERS_BVF(2, 2, 2, 4, 3, 1, 8), HERS_BVF(4, 2, 2, 4, 2, 1, 4),
    HERS_BVF(2, 2, 2, 2, 3, 1, 8),
    HERS_BVC(2, 2, 2, 4, 3, 1), HERS_BVC(4, 2, 2, 4, 2, 1), HERS_BVC(2, 2, 3, 4, 2, 1),
    HERS_BVC(2, 2, 2, 4, 2, 2),
};
#undef HERS_BV
#undef HERS_BVG
#undef HERS_BVP
#undef HERS_BVF
#undef HERS_BVC
constexpr int NUM_BATCH_VARIANTS = sizeof(kBatchVariants) / sizeof(kBatchVariants[0]);

static int batch_smem(const BatchVariant& v) {
    return v.stages * (v.groups * v.np + v.nb) * v.dps * 2 * TILE * 4;
}
static int batch_threads(const BatchVariant& v) { return v.groups * TILE + 32; }

int batch_variant_count() { return NUM_BATCH_VARIANTS; }
int batch_variant_np(int v) { return kBatchVariants[v].groups * kBatchVariants[v].np; }
int batch_variant_nb(int v) { return kBatchVariants[v].nb; }

// Direct launch of the persistent kernel of variant v over device tables.
cudaError_t launch_batched(int v, const BatchChunk* d_chunks, const BatchSeg* d_segs, uint32_t nsegs,
                           uint32_t nunits, uint32_t* d_counter, uint64_t* X, int* err, int device, cudaStream_t st) {
    // X: the X area of the pairs' workspace; the kernel writes uint32 accumulators
    // [pair][3][NUM_S][N] at its start
    if (v < 0 || v >= NUM_BATCH_VARIANTS) return cudaErrorInvalidValue;
    const BatchVariant& V = kBatchVariants[v];
    const int smem = batch_smem(V);
    cudaError_t e = cudaFuncSetAttribute(V.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    int per_sm = 0, sms = 0;
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, V.fn, batch_threads(V), smem);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const unsigned grid = (unsigned)std::min<uint64_t>((uint64_t)per_sm * sms, nunits ? nunits : 1);
    e = cudaMemsetAsync(d_counter, 0, sizeof(uint32_t), st);
    if (e != cudaSuccess) return e;
    V.fn<<<grid, batch_threads(V), smem, st>>>(d_chunks, d_segs, nsegs, nunits, d_counter, (uint32_t*)X, err);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace hers

using namespace hers;

struct hers_batch {
    hers_ctx* ctx;
    const hers_keys* keys;
    int variant;
    uint32_t ngroups, nunits;
    uint64_t npairs;
    uint64_t* scores;
    uint64_t* ws;
    void* dev;  // chunks, units and the counter, one allocation
    cudaGraph_t graph;
    cudaGraphExec_t exec;
    cudaEvent_t ev[3];  // traced runs: start, after the tensor kernel, end
    // launch parameters of the built variant (what the graph holds)
    BatchFn fn;
    unsigned grid;
    int smem, threads;
    BatchChunk* d_chunks;
    BatchSeg* d_segs;
    uint32_t nsegs;
    uint32_t* d_counter;
    double tune_ms[NUM_BATCH_VARIANTS];
};

namespace {

struct Plan {
    std::vector<BatchChunk> chunks;
    std::vector<BatchSeg> segs;
    uint32_t ngroups = 0;
    uint64_t npairs = 0, nunits = 0;
};

}  // namespace

namespace hers {

// Plans work over range items: item i searches blocks [begin_i, end_i) of the
// resident gallery at `gallery` (block 0) with dimension d; its pair of
// block b is pair_base_i + (b - begin_i).  For every gallery, the items' range
// end points cut the blocks into segments over which the set of covering items
// is constant; each segment with covering items is a group.
// Unit order within a segment: (limb, tile) outermost, then block, then probe
// chunk.  Units in flight at one time then share one (limb, tile): the probe
// rows they need (all the segment's probes, d x 4 KiB each) stay in L2 across
// blocks, and the chunks of one block run back to back, so a gallery run is
// read from HBM once and from L2 by the other chunks.
void plan_ranges(const RangeItem* items, uint32_t nitems, int np_max, int nb_max,
                 std::vector<BatchChunk>& chunks, std::vector<BatchSeg>& segs, uint32_t* ngroups,
                 uint64_t* nunits) {
    uint64_t unit = 0;
    std::map<std::pair<const uint64_t*, uint32_t>, std::vector<uint32_t>> by_gallery;
    std::vector<std::pair<const uint64_t*, uint32_t>> order;
    for (uint32_t i = 0; i < nitems; i++) {
        auto key = std::make_pair(items[i].gallery, items[i].d);
        if (!by_gallery.count(key)) order.push_back(key);
        by_gallery[key].push_back(i);
    }
    uint32_t groups = 0;
    for (const auto& key : order) {
        const std::vector<uint32_t>& its = by_gallery[key];
        std::vector<uint64_t> cuts;
        for (uint32_t i : its) {
            cuts.push_back(items[i].begin);
            cuts.push_back(items[i].end);
        }
        std::sort(cuts.begin(), cuts.end());
        cuts.erase(std::unique(cuts.begin(), cuts.end()), cuts.end());
        for (size_t c = 0; c + 1 < cuts.size(); c++) {
            const uint64_t s0 = cuts[c], s1 = cuts[c + 1];
            std::vector<uint32_t> cover;
            for (uint32_t i : its)
                if (items[i].begin <= s0 && items[i].end >= s1) cover.push_back(i);
            if (cover.empty()) continue;
            groups++;
            const uint32_t first = (uint32_t)chunks.size();
            for (size_t c0 = 0; c0 < cover.size(); c0 += np_max) {
                BatchChunk ch = {};
                ch.gallery = key.first;
                ch.d = key.second;
                ch.np = (uint32_t)std::min<size_t>(np_max, cover.size() - c0);
                for (uint32_t q = 0; q < ch.np; q++) {
                    const RangeItem& it = items[cover[c0 + q]];
                    ch.probe[q] = it.probe;
                    ch.pair[q] = it.pair_base - it.begin;  // + absolute block (mod 2^64)
                }
                chunks.push_back(ch);
            }
            const uint32_t nch = (uint32_t)chunks.size() - first;
            const uint32_t nbg = (uint32_t)((s1 - s0 + nb_max - 1) / nb_max);
            segs.push_back({(uint32_t)std::min<uint64_t>(unit, 0xFFFFFFFFull), first, nch, nbg, (uint32_t)s0,
                            (uint32_t)s1});
            unit += (uint64_t)NUM_S * NTILES * nbg * nch;
        }
    }
    if (ngroups) *ngroups = groups;
    if (nunits) *nunits = unit;
}

}  // namespace hers

namespace {

Plan make_plan(const hers_batch_item* items, uint32_t nitems, int np_max, int nb_max) {
    Plan P;
    std::vector<RangeItem> r(nitems);
    for (uint32_t i = 0; i < nitems; i++) {
        r[i] = {items[i].gallery, 0, items[i].nblocks, items[i].d, items[i].probe, P.npairs};
        P.npairs += items[i].nblocks;
    }
    plan_ranges(r.data(), nitems, np_max, nb_max, P.chunks, P.segs, &P.ngroups, &P.nunits);
    return P;
}

void batch_release(hers_batch* B) {
    if (B->exec) cudaGraphExecDestroy(B->exec);
    if (B->graph) cudaGraphDestroy(B->graph);
    if (B->dev) cudaFree(B->dev);
    B->exec = nullptr;
    B->graph = nullptr;
    B->dev = nullptr;
}

// The batch's launches: counter reset, persistent tensor kernel, epilogue.
// With `traced`, events go between them (used outside a graph only).
cudaError_t batch_launch(hers_batch* B, cudaStream_t st, bool traced) {
    uint64_t* X = B->ws;
    uint64_t* C = X + B->npairs * 15 * N;
    uint64_t* KS = C + B->npairs * 6 * N;
    cudaError_t e = cudaMemsetAsync(B->d_counter, 0, sizeof(uint32_t), st);
    if (traced) cudaEventRecord(B->ev[0], st);
    B->fn<<<B->grid, B->threads, B->smem, st>>>(B->d_chunks, B->d_segs, B->nsegs, B->nunits, B->d_counter,
                                                (uint32_t*)X, B->ctx->err);
    if (traced) cudaEventRecord(B->ev[1], st);
    if (e == cudaSuccess) e = cudaGetLastError();
    cudaError_t el = launch_epilogue(B->ctx->tw, B->keys->k, B->npairs, X, C, KS, B->scores, st, nullptr,
                                     nullptr, B->ctx->epi_variant);
    if (traced) cudaEventRecord(B->ev[2], st);
    return e != cudaSuccess ? e : el;
}

// Builds the device tables and the graph of one variant.
int batch_build(hers_batch* B, const hers_batch_item* items, uint32_t nitems, int v) {
    hers_ctx* ctx = B->ctx;
    const BatchVariant& V = kBatchVariants[v];
    Plan P = make_plan(items, nitems, V.groups * V.np, V.nb);
    if (P.nunits >= UNIT_STOP) return fail(ctx, HERS_E_INVAL, "hers_batch_create: too many units");
    const size_t cbytes = P.chunks.size() * sizeof(BatchChunk);
    const size_t ubytes = P.segs.size() * sizeof(BatchSeg);
    const size_t total = ((cbytes + 255) / 256) * 256 + ((ubytes + 255) / 256) * 256 + 256;
    cudaError_t e = cudaMalloc(&B->dev, total);
    if (e != cudaSuccess) return fail(ctx, HERS_E_NOMEM, "hers_batch_create: %s", cudaGetErrorString(e));
    BatchChunk* d_chunks = (BatchChunk*)B->dev;
    BatchSeg* d_segs = (BatchSeg*)((char*)B->dev + ((cbytes + 255) / 256) * 256);
    uint32_t* d_counter = (uint32_t*)((char*)d_segs + ((ubytes + 255) / 256) * 256);
    e = cudaMemcpy(d_chunks, P.chunks.data(), cbytes, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d_segs, P.segs.data(), ubytes, cudaMemcpyHostToDevice);
    const int smem = batch_smem(V);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(V.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    int per_sm = 0, sms = 0;
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, V.fn, batch_threads(V), smem);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "hers_batch_create: setup");
    if (per_sm < 1) {
        cudaFuncAttributes fa = {};
        cudaFuncGetAttributes(&fa, V.fn);
        return fail(ctx, HERS_E_CUDA,
                    "hers_batch_create: variant %s does not fit an SM (%d registers, %d threads max, "
                    "%d + %d bytes shared)",
                    V.name, fa.numRegs, fa.maxThreadsPerBlock, (int)fa.sharedSizeBytes, smem);
    }
    const unsigned grid = (unsigned)std::min<uint64_t>((uint64_t)per_sm * sms, P.nunits);

    B->fn = V.fn;
    B->grid = grid;
    B->smem = smem;
    B->threads = batch_threads(V);
    B->d_chunks = d_chunks;
    B->d_segs = d_segs;
    B->nsegs = (uint32_t)P.segs.size();
    B->d_counter = d_counter;
    B->variant = v;
    B->ngroups = P.ngroups;
    B->nunits = (uint32_t)P.nunits;
    B->npairs = P.npairs;
    cudaStream_t cs = ctx->stream;
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "hers_batch_create: begin capture");
    cudaError_t el = batch_launch(B, cs, false);
    e = cudaStreamEndCapture(cs, &B->graph);
    if (el != cudaSuccess) e = el;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&B->exec, B->graph, 0);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "hers_batch_create: graph");
    return HERS_OK;
}

}  // namespace

extern "C" {

int hers_batch_variants(void) { return NUM_BATCH_VARIANTS; }

const char* hers_batch_variant_name(int v) {
    return (v >= 0 && v < NUM_BATCH_VARIANTS) ? kBatchVariants[v].name : "";
}

uint64_t hers_batch_workspace_bytes(const hers_batch_item* items, uint32_t nitems) {
    uint64_t np = 0;
    for (uint32_t i = 0; items && i < nitems; i++) np += items[i].nblocks;
    return hers_search_workspace_bytes(np);
}

int hers_batch_create(hers_ctx* ctx, const hers_keys* keys, const hers_batch_item* items,
                      uint32_t nitems, uint64_t* scores_ct, void* workspace, uint64_t workspace_bytes,
                      uint32_t flags, hers_batch** out) {
    if (!ctx || !keys || !items || !scores_ct || !workspace || !out || nitems == 0)
        return fail(ctx, HERS_E_INVAL, "hers_batch_create: null argument or no items");
    *out = nullptr;
    for (uint32_t i = 0; i < nitems; i++) {
        const hers_batch_item& it = items[i];
        if (!it.gallery || !it.probe || it.nblocks == 0 || it.d == 0 || it.d > HERS_MAX_D)
            return fail(ctx, HERS_E_INVAL, "hers_batch_create: item %u is invalid", i);
    }
    if (workspace_bytes < hers_batch_workspace_bytes(items, nitems))
        return fail(ctx, HERS_E_NOMEM, "hers_batch_create: workspace too small");
    const int forced = (int)((flags >> 8) & 0xFF) - 1;
    if (forced >= NUM_BATCH_VARIANTS)
        return fail(ctx, HERS_E_INVAL, "hers_batch_create: variant %d not in [0, %d)", forced,
                    NUM_BATCH_VARIANTS);
    DeviceGuard g(ctx->device);
    hers_batch* B = new (std::nothrow) hers_batch();
    if (!B) return fail(ctx, HERS_E_NOMEM, "hers_batch_create: host allocation");
    B->ctx = ctx;
    B->keys = keys;
    B->scores = scores_ct;
    B->ws = (uint64_t*)workspace;
    for (int i = 0; i < 3; i++)
        if (cudaEventCreate(&B->ev[i]) != cudaSuccess) {
            for (int j = 0; j < i; j++) cudaEventDestroy(B->ev[j]);
            delete B;
            return fail(ctx, HERS_E_CUDA, "hers_batch_create: event creation");
        }
    for (int v = 0; v < NUM_BATCH_VARIANTS; v++) B->tune_ms[v] = -1;
    int rc = HERS_OK;
    if (forced >= 0 || !(flags & HERS_BATCH_AUTOTUNE)) {
        rc = batch_build(B, items, nitems, forced >= 0 ? forced : DEFAULT_BATCH_VARIANT);
    } else {
        // autotune: build every variant, time 3 graph launches each, keep the fastest
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        int best = -1;
        double best_ms = 0;
        for (int v = 0; v < NUM_BATCH_VARIANTS && rc == HERS_OK; v++) {
            rc = batch_build(B, items, nitems, v);
            if (rc != HERS_OK) break;
            cudaError_t e = cudaGraphLaunch(B->exec, ctx->stream);  // warm
            double vb = 0;
            for (int rep = 0; rep < 3 && e == cudaSuccess; rep++) {
                cudaEventRecord(e0, ctx->stream);
                e = cudaGraphLaunch(B->exec, ctx->stream);
                cudaEventRecord(e1, ctx->stream);
                if (e == cudaSuccess) e = cudaEventSynchronize(e1);
                float ms = 0;
                if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
                if (rep == 0 || ms < vb) vb = ms;
            }
            if (e != cudaSuccess) rc = cuda_fail(ctx, e, "hers_batch_create: autotune");
            B->tune_ms[v] = vb;
            if (rc == HERS_OK && (best < 0 || vb < best_ms)) {
                best = v;
                best_ms = vb;
            }
            batch_release(B);
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (rc == HERS_OK) rc = batch_build(B, items, nitems, best);
    }
    if (rc == HERS_OK) rc = hers_check(ctx, nullptr);
    if (rc != HERS_OK) {
        batch_release(B);
        for (int i = 0; i < 3; i++) cudaEventDestroy(B->ev[i]);
        delete B;
        return rc;
    }
    *out = B;
    return HERS_OK;
}

int hers_batch_trace(hers_batch* B, void* stream, double* tensor_ms, double* total_ms) {
    if (!B) return HERS_E_INVAL;
    DeviceGuard g(B->ctx->device);
    cudaError_t e = batch_launch(B, (cudaStream_t)stream, true);
    if (e == cudaSuccess) count_launches(8);
    if (e == cudaSuccess) e = cudaEventSynchronize(B->ev[2]);
    float t = 0, a = 0;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, B->ev[0], B->ev[1]);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&a, B->ev[0], B->ev[2]);
    if (e != cudaSuccess) return cuda_fail(B->ctx, e, "hers_batch_trace");
    if (tensor_ms) *tensor_ms = t;
    if (total_ms) *total_ms = a;
    return HERS_OK;
}

int hers_batch_run(hers_batch* B, void* stream) {
    if (!B) return HERS_E_INVAL;
    DeviceGuard g(B->ctx->device);
    cudaError_t e = cudaGraphLaunch(B->exec, (cudaStream_t)stream);
    if (e == cudaSuccess) count_launches(8);
    return e == cudaSuccess ? HERS_OK : cuda_fail(B->ctx, e, "hers_batch_run");
}

int hers_batch_info(const hers_batch* B, int* variant, uint32_t* ngroups, uint32_t* nunits,
                    uint64_t* npairs, double* tune_ms) {
    if (!B) return HERS_E_INVAL;
    if (variant) *variant = B->variant;
    if (ngroups) *ngroups = B->ngroups;
    if (nunits) *nunits = B->nunits;
    if (npairs) *npairs = B->npairs;
    if (tune_ms)
        for (int v = 0; v < NUM_BATCH_VARIANTS; v++) tune_ms[v] = B->tune_ms[v];
    return HERS_OK;
}

int hers_batch_free(hers_batch* B) {
    if (!B) return HERS_E_INVAL;
    {
        DeviceGuard g(B->ctx->device);
        cudaStreamSynchronize(B->ctx->stream);
        batch_release(B);
        for (int i = 0; i < 3; i++) cudaEventDestroy(B->ev[i]);
    }
    delete B;
    return HERS_OK;
}

}  // extern "C"
