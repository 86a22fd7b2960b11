// Stage 1 of the two-stage search (Sec. 3.2): the K gallery entries with the
// largest decrypted scores, ordered by score descending and, among equal
// scores, by index ascending.  The client runs it on the scores that
// hers_decrypt_scores leaves in device memory; its output feeds the re-rank.
//
// Exact radix selection.  Scores map to order-preserving 32-bit keys
// (s xor 2^31).  Three histogram passes over the keys (bits 31..20, 19..8,
// 7..0), each restricted to the keys that match the bits fixed so far, pin
// the K-th largest key T, the number of keys above it and how many of the
// keys equal to T belong to the top K.  When only some of those ties belong,
// a counting pass and a scan rank the ties by index.  A collection pass then
// gathers exactly K candidates, and one CTA sorts them.  No step waits on the
// host: the selection state lives in device memory.
#include <algorithm>

#include "hers.h"
#include "internal.h"

namespace hers {
namespace {

constexpr int TK_THREADS = 256;
constexpr uint32_t TK_MAXK = 4096;
constexpr int TK_SORT_THREADS = 1024;

struct TopkState {
    uint32_t prefix;  // key bits fixed so far
    uint32_t mask;    // which key bits are fixed
    uint32_t need;    // keys matching prefix/mask that still belong to the top K
    uint32_t above;   // keys known to lie above the prefix's range
    uint32_t ties;    // keys equal to the threshold (after the last level)
    uint32_t ncand;   // candidates collected
};

__device__ __forceinline__ uint32_t score_key(int32_t s) { return (uint32_t)s ^ 0x80000000u; }
__device__ __forceinline__ int level_shift(int level) { return level == 0 ? 20 : (level == 1 ? 8 : 0); }
__device__ __forceinline__ int level_bins(int level) { return level < 2 ? 4096 : 256; }

// CTA b owns the contiguous index range [lo, hi).
__device__ __forceinline__ void cta_range(uint64_t m, uint64_t& lo, uint64_t& hi) {
    const uint64_t chunk = (m + gridDim.x - 1) / gridDim.x;
    lo = (uint64_t)blockIdx.x * chunk;
    hi = lo + chunk < m ? lo + chunk : m;
    if (lo > m) lo = m;
}

__global__ void k_topk_init(TopkState* st, uint32_t k) {
    st->prefix = 0;
    st->mask = 0;
    st->need = k;
    st->above = 0;
    st->ties = 0;
    st->ncand = 0;
}

// Histogram of one level's key bits over the keys that match the prefix.
__global__ void __launch_bounds__(TK_THREADS) k_topk_hist(const int32_t* __restrict__ s, uint64_t m,
                                                          int level, const TopkState* __restrict__ st,
                                                          uint32_t* __restrict__ hist) {
    __shared__ uint32_t h[4096];
    const int nb = level_bins(level), sh = level_shift(level);
    for (int i = threadIdx.x; i < nb; i += TK_THREADS) h[i] = 0;
    const uint32_t prefix = st->prefix, mask = st->mask;
    __syncthreads();
    uint64_t lo, hi;
    cta_range(m, lo, hi);
    for (uint64_t i = lo + threadIdx.x; i < hi; i += TK_THREADS) {
        const uint32_t k = score_key(s[i]);
        if ((k & mask) == prefix) atomicAdd(&h[(k >> sh) & (uint32_t)(nb - 1)], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nb; i += TK_THREADS)
        if (h[i]) atomicAdd(&hist[i], h[i]);
}

// One CTA: the bin, counted from the top, that holds the need-th key; fixes
// its bits in the prefix and clears the histogram for the next level.
__global__ void __launch_bounds__(TK_THREADS) k_topk_select(int level, TopkState* st, uint32_t* hist) {
    __shared__ uint32_t part[TK_THREADS], before[TK_THREADS];
    __shared__ uint32_t s_need;
    const int nb = level_bins(level), sh = level_shift(level);
    const int per = nb / TK_THREADS;
    const int t = threadIdx.x;
    const int b_hi = nb - t * per;  // thread t owns bins [b_hi - per, b_hi), top bins first
    uint32_t sum = 0;
    for (int b = b_hi - per; b < b_hi; b++) sum += hist[b];
    part[t] = sum;
    if (t == 0) s_need = st->need;
    __syncthreads();
    if (t == 0) {
        uint32_t a = 0;
        for (int i = 0; i < TK_THREADS; i++) {
            before[i] = a;
            a += part[i];
        }
    }
    __syncthreads();
    const uint32_t need = s_need;
    if (before[t] < need && need <= before[t] + part[t]) {  // exactly one thread
        uint32_t a = before[t];
        for (int b = b_hi - 1; b >= b_hi - per; b--) {
            const uint32_t c = hist[b];
            if (a + c >= need) {
                st->prefix |= (uint32_t)b << sh;
                st->mask |= (uint32_t)(nb - 1) << sh;
                st->above += a;
                st->need = need - a;
                if (level == 2) st->ties = c;
                break;
            }
            a += c;
        }
    }
    __syncthreads();
    for (int b = t; b < 4096; b += TK_THREADS) hist[b] = 0;
}

// Keys equal to the threshold, per CTA (only when some of them are dropped).
__global__ void __launch_bounds__(TK_THREADS) k_topk_tiecount(const int32_t* __restrict__ s, uint64_t m,
                                                              const TopkState* __restrict__ st,
                                                              uint32_t* __restrict__ tiecnt) {
    __shared__ uint32_t c;
    if (st->need == st->ties) return;  // every tie is taken: no ranking needed
    const uint32_t T = st->prefix;
    if (threadIdx.x == 0) c = 0;
    __syncthreads();
    uint64_t lo, hi;
    cta_range(m, lo, hi);
    uint32_t mine = 0;
    for (uint64_t i = lo + threadIdx.x; i < hi; i += TK_THREADS) mine += score_key(s[i]) == T;
    for (int o = 16; o > 0; o >>= 1) mine += __shfl_down_sync(0xffffffffu, mine, o);
    if ((threadIdx.x & 31) == 0 && mine) atomicAdd(&c, mine);
    __syncthreads();
    if (threadIdx.x == 0) tiecnt[blockIdx.x] = c;
}

// Exclusive scan of the per-CTA tie counts (one thread; a few thousand CTAs).
__global__ void k_topk_tiescan(const TopkState* __restrict__ st, const uint32_t* __restrict__ tiecnt,
                               uint32_t* __restrict__ tiebase, uint32_t nctas) {
    if (st->need == st->ties) return;
    uint32_t a = 0;
    for (uint32_t i = 0; i < nctas; i++) {
        tiebase[i] = a;
        a += tiecnt[i];
    }
}

__device__ __forceinline__ uint64_t cand_word(uint32_t key, uint64_t i) {
    return ((uint64_t)key << 32) | (uint32_t)~(uint32_t)i;  // sorts by key desc, then index asc
}

// Gathers the keys above the threshold and the first `need` ties by index.
__global__ void __launch_bounds__(TK_THREADS) k_topk_collect(const int32_t* __restrict__ s, uint64_t m,
                                                             TopkState* st, const uint32_t* __restrict__ tiebase,
                                                             uint64_t* __restrict__ cand, uint32_t k) {
    __shared__ uint32_t warp_tot[TK_THREADS / 32];
    const uint32_t T = st->prefix, need = st->need;
    const bool all_ties = need == st->ties;
    uint64_t lo, hi;
    cta_range(m, lo, hi);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // every write stays inside the k-entry buffer; a count beyond k is caught
    // by the sort kernel's check of ncand
    auto push = [&](uint64_t w) {
        const uint32_t pos = atomicAdd(&st->ncand, 1u);
        if (pos < k) cand[pos] = w;
    };
    uint32_t running = all_ties ? 0 : tiebase[blockIdx.x];  // ties before this tile
    for (uint64_t base = lo; base < hi; base += TK_THREADS) {
        const uint64_t i = base + threadIdx.x;
        const bool valid = i < hi;
        const uint32_t key = valid ? score_key(s[i]) : 0u;
        if (valid && key > T) push(cand_word(key, i));
        const bool tie = valid && key == T;
        if (all_ties) {
            if (tie) push(cand_word(key, i));
            continue;
        }
        // rank of this tie among the ties of the tile, in index order
        const uint32_t bal = __ballot_sync(0xffffffffu, tie);
        if (lane == 0) warp_tot[warp] = __popc(bal);
        __syncthreads();
        uint32_t r = running + __popc(bal & ((1u << lane) - 1u));
        uint32_t tile_tot = 0;
        for (int w = 0; w < TK_THREADS / 32; w++) {
            if (w < warp) r += warp_tot[w];
            tile_tot += warp_tot[w];
        }
        if (tie && r < need) push(cand_word(key, i));
        running += tile_tot;
        __syncthreads();
    }
}

// One CTA: bitonic sort of the K candidates (descending), padded to a power
// of two with zero words, which sort last (every candidate word is > 0:
// indices are below 2^32 - 1).
__global__ void __launch_bounds__(TK_SORT_THREADS) k_topk_sort(const TopkState* __restrict__ st,
                                                               const uint64_t* __restrict__ cand, uint32_t k,
                                                               uint32_t P, int64_t* __restrict__ out_idx,
                                                               int32_t* __restrict__ out_score, int* err) {
    __shared__ uint64_t v[TK_MAXK];
    if (threadIdx.x == 0 && st->ncand != k) atomicOr(err, 8);  // the selection lost count
    for (uint32_t i = threadIdx.x; i < P; i += TK_SORT_THREADS) v[i] = i < k ? cand[i] : 0;
    __syncthreads();
    for (uint32_t size = 2; size <= P; size <<= 1)
        for (uint32_t stride = size >> 1; stride > 0; stride >>= 1) {
            for (uint32_t i = threadIdx.x; i < P / 2; i += TK_SORT_THREADS) {
                const uint32_t a = 2 * i - (i & (stride - 1)), b = a + stride;
                const bool desc = (a & size) == 0;
                const uint64_t x = v[a], y = v[b];
                if ((x < y) == desc) {
                    v[a] = y;
                    v[b] = x;
                }
            }
            __syncthreads();
        }
    for (uint32_t i = threadIdx.x; i < k; i += TK_SORT_THREADS) {
        const uint64_t w = v[i];
        out_idx[i] = (int64_t)(uint32_t)~(uint32_t)w;
        out_score[i] = (int32_t)((uint32_t)(w >> 32) ^ 0x80000000u);
    }
}

uint32_t topk_ctas(uint64_t m) {
    const uint64_t want = (m + TK_THREADS * 16 - 1) / (TK_THREADS * 16);
    return (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>(want, 2048));
}

struct TopkLayout {
    uint64_t state, hist, tiecnt, tiebase, cand, bytes;
};

TopkLayout topk_layout(uint64_t m) {
    TopkLayout L;
    const uint32_t g = topk_ctas(m);
    L.state = 0;
    L.hist = 256;
    L.tiecnt = L.hist + 4096 * 4;
    L.tiebase = L.tiecnt + ((uint64_t)g * 4 + 255) / 256 * 256;
    L.cand = L.tiebase + ((uint64_t)g * 4 + 255) / 256 * 256;
    L.bytes = L.cand + TK_MAXK * 8;
    return L;
}

}  // namespace
}  // namespace hers

using namespace hers;

extern "C" {

uint64_t hers_topk_workspace_bytes(uint64_t m) { return topk_layout(m).bytes; }

int hers_topk(hers_ctx* ctx, const int32_t* scores, uint64_t m, uint32_t k, int64_t* out_idx,
              int32_t* out_scores, void* workspace, uint64_t workspace_bytes, void* stream) {
    if (!ctx || !scores || !out_idx || !out_scores || !workspace)
        return fail(ctx, HERS_E_INVAL, "hers_topk: null argument");
    if (m == 0 || m >= 0xFFFFFFFFull)
        return fail(ctx, HERS_E_INVAL, "hers_topk: m = %llu not in [1, 2^32 - 1)", (unsigned long long)m);
    if (k == 0 || k > TK_MAXK || k > m)
        return fail(ctx, HERS_E_INVAL, "hers_topk: k = %u not in [1, min(m, %u)]", k, TK_MAXK);
    const TopkLayout L = topk_layout(m);
    if (workspace_bytes < L.bytes)
        return fail(ctx, HERS_E_NOMEM, "hers_topk: workspace %llu < %llu bytes",
                    (unsigned long long)workspace_bytes, (unsigned long long)L.bytes);
    DeviceGuard g(ctx->device);
    cudaStream_t st = stream ? (cudaStream_t)stream : (cudaStream_t)0;
    uint8_t* ws = (uint8_t*)workspace;
    TopkState* S = (TopkState*)(ws + L.state);
    uint32_t* hist = (uint32_t*)(ws + L.hist);
    uint32_t* tiecnt = (uint32_t*)(ws + L.tiecnt);
    uint32_t* tiebase = (uint32_t*)(ws + L.tiebase);
    uint64_t* cand = (uint64_t*)(ws + L.cand);
    const uint32_t ctas = topk_ctas(m);
    uint32_t P = 1;
    while (P < k) P <<= 1;
    cudaError_t e = cudaMemsetAsync(hist, 0, 4096 * 4, st);
    if (e == cudaSuccess) {
        k_topk_init<<<1, 1, 0, st>>>(S, k);
        for (int level = 0; level < 3; level++) {
            k_topk_hist<<<ctas, TK_THREADS, 0, st>>>(scores, m, level, S, hist);
            k_topk_select<<<1, TK_THREADS, 0, st>>>(level, S, hist);
        }
        k_topk_tiecount<<<ctas, TK_THREADS, 0, st>>>(scores, m, S, tiecnt);
        k_topk_tiescan<<<1, 1, 0, st>>>(S, tiecnt, tiebase, ctas);
        k_topk_collect<<<ctas, TK_THREADS, 0, st>>>(scores, m, S, tiebase, cand, k);
        k_topk_sort<<<1, TK_SORT_THREADS, 0, st>>>(S, cand, k, P, out_idx, out_scores, ctx->err);
        count_launches(11);
        e = cudaGetLastError();
    }
    return e == cudaSuccess ? HERS_OK : cuda_fail(ctx, e, "hers_topk");
}

}  // extern "C"
