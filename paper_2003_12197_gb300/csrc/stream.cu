// Streamed search over a gallery kept in canonical form (two limbs,
// coefficient domain: 32 d bytes per entry, the ciphertexts' own size) in
// host or device memory.  This is for galleries too large for the resident
// form: 100M entries at d = 64 are 204.8 GB canonical against 409.6 GB
// resident.
//
// Per chunk of blocks:
//   1. copy in (from host memory);
//   2. extend + NTT to the resident form, into a device chunk buffer;
//   3. one persistent batched tensor launch with every probe;
//   4. the epilogue;
//   5. the score ciphertexts are copied into their [probe][block] places.
// Two chunk slots alternate, fed from a ring of NSTAGE staging buffers.
// Three streams: the copies (a stream of their own, so the copy engine runs
// up to NSTAGE chunks ahead as soon as a staging buffer is free), the
// extensions (the context's stream) and the searches (the caller's stream).
// Chunk c+1's copy and extension overlap chunk c's search.
#include <algorithm>
#include <vector>

#include "common.cuh"
#include "hers.h"
#include "internal.h"

using namespace hers;

namespace {

// Staging buffers for host chunks: the copy stream may run this many chunks
// ahead of the extensions.
constexpr int NSTAGE = 4;

struct SlotLayout {
    uint64_t resident, X, C, KS, OUT, tables;  // word offsets in the slot
    uint64_t words;
    uint64_t staging_words;  // one staging buffer (after the two slots)
};

SlotLayout slot_layout(uint32_t d, uint32_t nprobes, uint32_t chunk, uint64_t table_bytes) {
    SlotLayout L;
    uint64_t w = 0;
    L.staging_words = ((uint64_t)chunk * d * 4 * N + 31) / 32 * 32;
    L.resident = w;
    w += (uint64_t)chunk * d * RES_WORDS_PER_DIM;
    const uint64_t pairs = (uint64_t)nprobes * chunk;
    L.X = w;
    w += pairs * 15 * N;
    L.C = w;
    w += pairs * 6 * N;
    L.KS = w;
    w += pairs * 4 * N;
    L.OUT = w;
    w += pairs * 4 * N;
    L.tables = w;
    w += (table_bytes + 7) / 8 + 64;
    L.words = (w + 31) / 32 * 32;  // 256-byte multiples
    return L;
}

uint64_t table_bytes_for(uint32_t nprobes, uint32_t chunk) {
    // at most one chunk record per probe and one segment per chunk (every probe
    // searches the whole chunk: one segment)
    (void)chunk;
    return (uint64_t)nprobes * sizeof(BatchChunk) + 256 + (uint64_t)nprobes * sizeof(BatchSeg) + 256 + 64;
}

}  // namespace

extern "C" {

uint64_t hers_search_stream_workspace_bytes(uint32_t d, uint32_t nprobes, uint32_t chunk_blocks) {
    const SlotLayout L = slot_layout(d, nprobes, chunk_blocks, table_bytes_for(nprobes, chunk_blocks));
    return (2 * L.words + NSTAGE * L.staging_words) * 8;
}

int hers_search_stream(hers_ctx* ctx, const hers_keys* keys, const uint64_t* gallery_ct,
                       int gallery_on_host, uint64_t nblocks, uint32_t d,
                       const uint64_t* const* probes, uint32_t nprobes, uint64_t* scores_ct,
                       uint32_t chunk_blocks, int variant, void* workspace, uint64_t workspace_bytes,
                       void* stream) {
    if (!ctx || !keys || !gallery_ct || !probes || !scores_ct || !workspace || nblocks == 0 ||
        nprobes == 0 || chunk_blocks == 0)
        return fail(ctx, HERS_E_INVAL, "hers_search_stream: null argument or empty sizes");
    if (d == 0 || d > HERS_MAX_D) return fail(ctx, HERS_E_INVAL, "hers_search_stream: d = %u", d);
    if (variant < 0 || variant >= batch_variant_count())
        return fail(ctx, HERS_E_INVAL, "hers_search_stream: variant %d", variant);
    for (uint32_t p = 0; p < nprobes; p++)
        if (!probes[p]) return fail(ctx, HERS_E_INVAL, "hers_search_stream: probe %u is null", p);
    const uint64_t tbytes = table_bytes_for(nprobes, chunk_blocks);
    const SlotLayout L = slot_layout(d, nprobes, chunk_blocks, tbytes);
    const uint64_t need = (2 * L.words + NSTAGE * L.staging_words) * 8;
    if (workspace_bytes < need)
        return fail(ctx, HERS_E_NOMEM, "hers_search_stream: workspace %llu < %llu bytes",
                    (unsigned long long)workspace_bytes, (unsigned long long)need);
    DeviceGuard g(ctx->device);
    cudaStream_t sm = (cudaStream_t)stream, sc = ctx->stream;
    uint64_t* slot[2] = {(uint64_t*)workspace, (uint64_t*)workspace + L.words};
    uint64_t* staging[NSTAGE];
    for (int k = 0; k < NSTAGE; k++) staging[k] = (uint64_t*)workspace + 2 * L.words + k * L.staging_words;
    const int np_var = batch_variant_np(variant);

    // Work tables: the same plan for every full chunk, one copy per slot (the
    // tables point at the slot's resident buffer); the last chunk may be shorter.
    auto plan = [&](int s, uint32_t nb, std::vector<BatchChunk>& ch, std::vector<BatchSeg>& un, uint64_t* nu) {
        std::vector<RangeItem> items(nprobes);
        for (uint32_t p = 0; p < nprobes; p++)
            items[p] = {slot[s] + L.resident, 0, nb, d, probes[p], (uint64_t)p * nb};
        uint32_t ng = 0;
        plan_ranges(items.data(), nprobes, np_var, batch_variant_nb(variant), ch, un, &ng, nu);
    };
    const uint64_t nchunks = (nblocks + chunk_blocks - 1) / chunk_blocks;
    const uint32_t last_nb = (uint32_t)(nblocks - (nchunks - 1) * chunk_blocks);
    struct Tables {
        BatchChunk* chunks;
        BatchSeg* units;
        uint32_t nsegs;
        uint32_t* counter;
        uint32_t nunits;
    };
    // table sets: [slot][full, last]; the "last" set lives in the same slot
    // area after a full chunk finished with it, so each slot holds the set
    // for the chunk it currently runs (re-uploaded when the size changes)
    Tables T[2][2];
    std::vector<BatchChunk> hc[2][2];
    std::vector<BatchSeg> hu[2][2];
    uint64_t nu[2][2] = {{0, 0}, {0, 0}};
    for (int s = 0; s < 2; s++) {
        plan(s, chunk_blocks, hc[s][0], hu[s][0], &nu[s][0]);
        plan(s, last_nb, hc[s][1], hu[s][1], &nu[s][1]);
        for (int k = 0; k < 2; k++) {
            uint8_t* tb = (uint8_t*)(slot[s] + L.tables);
            T[s][k].chunks = (BatchChunk*)tb;
            T[s][k].units = (BatchSeg*)(tb + (hc[s][k].size() * sizeof(BatchChunk) + 255) / 256 * 256);
            T[s][k].nsegs = (uint32_t)hu[s][k].size();
            T[s][k].counter = (uint32_t*)((uint8_t*)T[s][k].units +
                                          (hu[s][k].size() * sizeof(BatchSeg) + 255) / 256 * 256);
            T[s][k].nunits = (uint32_t)nu[s][k];
        }
    }

    // ev_copied[k]: staging k holds its chunk; ev_staged[k]: staging k has
    // been extended from and may be refilled; ev_ext[s]: slot s's resident
    // buffer and tables are ready; ev_free[s]: its resident buffer may be refilled
    cudaEvent_t ev_copied[NSTAGE], ev_staged[NSTAGE], ev_ext[2], ev_free[2], ev_join, ev_join2;
    cudaStream_t scp = nullptr;  // the copies' stream (host galleries)
    cudaError_t e = cudaSuccess;
    for (int s = 0; s < 2 && e == cudaSuccess; s++) {
        e = cudaEventCreateWithFlags(&ev_ext[s], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev_free[s], cudaEventDisableTiming);
    }
    for (int k = 0; k < NSTAGE && e == cudaSuccess; k++) {
        e = cudaEventCreateWithFlags(&ev_copied[k], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev_staged[k], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev_join, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev_join2, cudaEventDisableTiming);
    if (e == cudaSuccess && gallery_on_host) e = cudaStreamCreateWithFlags(&scp, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "hers_search_stream: events");
    // the side streams start after work already queued on the caller's stream
    cudaEventRecord(ev_join, sm);
    cudaStreamWaitEvent(sc, ev_join, 0);
    if (scp) cudaStreamWaitEvent(scp, ev_join, 0);

    int table_kind[2] = {-1, -1};
    for (uint64_t c = 0; c < nchunks && e == cudaSuccess; c++) {
        const int s = (int)(c & 1);
        const uint64_t b0 = c * chunk_blocks;
        const uint32_t nb = (uint32_t)std::min<uint64_t>(chunk_blocks, nblocks - b0);
        const int kind = (c == nchunks - 1 && nb != chunk_blocks) ? 1 : 0;
        uint64_t* base = slot[s];
        const uint64_t* src = gallery_ct + b0 * d * 4 * N;
        const uint64_t* cts = src;
        const int k = (int)(c % NSTAGE);
        if (gallery_on_host) {
            // copy stream: wait until staging k has been extended from
            if (c >= NSTAGE) cudaStreamWaitEvent(scp, ev_staged[k], 0);
            e = cudaMemcpyAsync(staging[k], src, (uint64_t)nb * d * 4 * N * 8, cudaMemcpyHostToDevice, scp);
            if (e == cudaSuccess) e = cudaEventRecord(ev_copied[k], scp);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(sc, ev_copied[k], 0);
            cts = staging[k];
        }
        // side stream: wait until the slot's previous chunk has been searched
        if (c >= 2) cudaStreamWaitEvent(sc, ev_free[s], 0);
        if (e == cudaSuccess) e = launch_extend_ntt(ctx->tw, cts, (uint64_t)nb * d, 0, d, base + L.resident, sc);
        if (e == cudaSuccess && gallery_on_host) e = cudaEventRecord(ev_staged[k], sc);
        if (e == cudaSuccess && table_kind[s] != kind) {
            const Tables& t = T[s][kind];
            e = cudaMemcpyAsync(t.chunks, hc[s][kind].data(), hc[s][kind].size() * sizeof(BatchChunk),
                                cudaMemcpyHostToDevice, sc);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(t.units, hu[s][kind].data(), hu[s][kind].size() * sizeof(BatchSeg),
                                    cudaMemcpyHostToDevice, sc);
            table_kind[s] = kind;  // a pageable source is staged before cudaMemcpyAsync returns
        }
        cudaEventRecord(ev_ext[s], sc);
        // caller's stream: search the chunk
        cudaStreamWaitEvent(sm, ev_ext[s], 0);
        const Tables& t = T[s][kind];
        const uint64_t npairs = (uint64_t)nprobes * nb;
        if (e == cudaSuccess)
            e = launch_batched(variant, t.chunks, t.units, t.nsegs, t.nunits, t.counter, base + L.X, ctx->err,
                               ctx->device, sm);
        cudaEventRecord(ev_free[s], sm);  // the resident chunk buffer may be refilled
        if (e == cudaSuccess)
            e = launch_epilogue(ctx->tw, keys->k, npairs, base + L.X, base + L.C, base + L.KS, base + L.OUT, sm,
                                nullptr, nullptr, ctx->epi_variant);
        for (uint32_t p = 0; p < nprobes && e == cudaSuccess; p++)
            e = cudaMemcpyAsync(scores_ct + ((uint64_t)p * nblocks + b0) * 4 * N,
                                base + L.OUT + (uint64_t)p * nb * 4 * N, (uint64_t)nb * 4 * N * 8,
                                cudaMemcpyDeviceToDevice, sm);
    }
    // join the side streams into the caller's
    cudaEventRecord(ev_join, sc);
    cudaStreamWaitEvent(sm, ev_join, 0);
    if (scp) {
        cudaEventRecord(ev_join2, scp);
        cudaStreamWaitEvent(sm, ev_join2, 0);
        cudaStreamDestroy(scp);  // destruction waits for its work to finish on the device
    }
    for (int s = 0; s < 2; s++) {
        cudaEventDestroy(ev_ext[s]);
        cudaEventDestroy(ev_free[s]);
    }
    for (int k = 0; k < NSTAGE; k++) {
        cudaEventDestroy(ev_copied[k]);
        cudaEventDestroy(ev_staged[k]);
    }
    cudaEventDestroy(ev_join);
    cudaEventDestroy(ev_join2);
    return e == cudaSuccess ? HERS_OK : cuda_fail(ctx, e, "hers_search_stream");
}

}  // extern "C"
