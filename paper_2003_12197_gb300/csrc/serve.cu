// Continuous-batching server for encrypted search requests (Alg 7's server
// side under load).  Requests (gallery, block range, probe ciphertexts in host
// memory) arrive at any time.  A scheduler thread admits them in arrival order
// as device memory allows, plans every admitted group of requests as one batch
// (overlapping ranges of one gallery share each gallery read: see
// plan_ranges), and issues the batch on one of three streams: probe copy-in and
// preparation, the persistent tensor kernel, the epilogue, and the score
// ciphertexts' copy-out to each request's host buffer.  Batches on the three
// streams overlap on the device; requests that arrive meanwhile form the next
// batch as soon as a stream and memory are free.  A request's latency runs
// from submission to its scores being in host memory.
//
// Device memory: one pool carved out of free HBM at creation, managed here by
// a first-fit allocator; a batch holds one contiguous range of it from launch
// to completion.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "common.cuh"
#include "hers.h"
#include "internal.h"

using namespace hers;
using Clock = std::chrono::steady_clock;

namespace {

// batches in flight, each on a stream of its own (three kept the tensor
// kernel fed best at saturation: 1.23-1.26G entries/s against 1.18-1.21G with
// two and 1.23G with four)
constexpr int SRV_STREAMS = 3;
constexpr uint64_t ALIGN = 256;

struct Request {
    uint64_t id;
    uint32_t gallery;
    uint64_t begin, end;
    const uint64_t* probe_ct_host;
    uint64_t* scores_host;
    Clock::time_point t_arrival, t_done;
    int status = 1;  // 1 pending, 0 done, < 0 failed
};

// First-fit allocator over [0, size) with coalescing.
struct Pool {
    std::map<uint64_t, uint64_t> free_;  // offset -> size
    void init(uint64_t size) { free_ = {{0, size}}; }
    bool alloc(uint64_t bytes, uint64_t* off) {
        bytes = (bytes + ALIGN - 1) / ALIGN * ALIGN;
        for (auto it = free_.begin(); it != free_.end(); ++it)
            if (it->second >= bytes) {
                *off = it->first;
                const uint64_t rest = it->second - bytes, roff = it->first + bytes;
                free_.erase(it);
                if (rest) free_[roff] = rest;
                return true;
            }
        return false;
    }
    void release(uint64_t off, uint64_t bytes) {
        bytes = (bytes + ALIGN - 1) / ALIGN * ALIGN;
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
};

struct Slot;

}  // namespace

struct hers_server {
    hers_ctx* ctx;
    const hers_keys* keys;
    std::vector<hers_server_gallery> gals;
    uint8_t* pool_base = nullptr;
    uint64_t pool_bytes = 0;
    Pool pool;
    uint32_t max_batch = 16;
    int variant = 1;
    cudaStream_t streams[SRV_STREAMS] = {};
    Slot* slots[SRV_STREAMS] = {};
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request*> pending;
    std::map<uint64_t, Request*> reqs;
    std::thread thr;
    bool stop = false;
    bool paused = false;  // admission held (requests queue up)
    uint64_t next_id = 1;
    uint64_t n_submitted = 0, n_completed = 0, n_batches = 0, n_entries = 0, max_batch_seen = 0;
    // time spent, summed over retired batches: device time of the kernels
    // (probe preparation, tensor, epilogue) and of the score copies to host
    // memory (CUDA events), and host time planning and issuing batches
    double t_kernels_ms = 0, t_copies_ms = 0, t_plan_ms = 0;
    int error = 0;
};

namespace {

// One stream's batch in flight.
struct Slot {
    hers_server* srv;
    int index;
    bool busy = false;
    bool done = false;  // set by the host callback
    uint64_t off = 0, bytes = 0;
    std::vector<Request*> reqs;
    BatchChunk* h_chunks = nullptr;  // pinned staging of the work tables
    BatchSeg* h_segs = nullptr;
    size_t cap_chunks = 0, cap_segs = 0;
    cudaEvent_t ev[3] = {};  // batch start, kernels done, copies done
};

void CUDART_CB on_batch_done(void* arg) {
    Slot* s = (Slot*)arg;
    hers_server* srv = s->srv;
    const Clock::time_point now = Clock::now();
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        for (Request* r : s->reqs) r->t_done = now;
        s->done = true;
    }
    srv->cv_work.notify_all();
}

uint64_t request_words(uint32_t d, uint64_t nblocks) {
    // probe cts + prepared probe + X/C/KS + output score cts
    return (uint64_t)d * (4 * N + RES_WORDS_PER_DIM) + nblocks * (SEARCH_WS_WORDS_PER_BLOCK + 4 * N);
}

bool ensure_staging(Slot* s, size_t nchunks, size_t nsegs) {
    if (nchunks > s->cap_chunks) {
        if (s->h_chunks) cudaFreeHost(s->h_chunks);
        s->cap_chunks = std::max(nchunks, 2 * s->cap_chunks);
        if (cudaMallocHost(&s->h_chunks, s->cap_chunks * sizeof(BatchChunk)) != cudaSuccess) {
            s->h_chunks = nullptr;
            s->cap_chunks = 0;
            return false;
        }
    }
    if (nsegs > s->cap_segs) {
        if (s->h_segs) cudaFreeHost(s->h_segs);
        s->cap_segs = std::max(nsegs, 2 * s->cap_segs);
        if (cudaMallocHost(&s->h_segs, s->cap_segs * sizeof(BatchSeg)) != cudaSuccess) {
            s->h_segs = nullptr;
            s->cap_segs = 0;
            return false;
        }
    }
    return true;
}

// Plans and issues one batch on slot s (called by the scheduler thread with
// the requests already removed from the queue; the lock is not held).
cudaError_t issue_batch(hers_server* srv, Slot* s, std::vector<BatchChunk>& chunks,
                        std::vector<BatchSeg>& segs, uint64_t nunits, const std::vector<RangeItem>& items,
                        uint64_t npairs) {
    hers_ctx* ctx = srv->ctx;
    cudaStream_t st = srv->streams[s->index];
    uint64_t* base = (uint64_t*)(srv->pool_base + s->off);
    // layout: per request [probe cts d*4N][probe d*RES_WORDS_PER_DIM]; then X, C, KS, OUT; then tables
    uint64_t* w = base;
    std::vector<uint64_t*> pct(s->reqs.size());
    for (size_t i = 0; i < s->reqs.size(); i++) {
        const uint32_t d = items[i].d;
        pct[i] = w;
        w += (uint64_t)d * (4 * N + RES_WORDS_PER_DIM);
    }
    uint64_t* X = w;
    uint64_t* C = X + npairs * 15 * N;
    uint64_t* KS = C + npairs * 6 * N;
    uint64_t* OUT = KS + npairs * 4 * N;
    uint8_t* tb = (uint8_t*)(OUT + npairs * 4 * N);
    BatchChunk* d_chunks = (BatchChunk*)tb;
    BatchSeg* d_segs = (BatchSeg*)(tb + (chunks.size() * sizeof(BatchChunk) + ALIGN - 1) / ALIGN * ALIGN);
    uint32_t* d_counter = (uint32_t*)((uint8_t*)d_segs + (segs.size() * sizeof(BatchSeg) + ALIGN - 1) / ALIGN * ALIGN);

    cudaError_t e = cudaEventRecord(s->ev[0], st);
    for (size_t i = 0; i < s->reqs.size() && e == cudaSuccess; i++) {
        const uint32_t d = items[i].d;
        e = cudaMemcpyAsync(pct[i], s->reqs[i]->probe_ct_host, (uint64_t)d * 4 * N * 8,
                            cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = launch_extend_ntt(ctx->tw, pct[i], d, 0, d, pct[i] + (uint64_t)d * 4 * N, st);
    }
    // the tables point at the prepared probes
    for (auto& ch : chunks)
        for (uint32_t q = 0; q < ch.np; q++)
            for (size_t i = 0; i < items.size(); i++)
                if (ch.probe[q] == items[i].probe) ch.probe[q] = pct[i] + (uint64_t)items[i].d * 4 * N;
    std::copy(chunks.begin(), chunks.end(), s->h_chunks);
    std::copy(segs.begin(), segs.end(), s->h_segs);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_chunks, s->h_chunks, chunks.size() * sizeof(BatchChunk), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_segs, s->h_segs, segs.size() * sizeof(BatchSeg), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = launch_batched(srv->variant, d_chunks, d_segs, (uint32_t)segs.size(), (uint32_t)nunits, d_counter, X, ctx->err,
                           ctx->device, st);
    if (e == cudaSuccess)
        e = launch_epilogue(ctx->tw, srv->keys->k, npairs, X, C, KS, OUT, st, nullptr, nullptr, ctx->epi_variant);
    if (e == cudaSuccess) e = cudaEventRecord(s->ev[1], st);
    for (size_t i = 0; i < s->reqs.size() && e == cudaSuccess; i++) {
        const Request* r = s->reqs[i];
        e = cudaMemcpyAsync(r->scores_host, OUT + items[i].pair_base * 4 * N,
                            (r->end - r->begin) * 4 * N * 8, cudaMemcpyDeviceToHost, st);
    }
    if (e == cudaSuccess) e = cudaEventRecord(s->ev[2], st);
    if (e == cudaSuccess) e = cudaLaunchHostFunc(st, on_batch_done, s);
    return e;
}

void scheduler(hers_server* srv) {
    DeviceGuard g(srv->ctx->device);
    std::unique_lock<std::mutex> lk(srv->mu);
    while (true) {
        // retire finished batches
        for (Slot* s : srv->slots)
            if (s->busy && s->done) {
                float k_ms = 0, c_ms = 0;
                if (cudaEventElapsedTime(&k_ms, s->ev[0], s->ev[1]) == cudaSuccess &&
                    cudaEventElapsedTime(&c_ms, s->ev[1], s->ev[2]) == cudaSuccess) {
                    srv->t_kernels_ms += k_ms;
                    srv->t_copies_ms += c_ms;
                }
                srv->pool.release(s->off, s->bytes);
                for (Request* r : s->reqs) {
                    r->status = 0;
                    srv->n_completed++;
                    srv->n_entries += (r->end - r->begin) * N;
                }
                s->reqs.clear();
                s->busy = s->done = false;
                srv->cv_done.notify_all();
            }
        if (srv->stop) {
            bool idle = true;
            for (Slot* s : srv->slots) idle = idle && !s->busy;
            if (idle) break;
        }
        Slot* freeslot = nullptr;
        for (Slot* s : srv->slots)
            if (!s->busy) {
                freeslot = s;
                break;
            }
        bool any_busy = false;
        for (Slot* s : srv->slots) any_busy = any_busy || s->busy;
        if (freeslot && !srv->pending.empty() && !srv->paused) {
            const Clock::time_point t_plan0 = Clock::now();
            // admit from the head of the queue while the batch fits in the pool
            size_t take = std::min<size_t>(srv->pending.size(), srv->max_batch);
            std::vector<BatchChunk> chunks;
            std::vector<BatchSeg> segs;
            uint64_t nunits = 0;
            std::vector<RangeItem> items;
            uint64_t npairs = 0, off = 0, bytes = 0;
            bool got = false;
            while (take > 0) {
                items.clear();
                chunks.clear();
                segs.clear();
                npairs = 0;
                uint64_t words = 0;
                for (size_t i = 0; i < take; i++) {
                    const Request* r = srv->pending[i];
                    const hers_server_gallery& G = srv->gals[r->gallery];
                    // placeholders for the probe pointers; issue_batch points them at the prepared probes
                    items.push_back({G.gallery, r->begin, r->end, G.d, (const uint64_t*)(uintptr_t)(i + 1), npairs});
                    npairs += r->end - r->begin;
                    words += request_words(G.d, r->end - r->begin);
                }
                uint32_t ng = 0;
                plan_ranges(items.data(), (uint32_t)items.size(), batch_variant_np(srv->variant),
                            batch_variant_nb(srv->variant), chunks, segs, &ng, &nunits);
                bytes = words * 8 + (chunks.size() * sizeof(BatchChunk) + ALIGN) +
                        (segs.size() * sizeof(BatchSeg) + ALIGN) + ALIGN;
                if (srv->pool.alloc(bytes, &off)) {
                    got = true;
                    break;
                }
                take--;
            }
            if (!got) {
                if (!any_busy) {  // the head request alone can never fit: fail it
                    Request* r = srv->pending.front();
                    srv->pending.pop_front();
                    r->status = HERS_E_NOMEM;
                    r->t_done = Clock::now();
                    srv->cv_done.notify_all();
                    continue;
                }
                srv->cv_work.wait_for(lk, std::chrono::microseconds(200));
                continue;
            }
            Slot* s = freeslot;
            s->reqs.assign(srv->pending.begin(), srv->pending.begin() + take);
            srv->pending.erase(srv->pending.begin(), srv->pending.begin() + take);
            s->off = off;
            s->bytes = bytes;
            s->busy = true;
            s->done = false;
            srv->n_batches++;
            srv->max_batch_seen = std::max<uint64_t>(srv->max_batch_seen, take);
            lk.unlock();
            // probe placeholders (i + 1) -> item order; issue_batch maps them to prepared probes
            for (size_t i = 0; i < items.size(); i++) items[i].probe = (const uint64_t*)(uintptr_t)(i + 1);
            cudaError_t e = ensure_staging(s, chunks.size(), segs.size()) ? cudaSuccess : cudaErrorMemoryAllocation;
            if (e == cudaSuccess && nunits >= 0xFFFFFFFFull) e = cudaErrorInvalidValue;
            if (e == cudaSuccess) e = issue_batch(srv, s, chunks, segs, nunits, items, npairs);
            lk.lock();
            srv->t_plan_ms += std::chrono::duration<double, std::milli>(Clock::now() - t_plan0).count();
            if (e != cudaSuccess) {
                srv->error = HERS_E_CUDA;
                for (Request* r : s->reqs) {
                    r->status = HERS_E_CUDA;
                    r->t_done = Clock::now();
                }
                srv->pool.release(s->off, s->bytes);
                s->reqs.clear();
                s->busy = false;
                srv->cv_done.notify_all();
            }
            continue;
        }
        srv->cv_work.wait_for(lk, std::chrono::microseconds(200));
    }
}

}  // namespace

extern "C" {

int hers_server_create(hers_ctx* ctx, const hers_keys* keys, const hers_server_gallery* gals,
                       uint32_t ngals, uint64_t workspace_bytes, uint32_t max_batch, int variant,
                       hers_server** out) {
    if (!ctx || !keys || !gals || ngals == 0 || !out) return fail(ctx, HERS_E_INVAL, "hers_server_create: null argument");
    *out = nullptr;
    for (uint32_t i = 0; i < ngals; i++)
        if (!gals[i].gallery || gals[i].nblocks == 0 || gals[i].d == 0 || gals[i].d > HERS_MAX_D)
            return fail(ctx, HERS_E_INVAL, "hers_server_create: gallery %u is invalid", i);
    if (variant < 0 || variant >= batch_variant_count())
        return fail(ctx, HERS_E_INVAL, "hers_server_create: variant %d", variant);
    DeviceGuard g(ctx->device);
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) return fail(ctx, HERS_E_CUDA, "hers_server_create: cudaMemGetInfo");
    const uint64_t reserve = 1ull << 30;  // left to the rest of the process
    const uint64_t avail = free_b > reserve ? free_b - reserve : 0;
    const uint64_t want = workspace_bytes ? std::min<uint64_t>(workspace_bytes, avail) : avail;
    if (want < (1ull << 20)) return fail(ctx, HERS_E_NOMEM, "hers_server_create: only %llu bytes of HBM free", (unsigned long long)avail);
    hers_server* srv = new (std::nothrow) hers_server();
    if (!srv) return fail(ctx, HERS_E_NOMEM, "hers_server_create: host allocation");
    srv->ctx = ctx;
    srv->keys = keys;
    srv->gals.assign(gals, gals + ngals);
    srv->max_batch = max_batch ? max_batch : 16;
    srv->variant = variant;
    cudaError_t e = cudaMalloc(&srv->pool_base, want);
    for (int i = 0; i < SRV_STREAMS && e == cudaSuccess; i++) {
        e = cudaStreamCreateWithFlags(&srv->streams[i], cudaStreamNonBlocking);
        Slot* s = new (std::nothrow) Slot();
        if (!s) e = cudaErrorMemoryAllocation;
        else {
            s->srv = srv;
            s->index = i;
            srv->slots[i] = s;
            for (int k = 0; k < 3 && e == cudaSuccess; k++) e = cudaEventCreate(&s->ev[k]);
        }
    }
    if (e != cudaSuccess) {
        for (int i = 0; i < SRV_STREAMS; i++) {
            if (srv->streams[i]) cudaStreamDestroy(srv->streams[i]);
            if (srv->slots[i])
                for (int k = 0; k < 3; k++)
                    if (srv->slots[i]->ev[k]) cudaEventDestroy(srv->slots[i]->ev[k]);
            delete srv->slots[i];
        }
        if (srv->pool_base) cudaFree(srv->pool_base);
        delete srv;
        return fail(ctx, HERS_E_NOMEM, "hers_server_create: %s", cudaGetErrorString(e));
    }
    srv->pool_bytes = want;
    srv->pool.init(want);
    srv->thr = std::thread(scheduler, srv);
    *out = srv;
    return HERS_OK;
}

int hers_server_submit(hers_server* srv, uint32_t gallery, uint64_t block_begin, uint64_t block_end,
                       const uint64_t* probe_ct_host, uint64_t* scores_ct_host, uint64_t* id) {
    if (!srv || !probe_ct_host || !scores_ct_host || !id) return HERS_E_INVAL;
    if (gallery >= srv->gals.size() || block_begin >= block_end || block_end > srv->gals[gallery].nblocks)
        return fail(srv->ctx, HERS_E_INVAL, "hers_server_submit: gallery %u blocks [%llu, %llu)", gallery,
                    (unsigned long long)block_begin, (unsigned long long)block_end);
    Request* r = new (std::nothrow) Request();
    if (!r) return HERS_E_NOMEM;
    r->gallery = gallery;
    r->begin = block_begin;
    r->end = block_end;
    r->probe_ct_host = probe_ct_host;
    r->scores_host = scores_ct_host;
    r->t_arrival = Clock::now();
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        r->id = srv->next_id++;
        srv->reqs[r->id] = r;
        srv->pending.push_back(r);
        srv->n_submitted++;
        *id = r->id;
    }
    srv->cv_work.notify_all();
    return HERS_OK;
}

int hers_server_wait(hers_server* srv, uint64_t id, uint32_t timeout_ms, double* latency_ms) {
    if (!srv) return HERS_E_INVAL;
    std::unique_lock<std::mutex> lk(srv->mu);
    auto it = srv->reqs.find(id);
    if (it == srv->reqs.end()) return HERS_E_INVAL;
    Request* r = it->second;
    const bool ok = srv->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), [&] { return r->status <= 0; });
    if (!ok) return HERS_E_TIMEOUT;
    const int st = r->status;
    if (latency_ms) *latency_ms = std::chrono::duration<double, std::milli>(r->t_done - r->t_arrival).count();
    srv->reqs.erase(it);
    delete r;
    return st;
}

int hers_server_pause(hers_server* srv, int paused) {
    if (!srv) return HERS_E_INVAL;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        srv->paused = paused != 0;
    }
    srv->cv_work.notify_all();
    return HERS_OK;
}

int hers_server_stats(hers_server* srv, uint64_t* submitted, uint64_t* completed, uint64_t* batches,
                      uint64_t* entries, uint64_t* max_batch_seen, uint64_t* pool_bytes) {
    if (!srv) return HERS_E_INVAL;
    std::lock_guard<std::mutex> lk(srv->mu);
    if (submitted) *submitted = srv->n_submitted;
    if (completed) *completed = srv->n_completed;
    if (batches) *batches = srv->n_batches;
    if (entries) *entries = srv->n_entries;
    if (max_batch_seen) *max_batch_seen = srv->max_batch_seen;
    if (pool_bytes) *pool_bytes = srv->pool_bytes;
    return srv->error;
}

int hers_server_timing(hers_server* srv, double* kernels_ms, double* copies_ms, double* plan_ms) {
    if (!srv) return HERS_E_INVAL;
    std::lock_guard<std::mutex> lk(srv->mu);
    if (kernels_ms) *kernels_ms = srv->t_kernels_ms;
    if (copies_ms) *copies_ms = srv->t_copies_ms;
    if (plan_ms) *plan_ms = srv->t_plan_ms;
    return HERS_OK;
}

int hers_server_free(hers_server* srv) {
    if (!srv) return HERS_E_INVAL;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        srv->stop = true;
    }
    srv->cv_work.notify_all();
    srv->thr.join();
    DeviceGuard g(srv->ctx->device);
    for (int i = 0; i < SRV_STREAMS; i++) {
        cudaStreamSynchronize(srv->streams[i]);
        cudaStreamDestroy(srv->streams[i]);
        if (srv->slots[i]) {
            if (srv->slots[i]->h_chunks) cudaFreeHost(srv->slots[i]->h_chunks);
            if (srv->slots[i]->h_segs) cudaFreeHost(srv->slots[i]->h_segs);
            for (int k = 0; k < 3; k++)
                if (srv->slots[i]->ev[k]) cudaEventDestroy(srv->slots[i]->ev[k]);
            delete srv->slots[i];
        }
    }
    cudaFree(srv->pool_base);
    for (auto& kv : srv->reqs) delete kv.second;  // every request not yet waited for, pending or done
    delete srv;
    return HERS_OK;
}

}  // extern "C"
