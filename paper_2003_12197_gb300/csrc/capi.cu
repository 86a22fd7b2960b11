// C ABI of the HERS library (declared in include/hers.h): contexts, keys,
// argument checking and the orchestration of the kernels in scheme.cu and
// search.cu.  No computation of the method runs on the host; the host only
// builds the NTT twiddle tables once per context.
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <atomic>
#include <new>
#include <vector>

#include "hers.h"
#include "hers_consts.h"
#include "internal.h"

using namespace hers;


namespace hers {
static std::atomic<uint64_t> g_launches{0};
void count_launches(uint64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
uint64_t launches_total() { return g_launches.load(std::memory_order_relaxed); }

int fail(hers_ctx* ctx, int code, const char* fmt, ...) {
    if (ctx) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(ctx->msg, sizeof ctx->msg, fmt, ap);
        va_end(ap);
    }
    return code;
}

int cuda_fail(hers_ctx* ctx, cudaError_t e, const char* where) {
    return fail(ctx, HERS_E_CUDA, "%s: %s", where, cudaGetErrorString(e));
}

DeviceGuard::DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
}
DeviceGuard::~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
}
}  // namespace hers


namespace {

const uint64_t H_MOD[NUM_MODS] = HERS_MOD_INIT;
const uint64_t H_PSI[NUM_MODS] = HERS_PSI_INIT;
const uint64_t H_SMOD[NUM_S] = HERS_SMOD_INIT;
const uint64_t H_SPSI[NUM_S] = HERS_SPSI_INIT;

typedef unsigned __int128 u128;

uint64_t h_mulmod(uint64_t a, uint64_t b, uint64_t p) { return (uint64_t)((u128)a * b % p); }

uint64_t h_pow(uint64_t b, uint64_t e, uint64_t p) {
    uint64_t r = 1;
    b %= p;
    while (e) {
        if (e & 1) r = h_mulmod(r, b, p);
        b = h_mulmod(b, b, p);
        e >>= 1;
    }
    return r;
}

int h_brev(int x, int bits) {
    int r = 0;
    for (int i = 0; i < bits; i++) {
        r = (r << 1) | (x & 1);
        x >>= 1;
    }
    return r;
}

cudaStream_t pick(hers_ctx*, void* stream) { return (cudaStream_t)stream; }

// Events of the next traced search call, or null when tracing is off / full.
cudaEvent_t* next_trace(hers_ctx* ctx) {
    if (ctx->tn >= ctx->tcap) return nullptr;
    return &ctx->tev[(size_t)(ctx->tn++) * SEARCH_EVENTS];
}

void ep_free(hers_ctx* ctx) {
    if (ctx->ep_ev[0]) cudaEventDestroy(ctx->ep_ev[0]);
    if (ctx->ep_ev[1]) cudaEventDestroy(ctx->ep_ev[1]);
    if (ctx->ep) cudaStreamDestroy(ctx->ep);
    ctx->ep = nullptr;
    ctx->ep_ev[0] = ctx->ep_ev[1] = nullptr;
}

void trace_free(hers_ctx* ctx) {
    for (cudaEvent_t e : ctx->tev) cudaEventDestroy(e);
    ctx->tev.clear();
    ctx->tcap = ctx->tn = 0;
}

}  // namespace

extern "C" {

int hers_default_params(hers_params* out) {
    if (!out) return HERS_E_INVAL;
    out->n = N;
    out->q[0] = H_MOD[0];
    out->q[1] = H_MOD[1];
    out->t = H_MOD[MOD_T];
    out->flags = 0;
    return HERS_OK;
}

const char* hers_status_string(int s) {
    switch (s) {
        case HERS_OK: return "HERS_OK";
        case HERS_E_INVAL: return "HERS_E_INVAL";
        case HERS_E_NOMEM: return "HERS_E_NOMEM";
        case HERS_E_CUDA: return "HERS_E_CUDA";
        case HERS_E_TIMEOUT: return "HERS_E_TIMEOUT";
        case HERS_E_PARAM: return "HERS_E_PARAM";
        case HERS_E_SAMPLER: return "HERS_E_SAMPLER";
        default: return "HERS_E_UNKNOWN";
    }
}

const char* hers_last_error(const hers_ctx* ctx) { return ctx ? ctx->msg : "null context"; }

uint64_t hers_ct_bytes(void) { return 4ull * N * 8; }
uint64_t hers_gallery_bytes(uint64_t nblocks, uint32_t d) { return nblocks * d * RES_WORDS_PER_DIM * 8; }
uint64_t hers_probe_bytes(uint32_t d) { return (uint64_t)d * RES_WORDS_PER_DIM * 8; }
uint64_t hers_search_workspace_bytes(uint64_t nblocks) { return nblocks * SEARCH_WS_WORDS_PER_BLOCK * 8; }
uint64_t hers_blocks_for(uint64_t m) { return (m + N - 1) / N; }
uint64_t hers_search_host_workspace_bytes(uint64_t nblocks, uint32_t d) {
    return hers_search_workspace_bytes(nblocks) + hers_probe_bytes(d) +
           (uint64_t)d * hers_ct_bytes() + nblocks * hers_ct_bytes();
}

int hers_create(const hers_params* p, int device, hers_ctx** out) {
    if (!out) return HERS_E_INVAL;
    *out = nullptr;
    hers_params def;
    hers_default_params(&def);
    // the plaintext modulus: the default t or the paper's (Sec. 4.1)
    int pm = 0;
    if (p) {
        if (p->n != def.n || p->q[0] != def.q[0] || p->q[1] != def.q[1] || p->flags != 0) return HERS_E_PARAM;
        if (p->t == H_MOD[MOD_T_PAPER]) pm = 1;
        else if (p->t != def.t) return HERS_E_PARAM;
    }
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return HERS_E_CUDA;
    hers_ctx* ctx = new (std::nothrow) hers_ctx();
    if (!ctx) return HERS_E_NOMEM;
    ctx->device = device;
    ctx->pm = pm;
    ctx->msg[0] = 0;
    DeviceGuard g(device);
    if (!g.ok) { delete ctx; return HERS_E_CUDA; }
    if (cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess) {
        delete ctx;
        return HERS_E_CUDA;
    }
    {   // the epilogue stream: the device's highest priority
        int least = 0, greatest = 0;
        if (cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess ||
            cudaStreamCreateWithPriority(&ctx->ep, cudaStreamNonBlocking, greatest) != cudaSuccess ||
            cudaEventCreateWithFlags(&ctx->ep_ev[0], cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&ctx->ep_ev[1], cudaEventDisableTiming) != cudaSuccess) {
            ep_free(ctx);
            cudaStreamDestroy(ctx->stream);
            delete ctx;
            return HERS_E_CUDA;
        }
    }
    // twiddles: [mod][forward, inverse][N] pairs (w, floor(w 2^64 / p)); entry 0
    // of the inverse table: the last inverse stage's twiddle times N^-1
    const size_t words = TW_WORDS;
    uint64_t* h = new (std::nothrow) uint64_t[words];
    if (!h) { ep_free(ctx); cudaStreamDestroy(ctx->stream); delete ctx; return HERS_E_NOMEM; }
    for (int i = 0; i < NUM_MODS; i++) {
        const uint64_t pm = H_MOD[i], psi = H_PSI[i], psi_inv = h_pow(psi, pm - 2, pm);
        uint64_t* f = h + (size_t)(4 * i) * N;
        for (int k = 0; k < N; k++) {
            const int r = h_brev(k, LOGN);
            const uint64_t w = h_pow(psi, (uint64_t)r, pm), wi = h_pow(psi_inv, (uint64_t)r, pm);
            f[2 * k] = w;
            f[2 * k + 1] = (uint64_t)(((u128)w << 64) / pm);
            f[2 * N + 2 * k] = wi;
            f[2 * N + 2 * k + 1] = (uint64_t)(((u128)wi << 64) / pm);
        }
        const uint64_t ninv = h_pow((uint64_t)N, pm - 2, pm);
        const uint64_t wl = h_mulmod(f[2 * N + 2], ninv, pm);  // inverse twiddle 1 times N^-1
        f[2 * N] = wl;
        f[2 * N + 1] = (uint64_t)(((u128)wl << 64) / pm);
    }
    // search basis: [i][forward, inverse][N] pairs of 32-bit words (w, floor(w 2^32 / r))
    uint32_t* h32 = (uint32_t*)(h + (size_t)NUM_MODS * 4 * N);
    for (int i = 0; i < NUM_S; i++) {
        const uint64_t r = H_SMOD[i], psi = H_SPSI[i], psi_inv = h_pow(psi, r - 2, r);
        uint32_t* f = h32 + (size_t)(4 * i) * N;
        for (int k = 0; k < N; k++) {
            const int b = h_brev(k, LOGN);
            const uint64_t w = h_pow(psi, (uint64_t)b, r), wi = h_pow(psi_inv, (uint64_t)b, r);
            f[2 * k] = (uint32_t)w;
            f[2 * k + 1] = (uint32_t)((w << 32) / r);
            f[2 * N + 2 * k] = (uint32_t)wi;
            f[2 * N + 2 * k + 1] = (uint32_t)((wi << 32) / r);
        }
        const uint64_t ninv = h_pow((uint64_t)N, r - 2, r);
        const uint64_t wl = h_mulmod(f[2 * N + 2], ninv, r);  // inverse twiddle 1 times N^-1
        f[2 * N] = (uint32_t)wl;
        f[2 * N + 1] = (uint32_t)((wl << 32) / r);
    }
    cudaError_t e = cudaMalloc(&ctx->tw, words * 8);
    if (e == cudaSuccess) e = cudaMemcpy(ctx->tw, h, words * 8, cudaMemcpyHostToDevice);
    delete[] h;
    if (e == cudaSuccess) e = cudaMalloc(&ctx->err, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(ctx->err, 0, sizeof(int));
    if (e != cudaSuccess) {
        cudaFree(ctx->tw);
        ep_free(ctx);
        cudaStreamDestroy(ctx->stream);
        delete ctx;
        return HERS_E_CUDA;
    }
    *out = ctx;
    return HERS_OK;
}

int hers_destroy(hers_ctx* ctx) {
    if (!ctx) return HERS_E_INVAL;
    {
        DeviceGuard g(ctx->device);
        cudaStreamSynchronize(ctx->stream);
        cudaStreamSynchronize(ctx->ep);
        cudaFree(ctx->tw);
        cudaFree(ctx->err);
        trace_free(ctx);
        ep_free(ctx);
        cudaStreamDestroy(ctx->stream);
    }
    delete ctx;
    return HERS_OK;
}

int hers_check(hers_ctx* ctx, void* stream) {
    if (!ctx) return HERS_E_INVAL;
    DeviceGuard g(ctx->device);
    cudaError_t e = cudaStreamSynchronize(pick(ctx, stream));
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "stream synchronize");
    int flag = 0;
    e = cudaMemcpy(&flag, ctx->err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "error flag read");
    if (flag) {
        cudaMemset(ctx->err, 0, sizeof(int));
        if (flag & 2) return fail(ctx, HERS_E_TIMEOUT, "a bounded device-side wait gave up");
        if (flag & 8) return fail(ctx, HERS_E_CUDA, "top-K selection: candidate count mismatch");
        return fail(ctx, HERS_E_SAMPLER, "a rejection sampler exhausted its attempts");
    }
    return HERS_OK;
}

int hers_keygen(hers_ctx* ctx, uint64_t seed, hers_keys** out) {
    if (!ctx || !out) return fail(ctx, HERS_E_INVAL, "hers_keygen: null argument");
    *out = nullptr;
    DeviceGuard g(ctx->device);
    hers_keys* K = new (std::nothrow) hers_keys();
    if (!K) return fail(ctx, HERS_E_NOMEM, "hers_keygen: host allocation");
    K->ctx = ctx;
    K->k.pm = ctx->pm;
    // sizes in words
    const size_t w_sk = N / 8, w_pk = 4 * N, w_evk = 8 * N, w_pkn = 8 * N, w_evkn = 16 * N, w_sn = 4 * N;
    const size_t total = w_sk + w_pk + w_evk + w_pkn + w_evkn + w_sn;
    cudaError_t e = cudaMalloc(&K->base, total * 8);
    if (e != cudaSuccess) { delete K; return fail(ctx, HERS_E_NOMEM, "hers_keygen: %s", cudaGetErrorString(e)); }
    uint64_t* b = (uint64_t*)K->base;
    K->k.pk = b;
    K->k.evk = b + w_pk;
    K->k.pk_ntt = K->k.evk + w_evk;
    K->k.evk_ntt = K->k.pk_ntt + w_pkn;
    K->k.s_ntt = K->k.evk_ntt + w_evkn;
    K->k.sk = (int8_t*)(K->k.s_ntt + w_sn);
    e = launch_keygen(ctx->tw, seed, K->k, ctx->err, ctx->stream);
    if (e != cudaSuccess) { cudaFree(K->base); delete K; return cuda_fail(ctx, e, "hers_keygen"); }
    int rc = hers_check(ctx, nullptr);
    if (rc != HERS_OK) { cudaFree(K->base); delete K; return rc; }
    *out = K;
    return HERS_OK;
}

int hers_keys_free(hers_keys* keys) {
    if (!keys) return HERS_E_INVAL;
    {
        DeviceGuard g(keys->ctx->device);
        cudaStreamSynchronize(keys->ctx->stream);
        cudaFree(keys->base);
        if (keys->evkw) cudaFree(keys->evkw);  // evkw and evkw_ntt share one allocation
    }
    delete keys;
    return HERS_OK;
}

uint32_t hers_basew_digits(uint32_t logw) {
    return (logw >= BASEW_MIN && logw <= BASEW_MAX) ? basew_digits(logw) : 0;
}

int hers_keys_add_basew(hers_ctx* ctx, hers_keys* keys, uint64_t seed, uint32_t logw) {
    if (!ctx || !keys) return fail(ctx, HERS_E_INVAL, "hers_keys_add_basew: null argument");
    if (!keys->k.sk) return fail(ctx, HERS_E_INVAL, "hers_keys_add_basew: the keys hold no secret key");
    if (logw < BASEW_MIN || logw > BASEW_MAX)
        return fail(ctx, HERS_E_INVAL, "hers_keys_add_basew: log2 w = %u not in [%u, %u]", logw, BASEW_MIN,
                    BASEW_MAX);
    DeviceGuard g(ctx->device);
    const uint32_t nd = basew_digits(logw);
    uint64_t* mem = nullptr;
    cudaError_t e = cudaMalloc(&mem, (size_t)nd * (4 + 8) * N * 8);
    if (e != cudaSuccess) return fail(ctx, HERS_E_NOMEM, "hers_keys_add_basew: %s", cudaGetErrorString(e));
    e = launch_keygen_w(ctx->tw, seed, logw, nd, keys->k, mem, mem + (size_t)nd * 4 * N, ctx->err, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) {
        cudaFree(mem);
        return cuda_fail(ctx, e, "hers_keys_add_basew");
    }
    if (keys->evkw) cudaFree(keys->evkw);
    keys->logw = logw;
    keys->ndig = nd;
    keys->evkw = mem;
    keys->evkw_ntt = mem + (size_t)nd * 4 * N;
    return HERS_OK;
}

int hers_keys_export_basew(hers_ctx* ctx, const hers_keys* keys, uint64_t* evkw) {
    if (!ctx || !keys || !evkw) return fail(ctx, HERS_E_INVAL, "hers_keys_export_basew: null argument");
    if (!keys->evkw) return fail(ctx, HERS_E_INVAL, "hers_keys_export_basew: no base-w keys");
    DeviceGuard g(ctx->device);
    cudaError_t e = cudaMemcpy(evkw, keys->evkw, (size_t)keys->ndig * 4 * N * 8, cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? HERS_OK : cuda_fail(ctx, e, "hers_keys_export_basew");
}

int hers_keys_export(hers_ctx* ctx, const hers_keys* keys, int8_t* sk, uint64_t* pk, uint64_t* evk) {
    if (!ctx || !keys) return fail(ctx, HERS_E_INVAL, "hers_keys_export: null argument");
    if (sk && !keys->k.sk) return fail(ctx, HERS_E_INVAL, "hers_keys_export: the keys hold no secret key");
    DeviceGuard g(ctx->device);
    cudaError_t e = cudaSuccess;
    if (sk) e = cudaMemcpy(sk, keys->k.sk, N, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && pk) e = cudaMemcpy(pk, keys->k.pk, 4 * N * 8, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && evk) e = cudaMemcpy(evk, keys->k.evk, 8 * N * 8, cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? HERS_OK : cuda_fail(ctx, e, "hers_keys_export");
}

int hers_encrypt_gallery(hers_ctx* ctx, const hers_keys* keys, const int8_t* feats, uint64_t m,
                         uint32_t d, uint64_t seed, uint64_t* gallery, uint64_t* gallery_ct,
                         void* stream) {
    if (!ctx || !keys || !feats || (!gallery && !gallery_ct))
        return fail(ctx, HERS_E_INVAL, "hers_encrypt_gallery: null argument");
    if (m == 0 || d == 0 || d > HERS_MAX_D)
        return fail(ctx, HERS_E_INVAL, "hers_encrypt_gallery: m = %llu, d = %u", (unsigned long long)m, d);
    DeviceGuard g(ctx->device);
    cudaStream_t st = pick(ctx, stream);
    const uint64_t nb = hers_blocks_for(m), nct = nb * d;
    // Encrypt in chunks of canonical cts (into gallery_ct, or a temporary
    // buffer), then extend each chunk to the resident form.
    const uint64_t chunk = 4096;  // cts per pass: 512 MiB of canonical cts at most
    uint64_t* tmp = nullptr;
    if (!gallery_ct) {
        cudaError_t e = cudaMallocAsync(&tmp, (nct < chunk ? nct : chunk) * 4 * N * 8, st);
        if (e != cudaSuccess) return fail(ctx, HERS_E_NOMEM, "hers_encrypt_gallery: %s", cudaGetErrorString(e));
    }
    cudaError_t e = cudaSuccess;
    for (uint64_t c0 = 0; c0 < nct && e == cudaSuccess; c0 += chunk) {
        const uint64_t n = nct - c0 < chunk ? nct - c0 : chunk;
        uint64_t* ct = gallery_ct ? gallery_ct + c0 * 4 * N : tmp;
        e = launch_encrypt(ctx->tw, keys->k, feats, m, d, c0, n, ENC_GALLERY, seed, ct, ctx->err, st);
        if (e == cudaSuccess && gallery) e = launch_extend_ntt(ctx->tw, ct, n, c0, d, gallery, st);
    }
    if (tmp) cudaFreeAsync(tmp, st);
    return e == cudaSuccess ? HERS_OK : cuda_fail(ctx, e, "hers_encrypt_gallery");
}

uint64_t hers_enroll_workspace_bytes(uint32_t d) { return 2ull * d * 4 * N * 8; }

int hers_enroll(hers_ctx* ctx, const hers_keys* keys, uint64_t* gallery, uint64_t nblocks, uint32_t d,
                uint64_t block, uint32_t slot, const int8_t* feats, uint64_t seed, void* workspace,
                uint64_t workspace_bytes, void* stream) {
    if (!ctx || !keys || !gallery || !feats || !workspace)
        return fail(ctx, HERS_E_INVAL, "hers_enroll: null argument");
    if (d == 0 || d > HERS_MAX_D) return fail(ctx, HERS_E_INVAL, "hers_enroll: d = %u", d);
    if (block >= nblocks || slot >= N)
        return fail(ctx, HERS_E_INVAL, "hers_enroll: block %llu of %llu, slot %u of %d",
                    (unsigned long long)block, (unsigned long long)nblocks, slot, N);
    if (workspace_bytes < hers_enroll_workspace_bytes(d))
        return fail(ctx, HERS_E_NOMEM, "hers_enroll: workspace %llu < %llu bytes",
                    (unsigned long long)workspace_bytes, (unsigned long long)hers_enroll_workspace_bytes(d));
    DeviceGuard g(ctx->device);
    cudaStream_t st = pick(ctx, stream);
    uint64_t* enc = (uint64_t*)workspace;        // d fresh ciphertexts of the entry
    uint64_t* upd = enc + (uint64_t)d * 4 * N;   // block b's updated canonical ciphertexts
    const uint64_t gslot = block * N + slot;
    cudaError_t e = launch_encrypt(ctx->tw, keys->k, feats, gslot, d, 0, d, ENC_SLOT, seed, enc, ctx->err, st);
    if (e == cudaSuccess) e = launch_resident_to_canonical_add(ctx->tw, gallery, block, d, enc, upd, st);
    if (e == cudaSuccess) e = launch_extend_ntt(ctx->tw, upd, d, block * d, d, gallery, st);
    return e == cudaSuccess ? HERS_OK : cuda_fail(ctx, e, "hers_enroll");
}

int hers_encrypt_probe(hers_ctx* ctx, const hers_keys* keys, const int8_t* q, uint32_t d,
                       uint64_t seed, uint64_t* probe_ct, void* stream) {
    if (!ctx || !keys || !q || !probe_ct) return fail(ctx, HERS_E_INVAL, "hers_encrypt_probe: null argument");
    if (d == 0 || d > HERS_MAX_D) return fail(ctx, HERS_E_INVAL, "hers_encrypt_probe: d = %u", d);
    DeviceGuard g(ctx->device);
    cudaError_t e = launch_encrypt(ctx->tw, keys->k, q, 0, d, 0, d, ENC_PROBE, seed, probe_ct, ctx->err,
                                   pick(ctx, stream));
    return e == cudaSuccess ? HERS_OK : cuda_fail(ctx, e, "hers_encrypt_probe");
}

int hers_probe_prepare(hers_ctx* ctx, const uint64_t* probe_ct, uint32_t d, uint64_t* probe,
                       void* stream) {
    if (!ctx || !probe_ct || !probe) return fail(ctx, HERS_E_INVAL, "hers_probe_prepare: null argument");
    if (d == 0 || d > HERS_MAX_D) return fail(ctx, HERS_E_INVAL, "hers_probe_prepare: d = %u", d);
    DeviceGuard g(ctx->device);
    cudaError_t e = launch_extend_ntt(ctx->tw, probe_ct, d, 0, d, probe, pick(ctx, stream), ctx->ext_cluster_max);
    return e == cudaSuccess ? HERS_OK : cuda_fail(ctx, e, "hers_probe_prepare");
}

int hers_search(hers_ctx* ctx, const hers_keys* keys, const uint64_t* gallery, uint64_t nblocks,
                uint32_t d, const uint64_t* probe, uint64_t* scores_ct, void* workspace,
                uint64_t workspace_bytes, void* stream) {
    if (!ctx || !keys || !gallery || !probe || !scores_ct || !workspace)
        return fail(ctx, HERS_E_INVAL, "hers_search: null argument");
    if (d == 0 || d > HERS_MAX_D) return fail(ctx, HERS_E_INVAL, "hers_search: d = %u", d);
    if (workspace_bytes < hers_search_workspace_bytes(nblocks))
        return fail(ctx, HERS_E_NOMEM, "hers_search: workspace %llu < %llu bytes",
                    (unsigned long long)workspace_bytes,
                    (unsigned long long)hers_search_workspace_bytes(nblocks));
    DeviceGuard g(ctx->device);
    const EpilogueStream ep = {ctx->ep, {ctx->ep_ev[0], ctx->ep_ev[1]}, ctx->tensor_first != 0};
    cudaError_t e = launch_search(ctx->tw, keys->k, gallery, nblocks, d, probe, scores_ct,
                                  (uint64_t*)workspace, ctx->err, pick(ctx, stream), next_trace(ctx),
                                  ctx->tensor_variant, nullptr, &ep, ctx->epi_variant);
    return e == cudaSuccess ? HERS_OK : cuda_fail(ctx, e, "hers_search");
}

int hers_search_rerand(hers_ctx* ctx, const hers_keys* keys, const uint64_t* gallery, uint64_t nblocks,
                       uint32_t d, const uint64_t* probe, uint64_t* scores_ct, void* workspace,
                       uint64_t workspace_bytes, uint64_t rerand_seed, void* stream) {
    int rc = hers_search(ctx, keys, gallery, nblocks, d, probe, scores_ct, workspace, workspace_bytes, stream);
    if (rc != HERS_OK || nblocks == 0) return rc;
    DeviceGuard g(ctx->device);
    cudaStream_t st = pick(ctx, stream);
    // the accumulator area of the workspace is free once the search is done
    uint64_t* z = (uint64_t*)workspace;
    cudaError_t e = launch_encrypt(ctx->tw, keys->k, nullptr, 0, 1, 0, nblocks, ENC_ZERO, rerand_seed, z,
                                   ctx->err, st);
    if (e == cudaSuccess) e = launch_ct_add(scores_ct, z, nblocks, st);
    return e == cudaSuccess ? HERS_OK : cuda_fail(ctx, e, "hers_search_rerand");
}

int hers_search_basew(hers_ctx* ctx, const hers_keys* keys, const uint64_t* gallery, uint64_t nblocks,
                      uint32_t d, const uint64_t* probe, uint64_t* scores_ct, void* workspace,
                      uint64_t workspace_bytes, void* stream) {
    if (!ctx || !keys || !gallery || !probe || !scores_ct || !workspace)
        return fail(ctx, HERS_E_INVAL, "hers_search_basew: null argument");
    if (!keys->evkw) return fail(ctx, HERS_E_INVAL, "hers_search_basew: the keys have no base-w keys");
    if (d == 0 || d > HERS_MAX_D) return fail(ctx, HERS_E_INVAL, "hers_search_basew: d = %u", d);
    if (workspace_bytes < hers_search_workspace_bytes(nblocks))
        return fail(ctx, HERS_E_NOMEM, "hers_search_basew: workspace too small");
    DeviceGuard g(ctx->device);
    const KeySwitchW ksw = {keys->evkw_ntt, keys->logw, keys->ndig};
    cudaError_t e = launch_search(ctx->tw, keys->k, gallery, nblocks, d, probe, scores_ct, (uint64_t*)workspace,
                                  ctx->err, pick(ctx, stream), next_trace(ctx), ctx->tensor_variant, &ksw, nullptr,
                                  ctx->epi_variant);
    return e == cudaSuccess ? HERS_OK : cuda_fail(ctx, e, "hers_search_basew");
}

}  // extern "C"

namespace {

// The host-buffer search step; waits for the copy back when `sync`.
int search_host(hers_ctx* ctx, const hers_keys* keys, const uint64_t* gallery, uint64_t nblocks,
                uint32_t d, const uint64_t* probe_ct_host, uint64_t* scores_ct_host, void* workspace,
                uint64_t workspace_bytes, void* stream, bool sync, const char* name) {
    if (!ctx || !keys || !gallery || !probe_ct_host || !scores_ct_host || !workspace)
        return fail(ctx, HERS_E_INVAL, "%s: null argument", name);
    if (d == 0 || d > HERS_MAX_D) return fail(ctx, HERS_E_INVAL, "%s: d = %u", name, d);
    if (workspace_bytes < hers_search_host_workspace_bytes(nblocks, d))
        return fail(ctx, HERS_E_NOMEM, "%s: workspace too small", name);
    DeviceGuard g(ctx->device);
    if (!sync) {
        // an asynchronous copy from or to pageable memory would not overlap
        // and could outlive the caller's buffer: require pinned memory
        const void* bufs[2] = {probe_ct_host, scores_ct_host};
        for (const void* b : bufs) {
            cudaPointerAttributes pa = {};
            if (cudaPointerGetAttributes(&pa, b) != cudaSuccess || pa.type != cudaMemoryTypeHost) {
                cudaGetLastError();
                return fail(ctx, HERS_E_INVAL, "%s: host buffers must be pinned", name);
            }
        }
    }
    cudaStream_t st = pick(ctx, stream);
    const EpilogueStream ep = {ctx->ep, {ctx->ep_ev[0], ctx->ep_ev[1]}, ctx->tensor_first != 0};
    // workspace: [search scratch][probe cts d*4N][probe form d*RES_WORDS_PER_DIM][score cts nblocks*4N]
    // (hers_search_host_workspace_bytes sums the same parts)
    uint64_t* ws = (uint64_t*)workspace;
    uint64_t* probe_ct = ws + nblocks * SEARCH_WS_WORDS_PER_BLOCK;
    uint64_t* probe = probe_ct + (uint64_t)d * 4 * N;
    uint64_t* out_dev = probe + (uint64_t)d * RES_WORDS_PER_DIM;
    cudaError_t e = cudaMemcpyAsync(probe_ct, probe_ct_host, (uint64_t)d * 4 * N * 8,
                                    cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = launch_extend_ntt(ctx->tw, probe_ct, d, 0, d, probe, st, ctx->ext_cluster_max);
    if (e == cudaSuccess)
        e = launch_search(ctx->tw, keys->k, gallery, nblocks, d, probe, out_dev, ws, ctx->err, st,
                          next_trace(ctx), ctx->tensor_variant, nullptr, &ep, ctx->epi_variant);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(scores_ct_host, out_dev, nblocks * 4 * N * 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && sync) e = cudaStreamSynchronize(st);
    return e == cudaSuccess ? HERS_OK : cuda_fail(ctx, e, name);
}

}  // namespace

extern "C" {

int hers_search_host(hers_ctx* ctx, const hers_keys* keys, const uint64_t* gallery,
                     uint64_t nblocks, uint32_t d, const uint64_t* probe_ct_host,
                     uint64_t* scores_ct_host, void* workspace, uint64_t workspace_bytes,
                     void* stream) {
    return search_host(ctx, keys, gallery, nblocks, d, probe_ct_host, scores_ct_host, workspace,
                       workspace_bytes, stream, true, "hers_search_host");
}

int hers_search_host_async(hers_ctx* ctx, const hers_keys* keys, const uint64_t* gallery,
                           uint64_t nblocks, uint32_t d, const uint64_t* probe_ct_host,
                           uint64_t* scores_ct_host, void* workspace, uint64_t workspace_bytes,
                           void* stream) {
    return search_host(ctx, keys, gallery, nblocks, d, probe_ct_host, scores_ct_host, workspace,
                       workspace_bytes, stream, false, "hers_search_host_async");
}

int hers_decrypt_scores(hers_ctx* ctx, const hers_keys* keys, const uint64_t* scores_ct,
                        uint64_t nblocks, int32_t* scores, uint64_t m, void* stream) {
    if (!ctx || !keys || !scores_ct || !scores) return fail(ctx, HERS_E_INVAL, "hers_decrypt_scores: null argument");
    if (!keys->k.sk) return fail(ctx, HERS_E_INVAL, "hers_decrypt_scores: the keys hold no secret key");
    if (m > nblocks * N) return fail(ctx, HERS_E_INVAL, "hers_decrypt_scores: m > nblocks N");
    DeviceGuard g(ctx->device);
    cudaError_t e = launch_decrypt(ctx->tw, keys->k, scores_ct, nblocks, scores, m, pick(ctx, stream));
    return e == cudaSuccess ? HERS_OK : cuda_fail(ctx, e, "hers_decrypt_scores");
}

int hers_trace_enable(hers_ctx* ctx, uint32_t max_calls) {
    if (!ctx) return HERS_E_INVAL;
    DeviceGuard g(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    trace_free(ctx);
    if (max_calls == 0) return HERS_OK;
    ctx->tev.resize((size_t)max_calls * SEARCH_EVENTS);
    for (size_t i = 0; i < ctx->tev.size(); i++) {
        cudaError_t e = cudaEventCreate(&ctx->tev[i]);
        if (e != cudaSuccess) {
            ctx->tev.resize(i);
            trace_free(ctx);
            return cuda_fail(ctx, e, "hers_trace_enable");
        }
    }
    ctx->tcap = max_calls;
    ctx->tn = 0;
    return HERS_OK;
}

int hers_trace_read(hers_ctx* ctx, uint32_t* ncalls, double* avg_ms) {
    if (!ctx || !ncalls || !avg_ms) return fail(ctx, HERS_E_INVAL, "hers_trace_read: null argument");
    DeviceGuard g(ctx->device);
    double sum[HERS_TRACE_PHASES] = {0, 0, 0, 0, 0};
    for (uint32_t c = 0; c < ctx->tn; c++) {
        cudaEvent_t* ev = &ctx->tev[(size_t)c * SEARCH_EVENTS];
        cudaError_t e = cudaEventSynchronize(ev[SEARCH_EVENTS - 1]);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "hers_trace_read");
        for (int ph = 0; ph < SEARCH_EVENTS - 1; ph++) {
            float ms = 0;
            e = cudaEventElapsedTime(&ms, ev[ph], ev[ph + 1]);
            if (e != cudaSuccess) return cuda_fail(ctx, e, "hers_trace_read");
            sum[ph] += ms;
        }
        float tot = 0;
        cudaEventElapsedTime(&tot, ev[0], ev[SEARCH_EVENTS - 1]);
        sum[HERS_TRACE_PHASES - 1] += tot;
    }
    *ncalls = ctx->tn;
    for (int ph = 0; ph < HERS_TRACE_PHASES; ph++) avg_ms[ph] = ctx->tn ? sum[ph] / ctx->tn : 0.0;
    ctx->tn = 0;
    return HERS_OK;
}

uint64_t hers_kernel_launches(void) { return launches_total(); }

int hers_tensor_variants(void) { return tensor_variant_count(); }

const char* hers_tensor_variant_name(int v) {
    const char* n = tensor_variant_name(v);
    return n ? n : "";
}

int hers_get_tensor_variant(const hers_ctx* ctx) { return ctx ? ctx->tensor_variant : -1; }

int hers_set_tensor_variant(hers_ctx* ctx, int v) {
    if (!ctx) return HERS_E_INVAL;
    if (v < 0 || v >= tensor_variant_count())
        return fail(ctx, HERS_E_INVAL, "hers_set_tensor_variant: %d not in [0, %d)", v,
                    tensor_variant_count());
    ctx->tensor_variant = v;
    return HERS_OK;
}

int hers_set_tensor_first(hers_ctx* ctx, int on) {
    if (!ctx) return HERS_E_INVAL;
    DeviceGuard g(ctx->device);
    // searches already enqueued keep their order; wait for them before the roles change
    cudaStreamSynchronize(ctx->ep);
    ctx->tensor_first = on ? 1 : 0;
    return HERS_OK;
}

int hers_get_tensor_first(const hers_ctx* ctx) { return ctx ? ctx->tensor_first : -1; }

int hers_autotune_extension(hers_ctx* ctx, uint32_t d, void* stream, int* cluster, double* ms) {
    if (!ctx) return HERS_E_INVAL;
    if (d == 0 || d > HERS_MAX_D) return fail(ctx, HERS_E_INVAL, "hers_autotune_extension: d = %u", d);
    DeviceGuard g(ctx->device);
    cudaStream_t st = pick(ctx, stream);
    // d canonical ciphertexts (zero residues are canonical; the work does not
    // depend on the values) and a prepared-probe buffer
    void* buf = nullptr;
    const uint64_t ct_bytes = (uint64_t)d * 4 * N * 8, pr_bytes = (uint64_t)d * RES_WORDS_PER_DIM * 8;
    cudaError_t e = cudaMallocAsync(&buf, ct_bytes + pr_bytes, st);
    if (e != cudaSuccess) return fail(ctx, HERS_E_NOMEM, "hers_autotune_extension: %s", cudaGetErrorString(e));
    uint64_t* cts = (uint64_t*)buf;
    uint64_t* pr = cts + (uint64_t)d * 4 * N;
    e = cudaMemsetAsync(cts, 0, ct_bytes, st);
    cudaEvent_t e0, e1;
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    double best[2] = {0, 0};
    // form 0: one CTA per polynomial; form 1: clusters (2 d polynomials <= the threshold)
    for (int form = 0; form < 2 && e == cudaSuccess; form++) {
        const uint64_t thr = form ? 2ull * d : 0;
        for (int rep = 0; rep < 6 && e == cudaSuccess; rep++) {
            e = cudaEventRecord(e0, st);
            for (int k = 0; k < 8 && e == cudaSuccess; k++) e = launch_extend_ntt(ctx->tw, cts, d, 0, d, pr, st, thr);
            if (e == cudaSuccess) e = cudaEventRecord(e1, st);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float t = 0;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
            if (rep == 1 || (rep > 1 && t / 8 < best[form])) best[form] = t / 8;  // rep 0 warms up
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFreeAsync(buf, st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "hers_autotune_extension");
    const bool use_cluster = best[1] < best[0];
    // the threshold: this size (2 d polynomials) and smaller take the cluster form when it won
    ctx->ext_cluster_max = use_cluster ? 2ull * d : (2ull * d > 2 ? 2ull * d - 2 : 0);
    if (ctx->ext_cluster_max > EXT_CLUSTER_MAX_POLYS && !use_cluster) ctx->ext_cluster_max = EXT_CLUSTER_MAX_POLYS;
    if (cluster) *cluster = use_cluster ? 1 : 0;
    if (ms) {
        ms[0] = best[0];
        ms[1] = best[1];
    }
    return HERS_OK;
}

int hers_epilogue_variants(void) { return EPI_VARIANTS; }

const char* hers_epilogue_variant_name(int v) {
    const char* n = epilogue_variant_name(v);
    return n ? n : "";
}

int hers_get_epilogue_variant(const hers_ctx* ctx) { return ctx ? ctx->epi_variant : -1; }

int hers_set_epilogue_variant(hers_ctx* ctx, int v) {
    if (!ctx) return HERS_E_INVAL;
    if (v < 0 || v >= EPI_VARIANTS)
        return fail(ctx, HERS_E_INVAL, "hers_set_epilogue_variant: %d not in [0, %d)", v, EPI_VARIANTS);
    ctx->epi_variant = v;
    return HERS_OK;
}

int hers_autotune_epilogue(hers_ctx* ctx, const hers_keys* keys, const uint64_t* gallery, uint64_t nblocks,
                           uint32_t d, const uint64_t* probe, void* workspace, uint64_t workspace_bytes,
                           void* stream, int* chosen, double* ms_per_variant) {
    if (!ctx || !keys || !gallery || !probe || !workspace || nblocks == 0)
        return fail(ctx, HERS_E_INVAL, "hers_autotune_epilogue: null argument or no blocks");
    if (d == 0 || d > HERS_MAX_D) return fail(ctx, HERS_E_INVAL, "hers_autotune_epilogue: d = %u", d);
    if (workspace_bytes < hers_search_workspace_bytes(nblocks))
        return fail(ctx, HERS_E_NOMEM, "hers_autotune_epilogue: workspace too small");
    DeviceGuard g(ctx->device);
    cudaStream_t st = pick(ctx, stream);
    uint64_t* ws = (uint64_t*)workspace;
    uint64_t* X = ws;
    uint64_t* C = X + nblocks * 15 * N;
    uint64_t* KS = C + nblocks * 6 * N;
    uint64_t* out = nullptr;
    cudaError_t e = cudaMallocAsync(&out, nblocks * 4 * N * 8, st);
    if (e != cudaSuccess) return fail(ctx, HERS_E_NOMEM, "hers_autotune_epilogue: %s", cudaGetErrorString(e));
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        cudaFreeAsync(out, st);
        return fail(ctx, HERS_E_CUDA, "hers_autotune_epilogue: event creation");
    }
    // each variant: the tensor kernel (untimed) to refill the accumulators,
    // then the epilogue timed; 1 warm-up and 3 timed rounds, minimum kept
    int best = -1;
    float best_ms = 0;
    for (int v = 0; v < EPI_VARIANTS && e == cudaSuccess; v++) {
        float vbest = 0;
        for (int rep = 0; rep < 4 && e == cudaSuccess; rep++) {
            e = launch_tensor(ctx->tensor_variant, gallery, nblocks, d, probe, (uint32_t*)X, ctx->err, st);
            if (e == cudaSuccess) e = cudaEventRecord(e0, st);
            if (e == cudaSuccess) e = launch_epilogue(ctx->tw, keys->k, nblocks, X, C, KS, out, st, nullptr, nullptr, v);
            if (e == cudaSuccess) e = cudaEventRecord(e1, st);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float ms = 0;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (rep == 1 || (rep > 1 && ms < vbest)) vbest = ms;
        }
        if (ms_per_variant) ms_per_variant[v] = vbest;
        if (e == cudaSuccess && (best < 0 || vbest < best_ms)) {
            best = v;
            best_ms = vbest;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFreeAsync(out, st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "hers_autotune_epilogue");
    ctx->epi_variant = best;
    if (chosen) *chosen = best;
    return HERS_OK;
}

int hers_autotune(hers_ctx* ctx, const hers_keys* keys, const uint64_t* gallery, uint64_t nblocks,
                  uint32_t d, const uint64_t* probe, void* workspace, uint64_t workspace_bytes,
                  void* stream, int* chosen, double* ms_per_variant) {
    if (!ctx || !keys || !gallery || !probe || !workspace || nblocks == 0)
        return fail(ctx, HERS_E_INVAL, "hers_autotune: null argument or no blocks");
    if (d == 0 || d > HERS_MAX_D) return fail(ctx, HERS_E_INVAL, "hers_autotune: d = %u", d);
    if (workspace_bytes < hers_search_workspace_bytes(nblocks))
        return fail(ctx, HERS_E_NOMEM, "hers_autotune: workspace too small");
    DeviceGuard g(ctx->device);
    cudaStream_t st = pick(ctx, stream);
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return fail(ctx, HERS_E_CUDA, "hers_autotune: event creation");
    int best = -1;
    float best_ms = 0;
    cudaError_t e = cudaSuccess;
    for (int v = 0; v < tensor_variant_count() && e == cudaSuccess; v++) {
        e = launch_tensor(v, gallery, nblocks, d, probe, (uint32_t*)workspace, ctx->err, st);  // warm
        float vbest = 0;
        for (int rep = 0; rep < 3 && e == cudaSuccess; rep++) {
            cudaEventRecord(e0, st);
            e = launch_tensor(v, gallery, nblocks, d, probe, (uint32_t*)workspace, ctx->err, st);
            cudaEventRecord(e1, st);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float ms = 0;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (rep == 0 || ms < vbest) vbest = ms;
        }
        if (ms_per_variant) ms_per_variant[v] = vbest;
        if (e == cudaSuccess && (best < 0 || vbest < best_ms)) {
            best = v;
            best_ms = vbest;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "hers_autotune");
    ctx->tensor_variant = best;
    if (chosen) *chosen = best;
    return HERS_OK;
}

}  // extern "C"
