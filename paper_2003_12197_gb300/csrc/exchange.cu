// Client/server exchange calls of the HERS C ABI (include/hers.h), following
// the paper's problem statement and protocols (Sec. 3.1: the client encrypts
// with pk and decrypts with sk, the server computes with pk and evk only;
// Algs 6-7: enrollment and search between the two):
//   - a server-side key handle built from the public and evaluation keys
//     alone, so the secret key never reaches the server's device;
//   - canonical ciphertexts in and out of the resident gallery form
//     (persistence and transfer of an encrypted gallery);
//   - host-buffer forms of gallery enrollment and of score decryption;
//   - a block range of a resident gallery as the search's extent.
// The arithmetic stays in the kernels of scheme.cu and search.cu; these calls
// check arguments, stage host buffers and order the launches.
#include <string.h>

#include <new>

#include "hers.h"
#include "hers_consts.h"
#include "internal.h"

using namespace hers;

namespace {

const uint64_t H_MODS[NUM_MODS] = HERS_MOD_INIT;  // q1, q2 first

// Staging budget of the host-buffer calls (bytes of device memory held for
// the duration of a call).
constexpr uint64_t STAGE_BYTES = 256ull << 20;

// True if every residue of `polys` canonical polynomials [..][2 limbs][N]
// lies in [0, q_l).
bool canonical(const uint64_t* x, uint64_t polys) {
    for (uint64_t p = 0; p < polys; p++) {
        const uint64_t q = H_MODS[p & 1];
        const uint64_t* r = x + p * N;
        for (int k = 0; k < N; k++)
            if (r[k] >= q) return false;
    }
    return true;
}

// Frees a stream-ordered allocation when the scope ends.
struct StageBuf {
    void* p = nullptr;
    cudaStream_t st;
    explicit StageBuf(cudaStream_t s) : st(s) {}
    cudaError_t alloc(uint64_t bytes) { return cudaMallocAsync(&p, bytes, st); }
    ~StageBuf() {
        if (p) cudaFreeAsync(p, st);
    }
};

}  // namespace

extern "C" {

int hers_keys_import(hers_ctx* ctx, const uint64_t* pk, const uint64_t* evk, hers_keys** out) {
    if (!ctx || !pk || !evk || !out) return fail(ctx, HERS_E_INVAL, "hers_keys_import: null argument");
    *out = nullptr;
    if (!canonical(pk, 4) || !canonical(evk, 8))
        return fail(ctx, HERS_E_INVAL, "hers_keys_import: a key residue is not in [0, q_l)");
    DeviceGuard g(ctx->device);
    hers_keys* K = new (std::nothrow) hers_keys();
    if (!K) return fail(ctx, HERS_E_NOMEM, "hers_keys_import: host allocation");
    K->ctx = ctx;
    K->k.pm = ctx->pm;
    // the public part of hers_keygen's layout: pk, evk, pk_ntt, evk_ntt (words)
    const size_t w_pk = 4 * N, w_evk = 8 * N, w_pkn = 8 * N, w_evkn = 16 * N;
    cudaError_t e = cudaMalloc(&K->base, (w_pk + w_evk + w_pkn + w_evkn) * 8);
    if (e != cudaSuccess) {
        delete K;
        return fail(ctx, HERS_E_NOMEM, "hers_keys_import: %s", cudaGetErrorString(e));
    }
    uint64_t* b = (uint64_t*)K->base;
    K->k.pk = b;
    K->k.evk = b + w_pk;
    K->k.pk_ntt = K->k.evk + w_evk;
    K->k.evk_ntt = K->k.pk_ntt + w_pkn;
    K->k.s_ntt = nullptr;  // no secret key on this handle
    K->k.sk = nullptr;
    e = cudaMemcpyAsync(K->k.pk, pk, w_pk * 8, cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(K->k.evk, evk, w_evk * 8, cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) e = launch_key_ntt(ctx->tw, K->k, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) {
        cudaFree(K->base);
        delete K;
        return cuda_fail(ctx, e, "hers_keys_import");
    }
    *out = K;
    return HERS_OK;
}

int hers_keys_has_secret(const hers_keys* keys) { return keys && keys->k.sk ? 1 : 0; }

int hers_search_range(hers_ctx* ctx, const hers_keys* keys, const uint64_t* gallery, uint64_t nblocks,
                      uint32_t d, uint64_t block_begin, uint64_t block_end, const uint64_t* probe,
                      uint64_t* scores_ct, void* workspace, uint64_t workspace_bytes, void* stream) {
    if (!ctx || !gallery) return fail(ctx, HERS_E_INVAL, "hers_search_range: null argument");
    if (block_begin > block_end || block_end > nblocks)
        return fail(ctx, HERS_E_INVAL, "hers_search_range: blocks [%llu, %llu) not inside [0, %llu)",
                    (unsigned long long)block_begin, (unsigned long long)block_end,
                    (unsigned long long)nblocks);
    if (d == 0 || d > HERS_MAX_D) return fail(ctx, HERS_E_INVAL, "hers_search_range: d = %u", d);
    return hers_search(ctx, keys, gallery + block_begin * d * RES_WORDS_PER_DIM, block_end - block_begin, d,
                       probe, scores_ct, workspace, workspace_bytes, stream);
}

int hers_encrypt_gallery_host(hers_ctx* ctx, const hers_keys* keys, const int8_t* feats_host, uint64_t m,
                              uint32_t d, uint64_t seed, uint64_t* gallery, uint64_t* gallery_ct,
                              void* stream) {
    if (!ctx || !keys || !feats_host || (!gallery && !gallery_ct))
        return fail(ctx, HERS_E_INVAL, "hers_encrypt_gallery_host: null argument");
    if (m == 0 || d == 0 || d > HERS_MAX_D)
        return fail(ctx, HERS_E_INVAL, "hers_encrypt_gallery_host: m = %llu, d = %u", (unsigned long long)m, d);
    DeviceGuard g(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    int rc = HERS_OK;
    {
        StageBuf f(st);
        cudaError_t e = f.alloc(m * d);
        if (e != cudaSuccess)
            return fail(ctx, HERS_E_NOMEM, "hers_encrypt_gallery_host: %s", cudaGetErrorString(e));
        e = cudaMemcpyAsync(f.p, feats_host, m * d, cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "hers_encrypt_gallery_host: copy");
        rc = hers_encrypt_gallery(ctx, keys, (const int8_t*)f.p, m, d, seed, gallery, gallery_ct, stream);
    }
    if (rc != HERS_OK) return rc;
    return hers_check(ctx, stream);
}

int hers_decrypt_scores_host(hers_ctx* ctx, const hers_keys* keys, const uint64_t* scores_ct_host,
                             uint64_t nblocks, int32_t* scores_host, uint64_t m) {
    if (!ctx || !keys || !scores_ct_host || !scores_host)
        return fail(ctx, HERS_E_INVAL, "hers_decrypt_scores_host: null argument");
    if (!keys->k.sk) return fail(ctx, HERS_E_INVAL, "hers_decrypt_scores_host: the keys hold no secret key");
    if (m > nblocks * N) return fail(ctx, HERS_E_INVAL, "hers_decrypt_scores_host: m > nblocks N");
    DeviceGuard g(ctx->device);
    cudaStream_t st = ctx->stream;
    const uint64_t ctb = 4ull * N * 8;
    const uint64_t per = STAGE_BYTES / (ctb + N * 4);  // blocks per pass
    StageBuf buf(st);
    cudaError_t e = buf.alloc(per * (ctb + N * 4));
    if (e != cudaSuccess) return fail(ctx, HERS_E_NOMEM, "hers_decrypt_scores_host: %s", cudaGetErrorString(e));
    uint64_t* cts = (uint64_t*)buf.p;
    int32_t* sc = (int32_t*)(cts + per * 4 * N);
    for (uint64_t b0 = 0; b0 * N < m && e == cudaSuccess; b0 += per) {
        const uint64_t nb = nblocks - b0 < per ? nblocks - b0 : per;
        const uint64_t mm = m - b0 * N < nb * N ? m - b0 * N : nb * N;
        e = cudaMemcpyAsync(cts, scores_ct_host + b0 * 4 * N, nb * ctb, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = launch_decrypt(ctx->tw, keys->k, cts, nb, sc, mm, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(scores_host + b0 * N, sc, mm * 4, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    }
    return e == cudaSuccess ? HERS_OK : cuda_fail(ctx, e, "hers_decrypt_scores_host");
}

int hers_export_ct(hers_ctx* ctx, const uint64_t* gallery, uint64_t nblocks, uint32_t d, uint64_t block_begin,
                   uint64_t block_end, uint64_t* ct_host) {
    if (!ctx || !gallery || !ct_host) return fail(ctx, HERS_E_INVAL, "hers_export_ct: null argument");
    if (d == 0 || d > HERS_MAX_D) return fail(ctx, HERS_E_INVAL, "hers_export_ct: d = %u", d);
    if (block_begin > block_end || block_end > nblocks)
        return fail(ctx, HERS_E_INVAL, "hers_export_ct: blocks [%llu, %llu) not inside [0, %llu)",
                    (unsigned long long)block_begin, (unsigned long long)block_end, (unsigned long long)nblocks);
    if (block_begin == block_end) return HERS_OK;
    DeviceGuard g(ctx->device);
    cudaStream_t st = ctx->stream;
    const uint64_t blk_bytes = (uint64_t)d * 4 * N * 8;
    uint64_t per = STAGE_BYTES / blk_bytes;
    if (per == 0) per = 1;
    if (per > 65535) per = 65535;
    StageBuf buf(st);
    cudaError_t e = buf.alloc(per * blk_bytes);
    if (e != cudaSuccess) return fail(ctx, HERS_E_NOMEM, "hers_export_ct: %s", cudaGetErrorString(e));
    for (uint64_t b0 = block_begin; b0 < block_end && e == cudaSuccess; b0 += per) {
        const uint64_t nb = block_end - b0 < per ? block_end - b0 : per;
        e = launch_resident_to_canonical_add(ctx->tw, gallery, b0, d, nullptr, (uint64_t*)buf.p, st,
                                             (uint32_t)nb);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(ct_host + (b0 - block_begin) * d * 4 * N, buf.p, nb * blk_bytes,
                                cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    }
    return e == cudaSuccess ? HERS_OK : cuda_fail(ctx, e, "hers_export_ct");
}

int hers_import_ct(hers_ctx* ctx, const uint64_t* ct_host, uint64_t nblocks, uint32_t d, uint64_t block_begin,
                   uint64_t block_end, uint64_t* gallery) {
    if (!ctx || !gallery || !ct_host) return fail(ctx, HERS_E_INVAL, "hers_import_ct: null argument");
    if (d == 0 || d > HERS_MAX_D) return fail(ctx, HERS_E_INVAL, "hers_import_ct: d = %u", d);
    if (block_begin > block_end || block_end > nblocks)
        return fail(ctx, HERS_E_INVAL, "hers_import_ct: blocks [%llu, %llu) not inside [0, %llu)",
                    (unsigned long long)block_begin, (unsigned long long)block_end, (unsigned long long)nblocks);
    if (block_begin == block_end) return HERS_OK;
    if (!canonical(ct_host, (block_end - block_begin) * d * 2))
        return fail(ctx, HERS_E_INVAL, "hers_import_ct: a ciphertext residue is not in [0, q_l)");
    DeviceGuard g(ctx->device);
    cudaStream_t st = ctx->stream;
    const uint64_t ct_bytes = 4ull * N * 8;
    const uint64_t per = STAGE_BYTES / ct_bytes;  // ciphertexts per pass
    StageBuf buf(st);
    cudaError_t e = buf.alloc(per * ct_bytes);
    if (e != cudaSuccess) return fail(ctx, HERS_E_NOMEM, "hers_import_ct: %s", cudaGetErrorString(e));
    const uint64_t c_begin = block_begin * d, c_end = block_end * d;
    for (uint64_t c0 = c_begin; c0 < c_end && e == cudaSuccess; c0 += per) {
        const uint64_t n = c_end - c0 < per ? c_end - c0 : per;
        e = cudaMemcpyAsync(buf.p, ct_host + (c0 - c_begin) * 4 * N, n * ct_bytes, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = launch_extend_ntt(ctx->tw, (const uint64_t*)buf.p, n, c0, d, gallery, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    }
    return e == cudaSuccess ? HERS_OK : cuda_fail(ctx, e, "hers_import_ct");
}

}  // extern "C"
