// Declarations shared by the library's translation units (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "hers_consts.h"

// The opaque context handle of include/hers.h.
struct hers_ctx {
    int device;
    cudaStream_t stream;  // the context's own stream (synchronous calls)
    uint64_t* tw;         // device twiddle tables [6][4][N]
    int* err;             // device flag: 1 = a sampler ran out of attempts, 2 = a wait gave up
    char msg[512];
    // tracing: SEARCH_EVENTS events per traced hers_search call
    std::vector<cudaEvent_t> tev;
    uint32_t tcap = 0, tn = 0;
    int tensor_variant = 1;  // tensor-kernel shape used by searches on this context
    int epi_variant = 0;     // epilogue form used by every search on this context (EPI_* flags)
    int tensor_first = 0;    // 1: the tensor kernel, not the epilogue, takes the high-priority stream
    uint64_t ext_cluster_max = 64;  // probe preparation: cluster form up to this many polynomials
    int pm = 0;              // plaintext modulus: 0 the default t, 1 the paper's t
    // the epilogue of a search runs on ep (the device's highest stream priority),
    // after ep_ev[0] (tensor done) and before ep_ev[1] (joined back to the caller)
    cudaStream_t ep = nullptr;
    cudaEvent_t ep_ev[2] = {nullptr, nullptr};
};

namespace hers {

// 64-bit words of the resident form per (gallery block, dimension): two
// polynomials of N int32 residues for each of the NUM_S primes of the search basis.
constexpr uint64_t RES_WORDS_PER_DIM = (uint64_t)NUM_S * N;
// Words of a context's twiddle tables: NUM_MODS moduli x (forward, inverse) x
// N pairs of 64-bit words, then NUM_S x 2 x N pairs of 32-bit words.
constexpr uint64_t TW_WORDS = (uint64_t)NUM_MODS * 4 * N + (uint64_t)NUM_S * 2 * N;

// Key material in device memory (all uint64 unless noted):
//   sk        int8 [N]                  ternary secret
//   pk        [2 polys][2 limbs][N]     canonical public key
//   evk       [2 j][2 polys][2 limbs][N] canonical relinearisation keys
//   pk_ntt    [2 polys][2 limbs][2][N]  NTT form and Shoup companion (encryption)
//   evk_ntt   [2 j][2 polys][2 limbs][2][N] NTT form + Shoup (key switch)
//   s_ntt     [2 limbs][2][N]           NTT form of s + Shoup (decryption)
struct DevKeys {
    int pm;  // plaintext modulus of the context: index into c_plain (0 default t, 1 the paper's t)
    int8_t* sk;
    uint64_t* pk;
    uint64_t* evk;
    uint64_t* pk_ntt;
    uint64_t* evk_ntt;
    uint64_t* s_ntt;
};
}  // namespace hers

// The opaque key handle of include/hers.h.
struct hers_keys {
    hers_ctx* ctx;
    hers::DevKeys k;
    void* base;  // single device allocation holding every key array
    // base-w gadget keys (hers_keys_add_basew), 0 / null when absent
    uint32_t logw = 0, ndig = 0;
    uint64_t* evkw = nullptr;      // [ndig][2 polys][2 limbs][N], canonical
    uint64_t* evkw_ntt = nullptr;  // [ndig][2][2][2][N]: NTT values and Shoup companions
};

namespace hers {
// Host helpers shared by the entry-point files.
int fail(hers_ctx* ctx, int code, const char* fmt, ...);
int cuda_fail(hers_ctx* ctx, cudaError_t e, const char* where);
// Makes a device current for the duration of a call, restoring the previous one.
struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev);
    ~DeviceGuard();
};

// scheme.cu
cudaError_t launch_keygen(const uint64_t* tw, uint64_t seed, DevKeys k, int* err, cudaStream_t st);
// NTT forms (with Shoup companions) of the canonical pk and evk in k.
cudaError_t launch_key_ntt(const uint64_t* tw, const DevKeys& k, cudaStream_t st);
// Base-w gadget (w = 2^logw): digits and key generation / key switch pieces.
constexpr uint32_t BASEW_MIN = 22, BASEW_MAX = 60;  // at most 5 digits: they fit the workspace
uint32_t basew_digits(uint32_t logw);
cudaError_t launch_keygen_w(const uint64_t* tw, uint64_t seed, uint32_t logw, uint32_t ndig, const DevKeys& k,
                            uint64_t* evkw, uint64_t* evkw_ntt, int* err, cudaStream_t st);
struct KeySwitchW {
    const uint64_t* evkw_ntt;
    uint32_t logw, ndig;
};
// Encryption modes of launch_encrypt: gallery blocks (Eq. 3), probe dimensions
// (Eq. 2), or encryptions of zero (output re-randomisation, obj = block).
// ENC_SLOT: one entry's d dimensions, each into the single slot `m` mod N of
// global slot m = b N + v (Alg 6's BatchEncode(.; v)); ciphertext c is dim c.
constexpr int ENC_GALLERY = 0, ENC_PROBE = 1, ENC_ZERO = 2, ENC_SLOT = 3;
cudaError_t launch_encrypt(const uint64_t* tw, const DevKeys& k, const int8_t* feats, uint64_t m,
                           uint32_t d, uint64_t ct_begin, uint64_t nct, int mode, uint64_t seed,
                           uint64_t* out_ct, int* err, cudaStream_t st);
// out[c] += add[c] mod q for nct canonical ciphertexts.
cudaError_t launch_ct_add(uint64_t* out, const uint64_t* add, uint64_t nct, cudaStream_t st);
// Canonical ciphertexts of blocks b .. b + nb - 1 (d each) recovered from the
// resident form (inverse NTTs and the CRT of the search basis), plus add[c]
// mod q when add is non-null, into out[c] (c counts from block b's first).
cudaError_t launch_resident_to_canonical_add(const uint64_t* tw, const uint64_t* resident, uint64_t b,
                                             uint32_t d, const uint64_t* add, uint64_t* out, cudaStream_t st,
                                             uint32_t nb = 1);
// Canonical cts ct[0 .. nct) (global indices ct_begin ..) of dimension d into
// the resident form at `out` (the base of block 0; RES_WORDS_PER_DIM words per
// (block, dimension)).
// Calls of at most cluster_max_polys polynomials take the cluster form
// (k_extend_ntt_cluster), larger ones one CTA per polynomial; both write the
// same bytes.
constexpr uint64_t EXT_CLUSTER_MAX_POLYS = 64;
cudaError_t launch_extend_ntt(const uint64_t* tw, const uint64_t* ct, uint64_t nct, uint64_t ct_begin,
                              uint32_t d, uint64_t* out, cudaStream_t st,
                              uint64_t cluster_max_polys = EXT_CLUSTER_MAX_POLYS);
cudaError_t launch_decrypt(const uint64_t* tw, const DevKeys& k, const uint64_t* scores_ct,
                           uint64_t nblocks, int32_t* scores, uint64_t m, cudaStream_t st);

// search.cu
// Workspace words per gallery block used by the search pipeline.
constexpr uint64_t SEARCH_WS_WORDS_PER_BLOCK = (15 + 6 + 4) * 4096ull;
// Phase boundaries recorded by launch_search when `ev` is non-null:
// ev[0] before the tensor kernel, ev[1] after it, ev[2] after the inverse
// NTTs, ev[3] after scale-and-round, ev[4] after the key switch.
constexpr int SEARCH_EVENTS = 5;
// `err` receives bit 2 if a bounded wait inside a streaming kernel gave up.
// `variant` selects the tensor-kernel shape (see tensor_variant_name).
constexpr int DEFAULT_TENSOR_VARIANT = 1;
// ksw (optional): key switch with the base-w gadget instead of the RNS one.
// ep (optional): the epilogue runs on ep.stream (a high-priority stream), so
// that its CTAs are dispatched ahead of pending CTAs of another search's
// tensor kernel; ep.ev[0] and ep.ev[1] fork from and join back to st.
// With tensor_first, the roles swap: the tensor kernel runs on ep.stream and
// the epilogue on st, so a search's tensor kernel is dispatched ahead of the
// previous search's epilogue and the epilogue fills what the SMs have left.
struct EpilogueStream {
    cudaStream_t stream;
    cudaEvent_t ev[2];
    bool tensor_first = false;
};
// Epilogue forms (every form computes the same bytes): EPI_INTT_SCALE_CLUSTER
// fuses the inverse NTTs with scale-and-round (clusters of NUM_S CTAs);
// EPI_KS_FUSED does the RNS key switch in one kernel per (pair, limb);
// EPI_INTT_SHFL makes the inverse NTTs' first exchange a warp-shuffle
// transpose instead of a pass through shared memory; EPI_LEAN compiles the
// split inverse NTTs and key-switch kernels for one more CTA per SM (fewer
// registers), so more of them run beside a persistent tensor kernel;
// EPI_KS_SHFL makes the in-warp exchange of the split key switch's 64-bit
// NTTs a warp-shuffle transpose.  Variant v is the OR of the flags,
// 0 <= v < EPI_VARIANTS.
constexpr int EPI_INTT_SCALE_CLUSTER = 1, EPI_KS_FUSED = 2, EPI_INTT_SHFL = 4, EPI_LEAN = 8, EPI_KS_SHFL = 16,
              EPI_VARIANTS = 32;
const char* epilogue_variant_name(int v);
cudaError_t launch_search(const uint64_t* tw, const DevKeys& k, const uint64_t* gallery,
                          uint64_t nblocks, uint32_t d, const uint64_t* probe, uint64_t* scores_ct,
                          uint64_t* ws, int* err, cudaStream_t st, cudaEvent_t* ev = nullptr,
                          int variant = DEFAULT_TENSOR_VARIANT, const KeySwitchW* ksw = nullptr,
                          const EpilogueStream* ep = nullptr, int epi = 0);
// Epilogue over npairs accumulators X (uint32 [npairs][3][NUM_S][N] at the
// start of the X area, 15 N words per pair); workspace C, KS as in
// launch_search; `ev` (optional) receives the boundaries after the inverse
// NTTs (ev[0]) and after scale-and-round (ev[1]).
// With ksw, the key switch uses the base-w gadget: its digits [npairs][ndig]
// [2][N] go after O in X (O [npairs][4][N] at X; 4 + 2 ndig <= 15 words per N).
cudaError_t launch_epilogue(const uint64_t* tw, const DevKeys& k, uint64_t npairs, uint64_t* X,
                            uint64_t* C, uint64_t* KS, uint64_t* out, cudaStream_t st,
                            cudaEvent_t* ev = nullptr, const KeySwitchW* ksw = nullptr, int epi = 0);
// The tensor kernel alone, into X [nblocks][3][NUM_S][N] (uint32).
cudaError_t launch_tensor(int variant, const uint64_t* gallery, uint64_t nblocks, uint32_t d,
                          const uint64_t* probe, uint32_t* X, int* err, cudaStream_t st);
int tensor_variant_count();
const char* tensor_variant_name(int v);

// A block range of one resident gallery against one prepared probe; the
// result of block b goes to pair pair_base + (b - begin).
struct RangeItem {
    const uint64_t* gallery;  // block 0 of the resident gallery
    uint64_t begin, end;
    uint32_t d;
    const uint64_t* probe;
    uint64_t pair_base;
};

// batch.cu: work tables of the persistent batched tensor kernel.
constexpr int BATCH_NPMAX = 16;
struct BatchChunk {  // up to BATCH_NPMAX probes sharing one gallery segment
    const uint64_t* gallery;
    const uint64_t* probe[BATCH_NPMAX];
    uint64_t pair[BATCH_NPMAX];  // pair of probe q at absolute block b: pair[q] + b (mod 2^64)
    uint32_t d, np;
};
// A segment: blocks [s0, s1) of one gallery, all searched by the same probes,
// cut into nch probe chunks.  Its work units are (limb, tile, block group of
// the kernel's NB blocks, chunk), numbered in that order from first_unit; the
// kernel decodes a unit index into them, so no per-unit table is built.
struct BatchSeg {
    uint32_t first_unit;
    uint32_t first_chunk, nch;
    uint32_t nbg;  // block groups: ceil((s1 - s0) / NB)
    uint32_t s0, s1;
};
// Plans range items into chunks and segments; *nunits receives the number of
// work units (HERS_E_INVAL-worthy when it reaches 2^32 - 1: the caller checks).
void plan_ranges(const RangeItem* items, uint32_t nitems, int np_max, int nb_max,
                 std::vector<BatchChunk>& chunks, std::vector<BatchSeg>& segs, uint32_t* ngroups,
                 uint64_t* nunits);
constexpr int DEFAULT_BATCH_VARIANT = 1;
int batch_variant_count();
int batch_variant_np(int v);
int batch_variant_nb(int v);
cudaError_t launch_batched(int v, const BatchChunk* d_chunks, const BatchSeg* d_segs, uint32_t nsegs,
                           uint32_t nunits, uint32_t* d_counter, uint64_t* X, int* err, int device, cudaStream_t st);

// Kernel launches issued by this library in this process (all contexts).
void count_launches(uint64_t n);
uint64_t launches_total();

}  // namespace hers
