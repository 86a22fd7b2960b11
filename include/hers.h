/*
 * hers.h -- C ABI of the GB300 HERS encrypted-search library (libhers.so).
 *
 * HERS (Engelsma, Jain, Boddeti) scores an encrypted probe q against an
 * encrypted gallery P = [p_1 .. p_m] of d-dimensional int8 features: the
 * server computes Enc(P^T q) (Sec. 3.1, Eq. 1) without decrypting either
 * side, and the client decrypts the m scores and takes the argmax (Alg 7).
 *
 * Scheme: FV (App. A, Algs 1-5) over R_q = Z_q[x]/(x^N + 1), N = 4096,
 * q = q1 q2 (two 54-bit NTT primes, 108 bits), plaintext modulus t = 4169729
 * by default or the paper's t = 1032193 (Sec. 4.1) as a context option (both
 * prime, t = 1 mod 2N, so plaintexts have N SIMD slots).  Gallery dimension
 * i of entries bN .. bN+N-1 is one plaintext (Eq. 3, one "block" b); probe
 * dimension i fills every slot (Eq. 2).  A block's score ciphertext is
 * sum_i ct_i (x) D_i^b (Eq. 4, Alg 7), with the degree-2 tensor accumulated
 * over i, scaled by t/q once and relinearised once (Alg 5's steps, moved
 * after the sum).
 *
 * Conventions common to every call:
 *  - Return value: HERS_OK (0) or a negative HERS_E_* status; on error the
 *    context's message is available from hers_last_error(ctx).
 *  - Pointers documented "device" are CUDA device pointers on the context's
 *    device, owned by the caller, who allocates them with the byte counts the
 *    hers_*_bytes() helpers give; pointers documented "host" are ordinary
 *    host memory, owned by the caller.  The library never frees caller memory.
 *  - stream: a cudaStream_t cast to void*; NULL is CUDA's default (legacy)
 *    stream.  Calls that only read/write device memory are asynchronous on
 *    that stream, so the caller keeps their buffers alive until the stream
 *    has run them; calls that write host memory return after the data is
 *    there.  Synchronous calls (hers_keygen) use the context's own stream.
 *  - Canonical ciphertext ("ct"): uint64 [2 polys][2 limbs][N], coefficient
 *    domain, limb 0 holds residues mod q1 in [0, q1), limb 1 mod q2 in [0, q2).
 *    This is the form ciphertexts are exchanged and compared in.
 *  - Handles (hers_ctx, hers_keys) are not safe for concurrent mutation from
 *    several host threads.
 *  - Every random draw (keys, encryption randomness) is a ChaCha20 (RFC 8439)
 *    stream keyed by the 64-bit seed argument, so identical seeds give
 *    identical bytes.
 */
#ifndef HERS_H
#define HERS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define HERS_OK 0
#define HERS_E_INVAL (-1)   /* bad argument (null pointer, size, d mismatch) */
#define HERS_E_NOMEM (-2)   /* device allocation failed or workspace too small */
#define HERS_E_CUDA (-3)    /* a CUDA call or kernel failed */
#define HERS_E_TIMEOUT (-4) /* a bounded device-side wait gave up */
#define HERS_E_PARAM (-5)   /* unsupported scheme parameters */
#define HERS_E_SAMPLER (-7) /* a rejection sampler exhausted its attempts */

#define HERS_N 4096u        /* ring degree n (Sec. 4.1) */
#define HERS_MAX_D 512u     /* largest feature dimension d accepted */

typedef struct hers_ctx hers_ctx;
typedef struct hers_keys hers_keys;

/* Scheme parameters (App. A; Sec. 4.1 fixes n and the paper's t, the rest is
 * this library's reading).  n and q must be the defaults; t is 4169729 (the
 * default: it holds every score of any int8 vectors, |score| <= d 127^2 < t/2
 * for d <= 128) or 1032193 (the paper's: it holds the scores of L2-normalised
 * int8 features, |score| < 131^2).  hers_create() checks. */
typedef struct hers_params {
    uint32_t n;       /* ring degree, 4096 */
    uint64_t q[2];    /* ciphertext modulus primes q1, q2 */
    uint64_t t;       /* plaintext modulus */
    uint32_t flags;   /* reserved, 0 */
} hers_params;

/* Fills *out with the default parameter set. */
int hers_default_params(hers_params* out);

/* Creates a context on CUDA device `device` with parameters p (NULL: the
 * defaults): uploads NTT twiddle tables and creates the context stream.  Keys
 * made on the context, and every call with them, use its plaintext modulus.
 * *out is owned by the caller, freed by hers_destroy.  HERS_E_PARAM for an
 * unsupported parameter set. */
int hers_create(const hers_params* p, int device, hers_ctx** out);
int hers_destroy(hers_ctx* ctx);

/* Message of the last failed call on ctx (never NULL; "" when none). */
const char* hers_last_error(const hers_ctx* ctx);
/* Static name of a status code. */
const char* hers_status_string(int status);

/* Buffer sizes, in bytes. */
uint64_t hers_ct_bytes(void);                                    /* one canonical ct: 2*2*N*8 */
uint64_t hers_gallery_bytes(uint64_t nblocks, uint32_t d);       /* resident gallery */
uint64_t hers_probe_bytes(uint32_t d);                           /* prepared probe */
uint64_t hers_search_workspace_bytes(uint64_t nblocks);          /* hers_search scratch */
uint64_t hers_blocks_for(uint64_t m);                            /* ceil(m / N) (Sec. 3.2 footnote) */

/*
 * Key generation (App. A, Alg 1).  Samples the ternary secret s, the public
 * key pk = ([-(a s + e)]_q, a) and two relinearisation keys
 * evk_j = ([-(a_j s + e_j) + g_j s^2]_q, a_j), g_j = (q/q_j) [(q/q_j)^-1]_{q_j}
 * (an RNS gadget: the base-w decomposition of Alg 1 with one digit per prime).
 * All key material stays in device memory inside *out (freed by
 * hers_keys_free): this is the client's handle, secret key included.  A
 * server builds its own handle from pk and evk alone (hers_keys_export on
 * the client, hers_keys_import on the server).  Synchronous.  HERS_E_SAMPLER if a sampler ran out of
 * attempts (probability below 2^-400).
 */
int hers_keygen(hers_ctx* ctx, uint64_t seed, hers_keys** out);
int hers_keys_free(hers_keys* keys);

/* Copies the keys to host memory in canonical form (for checking and
 * storage): sk int8[N] in {-1,0,1}; pk uint64[2][2][N]; evk uint64[2][2][2][N]
 * ([digit j][poly][limb][N]).  Any pointer may be NULL to skip it. */
int hers_keys_export(hers_ctx* ctx, const hers_keys* keys, int8_t* sk, uint64_t* pk,
                     uint64_t* evk);

/*
 * Server-side keys (Sec. 3.1: the server holds pk and evk, never sk; Alg 7's
 * server loop uses only evk, Alg 6's server side only pk).  Builds a key
 * handle on ctx from the canonical public key pk, host uint64 [2][2][N], and
 * relinearisation keys evk, host uint64 [2][2][2][N] ([digit j][poly][limb][N]),
 * as hers_keys_export writes them on the client.  Every residue must lie in
 * [0, q_l) (HERS_E_INVAL otherwise).  The handle serves every call that
 * encrypts or searches (hers_encrypt_*, hers_enroll, hers_search*,
 * hers_batch_*, hers_server_*, hers_search_stream); calls that need the secret
 * key (hers_decrypt_scores*, hers_keys_add_basew, hers_keys_export of sk)
 * return HERS_E_INVAL with it.  Synchronous; freed by hers_keys_free.
 * hers_keys_has_secret: 1 if the handle holds a secret key (hers_keygen), 0
 * if not (hers_keys_import) or keys is NULL.
 */
int hers_keys_import(hers_ctx* ctx, const uint64_t* pk, const uint64_t* evk, hers_keys** out);
int hers_keys_has_secret(const hers_keys* keys);

/*
 * Enrollment, batch form (Alg 6; Eq. 3 encoding; Alg 2 encryption).
 * feats: device int8 [m][d] row-major (entry-major).  Block b, dimension i
 * becomes the plaintext whose slot j holds feats[b N + j][i] (0 past m),
 * encrypted with randomness stream obj = b d + i.
 * gallery: device, hers_gallery_bytes(ceil(m/N), d) bytes: the resident form
 *   the search streams (the centred lift of every ciphertext coefficient, in
 *   the NTT domain of each of the library's eight 30-bit search primes, one
 *   int32 per residue; the layout is private to the library), or NULL to
 *   write the canonical cts only (for hers_search_stream).
 * gallery_ct: device uint64 [ceil(m/N)][d][2][2][N] canonical cts, or NULL
 *   (at least one of gallery, gallery_ct is non-NULL).
 * Asynchronous on stream; sampler failures are reported by the next
 * synchronous call on ctx (hers_check).
 */
int hers_encrypt_gallery(hers_ctx* ctx, const hers_keys* keys, const int8_t* feats, uint64_t m,
                         uint32_t d, uint64_t seed, uint64_t* gallery, uint64_t* gallery_ct,
                         void* stream);

/*
 * hers_encrypt_gallery with the features in host memory: feats_host, host
 * int8 [m][d] row-major, pageable or pinned.  The call stages them in a
 * temporary device buffer of m d bytes (stream-ordered allocation on
 * `stream`, freed before it returns), encrypts as hers_encrypt_gallery does,
 * and returns after the gallery is written (synchronous; sampler failures are
 * reported as HERS_E_SAMPLER).  Same gallery and gallery_ct arguments.
 */
int hers_encrypt_gallery_host(hers_ctx* ctx, const hers_keys* keys, const int8_t* feats_host, uint64_t m,
                              uint32_t d, uint64_t seed, uint64_t* gallery, uint64_t* gallery_ct,
                              void* stream);

/*
 * Persistence and transfer of a resident gallery in the exchange form (Alg 6:
 * the server stores the enrolled ciphertexts; a ciphertext is a pair of
 * polynomials in R_q, App. A).  The resident form is private to the library;
 * these calls convert blocks [block_begin, block_end) of a resident gallery of
 * nblocks blocks and dimension d to and from canonical ciphertexts in host
 * memory, ct_host uint64 [block_end - block_begin][d][2][2][N] (the layout of
 * hers_encrypt_gallery's gallery_ct).
 * hers_export_ct: resident -> canonical (inverse NTTs and the CRT of the
 *   search basis on the device), exactly the ciphertexts that were enrolled.
 * hers_import_ct: canonical -> resident (the extension of
 *   hers_encrypt_gallery); HERS_E_INVAL if a residue is not in [0, q_l).
 * Both are synchronous on the context's stream and use a device staging
 * buffer of at most 256 MiB for the duration of the call; host buffers may be
 * pageable.  An empty range does nothing.
 */
int hers_export_ct(hers_ctx* ctx, const uint64_t* gallery, uint64_t nblocks, uint32_t d, uint64_t block_begin,
                   uint64_t block_end, uint64_t* ct_host);
int hers_import_ct(hers_ctx* ctx, const uint64_t* ct_host, uint64_t nblocks, uint32_t d, uint64_t block_begin,
                   uint64_t block_end, uint64_t* gallery);

/*
 * Online single-entry enrollment (Alg 6): the entry's d int8 features (device
 * pointer `feats`) go into slot `slot` of resident block `block` of a gallery
 * of nblocks blocks and dimension d.  For each dimension i the call encrypts
 * the plaintext whose slot `slot` holds feats[i] and every other slot 0
 * (BatchEncode(.; v)), with u, e1, e2 from the streams (seed, 0x41..0x43,
 * (block N + slot) d + i), adds it to the block's ciphertext (CipherAdd), and
 * rewrites that ciphertext's resident form.  The block's canonical
 * ciphertexts are recovered from the resident form, so no canonical copy is
 * needed.  The slot should be empty (it holds 0 for padded slots); otherwise
 * its value becomes the sum.  workspace: device, hers_enroll_workspace_bytes(d)
 * bytes.  Asynchronous on `stream`.  HERS_E_INVAL for a block or slot out of
 * range.
 */
uint64_t hers_enroll_workspace_bytes(uint32_t d);
int hers_enroll(hers_ctx* ctx, const hers_keys* keys, uint64_t* gallery, uint64_t nblocks, uint32_t d,
                uint64_t block, uint32_t slot, const int8_t* feats, uint64_t seed, void* workspace,
                uint64_t workspace_bytes, void* stream);

/*
 * Probe encryption (Alg 7 client side; Eq. 2 encoding; Alg 2).
 * q: device int8 [d].  Dimension i is the constant plaintext q[i] (every slot
 * = q[i]), encrypted under pk with randomness stream obj = i.
 * probe_ct: device uint64 [d][2][2][N] canonical cts (what the client sends).
 */
int hers_encrypt_probe(hers_ctx* ctx, const hers_keys* keys, const int8_t* q, uint32_t d,
                       uint64_t seed, uint64_t* probe_ct, void* stream);

/* Server side: turns d received canonical probe cts (device) into the form
 * the search reads (device, hers_probe_bytes(d) bytes). */
int hers_probe_prepare(hers_ctx* ctx, const uint64_t* probe_ct, uint32_t d, uint64_t* probe,
                       void* stream);

/*
 * Encrypted search (Alg 7 server loop; Eq. 4; Alg 5), one probe against
 * blocks [0, nblocks) of a resident gallery of dimension d.
 * For every block b: X_k = sum_i tensor_k(ct_i, D_i^b) exactly (k = 0, 1, 2),
 * c_k = [round(t X_k / q)]_q, then one relinearisation with evk.
 * scores_ct: device uint64 [nblocks][2][2][N] canonical score cts.
 * workspace: device scratch of at least hers_search_workspace_bytes(nblocks).
 * Reads only the evaluation key of `keys`.  Asynchronous on stream: the
 * tensor kernel runs on `stream`; the rounding and relinearisation run on a
 * high-priority stream of the context, forked after the tensor kernel and
 * joined back to `stream` with events, so work enqueued on `stream` after
 * the call (or a synchronisation of `stream`) sees the finished scores.
 * Searches on several streams of one context may be in flight at once;
 * calls on one context must come from one host thread at a time.
 * nblocks = 0 is accepted and enqueues nothing (the pointers must still be
 * non-null).
 */
int hers_search(hers_ctx* ctx, const hers_keys* keys, const uint64_t* gallery, uint64_t nblocks,
                uint32_t d, const uint64_t* probe, uint64_t* scores_ct, void* workspace,
                uint64_t workspace_bytes, void* stream);
/*
 * hers_search over blocks [block_begin, block_end) of a resident gallery of
 * nblocks blocks (Alg 7's loop over the gallery's blocks, restricted to a
 * range): scores_ct receives [block_end - block_begin][2][2][N], the score
 * ciphertext of block block_begin first; the workspace is sized for
 * block_end - block_begin blocks.  HERS_E_INVAL if the range is not inside
 * [0, nblocks).  Otherwise as hers_search.
 */
int hers_search_range(hers_ctx* ctx, const hers_keys* keys, const uint64_t* gallery, uint64_t nblocks,
                      uint32_t d, uint64_t block_begin, uint64_t block_end, const uint64_t* probe,
                      uint64_t* scores_ct, void* workspace, uint64_t workspace_bytes, void* stream);

/*
 * Base-w relinearisation gadget (Alg 1 / Alg 5 with g_j = w^j, w = 2^logw),
 * as an option beside the default RNS gadget.
 *
 * hers_basew_digits(logw): the number of digits l = ceil(108 / logw) for
 * 22 <= logw <= 60 (at most 5 digits), else 0.
 * hers_keys_add_basew: generates evkw_j = ([-(a_j s + e_j) + w^j s^2]_q, a_j),
 * j < l, for the keys' secret key s, with a_j (uniform mod q, limb by limb)
 * and e_j from the streams (seed, 0x06, 2 j + limb) and (seed, 0x07, j), and
 * attaches them to `keys` (replacing earlier base-w keys).  Synchronous.
 * hers_keys_export_basew: copies them to host memory, [l][2][2][N] canonical.
 * hers_search_basew: hers_search with the one key switch per block done with
 * these keys: the coefficients of c2, as integers in [0, q), are cut into l
 * base-w digits D_j and (c0', c1') = (c0 + sum_j D_j evkw_j0, c1 + sum_j D_j
 * evkw_j1).  Same arguments, workspace and errors as hers_search;
 * HERS_E_INVAL when the keys have no base-w keys.
 */
uint32_t hers_basew_digits(uint32_t logw);
int hers_keys_add_basew(hers_ctx* ctx, hers_keys* keys, uint64_t seed, uint32_t logw);
int hers_keys_export_basew(hers_ctx* ctx, const hers_keys* keys, uint64_t* evkw);
int hers_search_basew(hers_ctx* ctx, const hers_keys* keys, const uint64_t* gallery, uint64_t nblocks,
                      uint32_t d, const uint64_t* probe, uint64_t* scores_ct, void* workspace,
                      uint64_t workspace_bytes, void* stream);

/*
 * hers_search with output re-randomisation (Alg 7's s <- Encrypt(0), as an
 * option): block b's score ciphertext gets a fresh encryption of zero added,
 * Enc(0) with u, e1, e2 drawn from the streams (rerand_seed, 0x31 + 0/1/2, b),
 * b counted from the first block of this call.  Decrypts to the same scores;
 * hides the noise left by the computation.  Same arguments, workspace and
 * errors as hers_search, plus rerand_seed.
 */
int hers_search_rerand(hers_ctx* ctx, const hers_keys* keys, const uint64_t* gallery, uint64_t nblocks,
                       uint32_t d, const uint64_t* probe, uint64_t* scores_ct, void* workspace,
                       uint64_t workspace_bytes, uint64_t rerand_seed, void* stream);

/*
 * hers_search without caller-supplied scratch, for callers that cannot
 * allocate device memory when they search: processes whose device memory is
 * owned by another framework, plugins handed buffers but no allocator, and
 * fixed-budget services that forbid allocation after start-up.  The paper
 * has no counterpart; the result is the same as hers_search's.
 *
 * The scratch is one array of HERS_NOALLOC_MAX_BLOCKS * 800 KiB (6.25 MiB)
 * compiled into the library.  Every GPU that loads the library holds it
 * until the process exits.  The call itself allocates nothing (no
 * cudaMalloc, cudaFree or allocating library routine).  The caller still
 * passes the gallery, the probe and scores_ct (device, [nblocks][2][2][N]).
 *  - nblocks above HERS_NOALLOC_MAX_BLOCKS is rejected with HERS_E_INVAL.
 *    Larger galleries are searched by calling once per range of at most
 *    that many blocks: gallery + b*hers_gallery_bytes(1, d)/8 words, scores_ct + b*4*N words.
 *  - The first call on a device looks up the array's device address
 *    (cudaGetSymbolAddress) with that device current.  Make that first call
 *    before any stream capture.  The address belongs to the CUDA context it
 *    was looked up in: after a device reset (cudaDeviceReset), or with
 *    another context current on the device, the next call looks it up again,
 *    so that call too should come before any stream capture.
 *  - Every call shares the one array and leaves its contents behind.
 *    Nothing in it needs to start at zero.  Calls that overlap on the GPU
 *    (other streams, other contexts on the same device, other host threads)
 *    race on it: serialise them.
 * Asynchronous on stream (NULL = CUDA's default stream).
 */
#define HERS_NOALLOC_MAX_BLOCKS 8u
int hers_search_noalloc(hers_ctx* ctx, const hers_keys* keys, const uint64_t* gallery,
                        uint64_t nblocks, uint32_t d, const uint64_t* probe, uint64_t* scores_ct,
                        void* stream);

/*
 * Batched search: many probes, each against its own subset of gallery
 * blocks, subsets uneven and of mixed dimensionality, in one persistent launch
 * captured with the rest of the pipeline as one CUDA graph.  This is Alg 7's
 * server loop run for many queries at once; every (probe, block) result equals
 * hers_search's.
 *
 * Item i = (gallery, nblocks, d, probe): blocks [0, nblocks) of a resident
 * gallery of dimension d against one prepared probe of dimension d.  Items
 * with the same (gallery, nblocks, d) form a group.  Each gallery byte a group
 * streams from HBM is used for up to NP of its probes at once (NP = 1, 2 or 4,
 * per variant).
 *
 * scores_ct: device [sum_i nblocks_i][2][2][N].  Item i's blocks start at
 * sum_{j<i} nblocks_j.  workspace: device, hers_batch_workspace_bytes().  The
 * plan keeps both pointers, and they must stay valid until hers_batch_free.
 *
 * flags:
 *  - HERS_BATCH_AUTOTUNE builds and times every variant and keeps the fastest
 *    (hers_batch_info reports the timings);
 *  - HERS_BATCH_VARIANT(v) forces variant v;
 *  - with neither, variant 1.
 *
 * hers_batch_create allocates the plan's work tables and instantiates the
 * graph (synchronous).  hers_batch_run launches the graph on `stream`
 * (asynchronous; NULL = CUDA's default stream).  Runs of one plan must not
 * overlap.
 */
typedef struct hers_batch_item {
    const uint64_t* gallery;  /* device: resident gallery of the subset */
    uint64_t nblocks;         /* blocks searched: [0, nblocks) */
    uint32_t d;               /* feature dimension of gallery and probe */
    const uint64_t* probe;    /* device: prepared probe (hers_probe_prepare) */
} hers_batch_item;
typedef struct hers_batch hers_batch;
#define HERS_BATCH_AUTOTUNE 1u
#define HERS_BATCH_VARIANT(v) ((uint32_t)((v) + 1) << 8)
uint64_t hers_batch_workspace_bytes(const hers_batch_item* items, uint32_t nitems);
int hers_batch_create(hers_ctx* ctx, const hers_keys* keys, const hers_batch_item* items,
                      uint32_t nitems, uint64_t* scores_ct, void* workspace,
                      uint64_t workspace_bytes, uint32_t flags, hers_batch** out);
int hers_batch_run(hers_batch* batch, void* stream);
/* variant, groups, work units, pairs (sum of nblocks) and, if tune_ms is
 * non-null, hers_batch_variants() autotune timings in ms (-1: not timed). */
int hers_batch_info(const hers_batch* batch, int* variant, uint32_t* ngroups, uint32_t* nunits,
                    uint64_t* npairs, double* tune_ms);
/* One traced run: the batch's launches issued directly on `stream` (outside
 * the graph, the same work) with CUDA events between them; returns after it
 * completes with the tensor kernel's and the whole run's device time in ms. */
int hers_batch_trace(hers_batch* batch, void* stream, double* tensor_ms, double* total_ms);
int hers_batch_free(hers_batch* batch);
int hers_batch_variants(void);
const char* hers_batch_variant_name(int v);

/*
 * Serving loop with continuous batching.  A server keeps the given resident
 * galleries and the evaluation key on the device.  It takes requests at any
 * time: (gallery, block range, probe ciphertexts in host memory).
 *
 * A scheduler thread admits queued requests in arrival order while their
 * device memory fits a pool carved out of free HBM at creation.  The pool is
 * workspace_bytes, or all free HBM minus 1 GiB when that is 0.  Each admitted
 * set of up to max_batch requests runs as one batch on one of three streams:
 *  - probe copy-in and preparation;
 *  - the persistent batched tensor kernel, where overlapping block ranges of
 *    one gallery share each gallery read;
 *  - the epilogue;
 *  - copy-out of each request's score ciphertexts.
 * Batches on the three streams overlap on the device.  Requests arriving
 * meanwhile form the next batch as soon as a stream and memory free up.  Every
 * result equals hers_search's on the same range.
 *
 * hers_server_submit: probe_ct_host is host [d][2][2][N] (pinned copies
 * faster).  scores_ct_host is host [end - begin][2][2][N], written when the
 * request completes.  Both must stay valid until hers_server_wait returns
 * for the id.
 * hers_server_wait: waits up to timeout_ms.  It returns the request's
 * status: HERS_OK, HERS_E_NOMEM if the request alone cannot fit the pool, or
 * HERS_E_TIMEOUT if the wait expired (the request then stays pending).
 * latency_ms receives the time from submission until its scores were in host
 * memory.  Each id is waited for once.
 * variant: the batched tensor-kernel shape (hers_batch_variant_name).
 * A request of dimension d over n blocks holds 8 (14 d N + 29 N n) bytes of
 * the pool while it runs, plus its share of the batch's work tables (a few
 * hundred bytes per segment of a gallery that one set of requests covers).
 */
typedef struct hers_server_gallery {
    const uint64_t* gallery;  /* device: resident gallery (block 0) */
    uint64_t nblocks;
    uint32_t d;
} hers_server_gallery;
typedef struct hers_server hers_server;
int hers_server_create(hers_ctx* ctx, const hers_keys* keys, const hers_server_gallery* galleries,
                       uint32_t ngalleries, uint64_t workspace_bytes, uint32_t max_batch, int variant,
                       hers_server** out);
int hers_server_submit(hers_server* srv, uint32_t gallery, uint64_t block_begin, uint64_t block_end,
                       const uint64_t* probe_ct_host, uint64_t* scores_ct_host, uint64_t* id);
int hers_server_wait(hers_server* srv, uint64_t id, uint32_t timeout_ms, double* latency_ms);
/* Holds (paused != 0) or resumes admission: while held, submitted requests
 * queue and batches already running finish. */
int hers_server_pause(hers_server* srv, int paused);
/* Counters since creation; returns a sticky error status (HERS_OK if none). */
int hers_server_stats(hers_server* srv, uint64_t* submitted, uint64_t* completed, uint64_t* batches,
                      uint64_t* entries, uint64_t* max_batch_seen, uint64_t* pool_bytes);
/* Where the server's time went, summed over its finished batches: device
 * time of each batch's kernels (probe preparation, tensor kernel, epilogue)
 * and of its score copies to host memory (CUDA events on the batch's stream;
 * batches on the three streams overlap, so the sums can exceed wall time), and
 * host time the scheduler spent planning and issuing batches.  Any pointer
 * may be NULL. */
int hers_server_timing(hers_server* srv, double* kernels_ms, double* copies_ms, double* plan_ms);
/* Finishes in-flight batches, drops queued requests and frees the server. */
int hers_server_free(hers_server* srv);

/*
 * Streamed search over a gallery kept in canonical form.  The canonical form
 * has 2 limbs in the coefficient domain, 32 d bytes per entry, i.e. the
 * ciphertexts' own size.  It is meant for galleries too large for the
 * resident form (64 d bytes per entry): 100M entries at d = 64 are 204.8 GB
 * canonical against 409.6 GB resident.
 *
 * The gallery is gallery_ct, [nblocks][d][2][2][N], in host memory when
 * gallery_on_host (pinned for full copy speed) or in device memory.
 * probes: host array of nprobes device pointers to prepared probes of
 * dimension d.  scores_ct: device [nprobes][nblocks][2][2][N].
 *
 * Per chunk of chunk_blocks blocks the call:
 *  - copies the chunk in;
 *  - extends it and NTTs it into the resident form in the workspace;
 *  - runs one persistent batched tensor launch with every probe (variant as
 *    hers_batch_variant_name) and the epilogue.
 * Two chunk slots alternate, so chunk c+1's copy and extension, on the
 * context's own stream, overlap chunk c's search on `stream`.
 *
 * workspace: device, hers_search_stream_workspace_bytes(d, nprobes,
 * chunk_blocks).  Asynchronous on `stream`: the work on both streams is joined
 * into `stream`.  Results equal hers_search's.
 */
uint64_t hers_search_stream_workspace_bytes(uint32_t d, uint32_t nprobes, uint32_t chunk_blocks);
int hers_search_stream(hers_ctx* ctx, const hers_keys* keys, const uint64_t* gallery_ct,
                       int gallery_on_host, uint64_t nblocks, uint32_t d,
                       const uint64_t* const* probes, uint32_t nprobes, uint64_t* scores_ct,
                       uint32_t chunk_blocks, int variant, void* workspace,
                       uint64_t workspace_bytes, void* stream);

/*
 * End-to-end server step with host buffers: copies the probe's d canonical
 * cts from host memory (probe_ct_host, [d][2][2][N]) to the device, prepares
 * them, searches blocks [0, nblocks) and copies the score cts back to host
 * memory (scores_ct_host, [nblocks][2][2][N]).  workspace: device scratch of
 * at least hers_search_host_workspace_bytes(nblocks, d) bytes (search scratch,
 * the probe's cts and prepared form, and the staged score cts); the call
 * allocates nothing.  Host buffers may be pageable; pinned ones copy faster.
 * Returns after the scores are in host memory.
 */
int hers_search_host(hers_ctx* ctx, const hers_keys* keys, const uint64_t* gallery,
                     uint64_t nblocks, uint32_t d, const uint64_t* probe_ct_host,
                     uint64_t* scores_ct_host, void* workspace, uint64_t workspace_bytes,
                     void* stream);
uint64_t hers_search_host_workspace_bytes(uint64_t nblocks, uint32_t d);
/*
 * hers_search_host without the final wait: the copies and kernels are
 * enqueued on `stream` (NULL = the CUDA default stream) and the call returns.
 * The scores are in host memory once `stream` reaches this point; the caller
 * synchronises (a stream or event wait) before reading them.  probe_ct_host
 * and scores_ct_host must be pinned host memory (cudaHostAlloc / registered)
 * and stay valid and unmodified until then; the workspace belongs to this call
 * until then too.  Calls on different streams with separate workspaces and
 * score buffers overlap: one call's copies run beside another's kernels.
 * Returns HERS_E_INVAL if a host buffer is not pinned.
 */
int hers_search_host_async(hers_ctx* ctx, const hers_keys* keys, const uint64_t* gallery,
                           uint64_t nblocks, uint32_t d, const uint64_t* probe_ct_host,
                           uint64_t* scores_ct_host, void* workspace, uint64_t workspace_bytes,
                           void* stream);

/*
 * Client-side decryption (App. A, Alg 3) and decoding of block score cts
 * (Alg 7 client side): pt = [round(t/q [c0 + c1 s]_q)]_t, slot j of block b
 * is entry bN + j, centred in [-(t-1)/2, (t-1)/2].
 * scores_ct: device [nblocks][2][2][N]; scores: device int32 [m] with
 * m <= nblocks N.  Asynchronous on stream.
 */
int hers_decrypt_scores(hers_ctx* ctx, const hers_keys* keys, const uint64_t* scores_ct,
                        uint64_t nblocks, int32_t* scores, uint64_t m, void* stream);

/*
 * Client-side decryption with host buffers (Alg 3; Alg 7's client side after
 * the server's response, Sec. 3.1's g with sk): scores_ct_host, host
 * [nblocks][2][2][N] (as hers_search_host writes them); scores_host, host
 * int32 [m], m <= nblocks N.  Synchronous on the context's stream, with a
 * device staging buffer of at most 256 MiB.  HERS_E_INVAL for keys without a
 * secret key.
 */
int hers_decrypt_scores_host(hers_ctx* ctx, const hers_keys* keys, const uint64_t* scores_ct_host,
                             uint64_t nblocks, int32_t* scores_host, uint64_t m);

/* Synchronises `stream` and the context's own stream, then reports deferred
 * device-side errors (sampler exhaustion) as a status. */
int hers_check(hers_ctx* ctx, void* stream);

/*
 * Tracing (no counterpart in the paper, which reports wall-clock times only).
 * hers_trace_enable(ctx, n) makes the next n hers_search / hers_search_host
 * calls on ctx record CUDA events at their phase boundaries on the stream they
 * run on (n = 0 turns tracing off).  hers_trace_read() waits for those events
 * and writes, into avg_ms[HERS_TRACE_PHASES], the average milliseconds per
 * call of: the tensor-accumulate kernel, the inverse NTTs, the exact
 * scale-and-round, the key switch (forward NTT, multiply, inverse NTT, add),
 * and the whole search; *ncalls is the number of calls averaged.  Reading
 * re-arms the n slots.
 */
#define HERS_TRACE_PHASES 5
int hers_trace_enable(hers_ctx* ctx, uint32_t max_calls);
int hers_trace_read(hers_ctx* ctx, uint32_t* ncalls, double* avg_ms);

/* Number of CUDA kernels this library has launched in this process. */
uint64_t hers_kernel_launches(void);

/*
 * Autotuner (no counterpart in the paper).  The tensor-accumulate kernel comes
 * in several shapes: gallery blocks per CTA, pipeline stages, dimensions per
 * stage, CTAs per SM.  Every shape computes the same exact result.
 * hers_autotune times each shape's kernel on the given search: 1 warm-up and
 * 3 timed launches each on `stream`, minimum kept.  It keeps the fastest shape
 * for later searches on ctx.  If ms_per_variant is non-null it receives
 * hers_tensor_variants() timings in ms.  workspace: as for hers_search.
 * Synchronous.  hers_set_tensor_variant selects a shape by index.
 */
int hers_tensor_variants(void);
const char* hers_tensor_variant_name(int v);
int hers_get_tensor_variant(const hers_ctx* ctx);
int hers_set_tensor_variant(hers_ctx* ctx, int v);
int hers_autotune(hers_ctx* ctx, const hers_keys* keys, const uint64_t* gallery, uint64_t nblocks,
                  uint32_t d, const uint64_t* probe, void* workspace, uint64_t workspace_bytes,
                  void* stream, int* chosen, double* ms_per_variant);

/*
 * Epilogue forms (no counterpart in the paper).  After the tensor kernel every
 * search runs the same epilogue arithmetic (inverse NTTs, exact
 * scale-and-round, key switch) in one of hers_epilogue_variants() forms, all
 * giving the same bytes: 0 "split" (one kernel per step), 1
 * "intt_scale_cluster" (inverse NTTs and scale-and-round in one kernel: a
 * cluster of eight CTAs per accumulator polynomial, residues exchanged in
 * distributed shared memory), 2 "ks_fused" (the key switch in one kernel per
 * block and limb), 3 both; adding 4 ("+shfl") makes the first data exchange
 * of every inverse NTT of the accumulators a warp-shuffle transpose instead
 * of a pass through shared memory, and adding 8 ("+lean") builds the split
 * inverse NTTs and the two-kernel key switch for one more CTA per SM (fewer
 * registers), so that more of them fit beside a persistent tensor kernel of
 * another search in flight, and adding 16 ("+ksshfl") makes the in-warp
 * exchange of the split key switch's 64-bit NTTs (a 16 x 16 transpose inside
 * each half-warp) a warp-shuffle transpose instead of a pass through shared
 * memory.  The context's form applies to every search on it
 * (hers_search*, hers_batch_*, hers_server_*, hers_search_stream).
 * hers_autotune_epilogue times each form's epilogue after the tensor kernel
 * of the given search (1 warm-up, 3 timed, minimum kept), keeps the fastest
 * on ctx and, if ms_per_variant is non-null, writes hers_epilogue_variants()
 * timings in ms.  It holds a temporary device buffer for nblocks score
 * ciphertexts during the call.  Synchronous.
 */
/*
 * Which half of a search takes the context's high-priority stream (no
 * counterpart in the paper).  By default (0) hers_search and the host-buffer
 * searches run the tensor kernel on the caller's stream and the epilogue on
 * the high-priority stream, so that one search's epilogue is dispatched ahead
 * of the next search's pending tensor CTAs.  With hers_set_tensor_first(ctx,
 * 1) the tensor kernel runs on the high-priority stream and the epilogue on
 * the caller's stream: a search's tensor kernel keeps its SMs and the
 * previous search's epilogue runs in the registers and shared memory it
 * leaves (useful with the one-CTA-per-SM tensor shapes).  Either way the call
 * is ordered on the caller's stream as documented for hers_search, and the
 * bytes are the same.  Setting it waits for the context's high-priority
 * stream.
 */
int hers_set_tensor_first(hers_ctx* ctx, int on);
int hers_get_tensor_first(const hers_ctx* ctx);
/*
 * Probe preparation form (no counterpart in the paper).  hers_probe_prepare
 * and the host-buffer searches extend a probe's 2 d polynomials to the
 * resident form either with one CTA per polynomial or with a cluster of eight
 * CTAs per polynomial (one per search prime, lifts shared through
 * distributed shared memory); both give the same bytes.  The context takes
 * the cluster form for calls of at most a threshold of polynomials (64 by
 * default: probes of d <= 32).  hers_autotune_extension times both forms for
 * a probe of dimension d (1 warm-up, 5 timed rounds of 8 preparations each,
 * minimum kept; zero ciphertexts, a temporary device buffer of d (4 N + 16
 * N) words), moves the threshold to this size's winner, and writes
 * *cluster = 1 if the cluster form won and ms[0], ms[1] = ms per preparation
 * (one CTA per polynomial, cluster).  Synchronous.
 */
int hers_autotune_extension(hers_ctx* ctx, uint32_t d, void* stream, int* cluster, double* ms);
int hers_epilogue_variants(void);
const char* hers_epilogue_variant_name(int v);
int hers_get_epilogue_variant(const hers_ctx* ctx);
int hers_set_epilogue_variant(hers_ctx* ctx, int v);
int hers_autotune_epilogue(hers_ctx* ctx, const hers_keys* keys, const uint64_t* gallery, uint64_t nblocks,
                           uint32_t d, const uint64_t* probe, void* workspace, uint64_t workspace_bytes,
                           void* stream, int* chosen, double* ms_per_variant);

/*
 * Stage 1 of the two-stage search (Sec. 3.2): the k entries with the largest
 * decrypted scores, ordered by score descending and, among equal scores, by
 * index ascending (the lowest index first).
 *
 * scores: device int32[m], e.g. hers_decrypt_scores' output (1 <= m < 2^32 - 1).
 * k: 1 <= k <= min(m, 4096).
 * out_idx: device int64[k]; out_scores: device int32[k].
 * workspace: device, hers_topk_workspace_bytes(m) bytes (selection state,
 * a histogram, per-CTA tie counts and the k candidates); the call allocates
 * nothing.  Asynchronous on `stream` (NULL = the CUDA default stream); no
 * step waits on the host.  Exact radix selection of the k-th largest score,
 * then a sort of the k candidates.  Returns HERS_E_INVAL for a size out of
 * range, HERS_E_NOMEM for a short workspace, HERS_E_CUDA on a CUDA error; an
 * internal count mismatch is reported by hers_check as HERS_E_CUDA.
 */
uint64_t hers_topk_workspace_bytes(uint64_t m);
int hers_topk(hers_ctx* ctx, const int32_t* scores, uint64_t m, uint32_t k, int64_t* out_idx,
              int32_t* out_scores, void* workspace, uint64_t workspace_bytes, void* stream);

/*
 * Diagnostic with no counterpart in the paper: sustained integer-pipe rate on
 * `device`, in operations per second over all SMs, for op 0 = 32x32 -> 64-bit
 * multiply-add (IMAD.WIDE.U32, the tensor kernel's inner operation), 1 =
 * 32-bit multiply-add, 2 = high half of a 64x64-bit product (__umul64hi, the
 * Shoup/Barrett step), 3 = signed 32x32 -> 64-bit multiply-add with both
 * factors in registers from shared memory into a 64-bit register sum (the
 * batched tensor kernel's form; 4 x 4 outer products, 16 per iteration).
 * Runs one kernel of `iters` iterations per thread;
 * allocates an 8-byte buffer for the duration of the call.
 */
int hers_probe_int_pipe(int device, uint32_t op, uint64_t iters, double* ops_per_s);

/*
 * Diagnostic with no counterpart in the paper: exercises the bounded wait
 * that every streaming kernel's producer and consumers use.  Launches one
 * CTA on ctx's stream whose thread waits on a shared-memory mbarrier that
 * nothing completes, with a budget of limit_ns nanoseconds of global time
 * (1e6 .. 2e9).  When the budget runs out the kernel sets bit 2 of the
 * context's device error flag and returns; the call then reads and clears the
 * flag as hers_check does.  Returns HERS_E_TIMEOUT, the expected outcome,
 * with *elapsed_ms the kernel's duration (CUDA events); HERS_E_INVAL for a
 * null argument or a limit out of range; HERS_E_CUDA on a CUDA error.  The
 * context stays usable afterwards.  Nothing faults: the wait is an ordinary
 * bounded loop that gives up.
 */
int hers_selftest_wait_timeout(hers_ctx* ctx, uint64_t limit_ns, double* elapsed_ms);

#ifdef __cplusplus
}
#endif

#endif /* HERS_H */
