// hers_search_noalloc: the search of hers_search for callers that cannot
// allocate device memory when they search.  Such callers include processes
// whose device memory is owned by another framework, plugins that are handed
// buffers but no allocator, and fixed-budget services that forbid allocation
// after start-up.  Its scratch is a file-scope device array compiled into the
// library instead of a caller-supplied workspace, so the call needs no
// cudaMalloc, cudaFree or other allocating routine.
#include <cuda.h>

#include <mutex>

#include "hers.h"
#include "internal.h"

namespace hers {

// Scratch of the search pipeline for up to HERS_NOALLOC_MAX_BLOCKS gallery
// blocks (SEARCH_WS_WORDS_PER_BLOCK words each: 6.25 MiB).  Every GPU that
// loads the library holds it until the process exits.
static __device__ __align__(256) uint64_t g_noalloc_scratch[HERS_NOALLOC_MAX_BLOCKS *
                                                            SEARCH_WS_WORDS_PER_BLOCK];

// Device address of g_noalloc_scratch per device.  In host code the array's
// name is only a host-side stand-in, so the address is looked up with the
// device current.  The address belongs to the CUDA context the module was
// loaded in: a device reset, or another context made current on the device,
// loads the module again at another address.  So each device's entry records
// the unique ID of the context it was looked up in (cuCtxGetId, reached
// through the runtime's driver entry points, no link to libcuda) and is looked
// up again when the current context's ID differs.
constexpr int MAX_DEVICES = 64;
struct ScratchSlot {
    uint64_t* ptr;
    unsigned long long ctx_id;
    bool keyed;  // ctx_id is valid
};
static ScratchSlot s_scratch[MAX_DEVICES];
static std::mutex s_scratch_mu;

typedef CUresult (*CtxGetCurrentFn)(CUcontext*);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long*);

// The unique ID of the calling thread's current context; false if there is
// none or the driver entry points are unavailable.
static bool current_context_id(unsigned long long* id) {
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            get_current = (CtxGetCurrentFn)f;
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            get_id = (CtxGetIdFn)f;
    });
    CUcontext c = nullptr;
    if (!get_current || !get_id || get_current(&c) != CUDA_SUCCESS || !c) return false;
    return get_id(c, id) == CUDA_SUCCESS;
}

static cudaError_t scratch_for(int device, uint64_t** out) {
    unsigned long long id = 0;
    bool have = current_context_id(&id);
    std::lock_guard<std::mutex> lk(s_scratch_mu);
    ScratchSlot& s = s_scratch[device];
    if (!s.ptr || !s.keyed || !have || s.ctx_id != id) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        if (!have) have = current_context_id(&id);  // the lookup made the primary context current
        s.ptr = (uint64_t*)p;
        s.ctx_id = id;
        s.keyed = have;  // without an ID the next call looks the address up again
    }
    *out = s.ptr;
    return cudaSuccess;
}

}  // namespace hers

extern "C" int hers_search_noalloc(hers_ctx* ctx, const hers_keys* keys, const uint64_t* gallery,
                                   uint64_t nblocks, uint32_t d, const uint64_t* probe,
                                   uint64_t* scores_ct, void* stream) {
    using namespace hers;
    if (!ctx || !keys || !gallery || !probe || !scores_ct)
        return fail(ctx, HERS_E_INVAL, "hers_search_noalloc: null argument");
    if (d == 0 || d > HERS_MAX_D) return fail(ctx, HERS_E_INVAL, "hers_search_noalloc: d = %u", d);
    if (nblocks > HERS_NOALLOC_MAX_BLOCKS)
        return fail(ctx, HERS_E_INVAL,
                    "hers_search_noalloc: %llu blocks exceed the built-in scratch of %u blocks; "
                    "call it once per range of at most %u blocks",
                    (unsigned long long)nblocks, HERS_NOALLOC_MAX_BLOCKS, HERS_NOALLOC_MAX_BLOCKS);
    if (ctx->device < 0 || ctx->device >= MAX_DEVICES)
        return fail(ctx, HERS_E_INVAL, "hers_search_noalloc: device %d", ctx->device);
    DeviceGuard g(ctx->device);
    uint64_t* ws = nullptr;
    cudaError_t e = scratch_for(ctx->device, &ws);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "hers_search_noalloc: scratch address");
    // launch_search writes every scratch word it later reads, so the contents
    // left by the previous call need no clearing.
    e = launch_search(ctx->tw, keys->k, gallery, nblocks, d, probe, scores_ct, ws, ctx->err,
                      (cudaStream_t)stream, nullptr, ctx->tensor_variant, nullptr, nullptr, ctx->epi_variant);
    return e == cudaSuccess ? HERS_OK : cuda_fail(ctx, e, "hers_search_noalloc");
}
