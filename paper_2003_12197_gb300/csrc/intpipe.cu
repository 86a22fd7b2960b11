// Integer-pipe throughput probe: the rates that bound the library's
// ALU-limited kernels (NTT butterflies, the tensor accumulate once gallery
// bytes are shared by many probes).  Each thread runs 8 independent
// dependent chains of one operation; ops/s = threads * iters * 8 / time.
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"
#include "hers.h"
#include "internal.h"

namespace hers {

template <int OP>
__global__ void __launch_bounds__(256) k_intpipe(uint64_t iters, uint32_t c, uint64_t* sink) {
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    uint64_t a[8];
    uint32_t b[8];
#pragma unroll
    for (int j = 0; j < 8; j++) {
        a[j] = (uint64_t)t * 0x9E3779B97F4A7C15ull + j;
        b[j] = t * 2654435761u + j;
    }
    for (uint64_t i = 0; i < iters; i++) {
#pragma unroll
        for (int j = 0; j < 8; j++) {
            if (OP == 0) a[j] += (uint64_t)(uint32_t)a[j] * c;          // IMAD.WIDE.U32
            else if (OP == 1) b[j] = b[j] * c + (uint32_t)j;            // IMAD (32-bit)
            else a[j] = __umul64hi(a[j], a[j] | 1) + (uint64_t)c;       // 64x64 high half
        }
    }
    uint64_t r = 0;
#pragma unroll
    for (int j = 0; j < 8; j++) r ^= a[j] ^ b[j];
    if (r == 0x123456789ull) sink[0] = r;  // keeps the chains live
}

// Op 3: the batched tensor kernel's instruction form, a signed 32x32->64
// multiply-add with both factors in registers (read from shared memory) into
// a 64-bit register sum, as the 4 x 4 outer product of 4 values of each side
// per iteration (16 sums per thread).  The compiler fuses only about half of
// these accumulates into the IMAD.WIDE (the rest take a separate 64-bit add),
// so this rate, not op 0's, is what such a loop can reach.
__global__ void __launch_bounds__(256) k_intpipe_outer(uint64_t iters, uint32_t c, uint64_t* sink) {
    __shared__ int32_t sa[1024], sb[1024];
    for (int i = threadIdx.x; i < 1024; i += blockDim.x) {
        sa[i] = (int32_t)((uint32_t)i * c) >> 3;
        sb[i] = (int32_t)((uint32_t)(i + 7) * (c ^ 0x5bd1e995u)) >> 3;
    }
    __syncthreads();
    int64_t acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) acc[i][j] = 0;
    const int t = threadIdx.x & 31;
    for (uint64_t it = 0; it < iters; it++) {
        const int base = (int)((it * 8) & 1023) & ~31;
        int32_t a[4], b[4];
#pragma unroll
        for (int i = 0; i < 4; i++) {
            a[i] = sa[(base + t + 32 * i) & 1023];
            b[i] = sb[(base + t + 32 * i + 7) & 1023];
        }
#pragma unroll
        for (int i = 0; i < 4; i++)
#pragma unroll
            for (int j = 0; j < 4; j++) asm("mad.wide.s32 %0, %1, %2, %0;" : "+l"(acc[i][j]) : "r"(a[i]), "r"(b[j]));
    }
    int64_t r = 0;
#pragma unroll
    for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) r ^= acc[i][j];
    if (r == 0x123456789ll) sink[0] = (uint64_t)r;  // keeps the sums live
}

// One thread waits on an mbarrier that nothing arrives on, with the same
// bounded wait the streaming kernels use; the give-up path is theirs too.
__global__ void k_wait_timeout(uint64_t limit_ns, int* err) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        mbar_fence_init();
    }
    __syncthreads();
    if (threadIdx.x == 0 && !mbar_wait(&bar, 0, limit_ns)) atomicOr(err, 2);
}

}  // namespace hers

extern "C" int hers_selftest_wait_timeout(hers_ctx* ctx, uint64_t limit_ns, double* elapsed_ms) {
    using namespace hers;
    if (!ctx || !elapsed_ms) return fail(ctx, HERS_E_INVAL, "hers_selftest_wait_timeout: null argument");
    if (limit_ns < 1000000ull || limit_ns > WAIT_NS)
        return fail(ctx, HERS_E_INVAL, "hers_selftest_wait_timeout: limit %llu ns not in [1e6, 2e9]",
                    (unsigned long long)limit_ns);
    DeviceGuard g(ctx->device);
    int rc = hers_check(ctx, nullptr);  // start from a clear error flag
    if (rc != HERS_OK) return rc;
    cudaEvent_t e0, e1;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "hers_selftest_wait_timeout: events");
    cudaEventRecord(e0, ctx->stream);
    k_wait_timeout<<<1, 32, 0, ctx->stream>>>(limit_ns, ctx->err);
    count_launches(1);
    e = cudaGetLastError();
    cudaEventRecord(e1, ctx->stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "hers_selftest_wait_timeout");
    *elapsed_ms = ms;
    return hers_check(ctx, ctx->stream);
}

extern "C" int hers_probe_int_pipe(int device, uint32_t op, uint64_t iters, double* ops_per_s) {
    using namespace hers;
    if (!ops_per_s || op > 3 || iters == 0) return HERS_E_INVAL;
    if (cudaSetDevice(device) != cudaSuccess) return HERS_E_CUDA;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess)
        return HERS_E_CUDA;
    const int blocks = sms * 8, threads = 256;
    uint64_t* sink = nullptr;
    cudaEvent_t e0, e1;
    if (cudaMalloc(&sink, 8) != cudaSuccess) return HERS_E_NOMEM;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    auto launch = [&](uint64_t it) {
        if (op == 0) k_intpipe<0><<<blocks, threads>>>(it, 0x9E3779B1u, sink);
        else if (op == 1) k_intpipe<1><<<blocks, threads>>>(it, 0x9E3779B1u, sink);
        else if (op == 2) k_intpipe<2><<<blocks, threads>>>(it, 0x9E3779B1u, sink);
        else k_intpipe_outer<<<blocks, threads>>>(it, 0x9E3779B1u, sink);
    };
    // op 3 does 16 multiply-adds per thread and iteration, the others 8
    const double per_iter = op == 3 ? 16.0 : 8.0;
    launch(iters / 8 + 1);  // warm-up
    cudaEventRecord(e0);
    launch(iters);
    cudaEventRecord(e1);
    cudaError_t e = cudaEventSynchronize(e1);
    float ms = 0;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    count_launches(2);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(sink);
    if (e != cudaSuccess || ms <= 0) return HERS_E_CUDA;
    *ops_per_s = (double)blocks * threads * (double)iters * per_iter / (ms * 1e-3);
    return HERS_OK;
}
