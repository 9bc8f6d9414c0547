// calib.cu -- measured costs of the three operations the batch-size cost
// model of Section 6.1 is written in: one random word, one multiplication
// (a Theorem 1 chain step, one die) and the exact threshold 2^64 mod B
// (the model's "division").  Each is run in registers by every thread of a
// full grid, with four independent streams per thread so that the loop is
// bound by issue rate, not latency, and timed with CUDA events on the
// caller's stream.  The results feed the cost model that picks the n_k.
#include "brr_common.cuh"
#include "internal.h"

namespace brr {

constexpr int kCalibThreads = 256;

// mode 0: words, 1: chain steps, 2: thresholds of B in [2^48, 2^64),
// 3: thresholds of B in [2^8, 2^40) (the 64-bit remainder path)
__global__ void __launch_bounds__(kCalibThreads) calib_kernel(int mode, uint32_t iters, uint64_t seed,
                                                              uint64_t *sink) {
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    uint64_t acc[4], r[4];
#pragma unroll
    for (int s = 0; s < 4; s++) {
        acc[s] = 0;
        r[s] = mix64(seed + tid * 4 + s);
    }
    for (uint32_t i = 0; i < iters; i++) {
#pragma unroll
        for (int s = 0; s < 4; s++) {
            if (mode == 0) {
                acc[s] ^= word(seed, tid * 4 + s, i & 0xFFFFu) + i;
            } else if (mode == 1) {
                acc[s] += chain_step(r[s], 0x9E3779B9u ^ (i * 2654435761u) | 1u);
            } else {
                // B from the running word: a fresh value every iteration
                const uint64_t h = r[s] = r[s] * 6364136223846793005ull + 1442695040888963407ull;
                const uint32_t bits = mode == 2 ? 49 + (uint32_t)(h >> 60) : 9 + (uint32_t)(h >> 59);
                const uint64_t B = (h >> (64 - bits)) | (1ull << (bits - 1));
                acc[s] += lemire_threshold(B);
            }
        }
    }
    const uint64_t x = acc[0] ^ acc[1] ^ acc[2] ^ acc[3] ^ r[0] ^ r[1] ^ r[2] ^ r[3];
    if (x == 0x5EED5EED5EED5EEDull) sink[0] = x;  // keeps the work; practically never stores
}

// Self-test of the bounded grid barrier: one block waits for `expected`
// arrivals, more than the grid holds, so the wait must run out after
// limit_ns and record BRR_ETIMEOUT.
__global__ void barrier_selftest_kernel(uint32_t *bar, int *err, uint32_t expected, uint64_t limit_ns) {
    if (grid_barrier_bounded(bar, err, expected, limit_ns)) record_error(err, BRR_EINVAL);  // cannot pass
}

}  // namespace brr

extern "C" brr_status brr_selftest_barrier_timeout(brr_ctx *ctx, uint64_t limit_ns, brr_stream_t stream_h) {
    using namespace brr;
    if (!ctx || limit_ns < 1000 || limit_ns > 100000000ull) return BRR_EINVAL;
    cudaStream_t stream = (cudaStream_t)stream_h;
    brr_status st = ensure_scratch(ctx, 256, stream);
    if (st != BRR_OK) return st;
    uint32_t *bar = static_cast<uint32_t *>(ctx->scratch);
    cudaError_t e = cudaMemsetAsync(bar, 0, 2 * sizeof(uint32_t), stream);
    if (e != cudaSuccess) return cuda_status(e);
    barrier_selftest_kernel<<<1, 32, 0, stream>>>(bar, ctx->d_err, 2, limit_ns);
    return cuda_status(cudaGetLastError());
}

extern "C" brr_status brr_calibrate(brr_ctx *ctx, double *ns_per_op, brr_stream_t stream_h) {
    using namespace brr;
    if (!ctx || !ns_per_op) return BRR_EINVAL;
    cudaStream_t stream = (cudaStream_t)stream_h;
    brr_status st = ensure_scratch(ctx, 256, stream);
    if (st != BRR_OK) return st;
    uint64_t *sink = static_cast<uint64_t *>(ctx->scratch);
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, calib_kernel, kCalibThreads, 0);
    if (e != cudaSuccess || per_sm < 1) return BRR_ECUDA;
    const uint32_t grid = (uint32_t)per_sm * ctx->num_sms;
    const uint32_t iters = 1u << 12;
    const double ops = (double)grid * kCalibThreads * 4.0 * iters;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return BRR_ECUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return BRR_ECUDA;
    }
    st = BRR_OK;
    for (int mode = 0; mode < 4 && st == BRR_OK; mode++) {
        calib_kernel<<<grid, kCalibThreads, 0, stream>>>(mode, 64, 7, sink);  // warm-up
        cudaEventRecord(e0, stream);
        calib_kernel<<<grid, kCalibThreads, 0, stream>>>(mode, iters, 11, sink);
        cudaEventRecord(e1, stream);
        float ms = 0.f;
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
            st = BRR_ECUDA;
            break;
        }
        ns_per_op[mode] = (double)ms * 1e6 / ops;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_status(e);
    return st;
}
