// CUDA-core fused multiply-add throughput of the GPU the context runs on: the denominator of the
// FP32 scoring form's roofline (its transforms, products and likelihood run on the FP32 pipe) and
// of the FP64 parts (per-pair constants and log-sum-exp accumulators).  The paper has no
// counterpart; this is a measurement hook.
//
// Each thread runs CH independent chains x <- x a + b (a = 1 - 2^-20, b = 2^-20: every chain
// converges to 1 and stays finite and normal), so the pipe is never waiting on a dependent
// result; the chains' sum is written only under a condition the host never meets, which keeps
// the arithmetic alive.  Timed with CUDA events on the context's stream, best of `reps` launches.
#include <math.h>

#include "bioem_internal.cuh"

namespace {

constexpr int kPeakThreads = 256;
constexpr int kPeakChains = 16;

template <int KIND>   // 0: FP32 FFMA, 1: FP32 packed FFMA2 (two lanes per instruction), 2: FP64 DFMA
__global__ void __launch_bounds__(kPeakThreads) k_fma_peak(int iters, float* sink32, double* sink64, int never) {
    if constexpr (KIND == 0) {
        float x[kPeakChains];
#pragma unroll
        for (int c = 0; c < kPeakChains; ++c) x[c] = 0.5f + 1e-3f * (float)((threadIdx.x + c) & 63);
        const float a = 1.0f - 9.5367431640625e-7f, b = 9.5367431640625e-7f;
#pragma unroll 1
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int c = 0; c < kPeakChains; ++c) x[c] = fmaf(x[c], a, b);
        }
        float s = 0.f;
#pragma unroll
        for (int c = 0; c < kPeakChains; ++c) s += x[c];
        if (never && s == 1234.5f) sink32[threadIdx.x] = s;
    } else if constexpr (KIND == 1) {
        float2 x[kPeakChains / 2];
#pragma unroll
        for (int c = 0; c < kPeakChains / 2; ++c)
            x[c] = make_float2(0.5f + 1e-3f * (float)((threadIdx.x + c) & 63), 0.25f + 1e-3f * (float)(c & 7));
        const float2 a = make_float2(1.0f - 9.5367431640625e-7f, 1.0f - 9.5367431640625e-7f);
        const float2 b = make_float2(9.5367431640625e-7f, 9.5367431640625e-7f);
#pragma unroll 1
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int c = 0; c < kPeakChains / 2; ++c) x[c] = __ffma2_rn(x[c], a, b);
        }
        float s = 0.f;
#pragma unroll
        for (int c = 0; c < kPeakChains / 2; ++c) s += x[c].x + x[c].y;
        if (never && s == 1234.5f) sink32[threadIdx.x] = s;
    } else {
        double x[kPeakChains];
#pragma unroll
        for (int c = 0; c < kPeakChains; ++c) x[c] = 0.5 + 1e-3 * (double)((threadIdx.x + c) & 63);
        const double a = 1.0 - 9.5367431640625e-7, b = 9.5367431640625e-7;
#pragma unroll 1
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int c = 0; c < kPeakChains; ++c) x[c] = fma(x[c], a, b);
        }
        double s = 0.0;
#pragma unroll
        for (int c = 0; c < kPeakChains; ++c) s += x[c];
        if (never && s == 1234.5) sink64[threadIdx.x] = s;
    }
}

template <int KIND>
cudaError_t launch_peak(int grid, int iters, cudaStream_t stream, float* s32, double* s64) {
    k_fma_peak<KIND><<<grid, kPeakThreads, 0, stream>>>(iters, s32, s64, 0);
    return cudaGetLastError();
}

cudaError_t launch_kind(int kind, int grid, int iters, cudaStream_t stream, float* s32, double* s64) {
    switch (kind) {
        case 0: return launch_peak<0>(grid, iters, stream, s32, s64);
        case 1: return launch_peak<1>(grid, iters, stream, s32, s64);
        default: return launch_peak<2>(grid, iters, stream, s32, s64);
    }
}

}  // namespace

extern "C" int bioem_fma_peak(bioem_ctx* ctx, int kind, int reps, double* flops_per_s) {
    if (!ctx || !flops_per_s || kind < 0 || kind > 2 || reps < 1 || reps > 1000) return BIOEM_ERR_INVALID_ARG;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return bioem_set_error(ctx, BIOEM_ERR_CUDA, "cudaSetDevice");
    int per_sm = 0;
    cudaError_t e = kind == 0   ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fma_peak<0>, kPeakThreads, 0)
                    : kind == 1 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fma_peak<1>, kPeakThreads, 0)
                                : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fma_peak<2>, kPeakThreads, 0);
    if (e != cudaSuccess || per_sm < 1) return bioem_check_cuda(ctx, e != cudaSuccess ? e : cudaErrorUnknown, "occupancy");
    const int grid = per_sm * ctx->num_sms;   // every SM full, one wave
    const double per_iter = (double)grid * kPeakThreads * kPeakChains * 2.0;   // flop per loop trip
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return bioem_check_cuda(ctx, cudaGetLastError(), "event");
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return bioem_check_cuda(ctx, cudaGetLastError(), "event");
    }
    // calibrate: a short launch, then iterations for ~20 ms per launch (bounded)
    int iters = kind == 2 ? 64 : 2048;
    double best = 0.0;
    int rc = BIOEM_OK;
    for (int r = -1; r < reps && rc == BIOEM_OK; ++r) {
        cudaEventRecord(e0, ctx->stream);
        e = launch_kind(kind, grid, iters, ctx->stream, nullptr, nullptr);
        cudaEventRecord(e1, ctx->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) {
            rc = bioem_check_cuda(ctx, e, "k_fma_peak");
            break;
        }
        if (r < 0) {
            const double scale = ms > 0.f ? 20.0 / ms : 64.0;
            const double it = (double)iters * (scale < 64.0 ? scale : 64.0);
            iters = (int)(it < 1.0 ? 1.0 : (it > 1e7 ? 1e7 : it));
            continue;
        }
        const double v = per_iter * iters / (ms * 1e-3);
        if (v > best) best = v;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    *flops_per_s = best;
    return BIOEM_OK;
}
