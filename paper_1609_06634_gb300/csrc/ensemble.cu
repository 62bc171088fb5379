// Posterior of a weighted ensemble of models over a set of images (Sec. 2, Eq. 10):
//   ln P(M | Omega) = sum_w ln sum_m w_m P_mw   (up to a constant)
// from the [models x images] matrix of ln P_mw, per-model posteriors sum_w ln P_mw, and weights
// raised by expectation-maximisation steps (responsibilities r_mw = w_m P_mw / sum_m' w_m' P_m'w,
// w_m <- mean_w r_mw; the objective is concave in w and the paper gives no optimiser).
//
// One pass = one launch of k_ens_pass (blocks of 256 threads over images, one image per thread
// per step; per-model sums reduced across lanes by a fixed shuffle tree and across warps and
// blocks in index order, so results are deterministic) and one single-block k_ens_update.
#include <math.h>

#include "bioem_internal.cuh"

namespace {

constexpr int kEnsThreads = 256;
constexpr int kEnsWarps = kEnsThreads / 32;
constexpr int kMaxModels = 512;

__device__ __forceinline__ double load_lp(const void* p, int elem_bytes, size_t i) {
    return elem_bytes == 8 ? __ldg(reinterpret_cast<const double*>(p) + i)
                           : (double)__ldg(reinterpret_cast<const float*>(p) + i);
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

// part[block][0 .. M)       sum over the block's images of r_mw
// part[block][M]            sum over the block's images of ln sum_m w_m P_mw
// part[block][M+1 .. 2M+1)  sum over the block's images of ln P_mw
// Shared memory: kEnsWarps x (2M + 1) doubles.
__global__ void __launch_bounds__(kEnsThreads) k_ens_pass(const void* __restrict__ logP, int elem_bytes, int M,
                                                          int n_img, const double* __restrict__ lw,
                                                          double* __restrict__ part) {
    extern __shared__ double ws[];   // [kEnsWarps][2M + 1]
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int stride = 2 * M + 1;
    for (int i = threadIdx.x; i < kEnsWarps * stride; i += blockDim.x) ws[i] = 0.0;
    __syncwarp();
    __syncthreads();
    double* mine = ws + warp * stride;
    for (int base = blockIdx.x * kEnsThreads; base < n_img; base += gridDim.x * kEnsThreads) {
        const int w = base + threadIdx.x;
        const bool ok = w < n_img;
        // ln sum_m w_m P_mw, by the running maximum
        double mx = -INFINITY, s = 0.0;
        if (ok) {
            for (int m = 0; m < M; ++m) {
                const double a = lw[m] + load_lp(logP, elem_bytes, (size_t)m * n_img + w);
                if (!(a > -INFINITY)) continue;
                if (a > mx) {
                    s = s * exp(mx - a) + 1.0;
                    mx = a;
                } else {
                    s += exp(a - mx);
                }
            }
        }
        const double lse = (ok && mx > -INFINITY) ? mx + log(s) : (ok ? -INFINITY : 0.0);
        const double t = warp_sum(lse);
        if (lane == 0) mine[M] += t;
        for (int m = 0; m < M; ++m) {
            const double lp = ok ? load_lp(logP, elem_bytes, (size_t)m * n_img + w) : 0.0;
            const double a = ok ? lw[m] + lp : -INFINITY;
            const double r = (ok && mx > -INFINITY && a > -INFINITY) ? exp(a - lse) : 0.0;
            const double rs = warp_sum(r);
            const double ls = warp_sum(lp);
            if (lane == 0) {
                mine[m] += rs;
                mine[M + 1 + m] += ls;
            }
        }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < stride; k += blockDim.x) {
        double v = 0.0;
        for (int wp = 0; wp < kEnsWarps; ++wp) v += ws[wp * stride + k];
        part[(size_t)blockIdx.x * stride + k] = v;
    }
}

// Folds the blocks' partial sums in block order.  update != 0: w_m = R_m / n_img and lw = ln w.
// Always: out[0] = sum_w ln sum_m w_m P_mw (for the weights the pass used), out[1 + m] = column sums.
__global__ void k_ens_update(const double* __restrict__ part, int n_blocks, int M, int n_img, int update,
                             double* __restrict__ weights, double* __restrict__ lw, double* __restrict__ out) {
    const int stride = 2 * M + 1;
    for (int m = threadIdx.x; m < M; m += blockDim.x) {
        double R = 0.0, L = 0.0;
        for (int b = 0; b < n_blocks; ++b) {
            R += part[(size_t)b * stride + m];
            L += part[(size_t)b * stride + M + 1 + m];
        }
        if (update) {
            const double wm = R / (double)n_img;
            weights[m] = wm;
            lw[m] = log(wm);
        }
        if (out) out[1 + m] = L;
    }
    if (threadIdx.x == 0 && out) {
        double T = 0.0;
        for (int b = 0; b < n_blocks; ++b) T += part[(size_t)b * stride + M];
        out[0] = T;
    }
}

// Normalise the caller's weights to sum 1 (in place) and write their logarithms.
__global__ void k_ens_normalize(double* __restrict__ weights, int M, double* __restrict__ lw, int* status) {
    __shared__ double tot;
    if (threadIdx.x == 0) {
        double s = 0.0;
        bool bad = false;
        for (int m = 0; m < M; ++m) {
            const double v = weights[m];
            if (!(v >= 0.0) || !isfinite(v)) bad = true;
            s += v;
        }
        if (bad || !(s > 0.0)) {
            atomicOr(status, BIOEM_DEV_NUMERIC);
            s = 0.0;
        }
        tot = s;
    }
    __syncthreads();
    for (int m = threadIdx.x; m < M; m += blockDim.x) {
        const double v = tot > 0.0 ? weights[m] / tot : 1.0 / M;
        weights[m] = v;
        lw[m] = log(v);
    }
}

}  // namespace

extern "C" int bioem_ensemble(bioem_ctx* ctx, const void* d_logP, int elem_bytes, int n_models, int n_img,
                              double* d_weights, int n_iter, double* d_out) {
    if (!ctx) return BIOEM_ERR_INVALID_ARG;
    if (!d_logP || !d_weights || !d_out || (elem_bytes != 4 && elem_bytes != 8) || n_models < 1 ||
        n_models > kMaxModels || n_img < 1 || n_iter < 0)
        return bioem_set_error(ctx, BIOEM_ERR_INVALID_ARG, "ensemble: bad argument");
    if (cudaSetDevice(ctx->device) != cudaSuccess) return bioem_set_error(ctx, BIOEM_ERR_CUDA, "cudaSetDevice");
    const int M = n_models;
    const int stride = 2 * M + 1;
    int n_blocks = (n_img + kEnsThreads - 1) / kEnsThreads;
    if (n_blocks > 4 * ctx->num_sms) n_blocks = 4 * ctx->num_sms;
    const size_t part_bytes = sizeof(double) * ((size_t)n_blocks * stride + M);
    double* part = nullptr;
    if (cudaMallocAsync((void**)&part, part_bytes, ctx->stream) != cudaSuccess) {
        cudaGetLastError();
        return bioem_set_error(ctx, BIOEM_ERR_OOM, "ensemble scratch");
    }
    double* lw = part + (size_t)n_blocks * stride;
    const size_t smem = sizeof(double) * kEnsWarps * stride;
    int rc = BIOEM_OK;
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(k_ens_pass, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        rc = bioem_check_cuda(ctx, cudaGetLastError(), "ensemble shared memory");
    if (!rc) {
        bioem_launch_begin(ctx, KID_ENSEMBLE);
        k_ens_normalize<<<1, 256, 0, ctx->stream>>>(d_weights, M, lw, ctx->d_status);
        bioem_launch_end(ctx, KID_ENSEMBLE);
        for (int it = 0; it <= n_iter && !rc; ++it) {
            const int update = it < n_iter;
            bioem_launch_begin(ctx, KID_ENSEMBLE);
            k_ens_pass<<<n_blocks, kEnsThreads, smem, ctx->stream>>>(d_logP, elem_bytes, M, n_img, lw, part);
            bioem_launch_end(ctx, KID_ENSEMBLE);
            bioem_launch_begin(ctx, KID_ENSEMBLE);
            k_ens_update<<<1, 256, 0, ctx->stream>>>(part, n_blocks, M, n_img, update, d_weights, lw,
                                                     update ? nullptr : d_out);
            bioem_launch_end(ctx, KID_ENSEMBLE);
            rc = bioem_check_cuda(ctx, cudaGetLastError(), "ensemble");
        }
    }
    cudaFreeAsync(part, ctx->stream);
    return rc;
}
