// C ABI entry points: argument validation, handle ownership, the device status word.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <new>

#include "bioem_internal.cuh"

int bioem_set_error(bioem_ctx* ctx, int code, const char* fmt, ...) {
    if (ctx) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(ctx->last_error, sizeof(ctx->last_error), fmt, ap);
        va_end(ap);
    }
    return code;
}

int bioem_check_cuda(bioem_ctx* ctx, cudaError_t e, const char* what) {
    if (e == cudaSuccess) return BIOEM_OK;
    if (e == cudaErrorMemoryAllocation) return bioem_set_error(ctx, BIOEM_ERR_OOM, "%s: %s", what, cudaGetErrorString(e));
    return bioem_set_error(ctx, BIOEM_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

const char* const bioem_kernel_names[KID_COUNT] = {
    "k_prepare_images", "k_project", "k_ctf_table", "k_psf_spectra", "k_psf_real",
    "k_score", "k_reduce_wave", "k_finalize", "k_pairs_out", "k_gemm_ops", "k_score_gemm", "k_ensemble",
    "k_lse_merge", "k_score_tc"};

void bioem_launch_begin(bioem_ctx* ctx, int kid) {
    if (!ctx->timing) return;
    bioem_timed_launch t{kid, nullptr, nullptr};
    if (cudaEventCreate(&t.start) != cudaSuccess || cudaEventCreate(&t.stop) != cudaSuccess) {
        cudaGetLastError();
        return;
    }
    cudaEventRecord(t.start, ctx->stream);
    ctx->pending.push_back(t);
}

void bioem_launch_end(bioem_ctx* ctx, int kid) {
    ctx->n_launches++;
    ctx->kid_launches[kid]++;
    if (!ctx->timing || ctx->pending.empty() || ctx->pending.back().kid != kid || !ctx->pending.back().stop) return;
    cudaEventRecord(ctx->pending.back().stop, ctx->stream);
}

// Fold the recorded event pairs into per-kernel totals (synchronises the stream).
static int collect_timings(bioem_ctx* ctx) {
    if (ctx->pending.empty()) return BIOEM_OK;
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    for (auto& t : ctx->pending) {
        float ms = 0.f;
        if (e == cudaSuccess && cudaEventElapsedTime(&ms, t.start, t.stop) == cudaSuccess) ctx->kid_ms[t.kid] += ms;
        cudaEventDestroy(t.start);
        cudaEventDestroy(t.stop);
    }
    ctx->pending.clear();
    cudaGetLastError();
    return e == cudaSuccess ? BIOEM_OK : bioem_check_cuda(ctx, e, "timing synchronisation");
}

float2* bioem_twiddles(bioem_ctx* ctx, int npix) {
    const int k = bioem_size_index(npix);
    return k < 0 ? nullptr : ctx->d_tw[k];
}

namespace {

const int kSizes[5] = {32, 64, 96, 128, 192};

int image_size_ok(int nx, int ny) {
    if (nx != ny) return 0;
    return nx == 32 || nx == 64 || nx == 96 || nx == 128 || nx == 192;
}

// Allocation with the stream-ordered allocator; memory is usable by later work on the stream.
template <class T>
int alloc(bioem_ctx* ctx, T** p, size_t count, const char* what) {
    *p = nullptr;
    if (count == 0) return BIOEM_OK;
    cudaError_t e = cudaMallocAsync((void**)p, sizeof(T) * count, ctx->stream);
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        return bioem_set_error(ctx, BIOEM_ERR_OOM, "cannot allocate %zu bytes for %s", sizeof(T) * count, what);
    }
    return BIOEM_OK;
}

void release(cudaStream_t stream, void* p) {
    if (p) cudaFreeAsync(p, stream);
}

}  // namespace

extern "C" {

const char* bioem_status_string(int status) {
    switch (status) {
        case BIOEM_OK: return "ok";
        case BIOEM_ERR_INVALID_ARG: return "invalid argument";
        case BIOEM_ERR_UNSUPPORTED_SIZE: return "unsupported size";
        case BIOEM_ERR_OOM: return "out of device memory";
        case BIOEM_ERR_CUDA: return "CUDA error";
        case BIOEM_ERR_TIMEOUT: return "device wait timed out";
        case BIOEM_ERR_NUMERIC: return "numerically degenerate input";
        default: return "unknown status";
    }
}

const char* bioem_last_error(const bioem_ctx* ctx) { return ctx ? ctx->last_error : "null context"; }

int bioem_create(bioem_ctx** out, int device, void* cuda_stream) {
    if (!out) return BIOEM_ERR_INVALID_ARG;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return BIOEM_ERR_INVALID_ARG;
    }
    bioem_ctx* ctx = new (std::nothrow) bioem_ctx();
    if (!ctx) return BIOEM_ERR_OOM;
    ctx->device = device;
    ctx->stream = (cudaStream_t)cuda_stream;
    ctx->scratch_limit = 2ull << 30;
    ctx->test_skip_chunk = -1;
    int rc = BIOEM_OK;
    if (cudaSetDevice(device) != cudaSuccess ||
        cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
        rc = BIOEM_ERR_CUDA;
    }
    if (!rc) {
        // keep stream-ordered allocations cached in the device pool between calls instead of
        // returning them to the driver at every synchronisation (projection sets are large)
        cudaMemPool_t pool;
        if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
            unsigned long long keep = ~0ull;
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        }
        cudaGetLastError();
    }
    if (!rc && cudaMalloc((void**)&ctx->d_status, sizeof(int)) != cudaSuccess) rc = BIOEM_ERR_OOM;
    if (!rc && cudaMemset(ctx->d_status, 0, sizeof(int)) != cudaSuccess) rc = BIOEM_ERR_CUDA;
    if (!rc && cudaMalloc((void**)&ctx->d_work, 4 * sizeof(int)) != cudaSuccess) rc = BIOEM_ERR_OOM;
    for (int k = 0; k < 5 && !rc; ++k) {
        const int n = kSizes[k];
        float2* h = (float2*)malloc(sizeof(float2) * n);
        if (!h) { rc = BIOEM_ERR_OOM; break; }
        for (int t = 0; t < n; ++t) {
            const double a = 2.0 * 3.14159265358979323846 * (double)t / (double)n;
            h[t] = make_float2((float)cos(a), (float)-sin(a));   // exp(-2 pi i t / n)
        }
        if (cudaMalloc((void**)&ctx->d_tw[k], sizeof(float2) * n) != cudaSuccess) rc = BIOEM_ERR_OOM;
        else if (cudaMemcpy(ctx->d_tw[k], h, sizeof(float2) * n, cudaMemcpyHostToDevice) != cudaSuccess) rc = BIOEM_ERR_CUDA;
        free(h);
    }
    if (!rc) rc = bioem_upload_score_twiddles(ctx);
    if (rc) {
        cudaGetLastError();
        bioem_destroy(ctx);
        return rc;
    }
    *out = ctx;
    return BIOEM_OK;
}

int bioem_set_stream(bioem_ctx* ctx, void* cuda_stream) {
    if (!ctx) return BIOEM_ERR_INVALID_ARG;
    ctx->stream = (cudaStream_t)cuda_stream;
    return BIOEM_OK;
}

int bioem_set_scratch_limit(bioem_ctx* ctx, unsigned long long bytes) {
    if (!ctx || bytes < 4096) return BIOEM_ERR_INVALID_ARG;
    ctx->scratch_limit = bytes;
    return BIOEM_OK;
}

void bioem_destroy(bioem_ctx* ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    if (ctx->d_rec) cudaFree(ctx->d_rec);
    if (ctx->d_acc) cudaFree(ctx->d_acc);
    if (ctx->d_status) cudaFree(ctx->d_status);
    if (ctx->d_work) cudaFree(ctx->d_work);
    for (int k = 0; k < 5; ++k)
        if (ctx->d_tw[k]) cudaFree(ctx->d_tw[k]);
    for (auto& t : ctx->pending) {
        cudaEventDestroy(t.start);
        cudaEventDestroy(t.stop);
    }
    cudaGetLastError();
    delete ctx;
}

int bioem_set_precision(bioem_ctx* ctx, int mode) {
    if (!ctx) return BIOEM_ERR_INVALID_ARG;
    if (mode < BIOEM_PRECISION_FP32 || mode > BIOEM_PRECISION_FP16X2_FFT)
        return bioem_set_error(ctx, BIOEM_ERR_INVALID_ARG, "unknown precision mode %d", mode);
    ctx->precision = mode;
    return BIOEM_OK;
}

int bioem_get_precision(const bioem_ctx* ctx) { return ctx ? ctx->precision : BIOEM_ERR_INVALID_ARG; }

int bioem_set_wait_test(bioem_ctx* ctx, long long skip_chunk, unsigned long long wait_ns) {
    if (!ctx || skip_chunk < -1 || (skip_chunk >= 0 && (wait_ns < 1000ull || wait_ns > 2000000000ull)))
        return BIOEM_ERR_INVALID_ARG;
    ctx->test_skip_chunk = skip_chunk;
    ctx->test_wait_ns = skip_chunk >= 0 ? wait_ns : 0;
    return BIOEM_OK;
}

int bioem_set_kernel_timing(bioem_ctx* ctx, int enable) {
    if (!ctx) return BIOEM_ERR_INVALID_ARG;
    ctx->timing = enable ? 1 : 0;
    return BIOEM_OK;
}

int bioem_kernel_time(bioem_ctx* ctx, const char* kernel, double* total_ms, unsigned long long* launches) {
    if (!ctx || !kernel) return BIOEM_ERR_INVALID_ARG;
    int kid = -1;
    for (int k = 0; k < KID_COUNT; ++k)
        if (strcmp(kernel, bioem_kernel_names[k]) == 0) kid = k;
    if (kid < 0) return bioem_set_error(ctx, BIOEM_ERR_INVALID_ARG, "unknown kernel name %s", kernel);
    cudaSetDevice(ctx->device);
    const int rc = collect_timings(ctx);
    if (total_ms) *total_ms = ctx->kid_ms[kid];
    if (launches) *launches = ctx->kid_launches[kid];
    return rc;
}

int bioem_reset_kernel_stats(bioem_ctx* ctx) {
    if (!ctx) return BIOEM_ERR_INVALID_ARG;
    cudaSetDevice(ctx->device);
    const int rc = collect_timings(ctx);
    ctx->n_launches = 0;
    for (int k = 0; k < KID_COUNT; ++k) {
        ctx->kid_launches[k] = 0;
        ctx->kid_ms[k] = 0.0;
    }
    return rc;
}

unsigned long long bioem_launch_count(const bioem_ctx* ctx) { return ctx ? ctx->n_launches : 0ull; }

int bioem_get_status(bioem_ctx* ctx, int* out_status) {
    if (!ctx || !out_status) return BIOEM_ERR_INVALID_ARG;
    cudaSetDevice(ctx->device);
    int h = 0;
    cudaError_t e = cudaMemcpyAsync(&h, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->d_status, 0, sizeof(int), ctx->stream);
    if (e != cudaSuccess) return bioem_check_cuda(ctx, e, "status read");
    *out_status = (h & BIOEM_DEV_TIMEOUT)   ? BIOEM_ERR_TIMEOUT
                  : (h & BIOEM_DEV_NUMERIC) ? BIOEM_ERR_NUMERIC
                  : (h ? BIOEM_ERR_CUDA : BIOEM_OK);
    return BIOEM_OK;
}

int bioem_prepare_images(bioem_ctx* ctx, const float* d_images, int n_img, int nx, int ny, double pixel_A,
                         bioem_images** out) {
    if (!ctx || !out) return BIOEM_ERR_INVALID_ARG;
    *out = nullptr;
    if (n_img < 0 || nx <= 0 || ny <= 0 || !(pixel_A > 0.0) || (n_img > 0 && !d_images))
        return bioem_set_error(ctx, BIOEM_ERR_INVALID_ARG, "prepare_images: bad argument");
    if (!image_size_ok(nx, ny))
        return bioem_set_error(ctx, BIOEM_ERR_UNSUPPORTED_SIZE, "prepare_images: %dx%d not supported", nx, ny);
    if (cudaSetDevice(ctx->device) != cudaSuccess) return bioem_set_error(ctx, BIOEM_ERR_CUDA, "cudaSetDevice");
    bioem_images* im = (bioem_images*)calloc(1, sizeof(bioem_images));
    if (!im) return BIOEM_ERR_OOM;
    im->ctx = ctx;
    im->device = ctx->device;
    im->stream = ctx->stream;
    im->n_img = n_img;
    im->nx = nx;
    im->ny = ny;
    im->pixel_A = pixel_A;
    int rc = alloc(ctx, &im->d_spec, (size_t)n_img * ny * (nx / 2 + 1), "image spectra");
    if (!rc) rc = alloc(ctx, &im->d_kA, (size_t)n_img, "image constants");
    if (!rc) rc = alloc(ctx, &im->d_amax, (size_t)n_img, "image constants");
    if (!rc && n_img > 0) rc = bioem_launch_prepare(ctx, d_images, im);
    if (rc) {
        bioem_free_images(im);
        return rc;
    }
    *out = im;
    return BIOEM_OK;
}

int bioem_project_model(bioem_ctx* ctx, const float* d_atoms, int n_atoms, double sigma_A, const float* d_quats, int nq,
                        const bioem_ctf* ctfs, int nctf, int nx, int ny, double pixel_A, bioem_projset** out) {
    if (!ctx || !out) return BIOEM_ERR_INVALID_ARG;
    *out = nullptr;
    if (n_atoms < 0 || nq < 0 || nctf <= 0 || !ctfs || !(sigma_A > 0.0) || !(pixel_A > 0.0) ||
        (n_atoms > 0 && !d_atoms) || (nq > 0 && !d_quats))
        return bioem_set_error(ctx, BIOEM_ERR_INVALID_ARG, "project_model: bad argument");
    for (int c = 0; c < nctf; ++c) {
        const bioem_ctf& f = ctfs[c];
        if (!(f.amp_contrast >= 0.0 && f.amp_contrast <= 1.0) || !(f.bfactor_A2 >= 0.0) || !(f.voltage_kV > 0.0) ||
            !isfinite(f.defocus_A))
            return bioem_set_error(ctx, BIOEM_ERR_INVALID_ARG, "project_model: bad CTF entry %d", c);
    }
    if (!image_size_ok(nx, ny))
        return bioem_set_error(ctx, BIOEM_ERR_UNSUPPORTED_SIZE, "project_model: %dx%d not supported", nx, ny);
    if ((long long)nq * nctf > 0x7fffffffll)
        return bioem_set_error(ctx, BIOEM_ERR_UNSUPPORTED_SIZE, "project_model: too many parameter sets");
    if (cudaSetDevice(ctx->device) != cudaSuccess) return bioem_set_error(ctx, BIOEM_ERR_CUDA, "cudaSetDevice");
    bioem_projset* ps = (bioem_projset*)calloc(1, sizeof(bioem_projset));
    if (!ps) return BIOEM_ERR_OOM;
    ps->ctx = ctx;
    ps->device = ctx->device;
    ps->stream = ctx->stream;
    ps->nq = nq;
    ps->nctf = nctf;
    ps->n_ps = nq * nctf;
    ps->nx = nx;
    ps->ny = ny;
    ps->pixel_A = pixel_A;
    int rc = alloc(ctx, &ps->d_spec, (size_t)ps->n_ps * ny * (nx / 2 + 1), "projection spectra");
    if (!rc) rc = alloc(ctx, &ps->d_kB, (size_t)ps->n_ps, "projection constants");
    if (!rc) rc = alloc(ctx, &ps->d_amax, (size_t)ps->n_ps, "projection constants");
    if (!rc && nq > 0) rc = bioem_launch_project(ctx, d_atoms, n_atoms, sigma_A, d_quats, nq, ctfs, nctf, ps);
    if (rc) {
        bioem_free_projset(ps);
        return rc;
    }
    *out = ps;
    return BIOEM_OK;
}

static int check_pair(bioem_ctx* ctx, const bioem_images* im, const bioem_projset* ps, int max_shift) {
    if (!ctx || !im || !ps) return BIOEM_ERR_INVALID_ARG;
    if (im->ctx != ctx || ps->ctx != ctx) return bioem_set_error(ctx, BIOEM_ERR_INVALID_ARG, "handle from another context");
    if (im->nx != ps->nx || im->ny != ps->ny || fabs(im->pixel_A - ps->pixel_A) > 1e-9 * im->pixel_A)
        return bioem_set_error(ctx, BIOEM_ERR_INVALID_ARG, "images and projections differ in size or pixel");
    if (max_shift < 0) return bioem_set_error(ctx, BIOEM_ERR_INVALID_ARG, "negative max_shift");
    const int supported = ctx->precision == BIOEM_PRECISION_FP32       ? bioem_score_supported(im->nx, max_shift)
                          : ctx->precision == BIOEM_PRECISION_FP16X2_FFT ? bioem_tc_supported(im->nx, max_shift)
                                                                         : bioem_gemm_supported(im->nx, max_shift);
    if (!supported)
        return bioem_set_error(ctx, BIOEM_ERR_UNSUPPORTED_SIZE, "max_shift %d unsupported at %d px in precision mode %d",
                               max_shift, im->nx, ctx->precision);
    if (ps->n_ps == 0) return bioem_set_error(ctx, BIOEM_ERR_INVALID_ARG, "empty parameter set");
    if (cudaSetDevice(ctx->device) != cudaSuccess) return bioem_set_error(ctx, BIOEM_ERR_CUDA, "cudaSetDevice");
    return BIOEM_OK;
}

int bioem_score_all(bioem_ctx* ctx, const bioem_images* images, const bioem_projset* projset, int max_shift,
                    double* d_logP, double* d_logP_per_orient, int* d_best_q, int* d_best_ctf, int* d_best_dx,
                    int* d_best_dy, double* d_best_logL) {
    int rc = check_pair(ctx, images, projset, max_shift);
    if (rc) return rc;
    if (images->n_img > 0 && !d_logP && !d_best_logL && !d_logP_per_orient)
        return bioem_set_error(ctx, BIOEM_ERR_INVALID_ARG, "score: no output");
    bioem_score_out out{};
    out.logP = d_logP;
    out.logP_orient = d_logP_per_orient;
    out.best_q = d_best_q;
    out.best_ctf = d_best_ctf;
    out.best_dx = d_best_dx;
    out.best_dy = d_best_dy;
    out.best_logL = d_best_logL;
    return bioem_launch_score(ctx, images, projset, max_shift, out);
}

int bioem_score(bioem_ctx* ctx, const bioem_images* images, const bioem_projset* projset, int max_shift,
                double* d_logP, double* d_logP_per_orient) {
    if (ctx && images && images->n_img > 0 && !d_logP)
        return bioem_set_error(ctx, BIOEM_ERR_INVALID_ARG, "score: d_logP is required");
    return bioem_score_all(ctx, images, projset, max_shift, d_logP, d_logP_per_orient, nullptr, nullptr, nullptr,
                           nullptr, nullptr);
}

int bioem_best_params(bioem_ctx* ctx, const bioem_images* images, const bioem_projset* projset, int max_shift,
                      int* d_best_q, int* d_best_ctf, int* d_best_dx, int* d_best_dy, double* d_best_logL) {
    if (ctx && images && images->n_img > 0 && !d_best_logL)
        return bioem_set_error(ctx, BIOEM_ERR_INVALID_ARG, "best_params: d_best_logL is required");
    return bioem_score_all(ctx, images, projset, max_shift, nullptr, nullptr, d_best_q, d_best_ctf, d_best_dx,
                           d_best_dy, d_best_logL);
}

int bioem_score_pairs(bioem_ctx* ctx, const bioem_images* images, const bioem_projset* projset, int max_shift,
                      int ps_begin, int ps_count, double* d_pair_max, double* d_pair_lse) {
    int rc = check_pair(ctx, images, projset, max_shift);
    if (rc) return rc;
    if (ps_begin < 0 || ps_count < 0 || (long long)ps_begin + ps_count > projset->n_ps ||
        (images->n_img > 0 && ps_count > 0 && !d_pair_max))
        return bioem_set_error(ctx, BIOEM_ERR_INVALID_ARG, "score_pairs: bad range or output");
    if (ps_count == 0 || images->n_img == 0) return BIOEM_OK;
    bioem_score_out out{};
    out.pair_max = d_pair_max;
    out.pair_lse = d_pair_lse;
    out.ps_begin = ps_begin;
    out.ps_count = ps_count;
    return bioem_launch_score(ctx, images, projset, max_shift, out);
}

int bioem_score_accumulate(bioem_ctx* ctx, const bioem_images* images, const bioem_projset* projset, int max_shift,
                           double* d_acc, int first) {
    int rc = check_pair(ctx, images, projset, max_shift);
    if (rc) return rc;
    if (images->n_img > 0 && !d_acc) return bioem_set_error(ctx, BIOEM_ERR_INVALID_ARG, "score_accumulate: d_acc");
    bioem_score_out out{};
    out.acc2 = d_acc;
    out.acc_first = first ? 1 : 0;
    return bioem_launch_score(ctx, images, projset, max_shift, out);
}

int bioem_synthetic_maps(bioem_ctx* ctx, const float* d_atoms, int n_atoms, double sigma_A, const float* d_quats,
                         const bioem_ctf* ctfs, int n, int nx, int ny, double pixel_A, float* d_out) {
    if (!ctx) return BIOEM_ERR_INVALID_ARG;
    if (n < 0 || n_atoms < 0 || !(sigma_A > 0.0) || !(pixel_A > 0.0) ||
        (n > 0 && (!d_quats || !ctfs || !d_out)) || (n_atoms > 0 && !d_atoms))
        return bioem_set_error(ctx, BIOEM_ERR_INVALID_ARG, "synthetic_maps: bad argument");
    if (!image_size_ok(nx, ny))
        return bioem_set_error(ctx, BIOEM_ERR_UNSUPPORTED_SIZE, "synthetic_maps: %dx%d not supported", nx, ny);
    if (n == 0) return BIOEM_OK;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return bioem_set_error(ctx, BIOEM_ERR_CUDA, "cudaSetDevice");
    return bioem_launch_synthetic(ctx, d_atoms, n_atoms, sigma_A, d_quats, ctfs, n, nx, pixel_A, d_out);
}

int bioem_images_count(const bioem_images* images) { return images ? images->n_img : -1; }
int bioem_projset_count(const bioem_projset* projset) { return projset ? projset->n_ps : -1; }

void bioem_free_images(bioem_images* im) {
    if (!im) return;
    cudaSetDevice(im->device);
    release(im->stream, im->d_spec);
    release(im->stream, im->d_kA);
    release(im->stream, im->d_amax);
    bioem_gemm_cache_free(&im->gemm, im->stream);
    free(im);
}

void bioem_free_projset(bioem_projset* ps) {
    if (!ps) return;
    cudaSetDevice(ps->device);
    release(ps->stream, ps->d_spec);
    release(ps->stream, ps->d_kB);
    release(ps->stream, ps->d_amax);
    bioem_gemm_cache_free(&ps->gemm, ps->stream);
    free(ps);
}

}  // extern "C"
