// Internal declarations shared by the translation units of the BioEM sm_103a library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/bioem.h"

// ------------------------------------------------------------------ kernel accounting
enum bioem_kernel_id {
    KID_PREPARE = 0, KID_PROJECT, KID_CTF_TABLE, KID_PSF_SPECTRA, KID_PSF_REAL, KID_SCORE, KID_REDUCE_WAVE,
    KID_FINALIZE, KID_PAIRS_OUT, KID_GEMM_OPS, KID_SCORE_GEMM, KID_ENSEMBLE, KID_LSE_MERGE, KID_SCORE_TC,
    KID_COUNT
};
extern const char* const bioem_kernel_names[KID_COUNT];

struct bioem_timed_launch {
    int kid;
    cudaEvent_t start, stop;
};

// ------------------------------------------------------------------ handles
struct bioem_ctx {
    int device;
    cudaStream_t stream;
    int num_sms;
    int* d_status;                      // device status word (BIOEM_ERR_* bits folded to a code)
    int* d_work;                        // work-item counter of the scoring kernel (reset before each launch)
    unsigned long long scratch_limit;   // bytes allowed for per-pair records
    // per-pair record scratch (grown on demand)
    void* d_rec;
    size_t rec_bytes;
    // per-image accumulators of the wave reduction
    void* d_acc;
    size_t acc_bytes;
    // twiddle tables (float2, W_N^k = exp(-2 pi i k / N)) for the direct transforms, by N
    float2* d_tw[5];
    char last_error[256];
    // launch accounting and optional per-launch CUDA-event timing on the context's stream
    unsigned long long n_launches;
    unsigned long long kid_launches[KID_COUNT];
    int timing;
    std::vector<bioem_timed_launch> pending;
    double kid_ms[KID_COUNT];
    int precision;   // BIOEM_PRECISION_*: the form bioem_score and its relatives use
    // failure-detection test hook, armed for the next tensor-core scoring launch only
    long long test_skip_chunk;            // -1: none
    unsigned long long test_wait_ns;      // 0: the default limit
};

// Operands of the split-precision GEMM scoring form, built from a handle's spectra on first use
// and kept with the handle (rebuilt when the precision or, for images, the shift window changes).
struct bioem_gemm_cache {
    void* d_ops;     // tile-ready hi/lo operand blocks
    size_t bytes;
    float* d_inv;    // per row (parameter set) or per image: 1 / power-of-two scale
    int mode;        // BIOEM_PRECISION_* it was built for (0: none)
    int shift;       // images: the displacement half-width of its columns
};

struct bioem_images {
    bioem_ctx* ctx;          // creating context (compared, never dereferenced after it is destroyed)
    int device;              // handles free their memory with their own device and stream
    cudaStream_t stream;
    int n_img, nx, ny;
    double pixel_A;
    float2* d_spec;   // [n_img][ny][nx/2 + 1] unit-norm half spectrum, DC = 0
    double* d_kA;     // [n_img] (3-n)/2 ln A + c(n)
    float* d_amax;    // [n_img] largest |coefficient| of the stored spectrum
    mutable bioem_gemm_cache gemm;
};

struct bioem_projset {
    bioem_ctx* ctx;
    int device;
    cudaStream_t stream;
    int nq, nctf, n_ps, nx, ny;
    double pixel_A;
    float2* d_spec;   // [n_ps][ny][nx/2 + 1] unit-norm PSF-filtered projection spectrum, DC = 0
    double* d_kB;     // [n_ps] -1/2 ln B
    float* d_amax;    // [n_ps] largest |coefficient| of the stored spectrum
    mutable bioem_gemm_cache gemm;
};

// ------------------------------------------------------------------ status codes inside kernels
#define BIOEM_DEV_NUMERIC 1
#define BIOEM_DEV_TIMEOUT 2

// ------------------------------------------------------------------ helpers
__host__ __device__ inline int bioem_size_index(int n) {
    switch (n) {
        case 32: return 0;
        case 64: return 1;
        case 96: return 2;
        case 128: return 3;
        case 192: return 4;
        default: return -1;
    }
}

__device__ __forceinline__ float2 c_add(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 c_sub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 c_mul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// conj(a) * b
__device__ __forceinline__ float2 c_mulc(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.x, b.y, -a.y * b.x));
}
__device__ __forceinline__ float2 c_scale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }

// t = ln(1 - x) for 0 <= x < 1 (x = rho^2, the per-displacement factor of the closed-form likelihood).
// Correlation coefficients of noisy images are small (rho^2 < 1e-2 for nearly every pair), and there
// the Taylor series -(x + x^2/2 + x^3/3 + x^4/4 + x^5/5) in Horner form is used: for x <= 1/32 its
// truncation error is below x^6/(6 (1 - x)), under 6e-9 of |t|, so the result is as accurate as the
// rounding of its five operations allows.  Larger x take the library's log1pf.
__device__ __forceinline__ float ln1m_series(float x) {
    float p = fmaf(x, 0.2f, 0.25f);
    p = fmaf(x, p, 0.33333334f);
    p = fmaf(x, p, 0.5f);
    p = fmaf(x, p, 1.0f);
    return -x * p;
}
__device__ __forceinline__ float ln1m(float x) {
    float t = ln1m_series(x);
    if (x > 0.03125f) t = log1pf(-x);
    return t;
}

// ------------------------------------------------------------------ launchers (defined in .cu files)
// prep_project.cu
int bioem_launch_prepare(bioem_ctx* ctx, const float* d_images, bioem_images* im);
int bioem_launch_project(bioem_ctx* ctx, const float* d_atoms, int n_atoms, double sigma_A,
                         const float* d_quats, int nq, const bioem_ctf* ctfs, int nctf,
                         bioem_projset* ps);
int bioem_launch_synthetic(bioem_ctx* ctx, const float* d_atoms, int n_atoms, double sigma_A,
                           const float* d_quats, const bioem_ctf* ctfs, int n, int npix,
                           double pixel_A, float* d_out);
double bioem_log_norm_constant(int n);
// zero-mean, unit-norm real-space images of `count` stored half spectra, and max |x| of each
int bioem_launch_spec_to_real(bioem_ctx* ctx, const float2* spec, int count, int npix, float* out, float* amax);

// score.cu
struct bioem_score_out {
    double* logP;
    double* logP_orient;
    int* best_q;
    int* best_ctf;
    int* best_dx;
    int* best_dy;
    double* best_logL;
    double* pair_max;   // score_pairs mode
    double* pair_lse;
    int ps_begin, ps_count;
    double* acc2;       // bioem_score_accumulate: caller's [n_img][2] (max, sum exp(. - max)) of ln L
    int acc_first;      // overwrite acc2 instead of folding into it
};
int bioem_score_supported(int npix, int max_shift);
int bioem_launch_score(bioem_ctx* ctx, const bioem_images* im, const bioem_projset* ps, int max_shift,
                       const bioem_score_out& out);
int bioem_upload_score_twiddles(bioem_ctx* ctx);

// gemm.cu (split-precision tensor-core form)
int bioem_gemm_supported(int npix, int max_shift);
int bioem_gemm_row_tile();
int bioem_gemm_prepare(bioem_ctx* ctx, const bioem_images* im, const bioem_projset* ps, int max_shift, int mode);
int bioem_gemm_records(bioem_ctx* ctx, const bioem_images* im, const bioem_projset* ps, int max_shift, int mode,
                       int ps_lo, int ps_hi, float* rec_t, float* rec_s, int* rec_d);
void bioem_gemm_cache_free(bioem_gemm_cache* c, cudaStream_t stream);

// score_tc.cu (FP32 scoring form with its column transforms as split-FP16 tensor-core products)
int bioem_tc_supported(int npix, int max_shift);
int bioem_tc_records(bioem_ctx* ctx, const bioem_images* im, const bioem_projset* ps, int max_shift, int wbegin,
                     int wl, float* rec_t, float* rec_s, int* rec_d);

// abi.cu
void bioem_launch_begin(bioem_ctx* ctx, int kid);   // call before a kernel launch
void bioem_launch_end(bioem_ctx* ctx, int kid);     // call after it (counts it; records the stop event)
int bioem_set_error(bioem_ctx* ctx, int code, const char* fmt, ...);
int bioem_check_cuda(bioem_ctx* ctx, cudaError_t e, const char* what);
float2* bioem_twiddles(bioem_ctx* ctx, int npix);
