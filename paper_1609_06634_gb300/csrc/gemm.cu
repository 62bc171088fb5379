// Split-precision scoring on the fifth-generation tensor cores.  The inverse transform restricted to
// the wanted displacements (Sec. 3.9 and Sec. 5: only some correlation coefficients are needed) is
// written as one dense real matrix product whose columns are displacements, with the conjugate
// Fourier product of Eq. 11 folded into the image-side operand:
//
//   rho_p(d) = Re sum_k w_kx conj(O(k)) C_p(k) exp(+2 pi i (ky dy + kx dx) / N)
//            = sum_k  Re C_p(k) Re G(k, d)  -  Im C_p(k) Im G(k, d),
//   G(k, d)  = w_kx conj(O(k)) exp(+2 pi i (ky dy + kx dx) / N),   w = 1 on kx = 0, N/2 and 2 elsewhere,
//
// O and C_p the unit-norm half spectra (DC = 0) of the image and of parameter set p, k = (ky, kx)
// over the N (N/2 + 1) stored coefficients.  So, with K = 2 N (N/2 + 1) real terms,
//   A [parameter sets x K]            row p:  (Re C_p(k), Im C_p(k)) for every k
//   B [image-displacement columns x K] column (w, d): (Re G_w(k, d), -Im G_w(k, d))
//   D = A B^T,  rho_p,w(d) = D[p][(w, d)]
// Each image owns NS^2 = (2 s + 1)^2 columns; a tile of 256 columns holds IPT = floor(256 / NS^2)
// images, a tile of 128 rows holds 128 parameter sets.  Both operands are split x = hi + lo into two
// 16-bit floats (BF16, or FP16 scaled by powers of two so the lo parts stay normal) and
//   D = A_hi B_hi + A_hi B_lo + A_lo B_hi     (FP32 accumulation in tensor memory; lo x lo dropped).
//
// The epilogue turns D into t(d) = log1p(-rho(d)^2) and writes, per (parameter set, image), the
// same (t_min, sum exp(c1 (t - t_min)), argmin d) record as the FP32 kernel, so the float64
// reductions that follow are shared.
//
// Kernel layout (one CTA per SM, persistent over 128 x 256 tiles): warp 0 streams operand chunks
// with bulk asynchronous copies into a four-stage shared-memory ring, warp 1 allocates 512 tensor-
// memory columns (two 256-column accumulators) and issues the MMAs from one thread, warps 2-9 drain
// an accumulator into FP32 registers (tcgen05.ld, then round-to-nearest adds) while the next group
// of K chunks accumulates into the other.  The tensor cores' own FP32 accumulation, run over the
// whole K of a tile, biased |rho| low by about 1e-5 (log P by -7e-3 at 128 px; one-signed, the
// same for BF16 and FP16 operands); restarting it every GROUP chunks (96 MMAs) and summing the
// partial products in registers removes most of that (restarting every 48 MMAs halves the rest but
// lets the epilogue's likelihood pass stall the MMAs at tile ends: 5-11 % slower).  Every wait on a
// barrier is bounded in time; on expiry the kernel sets a status bit and leaves cleanly.
//
// Operands are stored in global memory already in the tensor cores' shared-memory layout (K-major,
// no swizzle: 8-row x 16-byte core matrices, the 4 core matrices of a 32-element K chunk 128 B
// apart, 8-row groups 512 B apart), one contiguous block per (tile, K chunk), hi block then lo
// block, so one bulk copy moves each.
#include <math.h>
#include <stdio.h>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "bioem_internal.cuh"
#include "tc_util.cuh"

namespace {

constexpr int GM = 128;                        // parameter sets per tile (tensor-memory lanes)
constexpr int GN = 256;                        // image-displacement columns per tile
constexpr int KC = 32;                         // K elements per pipeline stage
constexpr int KSTEP = 16;                      // K per MMA instruction (16-bit operands)
constexpr int A_TERM = GM * KC * 2;            // bytes of one operand term of one stage: 8 KB
constexpr int B_TERM = GN * KC * 2;            // 16 KB
constexpr int RG_BYTES = KC * 16;              // one 8-row group: KC / 8 core matrices of 128 B
constexpr int STAGE = 2 * A_TERM + 2 * B_TERM; // 48 KB: A hi, A lo, B hi, B lo
constexpr int NSTAGE = 4;
constexpr int EPI_THREADS = 256;               // epilogue: 8 warps, two per tensor-memory lane quarter
constexpr int GEMM_THREADS = 64 + EPI_THREADS; // warp 0 copies, warp 1 MMAs, warps 2-9 epilogue
constexpr int GROUP = 16;                      // K chunks accumulated in tensor memory before a drain (96 MMAs)
constexpr size_t GEMM_SMEM = (size_t)NSTAGE * STAGE + 256;
constexpr int TMEM_COLS = 2 * GN;

static_assert(KC % KSTEP == 0, "whole MMA steps per stage");
static_assert(STAGE < (1 << 20), "transaction count of one barrier phase");

// ------------------------------------------------------------------ operand construction
// Scale exponent e with bound * 2^e < 2^15 (FP16 keeps its largest hi parts below 65504 and its lo
// parts, about 2^-11 of them, normal).
__device__ __forceinline__ int scale_exp(float bound) {
    if (!(bound > 0.f) || !isfinite(bound)) return 0;
    int e;
    frexpf(bound, &e);   // bound < 2^e
    return 15 - e;
}

// (x, y) -> hi = round(x, y) and lo = round(x - hi, y - hi), each a pair of 16-bit floats in one word
// (x in the low half: the lower K index).
__device__ __forceinline__ void split2(float x, float y, int fp16, uint32_t& hi, uint32_t& lo) {
    if (fp16) {
        const __half2 h = __floats2half2_rn(x, y);
        const float2 hf = __half22float2(h);
        const __half2 l = __floats2half2_rn(x - hf.x, y - hf.y);
        hi = *reinterpret_cast<const uint32_t*>(&h);
        lo = *reinterpret_cast<const uint32_t*>(&l);
    } else {
        const __nv_bfloat162 h = __floats2bfloat162_rn(x, y);
        const float2 hf = __bfloat1622float2(h);
        const __nv_bfloat162 l = __floats2bfloat162_rn(x - hf.x, y - hf.y);
        hi = *reinterpret_cast<const uint32_t*>(&h);
        lo = *reinterpret_cast<const uint32_t*>(&l);
    }
}

// A operand: one warp per core matrix (8 parameter sets x 4 coefficients = 8 x 8 K elements) of a
// (row tile, K chunk); lane = 4 (row % 8) + coefficient % 4, so each warp writes 128 contiguous bytes.
// ncoef = N (N/2 + 1) coefficients per spectrum.
__global__ void k_gemm_ops_ps(const float2* __restrict__ spec, const float* __restrict__ amax, int n_ps, int ncoef,
                              int n_chunks, int fp16, unsigned char* __restrict__ ops, size_t total_cm) {
    const int lane = threadIdx.x & 31;
    const size_t nw = (size_t)gridDim.x * (blockDim.x >> 5);
    for (size_t cm = (size_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); cm < total_cm; cm += nw) {
        const int kg = (int)(cm % (KC / 8));
        size_t rest = cm / (KC / 8);
        const int rg = (int)(rest % (GM / 8));
        rest /= (GM / 8);
        const int chunk = (int)(rest % n_chunks);
        const size_t tile = rest / n_chunks;
        const long long p = (long long)tile * GM + rg * 8 + (lane >> 2);
        const int c = chunk * (KC / 2) + kg * 4 + (lane & 3);
        float2 v = make_float2(0.f, 0.f);
        if (p < n_ps) {
            v = __ldg(spec + (size_t)p * ncoef + c);
            if (fp16) {
                const int e = scale_exp(__ldg(amax + p));
                v.x = ldexpf(v.x, e);
                v.y = ldexpf(v.y, e);
            }
        }
        uint32_t hi, lo;
        split2(v.x, v.y, fp16, hi, lo);
        unsigned char* blk = ops + (tile * n_chunks + chunk) * (size_t)(2 * A_TERM);
        const int off = rg * RG_BYTES + kg * 128 + lane * 4;
        *reinterpret_cast<uint32_t*>(blk + off) = hi;
        *reinterpret_cast<uint32_t*>(blk + A_TERM + off) = lo;
    }
}

// B operand: column n of image tile `tile` is displacement d = n - NS^2 ib of image w = IPT tile + ib;
// element pair (Re G, -Im G) of coefficient c = ky (N/2 + 1) + kx.  tw[t] = exp(-2 pi i t / N).
__global__ void k_gemm_ops_img(const float2* __restrict__ spec, const float* __restrict__ amax, int n_img, int npix,
                               int nh, int n_chunks, int smax, int ipt, int fp16, const float2* __restrict__ tw,
                               unsigned char* __restrict__ ops, size_t total_cm) {
    const int lane = threadIdx.x & 31;
    const int ns = 2 * smax + 1, ns2 = ns * ns;
    const size_t nw = (size_t)gridDim.x * (blockDim.x >> 5);
    for (size_t cm = (size_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); cm < total_cm; cm += nw) {
        const int kg = (int)(cm % (KC / 8));
        size_t rest = cm / (KC / 8);
        const int rg = (int)(rest % (GN / 8));
        rest /= (GN / 8);
        const int chunk = (int)(rest % n_chunks);
        const size_t tile = rest / n_chunks;
        const int n = rg * 8 + (lane >> 2);
        const int ib = n / ns2;
        const int d = n - ib * ns2;
        const long long w = (long long)tile * ipt + ib;
        const int c = chunk * (KC / 2) + kg * 4 + (lane & 3);
        float gx = 0.f, gy = 0.f;
        if (ib < ipt && w < n_img) {
            const int ky = c / nh, kx = c - (c / nh) * nh;
            const int dy = d / ns - smax, dx = d - (d / ns) * ns - smax;
            int t = (ky * dy + kx * dx) % npix;
            t += t < 0 ? npix : 0;
            const float2 e = __ldg(tw + t);                  // exp(-i theta): exp(+i theta) = conj(e)
            const float2 o = __ldg(spec + (size_t)w * npix * nh + c);
            const float wk = (kx == 0 || kx == npix / 2) ? 1.f : 2.f;
            // conj(o) conj(e) = conj(o e)
            const float re = o.x * e.x - o.y * e.y, im = o.x * e.y + o.y * e.x;
            gx = wk * re;    // Re G
            gy = wk * im;    // -Im G = +Im(o e)
            if (fp16) {
                const int es = scale_exp(2.8285f * __ldg(amax + w));   // |G| <= 2 |o| <= 2 sqrt(2) amax
                gx = ldexpf(gx, es);
                gy = ldexpf(gy, es);
            }
        }
        uint32_t hi, lo;
        split2(gx, gy, fp16, hi, lo);
        unsigned char* blk = ops + (tile * n_chunks + chunk) * (size_t)(2 * B_TERM);
        const int off = rg * RG_BYTES + kg * 128 + lane * 4;
        *reinterpret_cast<uint32_t*>(blk + off) = hi;
        *reinterpret_cast<uint32_t*>(blk + B_TERM + off) = lo;
    }
}

// B operand of the real-space form (Sec. 3.3's real-space variant: one correlation per
// displacement): column n of image tile `tile` is displacement d of image w; the K pair c holds
// pixels r = 2c, 2c + 1 (same row: N is even) of the displaced image o'(r - d), indices mod N.
// img: [n_img][N][N] zero-mean unit-norm real-space images; amax: max |o'| per image.
__global__ void k_gemm_ops_img_real(const float* __restrict__ img, const float* __restrict__ amax, int n_img,
                                    int npix, int n_chunks, int smax, int ipt, int fp16,
                                    unsigned char* __restrict__ ops, size_t total_cm) {
    const int lane = threadIdx.x & 31;
    const int ns = 2 * smax + 1, ns2 = ns * ns;
    const size_t nw = (size_t)gridDim.x * (blockDim.x >> 5);
    for (size_t cm = (size_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); cm < total_cm; cm += nw) {
        const int kg = (int)(cm % (KC / 8));
        size_t rest = cm / (KC / 8);
        const int rg = (int)(rest % (GN / 8));
        rest /= (GN / 8);
        const int chunk = (int)(rest % n_chunks);
        const size_t tile = rest / n_chunks;
        const int n = rg * 8 + (lane >> 2);
        const int ib = n / ns2;
        const int d = n - ib * ns2;
        const long long w = (long long)tile * ipt + ib;
        const int c = chunk * (KC / 2) + kg * 4 + (lane & 3);
        float gx = 0.f, gy = 0.f;
        if (ib < ipt && w < n_img) {
            const int r0 = 2 * c;
            const int y = r0 / npix, x0 = r0 - (r0 / npix) * npix;
            const int dy = d / ns - smax, dx = d - (d / ns) * ns - smax;
            int ys = (y - dy) % npix;
            ys += ys < 0 ? npix : 0;
            int xs = (x0 - dx) % npix;
            xs += xs < 0 ? npix : 0;
            const int xs1 = xs + 1 == npix ? 0 : xs + 1;
            const float* row = img + ((size_t)w * npix + ys) * npix;
            gx = __ldg(row + xs);
            gy = __ldg(row + xs1);
            if (fp16) {
                const int es = scale_exp(__ldg(amax + w));
                gx = ldexpf(gx, es);
                gy = ldexpf(gy, es);
            }
        }
        uint32_t hi, lo;
        split2(gx, gy, fp16, hi, lo);
        unsigned char* blk = ops + (tile * n_chunks + chunk) * (size_t)(2 * B_TERM);
        const int off = rg * RG_BYTES + kg * 128 + lane * 4;
        *reinterpret_cast<uint32_t*>(blk + off) = hi;
        *reinterpret_cast<uint32_t*>(blk + B_TERM + off) = lo;
    }
}

// 1 / (scale of parameter set p) and 1 / (scale of image w), exact powers of two.
__global__ void k_gemm_inv_scales(const float* __restrict__ amax, int n, float bound_factor, int fp16,
                                  float* __restrict__ inv) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        inv[i] = fp16 ? ldexpf(1.f, -scale_exp(bound_factor * amax[i])) : 1.f;
}

struct GemmArgs {
    const unsigned char* a_ops;   // [row tiles][chunks][hi, lo][128 x 64]
    const unsigned char* b_ops;   // [column tiles][chunks][hi, lo][256 x 64]
    const float* inv_ps;          // [row tiles * 128] 1 / scale of each parameter set
    const float* inv_img;         // [n_img]
    int n_chunks;
    int ptile0, n_ptiles;         // row tiles [ptile0, ptile0 + n_ptiles)
    int n_itiles, ipt, smax;      // column tiles, images per column tile, displacement half-width
    int n_img;
    int ps_lo, ps_hi;             // records for parameter sets [ps_lo, ps_hi)
    float c1;                     // (3 - n) / 2
    uint32_t idesc;
    long long skip_chunk;         // failure-detection test: the producer skips this chunk's copies (-1: none)
    unsigned long long wait_ns;   // limit of every barrier wait
    float* rec_t;                 // [n_img][ps_hi - ps_lo]
    float* rec_s;
    int* rec_d;
    int* status;
};

struct Part {
    float t;   // min ln(1 - rho^2)
    float s;   // sum exp(c1 (t(d) - t))
    int d;     // index of the minimum (lowest on ties)
};

__device__ __forceinline__ Part part_merge(Part a, Part b, float c1) {
    if (b.t > a.t || (b.t == a.t && b.d > a.d)) {
        const Part x = a;
        a = b;
        b = x;
    }
    if (!(a.t < INFINITY)) return b;
    return Part{b.t, b.s + a.s * __expf(c1 * (a.t - b.t)), b.d};
}

// One displacement's value into a running (t_min, sum, argmin): rho = v inv, t = ln(1 - rho^2).
// No data-dependent branch apart from ln1m's rarely taken one for rho^2 > 1/32 (the lanes of a warp
// hold different parameter sets, so a branch would serialise both sides on every column), one exponential: e = exp(c1 |t - t_min|) either rescales
// the sum to a new minimum (s e + 1) or is the new term (s + e).  r2max collects rho^2 for one
// |rho| >= 1 check per tile.
__device__ __forceinline__ void part_add(Part& st, float& r2max, float v, float inv, int j, float c1) {
    const float rho = v * inv;
    const float r2 = rho * rho;
    r2max = fmaxf(r2max, r2);
    const float tv = ln1m(fminf(r2, 1.0f - 5.9604645e-8f));
    const bool lower = tv < st.t;
    const float e = __expf(c1 * fabsf(tv - st.t));   // the first value: exp(-inf) = 0, s = 0 * 0 + 1
    st.s = lower ? fmaf(st.s, e, 1.f) : st.s + e;
    st.d = lower ? j : st.d;
    st.t = fminf(st.t, tv);
}

__device__ __forceinline__ bool warp_all(bool ok) { return __all_sync(0xffffffffu, ok) != 0; }

// OR of `flag` over the 256 epilogue threads (named barrier 1; every epilogue thread must arrive).
__device__ __forceinline__ bool epilogue_any(bool flag) {
    uint32_t r;
    asm volatile(
        "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.or.pred q, 1, %2, p;\n selp.u32 %0, 1, 0, q;\n}"
        : "=r"(r)
        : "r"((uint32_t)flag), "r"(EPI_THREADS)
        : "memory");
    return r != 0;
}

__device__ __forceinline__ void epilogue_sync() { asm volatile("bar.sync 1, %0;" ::"r"(EPI_THREADS) : "memory"); }

__global__ void __launch_bounds__(GEMM_THREADS, 1) k_score_gemm(const GemmArgs g) {
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t bar_full[NSTAGE], bar_empty[NSTAGE], bar_tfull[2], bar_tempty[2], bar_drain;
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_flag;
    __shared__ Part straddle[2][GM];   // the image cut by the column halves: each half's part, per row
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n_tiles = g.n_ptiles * g.n_itiles;
    const int n_groups = (g.n_chunks + GROUP - 1) / GROUP;

    if (threadIdx.x == 0) {
        for (int s = 0; s < NSTAGE; ++s) {
            mbar_init(smem_u32(&bar_full[s]), 1);
            mbar_init(smem_u32(&bar_empty[s]), 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(smem_u32(&bar_tfull[b]), 1);
            mbar_init(smem_u32(&bar_tempty[b]), EPI_THREADS);
        }
        mbar_init(smem_u32(&bar_drain), 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;
    volatile int* abort_v = &abort_flag;
    const uint32_t sbase = smem_u32(smem);

    if (warp == 0 && lane == 0) {
        // ---------------- producer: operand chunks into the stage ring
        uint32_t it = 0;
        for (int t = blockIdx.x; t < n_tiles; t += gridDim.x) {
            const int ptile = g.ptile0 + t / g.n_itiles, itile = t % g.n_itiles;
            const unsigned char* ga = g.a_ops + (size_t)ptile * g.n_chunks * (2 * A_TERM);
            const unsigned char* gb = g.b_ops + (size_t)itile * g.n_chunks * (2 * B_TERM);
            bool ok = true;
            for (int ch = 0; ch < g.n_chunks; ++ch, ++it) {
                const uint32_t s = it % NSTAGE, round = it / NSTAGE;
                if (round > 0 && !mbar_wait(smem_u32(&bar_empty[s]), (round - 1) & 1, abort_v, g.status, g.wait_ns)) {
                    ok = false;
                    break;
                }
                if ((long long)it == g.skip_chunk) continue;   // test: this stage's barrier never completes
                const uint32_t full = smem_u32(&bar_full[s]);
                mbar_expect_tx(full, STAGE);
                bulk_g2s(sbase + s * STAGE, ga + (size_t)ch * (2 * A_TERM), 2 * A_TERM, full);
                bulk_g2s(sbase + s * STAGE + 2 * A_TERM, gb + (size_t)ch * (2 * B_TERM), 2 * B_TERM, full);
            }
            if (!ok) break;
        }
        // copies still landing must not outlive the block: wait for the last phases issued
        for (uint32_t k = 1; k <= NSTAGE && k <= it; ++k) {
            const uint32_t i = it - k;
            if ((long long)i == g.skip_chunk) continue;
            mbar_drain(smem_u32(&bar_full[i % NSTAGE]), (i / NSTAGE) & 1, g.wait_ns);
        }
    } else if (warp == 1 && lane == 0) {
        // ---------------- MMA issue: each group of GROUP chunks into a fresh accumulator buffer
        const uint32_t lbo = 128, sbo = RG_BYTES;
        uint32_t it = 0, gi = 0;
        bool ok = true;
        for (int t = blockIdx.x; t < n_tiles && ok; t += gridDim.x) {
            for (int gr = 0; gr < n_groups && ok; ++gr, ++gi) {
                const uint32_t b = gi & 1, use = gi >> 1;
                if (use > 0 && !mbar_wait(smem_u32(&bar_tempty[b]), (use - 1) & 1, abort_v, g.status, g.wait_ns)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t d = tmem + b * GN;
                const int ch1 = min(g.n_chunks, (gr + 1) * GROUP);
                for (int ch = gr * GROUP; ch < ch1; ++ch, ++it) {
                    const uint32_t s = it % NSTAGE, round = it / NSTAGE;
                    if (!mbar_wait(smem_u32(&bar_full[s]), round & 1, abort_v, g.status, g.wait_ns)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t st = sbase + s * STAGE;
                    const bool first = ch == gr * GROUP;
#pragma unroll
                    for (int j = 0; j < KC / KSTEP; ++j) {
                        const uint64_t a_hi = sdesc(st + j * 256, lbo, sbo);
                        const uint64_t a_lo = sdesc(st + A_TERM + j * 256, lbo, sbo);
                        const uint64_t b_hi = sdesc(st + 2 * A_TERM + j * 256, lbo, sbo);
                        const uint64_t b_lo = sdesc(st + 2 * A_TERM + B_TERM + j * 256, lbo, sbo);
                        umma(d, a_hi, b_hi, g.idesc, (first && j == 0) ? 0u : 1u);
                        umma(d, a_hi, b_lo, g.idesc, 1u);
                        umma(d, a_lo, b_hi, g.idesc, 1u);
                    }
                    umma_commit(smem_u32(&bar_empty[s]));   // frees the stage once these MMAs have read it
                }
                if (ok) umma_commit(smem_u32(&bar_tfull[b]));
            }
        }
        // every MMA issued has completed before the block releases tensor memory
        umma_commit(smem_u32(&bar_drain));
        mbar_drain(smem_u32(&bar_drain), 0, g.wait_ns);
    } else if (warp >= 2) {
        // ---------------- epilogue: two threads per parameset (tensor-memory lane), 128 columns each
        const int e = warp - 2;
        const int q = warp & 3;             // lane quarter this warp may access
        const int h = e >> 2;               // column half
        const int row = 32 * q + lane;
        const uint32_t trow = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(128 * h);
        const int ns2 = (2 * g.smax + 1) * (2 * g.smax + 1);
        const int wl = g.ps_hi - g.ps_lo;
        const int col0 = 128 * h;
        // the image holding column 127 continues past it: its two parts meet in shared memory
        const int ib_cut = 127 / ns2;
        const bool cut = ib_cut < g.ipt && (ib_cut + 1) * ns2 > 128;
        uint32_t gi = 0;
        for (int t = blockIdx.x; t < n_tiles; t += gridDim.x) {
            float acc[128];
#pragma unroll
            for (int c = 0; c < 128; ++c) acc[c] = 0.f;
            bool fail = false;
            for (int gr = 0; gr < n_groups; ++gr, ++gi) {
                const uint32_t b = gi & 1, use = gi >> 1;
                if (!fail) fail = !warp_all(mbar_wait(smem_u32(&bar_tfull[b]), use & 1, abort_v, g.status, g.wait_ns));
                if (fail) continue;
                tc_fence_after();
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    float v[32];
                    tmem_ld32(trow + b * GN + 32 * i, v);
#pragma unroll
                    for (int k = 0; k < 32; ++k) acc[32 * i + k] += v[k];   // FP32, round to nearest
                }
                tc_fence_before();
                mbar_arrive(smem_u32(&bar_tempty[b]));
            }
            const int ptile = g.ptile0 + t / g.n_itiles, itile = t % g.n_itiles;
            const int p = ptile * GM + row;
            const bool p_ok = p >= g.ps_lo && p < g.ps_hi;
            const float inv_p = p_ok ? __ldg(g.inv_ps + p) : 0.f;
            // walk this thread's 128 columns image by image
            int ib = col0 / ns2;
            int j = col0 - ib * ns2;
            bool starts_here = j == 0;
            int w = itile * g.ipt + ib;
            float inv = (ib < g.ipt && w < g.n_img) ? inv_p * __ldg(g.inv_img + w) : 0.f;
            Part st{INFINITY, 0.f, 0x7fffffff};
            float r2max = 0.f;
            // 8 blocks of 16 columns in a rolled loop (the likelihood body exists once in the code:
            // unrolled over all 128 columns it crowded the instruction cache the MMA thread runs from)
#pragma unroll 1
            for (int blk = 0; blk < 8; ++blk) {
                float v[16];
#pragma unroll
                for (int k = 0; k < 16; ++k) v[k] = acc[k];
#pragma unroll
                for (int bb = 1; bb < 8; ++bb) {
                    if (blk == bb) {
#pragma unroll
                        for (int k = 0; k < 16; ++k) v[k] = acc[16 * bb + k];
                    }
                }
#pragma unroll
                for (int k = 0; k < 16; ++k) {
                if (j == ns2) {   // image ib complete
                    if (!fail && starts_here && ib < g.ipt && w < g.n_img && p_ok) {
                        const size_t o = (size_t)w * wl + (p - g.ps_lo);
                        g.rec_t[o] = st.t;
                        g.rec_s[o] = st.s;
                        g.rec_d[o] = st.d;
                    } else if (!starts_here) {
                        straddle[1][row] = st;   // second part of the cut image
                    }
                    ++ib;
                    ++w;
                    j = 0;
                    starts_here = true;
                    inv = (ib < g.ipt && w < g.n_img) ? inv_p * __ldg(g.inv_img + w) : 0.f;
                    st = Part{INFINITY, 0.f, 0x7fffffff};
                }
                if (ib < g.ipt) part_add(st, r2max, v[k], inv, j, g.c1);
                ++j;
                }
            }
            if (r2max >= 1.0f) atomicOr(g.status, BIOEM_DEV_NUMERIC);   // inv = 0 off the valid sets / images
            if (ib < g.ipt) {
                if (h == 0 && cut) {
                    straddle[0][row] = st;   // first part of the cut image
                } else if (h == 1 && !starts_here) {
                    straddle[1][row] = st;   // the cut image ends exactly at column 255
                } else if (!fail && w < g.n_img && p_ok && j == ns2) {
                    const size_t o = (size_t)w * wl + (p - g.ps_lo);
                    g.rec_t[o] = st.t;
                    g.rec_s[o] = st.s;
                    g.rec_d[o] = st.d;
                }
            }
            if (epilogue_any(fail)) break;   // uniform over the epilogue threads
            if (cut && h == 0) {
                const int wc = itile * g.ipt + ib_cut;
                if (wc < g.n_img && p_ok) {
                    const Part m = part_merge(straddle[0][row], straddle[1][row], g.c1);
                    const size_t o = (size_t)wc * wl + (p - g.ps_lo);
                    g.rec_t[o] = m.t;
                    g.rec_s[o] = m.s;
                    g.rec_d[o] = m.d;
                }
            }
            epilogue_sync();   // the parts are read before the next tile writes them
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
}

bool mode_fp16(int mode) { return mode == BIOEM_PRECISION_FP16X2 || mode == BIOEM_PRECISION_FP16X2_REAL; }
bool mode_real(int mode) { return mode == BIOEM_PRECISION_BF16X2_REAL || mode == BIOEM_PRECISION_FP16X2_REAL; }

// K / KC: Fourier form K = 2 N (N/2 + 1) (real and imaginary parts of the half spectrum); real-space
// form K = N^2 pixels.
int n_chunks_for(int npix, int mode) {
    return mode_real(mode) ? npix * npix / KC : npix * (npix / 2 + 1) * 2 / KC;
}

void release_cache(bioem_gemm_cache& c, cudaStream_t stream) {
    if (c.d_ops) cudaFreeAsync(c.d_ops, stream);
    if (c.d_inv) cudaFreeAsync(c.d_inv, stream);
    c = bioem_gemm_cache{};
}

int alloc_cache(bioem_ctx* ctx, bioem_gemm_cache& c, size_t ops_bytes, size_t n_inv, const char* what) {
    release_cache(c, ctx->stream);
    if (cudaMallocAsync(&c.d_ops, ops_bytes, ctx->stream) != cudaSuccess ||
        cudaMallocAsync((void**)&c.d_inv, sizeof(float) * (n_inv ? n_inv : 1), ctx->stream) != cudaSuccess) {
        cudaGetLastError();
        release_cache(c, ctx->stream);
        return bioem_set_error(ctx, BIOEM_ERR_OOM, "%s: %zu bytes", what, ops_bytes);
    }
    c.bytes = ops_bytes;
    return BIOEM_OK;
}

int grid_for(bioem_ctx* ctx, size_t warps_of_work) {
    const size_t blocks = (warps_of_work + 7) / 8;
    const size_t cap = (size_t)ctx->num_sms * 8;
    return (int)(blocks < cap ? (blocks > 0 ? blocks : 1) : cap);
}

}  // namespace

void bioem_gemm_cache_free(bioem_gemm_cache* c, cudaStream_t stream) { release_cache(*c, stream); }

int bioem_gemm_supported(int npix, int max_shift) {
    if (max_shift < 0 || 2 * max_shift >= npix) return 0;
    if ((2 * max_shift + 1) * (2 * max_shift + 1) > GN) return 0;
    return bioem_size_index(npix) >= 0 && (npix * (npix / 2 + 1) * 2) % KC == 0 && (npix * npix) % KC == 0;
}

int bioem_gemm_row_tile() { return GM; }

// Real-space zero-mean unit-norm arrays [count][N][N] and their max |x| for `count` spectra, in
// one stream-ordered temporary (freed by the caller with cudaFreeAsync).
static int real_space(bioem_ctx* ctx, const float2* spec, int count, int npix, float** out, float** amax) {
    const size_t n = (size_t)count * npix * npix;
    void* p = nullptr;
    if (cudaMallocAsync(&p, sizeof(float) * (n + (size_t)count + 64), ctx->stream) != cudaSuccess) {
        cudaGetLastError();
        return bioem_set_error(ctx, BIOEM_ERR_OOM, "real-space operand scratch (%zu floats)", n);
    }
    *out = (float*)p;
    *amax = (float*)p + n;
    const int rc = bioem_launch_spec_to_real(ctx, spec, count, npix, *out, *amax);
    if (rc) cudaFreeAsync(p, ctx->stream);
    return rc;
}

int bioem_gemm_prepare(bioem_ctx* ctx, const bioem_images* im, const bioem_projset* ps, int max_shift, int mode) {
    const int npix = im->nx, nh = npix / 2 + 1;
    const int n_chunks = n_chunks_for(npix, mode);
    const int fp16 = mode_fp16(mode) ? 1 : 0;
    const bool real = mode_real(mode);
    if (ps->gemm.mode != mode || !ps->gemm.d_ops) {
        const size_t n_ptiles = ((size_t)ps->n_ps + GM - 1) / GM;
        const size_t bytes = n_ptiles * n_chunks * (size_t)(2 * A_TERM);
        int rc = alloc_cache(ctx, ps->gemm, bytes, n_ptiles * GM, "parameter-set operand");
        if (rc) return rc;
        if (cudaMemsetAsync(ps->gemm.d_inv, 0, sizeof(float) * n_ptiles * GM, ctx->stream) != cudaSuccess)
            return bioem_check_cuda(ctx, cudaGetLastError(), "operand scales");
        // the A operand reads pairs of values: spectrum coefficients (Fourier form) or pairs of
        // adjacent pixels of the real-space projection (real-space form)
        const float2* src = ps->d_spec;
        const float* amax = ps->d_amax;
        float* tmp = nullptr;
        if (real) {
            float* ra = nullptr;
            rc = real_space(ctx, ps->d_spec, ps->n_ps, npix, &tmp, &ra);
            if (rc) return rc;
            src = reinterpret_cast<const float2*>(tmp);
            amax = ra;
        }
        const int ncoef = real ? npix * npix / 2 : npix * nh;
        const size_t total_cm = n_ptiles * n_chunks * (GM / 8) * (KC / 8);
        bioem_launch_begin(ctx, KID_GEMM_OPS);
        k_gemm_ops_ps<<<grid_for(ctx, total_cm), 256, 0, ctx->stream>>>(src, amax, ps->n_ps, ncoef, n_chunks, fp16,
                                                                       (unsigned char*)ps->gemm.d_ops, total_cm);
        bioem_launch_end(ctx, KID_GEMM_OPS);
        bioem_launch_begin(ctx, KID_GEMM_OPS);
        k_gemm_inv_scales<<<(ps->n_ps + 255) / 256, 256, 0, ctx->stream>>>(amax, ps->n_ps, 1.f, fp16, ps->gemm.d_inv);
        bioem_launch_end(ctx, KID_GEMM_OPS);
        if (tmp) cudaFreeAsync(tmp, ctx->stream);
        rc = bioem_check_cuda(ctx, cudaGetLastError(), "k_gemm_ops_ps");
        if (rc) return rc;
        ps->gemm.mode = mode;
        ps->gemm.shift = -1;
    }
    if (im->gemm.mode != mode || im->gemm.shift != max_shift || !im->gemm.d_ops) {
        const int ns2 = (2 * max_shift + 1) * (2 * max_shift + 1);
        const int ipt = GN / ns2;
        const size_t n_itiles = ((size_t)im->n_img + ipt - 1) / ipt;
        const size_t bytes = n_itiles * n_chunks * (size_t)(2 * B_TERM);
        int rc = alloc_cache(ctx, im->gemm, bytes, (size_t)im->n_img, "image operand");
        if (rc) return rc;
        const size_t total_cm = n_itiles * n_chunks * (GN / 8) * (KC / 8);
        if (real) {
            float *tmp = nullptr, *ra = nullptr;
            rc = real_space(ctx, im->d_spec, im->n_img, npix, &tmp, &ra);
            if (rc) return rc;
            bioem_launch_begin(ctx, KID_GEMM_OPS);
            k_gemm_ops_img_real<<<grid_for(ctx, total_cm), 256, 0, ctx->stream>>>(
                tmp, ra, im->n_img, npix, n_chunks, max_shift, ipt, fp16, (unsigned char*)im->gemm.d_ops, total_cm);
            bioem_launch_end(ctx, KID_GEMM_OPS);
            bioem_launch_begin(ctx, KID_GEMM_OPS);
            k_gemm_inv_scales<<<(im->n_img + 255) / 256, 256, 0, ctx->stream>>>(ra, im->n_img, 1.f, fp16,
                                                                                im->gemm.d_inv);
            bioem_launch_end(ctx, KID_GEMM_OPS);
            cudaFreeAsync(tmp, ctx->stream);
        } else {
            bioem_launch_begin(ctx, KID_GEMM_OPS);
            k_gemm_ops_img<<<grid_for(ctx, total_cm), 256, 0, ctx->stream>>>(
                im->d_spec, im->d_amax, im->n_img, npix, nh, n_chunks, max_shift, ipt, fp16,
                bioem_twiddles(ctx, npix), (unsigned char*)im->gemm.d_ops, total_cm);
            bioem_launch_end(ctx, KID_GEMM_OPS);
            bioem_launch_begin(ctx, KID_GEMM_OPS);
            k_gemm_inv_scales<<<(im->n_img + 255) / 256, 256, 0, ctx->stream>>>(im->d_amax, im->n_img, 2.8285f, fp16,
                                                                                im->gemm.d_inv);
            bioem_launch_end(ctx, KID_GEMM_OPS);
        }
        rc = bioem_check_cuda(ctx, cudaGetLastError(), "k_gemm_ops_img");
        if (rc) return rc;
        im->gemm.mode = mode;
        im->gemm.shift = max_shift;
    }
    return BIOEM_OK;
}

int bioem_gemm_records(bioem_ctx* ctx, const bioem_images* im, const bioem_projset* ps, int max_shift, int mode,
                       int ps_lo, int ps_hi, float* rec_t, float* rec_s, int* rec_d) {
    static_assert(GEMM_SMEM <= 227 * 1024, "shared memory per block");
    if (ps_hi <= ps_lo || im->n_img == 0) return BIOEM_OK;
    const int npix = im->nx;
    const int ns2 = (2 * max_shift + 1) * (2 * max_shift + 1);
    GemmArgs g{};
    g.a_ops = (const unsigned char*)ps->gemm.d_ops;
    g.b_ops = (const unsigned char*)im->gemm.d_ops;
    g.inv_ps = ps->gemm.d_inv;
    g.inv_img = im->gemm.d_inv;
    g.n_chunks = n_chunks_for(npix, mode);
    g.ptile0 = ps_lo / GM;
    g.n_ptiles = (ps_hi + GM - 1) / GM - g.ptile0;
    g.ipt = GN / ns2;
    g.n_itiles = (im->n_img + g.ipt - 1) / g.ipt;
    g.smax = max_shift;
    g.n_img = im->n_img;
    g.ps_lo = ps_lo;
    g.ps_hi = ps_hi;
    const int n = npix * npix;
    g.c1 = 0.5f * (3.0f - (float)n);
    const uint32_t fmt = mode_fp16(mode) ? 0u : 1u;   // 0 FP16, 1 BF16
    g.idesc = (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(GN >> 3) << 17) | ((uint32_t)(GM >> 4) << 24);
    g.rec_t = rec_t;
    g.rec_s = rec_s;
    g.rec_d = rec_d;
    g.status = ctx->d_status;
    g.skip_chunk = ctx->test_skip_chunk;
    g.wait_ns = ctx->test_wait_ns ? ctx->test_wait_ns : kWaitNs;
    ctx->test_skip_chunk = -1;   // armed for one launch
    ctx->test_wait_ns = 0;
    const long long n_tiles = (long long)g.n_ptiles * g.n_itiles;
    if (n_tiles > 0x7fffffffll) return bioem_set_error(ctx, BIOEM_ERR_UNSUPPORTED_SIZE, "too many GEMM tiles");
    if (cudaFuncSetAttribute(k_score_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)GEMM_SMEM) != cudaSuccess)
        return bioem_check_cuda(ctx, cudaGetLastError(), "GEMM shared memory attribute");
    const int grid = (int)(n_tiles < ctx->num_sms ? n_tiles : ctx->num_sms);
    bioem_launch_begin(ctx, KID_SCORE_GEMM);
    k_score_gemm<<<grid, GEMM_THREADS, GEMM_SMEM, ctx->stream>>>(g);
    bioem_launch_end(ctx, KID_SCORE_GEMM);
    return bioem_check_cuda(ctx, cudaGetLastError(), "k_score_gemm");
}
