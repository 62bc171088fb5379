// Fused scoring kernel: per (image, parameter set) pair, the Fourier-space product, the inverse
// transform evaluated on the displacement window only, and the closed-form likelihood with a
// log-sum-exp over displacements (Sec. 3.3, Eqs. 11-12; Sec. 3.9 and Sec. 5 note that the product,
// the inverse FFT and the likelihood were three kernels with the correlation map stored between
// them, and that only some output coefficients are needed: here they are one kernel and the map
// never leaves the SM).
//
// Spectra (both unit-norm, DC = 0, half spectrum kx = 0..N/2):
//   rho(d) = X(d) / sqrt(A B) = Re sum_{ky} sum_{kx<=N/2} w_kx conj(O(k)) C(k) exp(+2 pi i k.d / N)
// with w = 1 on the kx = 0 and kx = N/2 columns, 2 elsewhere.  Evaluated in two stages:
//   stage A (per column kx, along ky):  Q(dy, kx) = sum_ky conj(O) C exp(+2 pi i ky dy / N)
//   stage B (per row dy, along kx):     rho(dy, dx) = Re sum_kx w_kx Q(dy, kx) exp(+2 pi i kx dx / N)
// each as a pruned transform: the N (or N/2) inputs split into R interleaved sub-sequences of
// length L = 16, each transformed by an in-register radix-2 FFT, then recombined with twiddles for
// the 2 SMAX + 1 wanted outputs only.
//
// Likelihood (closed form of Eq. 8 integrated over N, mu, lambda):
//   ln L(d) = kA + kB + (3 - n)/2 ln(1 - rho(d)^2),  kA = (3-n)/2 ln A + c(n),  kB = -1/2 ln B.
// Per pair the kernel records t_min = min_d ln(1 - rho^2), s = sum_d exp((3-n)/2 (t(d) - t_min))
// and the argmin d; a float64 reduction (k_reduce_wave) turns the records into per-image and
// per-orientation log-sum-exps and maximising parameters.
#include <math.h>
#include <stdio.h>

#include <mutex>
#include <type_traits>

#include "bioem_internal.cuh"
#include "rdft16.cuh"

namespace {

constexpr int L = 16;   // sub-transform length
// Dynamic shared memory a scoring block may take: 227 KiB per block, less 1 KiB for the kernels'
// static shared variables.
constexpr size_t kScoreSmemLimit = 227u * 1024u - 1024u;

// W_M^t = exp(+2 pi i t / M), uploaded once per device.
__constant__ float2 c_w16[16];
__constant__ float2 c_w32[32];
__constant__ float2 c_w64[64];
__constant__ float2 c_w128[128];
__constant__ float2 c_w96[96];
__constant__ float2 c_w192[192];

template <int M>
__device__ __forceinline__ float2 cw(int t) {
    if constexpr (M == 16) return c_w16[t];
    else if constexpr (M == 32) return c_w32[t];
    else if constexpr (M == 64) return c_w64[t];
    else if constexpr (M == 96) return c_w96[t];
    else if constexpr (M == 192) return c_w192[t];
    else return c_w128[t];
}

template <int M>
__device__ __forceinline__ const float2* cw_table() {
    if constexpr (M == 16) return c_w16;
    else if constexpr (M == 32) return c_w32;
    else if constexpr (M == 64) return c_w64;
    else if constexpr (M == 96) return c_w96;
    else if constexpr (M == 192) return c_w192;
    else return c_w128;
}

// d * W_LL^t for a compile-time exponent t < LL / 2.
template <int LL, int T>
__device__ __forceinline__ float2 twiddle_mul(float2 d) {
    if constexpr (T == 0) {
        return d;
    } else if constexpr (4 * T == LL) {          // W^(LL/4) = i
        return make_float2(-d.y, d.x);
    } else if constexpr (8 * T == LL) {          // (1 + i) / sqrt 2
        const float r = 0.70710678118654752f;
        return make_float2((d.x - d.y) * r, (d.x + d.y) * r);
    } else if constexpr (8 * T == 3 * LL) {      // (-1 + i) / sqrt 2
        const float r = 0.70710678118654752f;
        return make_float2(-(d.x + d.y) * r, (d.x - d.y) * r);
    } else {
        return c_mul(d, cw<LL>(T));
    }
}

template <int LL, int HALF, int BLK, int J>
__device__ __forceinline__ void dif_butterflies(float2 (&x)[LL]) {
    if constexpr (BLK < LL) {
        if constexpr (J < HALF) {
            const float2 a = x[BLK + J], b = x[BLK + J + HALF];
            x[BLK + J] = __fadd2_rn(a, b);
            x[BLK + J + HALF] = twiddle_mul<LL, J * (LL / (2 * HALF))>(__ffma2_rn(b, make_float2(-1.f, -1.f), a));
            dif_butterflies<LL, HALF, BLK, J + 1>(x);
        } else {
            dif_butterflies<LL, HALF, BLK + 2 * HALF, 0>(x);
        }
    }
}

template <int LL, int HALF>
__device__ __forceinline__ void dif_stages(float2 (&x)[LL]) {
    if constexpr (HALF >= 1) {
        dif_butterflies<LL, HALF, 0, 0>(x);
        dif_stages<LL, HALF / 2>(x);
    }
}

// In-register DFT y[u] = sum_a x[a] W_LL^(a u), radix-2 decimation in frequency; on return
// y[u] is stored at x[bitrev(u)].
template <int LL>
__device__ __forceinline__ void fft_dif(float2 (&x)[LL]) {
    dif_stages<LL, LL / 2>(x);
}

template <int LL, int J>
__device__ __forceinline__ void first_stage_half_zero(float2 (&x)[LL]) {
    if constexpr (J < LL / 2) {
        x[J + LL / 2] = twiddle_mul<LL, J>(x[J]);
        first_stage_half_zero<LL, J + 1>(x);
    }
}

// fft_dif for inputs whose upper half x[LL/2 ..] is zero: the first stage's butterflies reduce to
// copies (a + 0 = a, a - 0 = a).
template <int LL>
__device__ __forceinline__ void fft_dif_half_zero(float2 (&x)[LL]) {
    first_stage_half_zero<LL, 0>(x);
    dif_stages<LL, LL / 4>(x);
}

__host__ __device__ constexpr int bitrev(int u, int bits) {
    int r = 0;
    for (int i = 0; i < bits; ++i) r |= ((u >> i) & 1) << (bits - 1 - i);
    return r;
}
__host__ __device__ constexpr int ilog2(int v) { return v <= 1 ? 0 : 1 + ilog2(v / 2); }
__host__ __device__ constexpr int pmod(int a, int m) { return ((a % m) + m) % m; }

template <int N_, int SMAX_, int PB_, int THREADS_, bool ALLOW_PACK_ = true, int BSPLIT_ = 1>
struct Cfg {
    static constexpr int N = N_;
    static constexpr int SMAX = SMAX_;
    static constexpr int PB = PB_;             // pairs per batch
    static constexpr int NC = N / 2;
    static constexpr int H = NC + 1;           // half-spectrum row length (kx = 0..N/2)
    static constexpr int NS = 2 * SMAX + 1;    // displacements per axis
    static constexpr int NROW = 2 * SMAX;      // stage-B transform rows per pair (dy < SMAX)
    static constexpr int R = N / L;            // sub-sequences per transform
    static constexpr int THREADS = THREADS_;   // threads doing the work (a block may have more)
    static constexpr int NWARPS = THREADS / 32;  // full warps (combine step)
    // stage-B threads per row: 2 when the block has two threads for every row (each sums half
    // of the sub-sequences, the halves are exchanged by a lane shuffle, and each evaluates the
    // likelihood for half of the dx outputs)
    static constexpr int BSPLIT = BSPLIT_;
    static_assert((BSPLIT == 1 || BSPLIT == 2) && THREADS >= PB * 2 * SMAX_ * BSPLIT, "stage-B threads");
    static constexpr bool PREFETCH = THREADS <= 320;   // stage-A projection prefetch (registers)
    static_assert(THREADS >= PB * NROW, "one stage-B row per thread");
    static_assert(NWARPS >= 1, "at least one full warp");
    static_assert(N % L == 0, "sub-transform length divides N");
    static constexpr int QS = H;               // Q row stride (complex); odd -> conflict-free columns
    static constexpr int NDIR = PB * NS;       // outputs of the dy = +SMAX row, evaluated directly
    static constexpr size_t SM_IMG = (size_t)N * H * sizeof(float2);
    static constexpr size_t SM_Q = (size_t)PB * NS * QS * sizeof(float2);
    static constexpr size_t SM_QA = (SM_Q + 15) / 16 * 16;   // the twiddle table starts 16-byte aligned
    // twiddle table twc[b][d] = W_N^(b d), d = 0..SMAX (the outputs -d use the conjugate), rows of
    // an even length TWS so that pairs (d, d + 1), d even, are read as one 16-byte load
    static constexpr int TWS = 2 * ((SMAX + 2) / 2);
    // the 128 px, +-16 px instance keeps a second table 2 W_N^(b d) for stage B (the weight 2 of
    // kx != 0 rides on the twiddles, exact, instead of scaling every input)
    static constexpr bool TW2 = N == 128 && SMAX == 16 && THREADS == 512;
    static constexpr size_t SM_TWC = (size_t)(TW2 ? 2 : 1) * R * TWS * sizeof(float2);
    static_assert((SM_IMG + SM_QA) % 16 == 0 && (TWS * sizeof(float2)) % 16 == 0, "16-byte twiddle pairs");
    static constexpr size_t SM_ROW = (size_t)PB * NROW * BSPLIT * (2 * sizeof(float) + sizeof(int));
    static constexpr size_t SM_DIR = (size_t)NDIR * sizeof(float);
    static constexpr size_t SM_BASE = SM_IMG + SM_QA + SM_TWC + SM_ROW + SM_DIR;
    // Packed edge columns: for real images and projections the product conj(O) C is Hermitian in
    // ky on the kx = 0 and kx = N/2 columns, so both columns' stage-A outputs are real, and one
    // complex transform of Z(ky) = P(ky, 0) + i P(ky, N/2) gives Q(dy, 0) as its real part and
    // Q(dy, N/2) as its imaginary part.  That leaves N/2 column tasks per pair (a multiple of the
    // block's warps); Z is formed for the batch in shared memory before stage A.  Used where Z fits.
    static constexpr size_t SM_Z_PACKED = (size_t)PB * N * sizeof(float2);
    static constexpr bool PACK = ALLOW_PACK_ && SM_BASE + SM_Z_PACKED <= kScoreSmemLimit;
    static constexpr int NCOL = PACK ? NC : H;      // stage-A column tasks per pair
    static constexpr int TASKS_A = PB * NCOL;       // stage-A column tasks per batch
    static constexpr size_t SM_Z = PACK ? SM_Z_PACKED : 0;
    // The dy = +SMAX row by real transforms (the 128 px, +-16 px instance): jobs (pair, Re / Im,
    // kx sub-sequence) on the last PB 2 R threads, each a real 16-point transform recombined into the
    // SMAX + 1 even (cosine) or odd (sine) outputs, summed over sub-sequences by lane shuffles; a
    // direct sum costs ~60 multiply-adds per output instead.
    static constexpr bool DIRFFT = PACK && N == 128 && SMAX == 16 && THREADS == 512 && PB == 8;
    static constexpr size_t SM_DTW = DIRFFT ? (size_t)2 * R * (SMAX + 1) * sizeof(float2) : 0;
    static constexpr size_t SM_DSUM = DIRFFT ? (size_t)PB * 2 * (SMAX + 1) * sizeof(float) : 0;
    static constexpr size_t SMEM = SM_BASE + SM_Z + SM_DTW + SM_DSUM;
    static_assert(SMEM <= kScoreSmemLimit, "dynamic shared memory per block");
    // Decoupled groups (the 128 px, +-16 px instance): the block's threads form NGROUP groups of
    // GT threads, group g owning pairs [g GPB, (g + 1) GPB) of every batch in every phase (packed
    // edge columns, stage A, stage B, the dy = +SMAX row, the combine), and within the batch loop
    // each group waits only on its own named barrier.  The groups drift apart, so that one group's
    // projection loads and barrier waits overlap the others' transform arithmetic instead of the
    // whole block moving through its phases in step (the FP32 pipe saturated in the transforms and
    // idle in between).  Measured per pair: 14.25 ns in step, 13.43 ns with two groups, 12.59 ns
    // with four, 13.17 ns with eight (one pair per group, the dy = +SMAX jobs on half a warp).
    static constexpr bool SPLIT = DIRFFT;
    static constexpr int NGROUP = SPLIT ? 4 : 1;
    static constexpr int GT = THREADS / NGROUP, GPB = PB / NGROUP;   // threads and pairs of one group
    static_assert(!SPLIT || (GT % 32 == 0 && GPB * NCOL == GT && GPB * NROW * BSPLIT == GT &&
                             ((GPB * 2 * R) % 32 == 0 || GPB * 2 * R == 16)),
                  "each group's tasks on its own threads, its dy = +SMAX jobs on whole warps or half a warp");
};

// The batch loop's barrier: the whole block, or with C::SPLIT the calling thread's group (named
// barrier 1 + group over C::GT threads).
template <class C>
__device__ __forceinline__ void batch_sync() {
    if constexpr (C::SPLIT) {
        asm volatile("bar.sync %0, %1;" ::"r"(1 + (int)threadIdx.x / C::GT), "n"(C::GT) : "memory");
    } else {
        __syncthreads();
    }
}

// Stage A for one column kx of one pair: Q(dy, kx) for dy = -SMAX..SMAX, with the rows ky = b + R a
// of sub-sequence b transformed by an in-register FFT and recombined with the twiddles
// twc[b][d] = W_N^(b d), d = 0..SMAX, and their conjugates (shared memory, the same address for every
// thread: broadcast).
// The projection column is read from global memory one sub-sequence ahead of its use.  With zcol
// set (the packed edge columns) the inputs are zcol[ky] instead of the product.
template <class C>
__device__ __forceinline__ void stage_a_column(float2 (&acc)[C::NS], const float2* __restrict__ img_col,
                                               const float2* __restrict__ ps_col, const float2* __restrict__ twc,
                                               const float2* __restrict__ zcol) {
    constexpr int H = C::H, R = C::R, NS = C::NS, SMAX = C::SMAX;
    float2 cn[L];
    if constexpr (C::PREFETCH) {
        if (!zcol) {
#pragma unroll
            for (int a = 0; a < L; ++a) cn[a] = __ldg(ps_col + (R * a) * H);
        }
    }
#pragma unroll 1
    for (int b = 0; b < R; ++b) {
        float2 x[L];
        if (zcol) {
#pragma unroll
            for (int a = 0; a < L; ++a) x[a] = zcol[R * a + b];
        } else if constexpr (C::PREFETCH) {
#pragma unroll
            for (int a = 0; a < L; ++a) x[a] = c_mulc(img_col[(R * a) * H], cn[a]);
            if (b + 1 < R) {
#pragma unroll
                for (int a = 0; a < L; ++a) cn[a] = __ldg(ps_col + (R * a + 1) * H);
            }
        } else {
#pragma unroll
            for (int a = 0; a < L; ++a) x[a] = c_mulc(img_col[(R * a) * H], __ldg(ps_col + (R * a) * H));
        }
        img_col += H;
        ps_col += H;
        fft_dif<L>(x);
        // W^(b d) and W^(-b d) are complex conjugates: one twiddle serves dy = +d and -d
        const float2* tw = twc + b * C::TWS;
#pragma unroll
        for (int d = 0; d <= SMAX; ++d) {
            const float2 w = tw[d];
            {
                const int mi = SMAX + d;
                const int u = bitrev(pmod(mi - SMAX, L), ilog2(L));
                acc[mi].x = fmaf(w.x, x[u].x, fmaf(-w.y, x[u].y, acc[mi].x));
                acc[mi].y = fmaf(w.x, x[u].y, fmaf(w.y, x[u].x, acc[mi].y));
            }
            if (d > 0) {
                const int mi = SMAX - d;
                const int u = bitrev(pmod(mi - SMAX, L), ilog2(L));
                acc[mi].x = fmaf(w.x, x[u].x, fmaf(w.y, x[u].y, acc[mi].x));
                acc[mi].y = fmaf(w.x, x[u].y, fmaf(-w.y, x[u].x, acc[mi].y));
            }
        }
    }
}

// Stage B for one row: rho-part(dx) = Re sum_{kx < N/2} w_kx Q(dy, kx) W_N^(kx dx), kx = b + R a;
// only a < L/2 carries data (kx < N/2 for every b < R).  With C::TW2, twc holds 2 W_N^(b d) (the
// weight w = 2 of kx != 0) and the kx = 0 term enters halved; scaling by 2 is exact, so the sums
// are those of the scaled inputs bit for bit.
template <class C>
__device__ __forceinline__ void stage_b_row(float (&acc)[C::NS], const float2* __restrict__ qrow,
                                            const float2* __restrict__ twc, int b0, int b1) {
    constexpr int R = C::R, NS = C::NS, SMAX = C::SMAX;
#pragma unroll 1
    for (int b = b0; b < b1; ++b) {
        float2 x[L];
#pragma unroll
        for (int a = 0; a < L / 2; ++a) x[a] = C::TW2 ? qrow[b + R * a] : c_scale(qrow[b + R * a], 2.f);
        if (b == 0) x[0] = make_float2((C::TW2 ? 0.5f : 1.f) * qrow[0].x, 0.f);   // kx = 0: weight 1, real
        fft_dif_half_zero<L>(x);
        const float2* tw = twc + b * C::TWS;   // conjugate pairs, as in stage A
#pragma unroll
        for (int d = 0; d <= SMAX; ++d) {
            const float2 w = tw[d];
            {
                const int mi = SMAX + d;
                const int u = bitrev(pmod(mi - SMAX, L), ilog2(L));
                acc[mi] = fmaf(w.x, x[u].x, fmaf(-w.y, x[u].y, acc[mi]));
            }
            if (d > 0) {
                const int mi = SMAX - d;
                const int u = bitrev(pmod(mi - SMAX, L), ilog2(L));
                acc[mi] = fmaf(w.x, x[u].x, fmaf(w.y, x[u].y, acc[mi]));
            }
        }
    }
}

// 2^x by the PTX instruction ex2.approx (relative error about 2^-22; results below 2^-126 flush to
// zero, far below the FP32 resolution of a sum that holds a term equal to 1).  The stage-B sum of
// exp((3 - n)/2 (t - t_min)) takes it with the factor (3 - n)/2 log2(e) folded into one constant:
// one instruction per displacement (6.5 % less k_score time than __expf at 128 px, +-16 px).
__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

struct Part {
    float t;   // min ln(1 - rho^2)
    float s;   // sum exp(c1 (t(d) - t))
    int d;     // index of the minimum, (dy + SMAX) * NS + (dx + SMAX)
};

__device__ __forceinline__ Part merge(Part a, Part b, float c1) {
    if (b.t > a.t || (b.t == a.t && b.d > a.d)) {
        const Part tmp = a;
        a = b;
        b = tmp;
    }
    // now b.t <= a.t (b holds the minimum, lowest index on ties)
    if (!(a.t < INFINITY)) return b;
    Part r;
    r.t = b.t;
    r.d = b.d;
    r.s = b.s + a.s * __expf(c1 * (a.t - b.t));
    return r;
}

// t = ln(1 - rho^2) as ln1m gives it, with |rho| >= 1 (no finite likelihood) flagged in the status
// word and clamped; both tests sit on the rarely taken rho^2 > 1/32 branch.
__device__ __forceinline__ float loglik_t(float rho, int* status) {
    float r2 = rho * rho;
    float t = ln1m_series(r2);
    if (r2 > 0.03125f) {
        if (r2 >= 1.0f) {
            atomicOr(status, BIOEM_DEV_NUMERIC);
            r2 = 1.0f - 5.9604645e-8f;
        }
        t = log1pf(-r2);
    }
    return t;
}

// Stage B (row transforms), the dy = +SMAX row, the likelihood epilogue and the per-pair combine of
// one batch whose Q (stage-A output, [pair][dy][kx]) is in q_s; records for pairs p0 .. hi-1.
template <class C>
__device__ __forceinline__ void score_tail(const float2* __restrict__ q_s, const float2* __restrict__ twc_s,
                                           float* row_t, float* row_s, int* row_d, float* dir_t,
                                           const float2* __restrict__ dtw, float* dsum,
                                           const float2* __restrict__ gtw, int p0, int hi, int s, float c1,
                                           float* __restrict__ rec_t, float* __restrict__ rec_s,
                                           int* __restrict__ rec_d, int* __restrict__ status) {
    constexpr int N = C::N, NC = C::NC, NS = C::NS, SMAX = C::SMAX, NROW = C::NROW;
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const bool active = tid < C::THREADS;
    // ---------------- stage B: one row (dy = -SMAX .. SMAX-1) of one pair per thread (per two
    // adjacent threads with BSPLIT = 2)
    if (tid < C::PB * NROW * C::BSPLIT) {
        constexpr int BS = C::BSPLIT;
        static_assert(BS == 1 || (C::PB * NROW * BS) % 32 == 0, "split rows fill whole warps");
        const int rr = tid / BS;
        const int h = tid - rr * BS;
        const int j = rr / NROW;
        const int r = rr - j * NROW;
        const float2* qrow = q_s + ((size_t)j * NS + r) * C::QS;
        float acc[NS];
#pragma unroll
        for (int m = 0; m < NS; ++m) acc[m] = 0.f;
        stage_b_row<C>(acc, qrow, twc_s + (C::TW2 ? C::R * C::TWS : 0), h * (C::R / BS), (h + 1) * (C::R / BS));
        constexpr int MH = BS == 2 ? (NS + 1) / 2 : NS;   // outputs evaluated by this thread
        int m0 = 0;
        if constexpr (BS == 2) {
#pragma unroll
            for (int m = 0; m < NS; ++m) acc[m] += __shfl_xor_sync(0xffffffffu, acc[m], 1);
            // the second thread moves its outputs m = MH .. NS-1 to acc[0 ..]
#pragma unroll
            for (int i = 0; i < MH; ++i) acc[i] = h ? (i + MH < NS ? acc[i + MH] : 0.f) : acc[i];
            m0 = h * MH;
        }
        const float qn = C::PACK ? qrow[0].y : qrow[NC].x;   // Nyquist column, weight 1, phase (-1)^dx
        const bool row_ok = abs(r - SMAX) <= s;
        float tmin = INFINITY;
        int arg = 0x7fffffff;
        // the full window (s = SMAX, uniform over the block) needs no per-output window test
        const float qa = ((m0 - SMAX) & 1) ? -qn : qn;   // the Nyquist term of output i is (-1)^i qa
        const float c1l = c1 * 1.44269504088896341f;
        float ssum = 0.f;
        auto eval = [&](auto full) {
#pragma unroll
            for (int i = 0; i < MH; ++i) {
                const int m = m0 + i;
                const float rho = acc[i] + ((i & 1) ? -qa : qa);
                // full window: every output but the second thread's padding slot (m = NS) counts
                const bool ok = decltype(full)::value ? (i < MH - 1 || m < NS)
                                                      : (row_ok && m < NS && abs(m - SMAX) <= s);
                const float t = ok ? loglik_t(rho, status) : INFINITY;
                acc[i] = t;
                if (t < tmin) {
                    tmin = t;
                    arg = r * NS + m;
                }
            }
            // with the full window t_min is finite, and a left-out output's +inf gives 2^-inf = 0
#pragma unroll
            for (int i = 0; i < MH; ++i) {
                if constexpr (decltype(full)::value)
                    ssum += ex2_approx(c1l * (acc[i] - tmin));
                else
                    ssum += (acc[i] < INFINITY) ? ex2_approx(c1l * (acc[i] - tmin)) : 0.f;
            }
        };
        if (s >= SMAX)
            eval(std::true_type{});
        else
            eval(std::false_type{});
        row_t[tid] = tmin;
        row_s[tid] = ssum;
        row_d[tid] = arg;
    }
    // ---------------- the dy = +SMAX row by real transforms (see Cfg::DIRFFT)
    if constexpr (C::DIRFFT) {
        constexpr int NJ = C::PB * 2 * C::R;   // jobs: (pair j, component c, sub-sequence b)
        static_assert(C::R == 8 && NJ % 32 == 0 && NJ <= C::THREADS, "one job per thread, whole warps");
        // the last NJ threads, or with C::SPLIT the last NJ / NGROUP threads of each group for its
        // pairs (the upper half of a warp when that is 16)
        constexpr int NJG = C::SPLIT ? NJ / C::NGROUP : NJ;
        constexpr unsigned JM = NJG >= 32 ? 0xffffffffu : (0xffffffffu << (32 - NJG));   // job lanes
        const int grp = C::SPLIT ? tid / C::GT : 0;
        const int tj = C::SPLIT ? tid - grp * C::GT - (C::GT - NJG) : tid - (C::THREADS - NJ);
        const int b = tj & 7, c = (tj >> 3) & 1, j = grp * C::GPB + (tj >> 4);
        const float2* qrow = q_s + ((size_t)j * NS + 2 * SMAX) * C::QS;
        if (tj >= 0) {
            float x[8], yr[9], yi[9], a17[SMAX + 1];
#pragma unroll
            for (int a = 0; a < 8; ++a) {
                const float2 v = qrow[b + 8 * a];
                x[a] = c ? v.y : v.x;
            }
            // packed column 0 = (Q(dy, 0), Q(dy, N/2)): weight 1 (the table carries 2), the Nyquist
            // part enters as (-1)^dx Q(dy, N/2) below
            if (b == 0) x[0] = c ? 0.f : 0.5f * x[0];
            rdft16(x, yr, yi);
#pragma unroll
            for (int k = 0; k <= SMAX; ++k) a17[k] = 0.f;
            recombine<SMAX + 1>(a17, yr, yi, dtw + (c * C::R + b) * (SMAX + 1));
#pragma unroll
            for (int k = 0; k <= SMAX; ++k) {
                a17[k] += __shfl_xor_sync(JM, a17[k], 1);
                a17[k] += __shfl_xor_sync(JM, a17[k], 2);
                a17[k] += __shfl_xor_sync(JM, a17[k], 4);
            }
            if (b == 0) {
#pragma unroll
                for (int k = 0; k <= SMAX; ++k) dsum[(j * 2 + c) * (SMAX + 1) + k] = a17[k];
            }
            __syncwarp(JM);
            // lane (c, b) of pair j: dx = b and b + 8 (and 16 for b = 0), sign + for c = 0, - for c = 1
            const float qn = qrow[0].y;
            const bool row_ok = SMAX <= s;
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                const int dx = r == 0 ? b : (r == 1 ? b + 8 : 2 * 8);
                if ((r == 2 && b != 0) || (c == 1 && dx == 0)) continue;
                const float cv = dsum[(j * 2) * (SMAX + 1) + dx], sv = dsum[(j * 2 + 1) * (SMAX + 1) + dx];
                const float rho = cv + (c ? sv : -sv) + ((dx & 1) ? -qn : qn);
                const int dxs = c ? -dx : dx;
                dir_t[j * NS + dxs + SMAX] = (row_ok && abs(dxs) <= s) ? loglik_t(rho, status) : INFINITY;
            }
        }
    }
    // ---------------- the dy = +SMAX row, one output per task, evaluated directly; the
    // threads without a stage-B row (tid >= PB NROW) take the first outputs so that few
    // threads with a row get two
    if (active && !C::DIRFFT) {
#pragma unroll 1
        for (int i = (tid + C::THREADS - C::PB * NROW * C::BSPLIT) % C::THREADS; i < C::NDIR; i += C::THREADS) {
            const int j = i / NS;
            const int mi = i - j * NS;
            const int dx = mi - SMAX;
            const float2* qrow = q_s + ((size_t)j * NS + 2 * SMAX) * C::QS;
            float accv = 0.f;
            int idx = pmod(dx, N);
            const int step = idx;
            for (int kx = 1; kx < NC; ++kx) {
                const float2 v = qrow[kx];
                const float2 wv = __ldg(gtw + idx);   // exp(-i theta): Re(v exp(+i theta)) = v.x w.x + v.y w.y
                accv = fmaf(v.x, wv.x, fmaf(v.y, wv.y, accv));
                idx += step;
                idx -= (idx >= N) ? N : 0;
            }
            const float qn = C::PACK ? qrow[0].y : qrow[NC].x;
            const float rho = qrow[0].x + 2.f * accv + ((dx & 1) ? -qn : qn);
            const bool ok = SMAX <= s && abs(dx) <= s;
            dir_t[i] = ok ? loglik_t(rho, status) : INFINITY;
        }
    }
    batch_sync<C>();
    // ---------------- combine the pieces of each pair (one full warp per pair; with C::SPLIT the
    // first warps of each group for its pairs)
    const int jw = C::SPLIT ? (tid / C::GT) * C::GPB + (warp - (tid / C::GT) * (C::GT / 32)) : warp;
    const int jend = C::SPLIT ? (tid / C::GT + 1) * C::GPB : C::PB;
    for (int j = jw; warp < C::NWARPS && j < jend; j += C::NWARPS) {
        const int p = p0 + j;
        if (p >= hi) continue;
        Part acc{INFINITY, 0.f, 0x7fffffff};
        constexpr int NR = NROW * C::BSPLIT;
        for (int r = lane; r < NR; r += 32)
            acc = merge(acc, Part{row_t[j * NR + r], row_s[j * NR + r], row_d[j * NR + r]}, c1);
        for (int mi = lane; mi < NS; mi += 32) {
            const float t = dir_t[j * NS + mi];
            acc = merge(acc, Part{t, t < INFINITY ? 1.f : 0.f, 2 * SMAX * NS + mi}, c1);
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            Part o;
            o.t = __shfl_xor_sync(0xffffffffu, acc.t, off);
            o.s = __shfl_xor_sync(0xffffffffu, acc.s, off);
            o.d = __shfl_xor_sync(0xffffffffu, acc.d, off);
            acc = merge(acc, o, c1);   // merge orders its operands, so both lanes agree
        }
        if (lane == 0) {
            rec_t[p] = acc.t;
            rec_s[p] = acc.s;
            rec_d[p] = acc.d;
        }
    }
}

// One work item: image w against parameter sets [lo, hi) of the wave starting at ps_begin.
// img: the image's spectrum; rec_*: the image's record row (indexed by the wave-relative set);
// gtw: exp(-2 pi i t / N), t < N, in global memory (the direct row's twiddles, L1-resident).
// Threads with tid >= C::THREADS only take part in the barriers.
template <class C>
__device__ __forceinline__ void score_item(unsigned char* smem, const float2* __restrict__ gtw,
                                           const float2* __restrict__ img, const int* __restrict__ ps_idx,
                                           const float2* __restrict__ ps_spec, int ps_begin, int lo, int hi, int s,
                                           float c1, float* __restrict__ rec_t, float* __restrict__ rec_s,
                                           int* __restrict__ rec_d, int* __restrict__ status) {
    constexpr int N = C::N, NC = C::NC, H = C::H, NS = C::NS, SMAX = C::SMAX, NROW = C::NROW;
    float2* img_s = reinterpret_cast<float2*>(smem);
    float2* q_s = reinterpret_cast<float2*>(smem + C::SM_IMG);
    float2* twc_s = reinterpret_cast<float2*>(smem + C::SM_IMG + C::SM_QA);
    float2* z_s = reinterpret_cast<float2*>(smem + C::SM_IMG + C::SM_QA + C::SM_TWC);   // [PB][N] (C::PACK)
    float* row_t = reinterpret_cast<float*>(z_s + (C::PACK ? C::PB * N : 0));
    float* row_s = row_t + C::PB * NROW * C::BSPLIT;
    int* row_d = reinterpret_cast<int*>(row_s + C::PB * NROW * C::BSPLIT);
    float* dir_t = reinterpret_cast<float*>(row_d + C::PB * NROW * C::BSPLIT);
    float2* dtw = reinterpret_cast<float2*>(reinterpret_cast<unsigned char*>(smem) + C::SM_BASE + C::SM_Z);
    float* dsum = reinterpret_cast<float*>(reinterpret_cast<unsigned char*>(dtw) + C::SM_DTW);

    const int tid = threadIdx.x;
    const bool active = tid < C::THREADS;
    __syncthreads();   // the previous item's readers of shared memory are done
    {
        const float2* cwN = cw_table<N>();
        for (int i = tid; i < C::R * C::TWS; i += blockDim.x) {
            const int b = i / C::TWS, d = i - (i / C::TWS) * C::TWS;
            const float2 w = d <= SMAX ? cwN[pmod(b * d, N)] : make_float2(0.f, 0.f);
            twc_s[i] = w;
            if constexpr (C::TW2) twc_s[C::R * C::TWS + i] = make_float2(2.f * w.x, 2.f * w.y);
        }
        const float4* src = reinterpret_cast<const float4*>(img);
        float4* dst = reinterpret_cast<float4*>(img_s);
        for (int i = tid; i < N * H / 2; i += blockDim.x) dst[i] = __ldg(src + i);
        if constexpr (C::DIRFFT) {
            // (T1, T2) x 2 (the weight of kx != 0) for component c, sub-sequence b, output dx
            const float2* cwN = cw_table<N>();
            for (int i = tid; i < 2 * C::R * (SMAX + 1); i += blockDim.x) {
                const int c = i / (C::R * (SMAX + 1)), b = (i / (SMAX + 1)) % C::R, dx = i % (SMAX + 1);
                const int u = dx & 15;
                const bool cj = u > 8;
                const float2 w = cwN[(b * dx) % N];   // (cos, sin) of 2 pi b dx / N
                const float t1 = c == 0 ? w.x : w.y;
                const float t2 = c == 0 ? (cj ? w.y : -w.y) : (cj ? -w.x : w.x);
                dtw[i] = make_float2(2.f * t1, 2.f * t2);
            }
        }
    }
    __syncthreads();
    for (int p0 = lo; p0 < hi; p0 += C::PB) {
        // ---------------- packed edge columns Z(ky) = P(ky, 0) + i P(ky, N/2) of the batch's pairs
        if constexpr (C::PACK) {
            // with C::SPLIT each group forms its own pairs' columns
            const int i0 = C::SPLIT ? (tid / C::GT) * C::GPB * N + tid % C::GT : tid;
            const int i1 = C::SPLIT ? (tid / C::GT + 1) * C::GPB * N : C::PB * N;
            const int istep = C::SPLIT ? C::GT : blockDim.x;
            for (int i = i0; i < i1; i += istep) {
                const int j = i / N;
                const int ky = i - j * N;
                const int p = min(p0 + j, hi - 1);
                const int gp = ps_idx ? __ldg(ps_idx + p) : ps_begin + p;
                const float2* ps_row = ps_spec + (size_t)gp * N * H + (size_t)ky * H;
                const float2 e0 = c_mulc(img_s[ky * H], __ldg(ps_row));
                const float2 e1 = c_mulc(img_s[ky * H + NC], __ldg(ps_row + NC));
                z_s[i] = make_float2(e0.x - e1.y, e0.y + e1.x);
            }
            batch_sync<C>();
        }
        // ---------------- stage A: one column of one pair per task
        if (active) {
#pragma unroll 1
            for (int task = tid; task < C::TASKS_A; task += C::THREADS) {
                const int j = task / C::NCOL;
                const int kx = task - j * C::NCOL;
                const int p = min(p0 + j, hi - 1);
                const int gp = ps_idx ? __ldg(ps_idx + p) : ps_begin + p;
                const float2* ps_col = ps_spec + (size_t)gp * N * H + kx;
                float2 acc[NS];
#pragma unroll
                for (int m = 0; m < NS; ++m) acc[m] = make_float2(0.f, 0.f);
                stage_a_column<C>(acc, img_s + kx, ps_col, twc_s, (C::PACK && kx == 0) ? z_s + j * N : nullptr);
                float2* qdst = q_s + (size_t)j * NS * C::QS + kx;
#pragma unroll
                for (int m = 0; m < NS; ++m) qdst[m * C::QS] = acc[m];
            }
        }
        batch_sync<C>();
        score_tail<C>(q_s, twc_s, row_t, row_s, row_d, dir_t, dtw, dsum, gtw, p0, hi, s, c1, rec_t, rec_s, rec_d,
                      status);
    }
}

// Work items (chunk ci, image w), item = ci n_img + w, are taken in index order from a global counter
// (zero at launch): the items in flight stay within one or two chunks of parameter sets, so a chunk
// is read from DRAM about once (a fixed item-per-block assignment let the blocks drift apart over
// thousands of items until several chunks competed for the L2; visiting two chunks per image before
// the next image, to reuse each image, made the two chunks compete the same way).
template <class C>
__global__ void __launch_bounds__(C::THREADS, 1)
k_score(const float2* __restrict__ gtw, const float2* __restrict__ img_spec, int n_img,
        const float2* __restrict__ ps_spec, int ps_begin, int ps_count, int chunk, int n_items, int s, float c1,
        float* __restrict__ rec_t, float* __restrict__ rec_s, int* __restrict__ rec_d, int* __restrict__ status,
        int* __restrict__ work) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int next_item;
    for (;;) {
        if (threadIdx.x == 0) next_item = atomicAdd(work, 1);
        __syncthreads();
        const int item = next_item;   // read by every thread before score_item's first barrier
        if (item >= n_items) break;
        const int ci = item / n_img;
        const int w = item - ci * n_img;
        const int lo = ci * chunk;
        const int hi = min(lo + chunk, ps_count);
        const size_t row = (size_t)w * ps_count;
        score_item<C>(smem, gtw, img_spec + (size_t)w * C::N * C::H, nullptr, ps_spec, ps_begin, lo, hi, s, c1, rec_t + row,
                      rec_s + row, rec_d + row, status);
    }
}

// ---------------------------------------------------------------------------- reductions (float64)
struct Acc {
    double M;    // running max
    double S;    // sum exp(. - M)
    double bv;   // best ln L
    int bp;      // its parameter set
    int bd;      // its displacement index
};

__device__ __forceinline__ void acc_add(Acc& a, double m, double s, int p, int d) {
    if (!(m > -INFINITY)) return;
    if (m > a.M) {
        a.S = a.S * exp(a.M - m) + s;
        a.M = m;
    } else {
        a.S += s * exp(m - a.M);
    }
    if (m > a.bv || (m == a.bv && p < a.bp)) {
        a.bv = m;
        a.bp = p;
        a.bd = d;
    }
}

__device__ __forceinline__ void acc_merge(Acc& a, const Acc& b) {
    if (b.M > -INFINITY) {
        if (b.M > a.M) {
            a.S = a.S * exp(a.M - b.M) + b.S;
            a.M = b.M;
        } else {
            a.S += b.S * exp(b.M - a.M);
        }
    }
    if (b.bv > a.bv || (b.bv == a.bv && b.bp < a.bp)) {
        a.bv = b.bv;
        a.bp = b.bp;
        a.bd = b.bd;
    }
}

constexpr int kRedThreads = 256;

// One block per image: fold the wave's pair records into the image's running accumulator and,
// if requested, write the per-orientation posteriors of the wave's orientations.
__global__ void __launch_bounds__(kRedThreads) k_reduce_wave(
    const float* __restrict__ rec_t, const float* __restrict__ rec_s, const int* __restrict__ rec_d,
    const double* __restrict__ kA, const double* __restrict__ kB, int ps_begin, int wave_len, int nctf,
    int nq, double c1, double log_norm_orient, Acc* __restrict__ acc, int first, double* __restrict__ logP_orient) {
    __shared__ Acc red[kRedThreads];
    const int w = blockIdx.x;
    const double ka = kA[w];
    Acc a{-INFINITY, 0.0, -INFINITY, 0x7fffffff, 0};
    const size_t base = (size_t)w * wave_len;
    for (int p = threadIdx.x; p < wave_len; p += blockDim.x) {
        const double m = ka + kB[ps_begin + p] + c1 * (double)rec_t[base + p];
        acc_add(a, m, (double)rec_s[base + p], ps_begin + p, rec_d[base + p]);
    }
    red[threadIdx.x] = a;
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if (threadIdx.x < st) acc_merge(red[threadIdx.x], red[threadIdx.x + st]);
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        Acc r = red[0];
        if (!first) {
            Acc prev = acc[w];
            acc_merge(prev, r);
            r = prev;
        }
        acc[w] = r;
    }
    if (logP_orient) {
        const int q0 = ps_begin / nctf;
        for (int ql = threadIdx.x; ql < wave_len / nctf; ql += blockDim.x) {
            double M = -INFINITY, S = 0.0;
            for (int c = 0; c < nctf; ++c) {
                const int p = ql * nctf + c;
                const double m = ka + kB[ps_begin + p] + c1 * (double)rec_t[base + p];
                const double s = rec_s[base + p];
                if (!(m > -INFINITY)) continue;
                if (m > M) { S = S * exp(M - m) + s; M = m; }
                else S += s * exp(m - M);
            }
            logP_orient[(size_t)w * nq + q0 + ql] = M + log(S) - log_norm_orient;
        }
    }
}

__global__ void k_finalize(const Acc* __restrict__ acc, int n_img, double log_norm, int nctf, int nsk, int smax,
                           double* logP, int* best_q, int* best_ctf, int* best_dx, int* best_dy, double* best_logL) {
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= n_img) return;
    const Acc a = acc[w];
    if (logP) logP[w] = a.M + log(a.S) - log_norm;
    if (best_q) best_q[w] = a.bp / nctf;
    if (best_ctf) best_ctf[w] = a.bp % nctf;
    if (best_dy) best_dy[w] = a.bd / nsk - smax;
    if (best_dx) best_dx[w] = a.bd % nsk - smax;
    if (best_logL) best_logL[w] = a.bv;
}

// pair_max[w][col0 + p] = max_d ln L and pair_lse[w][col0 + p] = ln sum_d L for the wave's records.
__global__ void k_pairs_out(const float* __restrict__ rec_t, const float* __restrict__ rec_s,
                            const double* __restrict__ kA, const double* __restrict__ kB, int n_img, int ps_begin,
                            int count, double c1, double* pair_max, double* pair_lse, int row_stride, int col0) {
    const size_t total = (size_t)n_img * count;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const int w = (int)(i / count);
        const int p = (int)(i - (size_t)w * count);
        const double m = kA[w] + kB[ps_begin + p] + c1 * (double)rec_t[i];
        const size_t o = (size_t)w * row_stride + col0 + p;
        pair_max[o] = m;
        if (pair_lse) pair_lse[o] = m + log((double)rec_s[i]);
    }
}

// Fold this call's per-image (max, sum) into the caller's running pairs acc2[w] = (M, S), ln sum L =
// M + ln S; first != 0 overwrites.
__global__ void k_fold_acc(const Acc* __restrict__ acc, int n_img, double* __restrict__ acc2, int first) {
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= n_img) return;
    double M = acc[w].M, S = acc[w].S;
    if (!first) {
        const double M0 = acc2[2 * w], S0 = acc2[2 * w + 1];
        if (M0 > -INFINITY) {
            if (!(M > -INFINITY)) { M = M0; S = S0; }
            else if (M0 > M) { S = S * exp(M - M0) + S0; M = M0; }
            else S += S0 * exp(M0 - M);
        }
    }
    acc2[2 * w] = M;
    acc2[2 * w + 1] = S;
}

// ---------------------------------------------------------------------------- host side
// The wave loop shared by the scoring forms: parameter sets [range) in waves whose per-pair records
// (n_img x wave) fit the scratch limit; `records(wbegin, wl, rec_t, rec_s, rec_d)` enqueues the
// kernel(s) writing the records of sets [wbegin, wbegin + wl), then the float64 reductions fold
// them.  Records name displacements d = (dy + smax) ns + (dx + smax), ns = 2 smax + 1 (smax: the
// record kernel's window, which may exceed the scored max_shift); the posterior is normalised by the
// S = (2 max_shift + 1)^2 scored displacements.  Waves are multiples of `align` parameter sets (whole
// orientations when per-orientation output is wanted).
template <class Records>
int run_waves(bioem_ctx* ctx, const bioem_images* im, const bioem_projset* ps, int max_shift, int smax, int align,
              const bioem_score_out& out, Records&& records) {
    const int n_img = im->n_img;
    const int n = im->nx * im->ny;
    const int nsk = 2 * smax + 1;
    const bool pairs_mode = out.pair_max != nullptr;
    const int range_begin = pairs_mode ? out.ps_begin : 0;
    const int range_len = pairs_mode ? out.ps_count : ps->n_ps;
    const int nctf = ps->nctf;
    if (n_img == 0 || range_len == 0) return BIOEM_OK;

    // wave length: records of n_img x wave must fit the scratch limit; a multiple of `align`
    const unsigned long long per_ps = (unsigned long long)n_img * 12ull;
    long long wave = (long long)(ctx->scratch_limit / per_ps);
    if (wave >= align) wave -= wave % align;
    const long long min_wave = pairs_mode ? 1 : nctf;
    if (wave < min_wave) wave = min_wave;
    if (!pairs_mode) wave -= wave % nctf;
    if (wave > range_len) wave = range_len;
    const size_t rec_need = (size_t)n_img * (size_t)wave * 12;
    if (ctx->rec_bytes < rec_need) {
        if (ctx->d_rec) cudaFreeAsync(ctx->d_rec, ctx->stream);
        ctx->d_rec = nullptr;
        ctx->rec_bytes = 0;
        if (cudaMallocAsync(&ctx->d_rec, rec_need, ctx->stream) != cudaSuccess)
            return bioem_set_error(ctx, BIOEM_ERR_OOM, "record scratch of %zu bytes", rec_need);
        ctx->rec_bytes = rec_need;
    }
    const size_t acc_need = sizeof(Acc) * (size_t)n_img;
    if (!pairs_mode && ctx->acc_bytes < acc_need) {
        if (ctx->d_acc) cudaFreeAsync(ctx->d_acc, ctx->stream);
        ctx->d_acc = nullptr;
        ctx->acc_bytes = 0;
        if (cudaMallocAsync(&ctx->d_acc, acc_need, ctx->stream) != cudaSuccess)
            return bioem_set_error(ctx, BIOEM_ERR_OOM, "accumulator scratch");
        ctx->acc_bytes = acc_need;
    }
    float* rec_t = reinterpret_cast<float*>(ctx->d_rec);
    float* rec_s = rec_t + (size_t)n_img * wave;
    int* rec_d = reinterpret_cast<int*>(rec_s + (size_t)n_img * wave);
    const double c1 = 0.5 * (3.0 - (double)n);
    const int S = (2 * max_shift + 1) * (2 * max_shift + 1);

    for (long long w0 = 0; w0 < range_len; w0 += wave) {
        const int wl = (int)(range_len - w0 < wave ? range_len - w0 : wave);
        const int wbegin = range_begin + (int)w0;
        int rc = records(wbegin, wl, rec_t, rec_s, rec_d);
        if (rc) return rc;
        if (pairs_mode) {
            bioem_launch_begin(ctx, KID_PAIRS_OUT);
            k_pairs_out<<<1024, 256, 0, ctx->stream>>>(rec_t, rec_s, im->d_kA, ps->d_kB, n_img, wbegin, wl, c1,
                                                       out.pair_max, out.pair_lse, range_len, (int)w0);
            bioem_launch_end(ctx, KID_PAIRS_OUT);
        } else {
            const double log_norm_orient = log((double)nctf * S);
            bioem_launch_begin(ctx, KID_REDUCE_WAVE);
            k_reduce_wave<<<n_img, kRedThreads, 0, ctx->stream>>>(rec_t, rec_s, rec_d, im->d_kA, ps->d_kB, wbegin, wl,
                                                                  nctf, ps->nq, c1, log_norm_orient,
                                                                  reinterpret_cast<Acc*>(ctx->d_acc), w0 == 0,
                                                                  out.logP_orient);
            bioem_launch_end(ctx, KID_REDUCE_WAVE);
        }
        rc = bioem_check_cuda(ctx, cudaGetLastError(), "reduction");
        if (rc) return rc;
    }
    if (!pairs_mode) {
        const double log_norm = log((double)ps->n_ps * S);
        bioem_launch_begin(ctx, KID_FINALIZE);
        k_finalize<<<(n_img + 255) / 256, 256, 0, ctx->stream>>>(reinterpret_cast<const Acc*>(ctx->d_acc), n_img, log_norm,
                                                                  nctf, nsk, smax, out.logP, out.best_q, out.best_ctf,
                                                                  out.best_dx, out.best_dy, out.best_logL);
        bioem_launch_end(ctx, KID_FINALIZE);
        if (out.acc2) {
            bioem_launch_begin(ctx, KID_FINALIZE);
            k_fold_acc<<<(n_img + 255) / 256, 256, 0, ctx->stream>>>(reinterpret_cast<const Acc*>(ctx->d_acc), n_img,
                                                                     out.acc2, out.acc_first);
            bioem_launch_end(ctx, KID_FINALIZE);
        }
        return bioem_check_cuda(ctx, cudaGetLastError(), "k_finalize");
    }
    return BIOEM_OK;
}

// Resident blocks of k_score<C> on the whole GPU (sets the kernel's shared-memory attribute).
template <class C>
int score_slots(bioem_ctx* ctx, int* slots) {
    const size_t smem = C::SMEM;
    if (cudaFuncSetAttribute(k_score<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return bioem_set_error(ctx, BIOEM_ERR_CUDA, "shared memory attribute (%zu bytes)", smem);
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_score<C>, C::THREADS, smem) != cudaSuccess || per_sm < 1)
        return bioem_set_error(ctx, BIOEM_ERR_CUDA, "occupancy query");
    *slots = per_sm * ctx->num_sms;
    return BIOEM_OK;
}

// One k_score<C> launch writing the records of parameter sets [wbegin, wbegin + wl) for every image.
// Chunk: enough work items to keep every slot busy, at most 512 parameter sets, whole batches.
template <class C>
int launch_score_records(bioem_ctx* ctx, const bioem_images* im, const bioem_projset* ps, int slots, int wbegin,
                         int wl, int max_shift, float* rec_t, float* rec_s, int* rec_d) {
    const int n_img = im->n_img;
    const long long target_items = 4ll * slots;
    const long long per_img = (target_items + n_img - 1) / n_img;
    long long chunk = (wl + per_img - 1) / per_img;
    chunk = ((chunk + C::PB - 1) / C::PB) * C::PB;
    if (chunk > 512) chunk = 512 / C::PB * C::PB;
    if (chunk < C::PB) chunk = C::PB;
    const long long n_chunks = (wl + chunk - 1) / chunk;
    const long long n_items = n_chunks * n_img;
    if (n_items > 0x7fffffffll) return bioem_set_error(ctx, BIOEM_ERR_UNSUPPORTED_SIZE, "too many work items");
    const int grid = (int)(n_items < slots ? n_items : slots);
    const float c1f = 0.5f * (3.0f - (float)(C::N * C::N));
    bioem_launch_begin(ctx, KID_SCORE);
    if (cudaMemsetAsync(ctx->d_work, 0, sizeof(int), ctx->stream) != cudaSuccess)
        return bioem_check_cuda(ctx, cudaGetLastError(), "work counter");
    k_score<C><<<grid, C::THREADS, C::SMEM, ctx->stream>>>(bioem_twiddles(ctx, C::N), im->d_spec, n_img, ps->d_spec,
                                                            wbegin, wl, (int)chunk, (int)n_items, max_shift, c1f,
                                                            rec_t, rec_s, rec_d, ctx->d_status, ctx->d_work);
    bioem_launch_end(ctx, KID_SCORE);
    return bioem_check_cuda(ctx, cudaGetLastError(), "k_score");
}

// The FP32 form: k_score<C> writes the records (displacements named in C's compile-time window).
template <class C>
int run_score(bioem_ctx* ctx, const bioem_images* im, const bioem_projset* ps, int max_shift,
              const bioem_score_out& out) {
    int slots = 0;
    const int rc = score_slots<C>(ctx, &slots);
    if (rc) return rc;
    auto records = [&](int wbegin, int wl, float* rec_t, float* rec_s, int* rec_d) -> int {
        return launch_score_records<C>(ctx, im, ps, slots, wbegin, wl, max_shift, rec_t, rec_s, rec_d);
    };
    return run_waves(ctx, im, ps, max_shift, C::SMAX, ps->nctf, out, records);
}

// The split-precision tensor-core form (gemm.cu writes the records, window = max_shift); waves are
// whole 128-set row tiles where the scratch allows.
int run_score_gemm(bioem_ctx* ctx, const bioem_images* im, const bioem_projset* ps, int max_shift,
                   const bioem_score_out& out) {
    const int mode = ctx->precision;
    int rc = bioem_gemm_prepare(ctx, im, ps, max_shift, mode);
    if (rc) return rc;
    const int tile = bioem_gemm_row_tile();
    int a = tile, b = ps->nctf;
    while (b) { const int t = a % b; a = b; b = t; }
    const int align = tile / a * ps->nctf;   // lcm(row tile, PSFs per orientation)
    auto records = [&](int wbegin, int wl, float* rec_t, float* rec_s, int* rec_d) -> int {
        return bioem_gemm_records(ctx, im, ps, max_shift, mode, wbegin, wbegin + wl, rec_t, rec_s, rec_d);
    };
    return run_waves(ctx, im, ps, max_shift, max_shift, align, out, records);
}

// <N, SMAX, pairs per batch, threads[, packed edge columns allowed]>: the threads divide the
// stage-A tasks (PB N/2 with the packed edge columns, PB (N/2 + 1) without) into whole rounds.
// Packed edge columns where they measured faster (128 px: 2 % at s = 4, 6 % at s = 16); at 32-96
// px the transforms are short enough that forming Z costs about as much as the column it saves
// (unpacked 4-9 % faster there).
using C32_4 = Cfg<32, 4, 32, 272, false>;
using C64_4 = Cfg<64, 4, 32, 264, false>;
using C64_8 = Cfg<64, 8, 16, 264, false>;
using C96_12 = Cfg<96, 12, 10, 245, false>;
using C128_4 = Cfg<128, 4, 24, 256>;
// 128 px, s <= 16: 512 threads (four warps per scheduler, 128 registers), one stage-A column per
// thread and two threads per stage-B row, in four decoupled groups of two pairs (Cfg::SPLIT); 11 %
// faster than 256 threads with one row per thread, which left the kernel waiting on
// dependent-instruction latency at two warps per scheduler.
using C128_16 = Cfg<128, 16, 8, 512, true, 2>;
using C192_24 = Cfg<192, 24, 2, 194>;
static_assert(C128_4::PACK && C128_16::PACK, "packed edge columns fit");
static_assert(C128_16::TASKS_A % C128_16::THREADS == 0 && C128_4::TASKS_A % C128_4::THREADS == 0 &&
              C64_8::TASKS_A % C64_8::THREADS == 0 && C64_4::TASKS_A % C64_4::THREADS == 0 &&
              C32_4::TASKS_A % C32_4::THREADS == 0 && C96_12::TASKS_A % C96_12::THREADS == 0 &&
              C192_24::TASKS_A % C192_24::THREADS == 0, "whole stage-A rounds");

}  // namespace

int bioem_score_supported(int npix, int max_shift) {
    if (max_shift < 0 || 2 * max_shift >= npix) return 0;
    switch (npix) {
        case 32: return max_shift <= 4;
        case 64: return max_shift <= 8;
        case 96: return max_shift <= 12;
        case 128: return max_shift <= 16;
        case 192: return max_shift <= 24;
        default: return 0;
    }
}

int bioem_launch_score(bioem_ctx* ctx, const bioem_images* im, const bioem_projset* ps, int max_shift,
                       const bioem_score_out& out) {
    if (ctx->precision == BIOEM_PRECISION_FP16X2_FFT) {
        if (!bioem_tc_supported(im->nx, max_shift))
            return bioem_set_error(ctx, BIOEM_ERR_UNSUPPORTED_SIZE,
                                   "tensor-core column transforms: 128 px and max_shift <= 16 only (%d px, %d)",
                                   im->nx, max_shift);
        auto records = [&](int wbegin, int wl, float* rec_t, float* rec_s, int* rec_d) -> int {
            return bioem_tc_records(ctx, im, ps, max_shift, wbegin, wl, rec_t, rec_s, rec_d);
        };
        return run_waves(ctx, im, ps, max_shift, 16, ps->nctf, out, records);
    }
    if (ctx->precision != BIOEM_PRECISION_FP32) {
        if (!bioem_gemm_supported(im->nx, max_shift))
            return bioem_set_error(ctx, BIOEM_ERR_UNSUPPORTED_SIZE,
                                   "split-precision form: max_shift %d at %d px exceeds 256 columns per image", max_shift,
                                   im->nx);
        return run_score_gemm(ctx, im, ps, max_shift, out);
    }
    switch (im->nx) {
        case 32: return run_score<C32_4>(ctx, im, ps, max_shift, out);
        case 64: return max_shift <= 4 ? run_score<C64_4>(ctx, im, ps, max_shift, out)
                                       : run_score<C64_8>(ctx, im, ps, max_shift, out);
        case 96: return run_score<C96_12>(ctx, im, ps, max_shift, out);
        case 128: return max_shift <= 4 ? run_score<C128_4>(ctx, im, ps, max_shift, out)
                                        : run_score<C128_16>(ctx, im, ps, max_shift, out);
        case 192: return run_score<C192_24>(ctx, im, ps, max_shift, out);
        default: return bioem_set_error(ctx, BIOEM_ERR_UNSUPPORTED_SIZE, "unsupported image size %d", im->nx);
    }
}

int bioem_upload_score_twiddles(bioem_ctx* ctx) {
    const int sizes[6] = {16, 32, 64, 96, 128, 192};
    for (int k = 0; k < 6; ++k) {
        const int M = sizes[k];
        float2 h[192];
        for (int t = 0; t < M; ++t) {
            const double a = 2.0 * 3.14159265358979323846 * (double)t / (double)M;
            h[t] = make_float2((float)cos(a), (float)sin(a));
        }
        cudaError_t e;
        switch (M) {
            case 16: e = cudaMemcpyToSymbol(c_w16, h, sizeof(float2) * 16); break;
            case 32: e = cudaMemcpyToSymbol(c_w32, h, sizeof(float2) * 32); break;
            case 64: e = cudaMemcpyToSymbol(c_w64, h, sizeof(float2) * 64); break;
            case 96: e = cudaMemcpyToSymbol(c_w96, h, sizeof(float2) * 96); break;
            case 192: e = cudaMemcpyToSymbol(c_w192, h, sizeof(float2) * 192); break;
            default: e = cudaMemcpyToSymbol(c_w128, h, sizeof(float2) * 128); break;
        }
        if (e != cudaSuccess) return bioem_check_cuda(ctx, e, "twiddle upload");
    }
    return BIOEM_OK;
}

// ---------------------------------------------------------------------------- allocation-free scoring
// Scratch for bioem_score_noalloc: per-image accumulators followed by per-pair records, reserved
// statically in device memory on every GPU this library is loaded on, for the life of the process.
// Host code must not use the symbol's host-side address: each device's address is looked up once
// with cudaGetSymbolAddress while that device is current.

namespace {

constexpr size_t kNoAllocBytes = 16u << 20;   // 16 MiB
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mutex;
void* g_noalloc_ptr[kMaxDevices] = {};

// Device address of the static scratch on the current device.  Looked up again on every call made
// outside a stream capture (a device reset between calls reloads the module, possibly at another
// address); a call made while the stream is capturing uses the address of the last such lookup.
int noalloc_scratch(bioem_ctx* ctx, void** out) {
    if (ctx->device < 0 || ctx->device >= kMaxDevices)
        return bioem_set_error(ctx, BIOEM_ERR_UNSUPPORTED_SIZE, "device ordinal %d too large", ctx->device);
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(ctx->stream, &cs) != cudaSuccess) {
        cudaGetLastError();
        cs = cudaStreamCaptureStatusActive;   // unknown: do not call into the runtime's module table
    }
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (cs == cudaStreamCaptureStatusNone) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) return bioem_check_cuda(ctx, e != cudaSuccess ? e : cudaErrorInvalidSymbol,
                                                             "cudaGetSymbolAddress(static scoring scratch)");
        g_noalloc_ptr[ctx->device] = p;
    } else if (!g_noalloc_ptr[ctx->device]) {
        return bioem_set_error(ctx, BIOEM_ERR_INVALID_ARG,
                               "allocation-free scoring: the first call on a device must come before any stream capture");
    }
    *out = g_noalloc_ptr[ctx->device];
    return BIOEM_OK;
}

// The wave loop of bioem_score (log P only) with records and accumulators in the static scratch.
template <class C>
int run_score_noalloc(bioem_ctx* ctx, const bioem_images* im, const bioem_projset* ps, int max_shift, double* logP) {
    const int n_img = im->n_img;
    const int nctf = ps->nctf;
    if (n_img == 0) return BIOEM_OK;
    const size_t acc_bytes = ((sizeof(Acc) * (size_t)n_img + 255) / 256) * 256;
    const size_t per_ps = (size_t)n_img * 12;
    if (acc_bytes + per_ps * nctf > kNoAllocBytes)
        return bioem_set_error(ctx, BIOEM_ERR_UNSUPPORTED_SIZE,
                               "allocation-free scoring: %d images x %d PSFs need %zu bytes of scratch, more than "
                               "the static %zu", n_img, nctf, acc_bytes + per_ps * nctf, kNoAllocBytes);
    void* base = nullptr;
    int rc = noalloc_scratch(ctx, &base);
    if (rc) return rc;
    long long wave = (long long)((kNoAllocBytes - acc_bytes) / per_ps);
    wave -= wave % nctf;
    if (wave > ps->n_ps) wave = ps->n_ps;
    Acc* acc = reinterpret_cast<Acc*>(base);
    float* rec_t = reinterpret_cast<float*>(static_cast<unsigned char*>(base) + acc_bytes);
    float* rec_s = rec_t + (size_t)n_img * wave;
    int* rec_d = reinterpret_cast<int*>(rec_s + (size_t)n_img * wave);

    int slots = 0;
    rc = score_slots<C>(ctx, &slots);
    if (rc) return rc;
    const int n = C::N * C::N;
    const double c1 = 0.5 * (3.0 - (double)n);
    const int S = (2 * max_shift + 1) * (2 * max_shift + 1);
    for (long long w0 = 0; w0 < ps->n_ps; w0 += wave) {
        const int wl = (int)(ps->n_ps - w0 < wave ? ps->n_ps - w0 : wave);
        rc = launch_score_records<C>(ctx, im, ps, slots, (int)w0, wl, max_shift, rec_t, rec_s, rec_d);
        if (rc) return rc;
        bioem_launch_begin(ctx, KID_REDUCE_WAVE);
        k_reduce_wave<<<n_img, kRedThreads, 0, ctx->stream>>>(rec_t, rec_s, rec_d, im->d_kA, ps->d_kB, (int)w0, wl,
                                                              nctf, ps->nq, c1, log((double)nctf * S), acc, w0 == 0,
                                                              nullptr);
        bioem_launch_end(ctx, KID_REDUCE_WAVE);
        rc = bioem_check_cuda(ctx, cudaGetLastError(), "k_reduce_wave");
        if (rc) return rc;
    }
    bioem_launch_begin(ctx, KID_FINALIZE);
    k_finalize<<<(n_img + 255) / 256, 256, 0, ctx->stream>>>(acc, n_img, log((double)ps->n_ps * S), nctf, C::NS,
                                                              C::SMAX, logP, nullptr, nullptr, nullptr, nullptr,
                                                              nullptr);
    bioem_launch_end(ctx, KID_FINALIZE);
    return bioem_check_cuda(ctx, cudaGetLastError(), "k_finalize");
}

}  // namespace

extern "C" int bioem_score_noalloc(bioem_ctx* ctx, const bioem_images* images, const bioem_projset* projset,
                                   int max_shift, double* d_logP) {
    if (!ctx || !images || !projset) return BIOEM_ERR_INVALID_ARG;
    if (images->ctx != ctx || projset->ctx != ctx)
        return bioem_set_error(ctx, BIOEM_ERR_INVALID_ARG, "handle from another context");
    if (images->nx != projset->nx || images->ny != projset->ny ||
        fabs(images->pixel_A - projset->pixel_A) > 1e-9 * images->pixel_A)
        return bioem_set_error(ctx, BIOEM_ERR_INVALID_ARG, "images and projections differ in size or pixel");
    if (max_shift < 0) return bioem_set_error(ctx, BIOEM_ERR_INVALID_ARG, "negative max_shift");
    if (!bioem_score_supported(images->nx, max_shift))
        return bioem_set_error(ctx, BIOEM_ERR_UNSUPPORTED_SIZE, "max_shift %d unsupported at %d px", max_shift,
                               images->nx);
    if (projset->n_ps == 0) return bioem_set_error(ctx, BIOEM_ERR_INVALID_ARG, "empty parameter set");
    if (images->n_img > 0 && !d_logP) return bioem_set_error(ctx, BIOEM_ERR_INVALID_ARG, "d_logP is required");
    if (cudaSetDevice(ctx->device) != cudaSuccess) return bioem_set_error(ctx, BIOEM_ERR_CUDA, "cudaSetDevice");
    switch (images->nx) {
        case 32: return run_score_noalloc<C32_4>(ctx, images, projset, max_shift, d_logP);
        case 64: return max_shift <= 4 ? run_score_noalloc<C64_4>(ctx, images, projset, max_shift, d_logP)
                                       : run_score_noalloc<C64_8>(ctx, images, projset, max_shift, d_logP);
        case 96: return run_score_noalloc<C96_12>(ctx, images, projset, max_shift, d_logP);
        case 128: return max_shift <= 4 ? run_score_noalloc<C128_4>(ctx, images, projset, max_shift, d_logP)
                                        : run_score_noalloc<C128_16>(ctx, images, projset, max_shift, d_logP);
        case 192: return run_score_noalloc<C192_24>(ctx, images, projset, max_shift, d_logP);
        default: return bioem_set_error(ctx, BIOEM_ERR_UNSUPPORTED_SIZE, "unsupported image size %d", images->nx);
    }
}

// ---------------------------------------------------------------------------- batched scoring
// Several models against several image stacks of mixed sizes in one persistent launch.  A segment
// is one (model, stack) pair: the stack's image spectra against that model's parameter sets for
// that stack.  Work items of all segments form one list; every item runs the instance for its
// image size.  All instances here use 256 threads (2 warps per scheduler keep the 96 / 192 px
// paths at their register counts).
#include <string>
#include <vector>

namespace {

// (unpacked edge columns: the four instances share one kernel's registers, and with the packed
// columns they spill)
using M64 = Cfg<64, 8, 15, 256, false>;
using M96 = Cfg<96, 12, 10, 256, false>;
using M128 = Cfg<128, 16, 7, 256, false>;
using M192 = Cfg<192, 24, 2, 256, false>;
constexpr int kMultiThreads = 256;

constexpr size_t cmax(size_t a, size_t b) { return a > b ? a : b; }
constexpr size_t kMultiSmem = cmax(cmax(M64::SMEM, M96::SMEM), cmax(M128::SMEM, M192::SMEM));

struct SegDesc {
    const float2* img;    // [n_img][N][N/2+1]
    const float2* ps;     // [n_ps][N][N/2+1]
    const float2* gtw;    // exp(-2 pi i t / N)
    const double* kA;     // [n_img]
    const double* kB;     // [n_ps]
    float* rec_t;         // [n_img][n_ps] records
    float* rec_s;
    int* rec_d;
    long long item_begin; // first global item of this segment
    long long row_begin;  // first global reduction row (image) of this segment
    int n_img, n_ps, chunk, n_chunks, s, npix, nctf;
    int out_row;          // model index (row of the output matrix)
    int out_col;          // column of the segment's first image in the output matrix
    float c1;
    double log_norm;      // ln(n_ps S)
};

__device__ __forceinline__ int find_seg(const SegDesc* segs, int n, long long x, bool rows) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        const long long b = rows ? segs[mid].row_begin : segs[mid].item_begin;
        if (b <= x) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__global__ void __launch_bounds__(kMultiThreads, 1)
k_score_multi(const SegDesc* __restrict__ segs, int n_segs, long long n_items, int* __restrict__ status,
              unsigned long long* __restrict__ work) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ long long next_item;
    for (;;) {
        // items in index order from a global counter (zero at launch), as in k_score
        if (threadIdx.x == 0) next_item = (long long)atomicAdd(work, 1ull);
        __syncthreads();
        const long long item = next_item;
        if (item >= n_items) break;
        const int g = find_seg(segs, n_segs, item, false);
        const SegDesc& sd = segs[g];
        const long long local = item - sd.item_begin;
        const int ci = (int)(local / sd.n_img);
        const int w = (int)(local - (long long)ci * sd.n_img);
        const int lo = ci * sd.chunk;
        const int hi = min(lo + sd.chunk, sd.n_ps);
        const size_t row = (size_t)w * sd.n_ps;
        switch (sd.npix) {
            case 64:
                score_item<M64>(smem, sd.gtw, sd.img + (size_t)w * 64 * 33, nullptr, sd.ps, 0, lo, hi, sd.s, sd.c1,
                                sd.rec_t + row, sd.rec_s + row, sd.rec_d + row, status);
                break;
            case 96:
                score_item<M96>(smem, sd.gtw, sd.img + (size_t)w * 96 * 49, nullptr, sd.ps, 0, lo, hi, sd.s, sd.c1,
                                sd.rec_t + row, sd.rec_s + row, sd.rec_d + row, status);
                break;
            case 128:
                score_item<M128>(smem, sd.gtw, sd.img + (size_t)w * 128 * 65, nullptr, sd.ps, 0, lo, hi, sd.s, sd.c1,
                                 sd.rec_t + row, sd.rec_s + row, sd.rec_d + row, status);
                break;
            default:
                score_item<M192>(smem, sd.gtw, sd.img + (size_t)w * 192 * 97, nullptr, sd.ps, 0, lo, hi, sd.s, sd.c1,
                                 sd.rec_t + row, sd.rec_s + row, sd.rec_d + row, status);
                break;
        }
    }
}

// One block per (segment, image): float64 log-sum-exp over the image's records, written as float32
// into out[model][column].
__global__ void __launch_bounds__(kRedThreads) k_reduce_multi(const SegDesc* __restrict__ segs, int n_segs,
                                                              float* __restrict__ out, int out_ld) {
    __shared__ double redM[kRedThreads], redS[kRedThreads];
    const long long row = blockIdx.x;
    const int g = find_seg(segs, n_segs, row, true);
    const SegDesc& sd = segs[g];
    const int w = (int)(row - sd.row_begin);
    const double ka = sd.kA[w];
    const double c1 = (double)sd.c1;
    double M = -INFINITY, S = 0.0;
    const size_t base = (size_t)w * sd.n_ps;
    for (int p = threadIdx.x; p < sd.n_ps; p += blockDim.x) {
        const double m = ka + sd.kB[p] + c1 * (double)sd.rec_t[base + p];
        const double s = sd.rec_s[base + p];
        if (!(m > -INFINITY)) continue;
        if (m > M) { S = S * exp(M - m) + s; M = m; }
        else S += s * exp(m - M);
    }
    redM[threadIdx.x] = M;
    redS[threadIdx.x] = S;
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if (threadIdx.x < st) {
            const double m2 = redM[threadIdx.x + st], s2 = redS[threadIdx.x + st];
            double m1 = redM[threadIdx.x], s1 = redS[threadIdx.x];
            if (m2 > -INFINITY) {
                if (m2 > m1) { s1 = s1 * exp(m1 - m2) + s2; m1 = m2; }
                else s1 += s2 * exp(m2 - m1);
            }
            redM[threadIdx.x] = m1;
            redS[threadIdx.x] = s1;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0)
        out[(size_t)sd.out_row * out_ld + sd.out_col + w] = (float)(redM[0] + log(redS[0]) - sd.log_norm);
}

struct TuneEntry {
    int npix, s, chunk;
};

int default_chunk(int npix) { return npix >= 192 ? 64 : 256; }

int tuned_chunk(const std::vector<TuneEntry>& t, int npix, int s) {
    for (const auto& e : t)
        if (e.npix == npix && e.s == s) return e.chunk;
    return default_chunk(npix);
}

int multi_pb(int npix) {
    switch (npix) {
        case 64: return M64::PB;
        case 96: return M96::PB;
        case 128: return M128::PB;
        default: return M192::PB;
    }
}

int multi_smax(int npix) {
    switch (npix) {
        case 64: return M64::SMAX;
        case 96: return M96::SMAX;
        case 128: return M128::SMAX;
        default: return M192::SMAX;
    }
}

}  // namespace

struct bioem_batch {
    bioem_ctx* ctx;
    int device;            // bioem_batch_free uses these, never the (possibly destroyed) context
    cudaStream_t stream;
    int n_models, n_stacks, n_cols;
    std::vector<SegDesc> segs;
    SegDesc* d_segs;
    void* d_rec;
    unsigned long long* d_work;   // work-item counter of the scoring launch
    long long n_items, n_rows;
    float* d_out;
    cudaStream_t cap_stream;
    cudaGraph_t graph;
    cudaGraphExec_t exec;
    int grid;
};

// tune table kept per process (per image size and shift window)
static std::mutex g_tune_mutex;
static std::vector<TuneEntry> g_tune;

// An entry the batched launch can use: a batched image size, a shift window its instance covers,
// and a chunk that is a whole number of that instance's batches, at most 4096 parameter sets.
static bool tune_entry_valid(int npix, int s, int chunk) {
    if (npix != 64 && npix != 96 && npix != 128 && npix != 192) return false;
    if (s < 0 || s > multi_smax(npix) || 2 * s >= npix) return false;
    const int pb = multi_pb(npix);
    return chunk > 0 && chunk <= 4096 && chunk % pb == 0;
}

// Read "npix shift chunk" lines into the process table.  Lines that are not three integers, or
// whose entry is not valid, are skipped (a corrupted or foreign cache file then only costs a new
// tuning run); returns the number of entries taken (-1 if the file cannot be opened) and, in
// *skipped, the number of non-blank lines skipped.
static int tune_load(const char* path, int* skipped = nullptr) {
    if (skipped) *skipped = 0;
    FILE* f = fopen(path, "r");
    if (!f) return -1;
    char line[256];
    int n = 0;
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    while (fgets(line, sizeof line, f)) {
        int npix, s, chunk;
        char extra;
        const int got = sscanf(line, "%d %d %d %c", &npix, &s, &chunk, &extra);
        if (got != 3 || !tune_entry_valid(npix, s, chunk)) {
            bool blank = true;
            for (const char* c = line; *c; ++c)
                if (*c != ' ' && *c != '\t' && *c != '\n' && *c != '\r') blank = false;
            if (!blank && skipped) ++*skipped;
            continue;
        }
        bool found = false;
        for (auto& e : g_tune)
            if (e.npix == npix && e.s == s) { e.chunk = chunk; found = true; }
        if (!found) g_tune.push_back({npix, s, chunk});
        ++n;
    }
    fclose(f);
    return n;
}

static int batch_build(bioem_batch* b, int grid_override) {
    bioem_ctx* ctx = b->ctx;
    const size_t nb = sizeof(SegDesc) * b->segs.size();
    if (cudaMalloc((void**)&b->d_segs, nb) != cudaSuccess) return bioem_set_error(ctx, BIOEM_ERR_OOM, "segment table");
    if (cudaMemcpy(b->d_segs, b->segs.data(), nb, cudaMemcpyHostToDevice) != cudaSuccess)
        return bioem_set_error(ctx, BIOEM_ERR_CUDA, "segment table upload");
    if (cudaMalloc((void**)&b->d_work, sizeof(unsigned long long)) != cudaSuccess)
        return bioem_set_error(ctx, BIOEM_ERR_OOM, "work counter");
    if (cudaFuncSetAttribute(k_score_multi, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMultiSmem) != cudaSuccess)
        return bioem_set_error(ctx, BIOEM_ERR_CUDA, "shared memory attribute (%zu bytes)", kMultiSmem);
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_score_multi, kMultiThreads, kMultiSmem) != cudaSuccess ||
        per_sm < 1)
        return bioem_set_error(ctx, BIOEM_ERR_CUDA, "occupancy query");
    long long g = (long long)per_sm * ctx->num_sms;
    if (grid_override > 0) g = grid_override;
    if (g > b->n_items) g = b->n_items;
    b->grid = (int)g;
    if (cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking) != cudaSuccess)
        return bioem_set_error(ctx, BIOEM_ERR_CUDA, "capture stream");
    if (cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
        return bioem_set_error(ctx, BIOEM_ERR_CUDA, "begin capture");
    cudaMemsetAsync(b->d_work, 0, sizeof(unsigned long long), b->cap_stream);
    k_score_multi<<<b->grid, kMultiThreads, kMultiSmem, b->cap_stream>>>(b->d_segs, (int)b->segs.size(), b->n_items,
                                                                        ctx->d_status, b->d_work);
    k_reduce_multi<<<(unsigned)b->n_rows, kRedThreads, 0, b->cap_stream>>>(b->d_segs, (int)b->segs.size(), b->d_out,
                                                                           b->n_cols);
    cudaError_t e = cudaStreamEndCapture(b->cap_stream, &b->graph);
    if (e != cudaSuccess) return bioem_check_cuda(ctx, e, "end capture");
    e = cudaGraphInstantiate(&b->exec, b->graph, 0);
    if (e != cudaSuccess) return bioem_check_cuda(ctx, e, "graph instantiate");
    return BIOEM_OK;
}

extern "C" {

int bioem_autotune_load(const char* cache_path, int* n_taken, int* n_skipped) {
    if (!cache_path) return BIOEM_ERR_INVALID_ARG;
    int skipped = 0;
    const int n = tune_load(cache_path, &skipped);
    if (n_taken) *n_taken = n < 0 ? 0 : n;
    if (n_skipped) *n_skipped = skipped;
    return n < 0 ? BIOEM_ERR_INVALID_ARG : BIOEM_OK;
}

int bioem_autotune(bioem_ctx* ctx, const bioem_images* images, const bioem_projset* projset, int max_shift,
                   const char* cache_path, int* out_chunk) {
    if (!ctx || !images || !projset) return BIOEM_ERR_INVALID_ARG;
    if (cache_path && tune_load(cache_path) > 0) {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        for (const auto& e : g_tune)
            if (e.npix == images->nx && e.s == max_shift) {
                if (out_chunk) *out_chunk = e.chunk;
                return BIOEM_OK;
            }
    }
    const int npix = images->nx;
    if (npix != 64 && npix != 96 && npix != 128 && npix != 192)
        return bioem_set_error(ctx, BIOEM_ERR_UNSUPPORTED_SIZE, "autotune: batched sizes are 64, 96, 128, 192");
    if (max_shift < 0 || max_shift > multi_smax(npix) || images->nx != projset->nx || images->n_img == 0 ||
        projset->n_ps == 0)
        return bioem_set_error(ctx, BIOEM_ERR_INVALID_ARG, "autotune: bad case");
    if (cudaSetDevice(ctx->device) != cudaSuccess) return bioem_set_error(ctx, BIOEM_ERR_CUDA, "cudaSetDevice");
    // trial: the first images (up to 2 per SM) against up to 4096 parameter sets, one segment
    const int n_img = images->n_img < 2 * ctx->num_sms ? images->n_img : 2 * ctx->num_sms;
    const int n_ps = projset->n_ps < 4096 ? projset->n_ps : 4096;
    const int pb = multi_pb(npix);
    const int cands[5] = {pb * 2, pb * 8, pb * 32, pb * 64, pb * 128};
    void* rec = nullptr;
    const size_t rec_bytes = (size_t)n_img * n_ps * 12;
    if (cudaMalloc(&rec, rec_bytes) != cudaSuccess) return bioem_set_error(ctx, BIOEM_ERR_OOM, "autotune records");
    double best_ms = 1e300;
    int best = default_chunk(npix);
    int rc = BIOEM_OK;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    for (int k = 0; k < 5 && rc == BIOEM_OK; ++k) {
        const int chunk = cands[k];
        if (chunk > 2 * n_ps && k > 0) break;
        bioem_batch b{};
        b.ctx = ctx;
        b.n_models = 1;
        b.n_stacks = 1;
        SegDesc sd{};
        sd.img = images->d_spec;
        sd.ps = projset->d_spec;
        sd.gtw = bioem_twiddles(ctx, npix);
        sd.kA = images->d_kA;
        sd.kB = projset->d_kB;
        sd.rec_t = static_cast<float*>(rec);
        sd.rec_s = sd.rec_t + (size_t)n_img * n_ps;
        sd.rec_d = reinterpret_cast<int*>(sd.rec_s + (size_t)n_img * n_ps);
        sd.n_img = n_img;
        sd.n_ps = n_ps;
        sd.chunk = chunk;
        sd.n_chunks = (n_ps + chunk - 1) / chunk;
        sd.s = max_shift;
        sd.npix = npix;
        sd.nctf = projset->nctf;
        sd.c1 = 0.5f * (3.0f - (float)(npix * npix));
        sd.log_norm = 0.0;
        b.n_items = (long long)sd.n_chunks * n_img;
        b.segs.push_back(sd);
        SegDesc* d_seg = nullptr;
        if (cudaMalloc((void**)&d_seg, sizeof(SegDesc)) != cudaSuccess) { rc = BIOEM_ERR_OOM; break; }
        cudaMemcpy(d_seg, &sd, sizeof(SegDesc), cudaMemcpyHostToDevice);
        cudaFuncSetAttribute(k_score_multi, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMultiSmem);
        const int grid = (int)(b.n_items < ctx->num_sms ? b.n_items : ctx->num_sms);
        double ms_best_rep = 1e300;
        for (int rep = 0; rep < 3; ++rep) {
            cudaEventRecord(e0, ctx->stream);
            cudaMemsetAsync(ctx->d_work, 0, sizeof(unsigned long long), ctx->stream);
            k_score_multi<<<grid, kMultiThreads, kMultiSmem, ctx->stream>>>(
                d_seg, 1, b.n_items, ctx->d_status, reinterpret_cast<unsigned long long*>(ctx->d_work));
            cudaEventRecord(e1, ctx->stream);
            if (cudaEventSynchronize(e1) != cudaSuccess) { rc = bioem_check_cuda(ctx, cudaGetLastError(), "autotune"); break; }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep > 0 && ms < ms_best_rep) ms_best_rep = ms;   // first repetition warms up
        }
        cudaFree(d_seg);
        if (ms_best_rep < best_ms) {
            best_ms = ms_best_rep;
            best = chunk;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(rec);
    if (rc) return rc;
    {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        bool found = false;
        for (auto& e : g_tune)
            if (e.npix == npix && e.s == max_shift) { e.chunk = best; found = true; }
        if (!found) g_tune.push_back({npix, max_shift, best});
        if (cache_path) {
            FILE* f = fopen(cache_path, "w");
            if (f) {
                for (const auto& e : g_tune) fprintf(f, "%d %d %d\n", e.npix, e.s, e.chunk);
                fclose(f);
            }
        }
    }
    if (out_chunk) *out_chunk = best;
    return BIOEM_OK;
}

int bioem_batch_create(bioem_ctx* ctx, int n_models, int n_stacks, const bioem_images* const* stacks,
                       const bioem_projset* const* projsets, const int* max_shift, float* d_logP_matrix,
                       bioem_batch** out) {
    if (!ctx || !out || n_models <= 0 || n_stacks <= 0 || !stacks || !projsets || !max_shift || !d_logP_matrix)
        return BIOEM_ERR_INVALID_ARG;
    *out = nullptr;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return bioem_set_error(ctx, BIOEM_ERR_CUDA, "cudaSetDevice");
    bioem_batch* b = new (std::nothrow) bioem_batch();
    if (!b) return BIOEM_ERR_OOM;
    b->ctx = ctx;
    b->device = ctx->device;
    b->stream = ctx->stream;
    b->n_models = n_models;
    b->n_stacks = n_stacks;
    b->d_out = d_logP_matrix;
    int col = 0;
    size_t rec_total = 0;
    std::vector<int> cols(n_stacks);
    for (int k = 0; k < n_stacks; ++k) {
        const bioem_images* im = stacks[k];
        if (!im || im->ctx != ctx) { delete b; return bioem_set_error(ctx, BIOEM_ERR_INVALID_ARG, "stack %d", k); }
        const int npix = im->nx;
        if ((npix != 64 && npix != 96 && npix != 128 && npix != 192) || max_shift[k] < 0 ||
            max_shift[k] > multi_smax(npix) || 2 * max_shift[k] >= npix) {
            delete b;
            return bioem_set_error(ctx, BIOEM_ERR_UNSUPPORTED_SIZE, "stack %d: %d px, shift %d", k, npix, max_shift[k]);
        }
        cols[k] = col;
        col += im->n_img;
    }
    b->n_cols = col;
    long long items = 0, rows = 0;
    for (int m = 0; m < n_models; ++m) {
        for (int k = 0; k < n_stacks; ++k) {
            const bioem_images* im = stacks[k];
            const bioem_projset* ps = projsets[(size_t)m * n_stacks + k];
            if (!ps || ps->ctx != ctx || ps->nx != im->nx || fabs(ps->pixel_A - im->pixel_A) > 1e-9 * im->pixel_A ||
                ps->n_ps == 0) {
                delete b;
                return bioem_set_error(ctx, BIOEM_ERR_INVALID_ARG, "projection set (%d, %d) does not match", m, k);
            }
            if (im->n_img == 0) continue;
            SegDesc sd{};
            sd.img = im->d_spec;
            sd.ps = ps->d_spec;
            sd.gtw = bioem_twiddles(ctx, im->nx);
            sd.kA = im->d_kA;
            sd.kB = ps->d_kB;
            sd.n_img = im->n_img;
            sd.n_ps = ps->n_ps;
            {
                std::lock_guard<std::mutex> lock(g_tune_mutex);
                sd.chunk = tuned_chunk(g_tune, im->nx, max_shift[k]);
            }
            sd.n_chunks = (sd.n_ps + sd.chunk - 1) / sd.chunk;
            sd.s = max_shift[k];
            sd.npix = im->nx;
            sd.nctf = ps->nctf;
            sd.out_row = m;
            sd.out_col = cols[k];
            sd.c1 = 0.5f * (3.0f - (float)(im->nx * im->nx));
            const int S = (2 * max_shift[k] + 1) * (2 * max_shift[k] + 1);
            sd.log_norm = log((double)ps->n_ps * S);
            sd.item_begin = items;
            sd.row_begin = rows;
            items += (long long)sd.n_chunks * sd.n_img;
            rows += sd.n_img;
            rec_total += (size_t)sd.n_img * sd.n_ps * 12;
            b->segs.push_back(sd);
        }
    }
    b->n_items = items;
    b->n_rows = rows;
    if (b->segs.empty()) { delete b; return bioem_set_error(ctx, BIOEM_ERR_INVALID_ARG, "no images"); }
    if (rows > 0x7fffffffll) { delete b; return bioem_set_error(ctx, BIOEM_ERR_UNSUPPORTED_SIZE, "too many rows"); }
    if (cudaMalloc(&b->d_rec, rec_total) != cudaSuccess) {
        delete b;
        return bioem_set_error(ctx, BIOEM_ERR_OOM, "batch records of %zu bytes", rec_total);
    }
    size_t off = 0;
    for (auto& sd : b->segs) {
        const size_t npair = (size_t)sd.n_img * sd.n_ps;
        float* base = reinterpret_cast<float*>(static_cast<unsigned char*>(b->d_rec) + off);
        sd.rec_t = base;
        sd.rec_s = base + npair;
        sd.rec_d = reinterpret_cast<int*>(base + 2 * npair);
        off += npair * 12;
    }
    const int rc = batch_build(b, 0);
    if (rc) {
        bioem_batch_free(b);
        return rc;
    }
    *out = b;
    return BIOEM_OK;
}

int bioem_batch_run(bioem_batch* b) {
    if (!b) return BIOEM_ERR_INVALID_ARG;
    bioem_ctx* ctx = b->ctx;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return bioem_set_error(ctx, BIOEM_ERR_CUDA, "cudaSetDevice");
    ctx->n_launches += 2;
    ctx->kid_launches[KID_SCORE] += 1;
    ctx->kid_launches[KID_REDUCE_WAVE] += 1;
    return bioem_check_cuda(ctx, cudaGraphLaunch(b->exec, ctx->stream), "graph launch");
}

long long bioem_batch_evals(const bioem_batch* b) {
    if (!b) return -1;
    long long e = 0;
    for (const auto& sd : b->segs) e += (long long)sd.n_img * sd.n_ps;
    return e;
}

void bioem_batch_free(bioem_batch* b) {
    if (!b) return;
    cudaSetDevice(b->device);
    cudaStreamSynchronize(b->stream);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    if (b->d_segs) cudaFree(b->d_segs);
    if (b->d_rec) cudaFree(b->d_rec);
    if (b->d_work) cudaFree(b->d_work);
    cudaGetLastError();
    delete b;
}

}  // extern "C"

// ---------------------------------------------------------------------------- gathered scoring
// Each image against its own list of parameter sets (CSR: offsets[n_img + 1], ps_idx[nnz] into the
// projection set), folded into running per-image float64 (max, sum) accumulators.
namespace {

template <class C>
__global__ void __launch_bounds__(C::THREADS, 1)
k_score_gathered(const float2* __restrict__ gtw, const float2* __restrict__ img_spec, int n_img,
                 const int* __restrict__ offsets, const int* __restrict__ ps_idx, const float2* __restrict__ ps_spec,
                 int chunk, int chunks_per_img, int s, float c1, float* __restrict__ rec_t, float* __restrict__ rec_s,
                 int* __restrict__ rec_d, int* __restrict__ status) {
    extern __shared__ __align__(16) unsigned char smem[];
    const long long n_items = (long long)n_img * chunks_per_img;
    for (long long item = blockIdx.x; item < n_items; item += gridDim.x) {
        const int ci = (int)(item / n_img);
        const int w = (int)(item - (long long)ci * n_img);
        const int b0 = offsets[w], b1 = offsets[w + 1];
        const int lo = ci * chunk;
        const int hi = min(lo + chunk, b1 - b0);
        if (lo >= hi) continue;   // uniform across the block: no barrier is skipped by a subset
        score_item<C>(smem, gtw, img_spec + (size_t)w * C::N * C::H, ps_idx + b0, ps_spec, 0, lo, hi, s, c1,
                      rec_t + b0, rec_s + b0, rec_d + b0, status);
    }
}

__global__ void __launch_bounds__(kRedThreads) k_fold_gathered(const int* __restrict__ offsets,
                                                               const int* __restrict__ ps_idx,
                                                               const float* __restrict__ rec_t,
                                                               const float* __restrict__ rec_s,
                                                               const double* __restrict__ kA,
                                                               const double* __restrict__ kB, double c1,
                                                               double* __restrict__ acc, int first) {
    __shared__ double redM[kRedThreads], redS[kRedThreads];
    const int w = blockIdx.x;
    const int b0 = offsets[w], b1 = offsets[w + 1];
    double M = -INFINITY, S = 0.0;
    for (int i = b0 + threadIdx.x; i < b1; i += blockDim.x) {
        const double m = kA[w] + kB[ps_idx[i]] + c1 * (double)rec_t[i];
        const double sv = rec_s[i];
        if (!(m > -INFINITY)) continue;
        if (m > M) { S = S * exp(M - m) + sv; M = m; }
        else S += sv * exp(m - M);
    }
    redM[threadIdx.x] = M;
    redS[threadIdx.x] = S;
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if (threadIdx.x < st) {
            const double m2 = redM[threadIdx.x + st], s2 = redS[threadIdx.x + st];
            double m1 = redM[threadIdx.x], s1 = redS[threadIdx.x];
            if (m2 > -INFINITY) {
                if (m2 > m1) { s1 = s1 * exp(m1 - m2) + s2; m1 = m2; }
                else s1 += s2 * exp(m2 - m1);
            }
            redM[threadIdx.x] = m1;
            redS[threadIdx.x] = s1;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        double m1 = redM[0], s1 = redS[0];
        if (!first) {
            const double m2 = acc[2 * w], s2 = acc[2 * w + 1];
            if (m2 > -INFINITY) {
                if (m2 > m1) { s1 = s1 * exp(m1 - m2) + s2; m1 = m2; }
                else s1 += s2 * exp(m2 - m1);
            }
        }
        acc[2 * w] = m1;
        acc[2 * w + 1] = s1;
    }
}

__global__ void k_acc_logP(const double* __restrict__ acc, int n_img, double log_norm, double* __restrict__ logP) {
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w < n_img) logP[w] = acc[2 * w] + log(acc[2 * w + 1]) - log_norm;
}

// Eq. 9's sum over disjoint parts of a grid: out[w] = the (M, S) pair of the union of the n_parts
// accumulators parts[k][w] (each ln sum L = M + ln S; an empty part has M = -inf), folded in index
// order k = 0, 1, ... so the result does not depend on the launch.  out may be parts (part 0).
__global__ void k_acc_merge(const double* __restrict__ parts, int n_parts, int n, double* out) {
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= n) return;
    double M = -INFINITY, S = 0.0;
    for (int k = 0; k < n_parts; ++k) {
        const double m2 = parts[((size_t)k * n + w) * 2], s2 = parts[((size_t)k * n + w) * 2 + 1];
        if (!(m2 > -INFINITY)) continue;
        if (m2 > M) { S = S * exp(M - m2) + s2; M = m2; }
        else S += s2 * exp(m2 - M);
    }
    out[2 * w] = M;
    out[2 * w + 1] = S;
}

// out[g] = ln sum_j exp(v[g len + j]) for consecutive groups of len values (a sum of Eq. 9 over a
// few grid points, e.g. the B-factors of one orientation and defocus), max-shifted in float64.
__global__ void k_group_lse(const double* __restrict__ v, long long n_groups, int len, double* __restrict__ out) {
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < n_groups;
         g += (long long)gridDim.x * blockDim.x) {
        const double* x = v + g * len;
        double m = -INFINITY;
        for (int j = 0; j < len; ++j) m = fmax(m, x[j]);
        if (!(m > -INFINITY)) {
            out[g] = m;
            continue;
        }
        double s = 0.0;
        for (int j = 0; j < len; ++j) s += exp(x[j] - m);
        out[g] = m + log(s);
    }
}

// Per listed pair i of image w: ln sum_d L(w | ps_idx[i], d) = kA + kB + c1 t_min + ln s (one block per image).
__global__ void __launch_bounds__(kRedThreads) k_gathered_pairs_out(const int* __restrict__ offsets,
                                                                    const int* __restrict__ ps_idx,
                                                                    const float* __restrict__ rec_t,
                                                                    const float* __restrict__ rec_s,
                                                                    const double* __restrict__ kA,
                                                                    const double* __restrict__ kB, double c1,
                                                                    double* __restrict__ pair_lse) {
    const int w = blockIdx.x;
    const int b0 = offsets[w], b1 = offsets[w + 1];
    for (int i = b0 + threadIdx.x; i < b1; i += blockDim.x)
        pair_lse[i] = kA[w] + kB[ps_idx[i]] + c1 * (double)rec_t[i] + log((double)rec_s[i]);
}

template <class C>
int run_gathered(bioem_ctx* ctx, const bioem_images* im, const bioem_projset* ps, int max_shift, const int* offsets,
                 const int* ps_idx, int nnz, int max_per_image, double* acc, int first, double* pair_lse) {
    const int n_img = im->n_img;
    const size_t need = (size_t)nnz * 12;
    if (ctx->rec_bytes < need) {
        if (ctx->d_rec) cudaFreeAsync(ctx->d_rec, ctx->stream);
        ctx->d_rec = nullptr;
        ctx->rec_bytes = 0;
        if (cudaMallocAsync(&ctx->d_rec, need, ctx->stream) != cudaSuccess)
            return bioem_set_error(ctx, BIOEM_ERR_OOM, "record scratch of %zu bytes", need);
        ctx->rec_bytes = need;
    }
    float* rec_t = reinterpret_cast<float*>(ctx->d_rec);
    float* rec_s = rec_t + nnz;
    int* rec_d = reinterpret_cast<int*>(rec_s + nnz);
    const size_t smem = C::SMEM;
    if (cudaFuncSetAttribute(k_score_gathered<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return bioem_set_error(ctx, BIOEM_ERR_CUDA, "shared memory attribute");
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_score_gathered<C>, C::THREADS, smem);
    if (per_sm < 1) per_sm = 1;
    const int chunk = 256 / C::PB * C::PB;   // whole batches
    const int cpi = (max_per_image + chunk - 1) / chunk;
    const long long items = (long long)n_img * cpi;
    const int grid = (int)(items < (long long)per_sm * ctx->num_sms ? items : (long long)per_sm * ctx->num_sms);
    const int n = C::N * C::N;
    if (grid > 0) {
        bioem_launch_begin(ctx, KID_SCORE);
        k_score_gathered<C><<<grid, C::THREADS, smem, ctx->stream>>>(bioem_twiddles(ctx, C::N), im->d_spec, n_img, offsets,
                                                                     ps_idx, ps->d_spec, chunk, cpi, max_shift,
                                                                     0.5f * (3.0f - (float)n), rec_t, rec_s, rec_d,
                                                                     ctx->d_status);
        bioem_launch_end(ctx, KID_SCORE);
        int rc = bioem_check_cuda(ctx, cudaGetLastError(), "k_score_gathered");
        if (rc) return rc;
    }
    bioem_launch_begin(ctx, KID_REDUCE_WAVE);
    if (pair_lse)
        k_gathered_pairs_out<<<n_img, kRedThreads, 0, ctx->stream>>>(offsets, ps_idx, rec_t, rec_s, im->d_kA, ps->d_kB,
                                                                    0.5 * (3.0 - (double)n), pair_lse);
    else
        k_fold_gathered<<<n_img, kRedThreads, 0, ctx->stream>>>(offsets, ps_idx, rec_t, rec_s, im->d_kA, ps->d_kB,
                                                               0.5 * (3.0 - (double)n), acc, first);
    bioem_launch_end(ctx, KID_REDUCE_WAVE);
    return bioem_check_cuda(ctx, cudaGetLastError(), "k_fold_gathered");
}

}  // namespace

extern "C" {

static int gathered(bioem_ctx* ctx, const bioem_images* images, const bioem_projset* projset, int max_shift,
                    const int* d_offsets, const int* d_ps_idx, int nnz, int max_per_image, double* d_acc, int first,
                    double* d_pair_lse) {
    if (!ctx || !images || !projset || !d_offsets || (!d_acc && !d_pair_lse) || nnz < 0 || max_per_image < 0 ||
        (nnz > 0 && !d_ps_idx))
        return BIOEM_ERR_INVALID_ARG;
    if (images->ctx != ctx || projset->ctx != ctx || images->nx != projset->nx)
        return bioem_set_error(ctx, BIOEM_ERR_INVALID_ARG, "images and projections do not match");
    if (!bioem_score_supported(images->nx, max_shift))
        return bioem_set_error(ctx, BIOEM_ERR_UNSUPPORTED_SIZE, "max_shift %d unsupported at %d px", max_shift,
                               images->nx);
    if (images->n_img == 0) return BIOEM_OK;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return bioem_set_error(ctx, BIOEM_ERR_CUDA, "cudaSetDevice");
#define G(C) run_gathered<C>(ctx, images, projset, max_shift, d_offsets, d_ps_idx, nnz, max_per_image, d_acc, first, d_pair_lse)
    switch (images->nx) {
        case 32: return G(C32_4);
        case 64: return max_shift <= 4 ? G(C64_4) : G(C64_8);
        case 96: return G(C96_12);
        case 128: return max_shift <= 4 ? G(C128_4) : G(C128_16);
        default: return G(C192_24);
    }
#undef G
}

int bioem_score_gathered(bioem_ctx* ctx, const bioem_images* images, const bioem_projset* projset, int max_shift,
                         const int* d_offsets, const int* d_ps_idx, int nnz, int max_per_image, double* d_acc,
                         int first) {
    if (!d_acc) return BIOEM_ERR_INVALID_ARG;
    return gathered(ctx, images, projset, max_shift, d_offsets, d_ps_idx, nnz, max_per_image, d_acc, first, nullptr);
}

int bioem_score_gathered_pairs(bioem_ctx* ctx, const bioem_images* images, const bioem_projset* projset, int max_shift,
                               const int* d_offsets, const int* d_ps_idx, int nnz, int max_per_image,
                               double* d_pair_lse) {
    if (!d_pair_lse && nnz > 0) return BIOEM_ERR_INVALID_ARG;
    if (nnz == 0) return BIOEM_OK;
    return gathered(ctx, images, projset, max_shift, d_offsets, d_ps_idx, nnz, max_per_image, nullptr, 0, d_pair_lse);
}

int bioem_acc_merge(bioem_ctx* ctx, const double* d_parts, int n_parts, int n, double* d_out) {
    if (!ctx || n_parts < 1 || n < 0 || (n > 0 && (!d_parts || !d_out))) return BIOEM_ERR_INVALID_ARG;
    if (n == 0) return BIOEM_OK;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return bioem_set_error(ctx, BIOEM_ERR_CUDA, "cudaSetDevice");
    bioem_launch_begin(ctx, KID_LSE_MERGE);
    k_acc_merge<<<(n + 255) / 256, 256, 0, ctx->stream>>>(d_parts, n_parts, n, d_out);
    bioem_launch_end(ctx, KID_LSE_MERGE);
    return bioem_check_cuda(ctx, cudaGetLastError(), "k_acc_merge");
}

int bioem_group_logsumexp(bioem_ctx* ctx, const double* d_values, long long n_groups, int group_len, double* d_out) {
    if (!ctx || n_groups < 0 || group_len < 1 || (n_groups > 0 && (!d_values || !d_out))) return BIOEM_ERR_INVALID_ARG;
    if (n_groups == 0) return BIOEM_OK;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return bioem_set_error(ctx, BIOEM_ERR_CUDA, "cudaSetDevice");
    const long long blocks = (n_groups + 255) / 256;
    bioem_launch_begin(ctx, KID_LSE_MERGE);
    k_group_lse<<<(unsigned)(blocks < 4096 ? blocks : 4096), 256, 0, ctx->stream>>>(d_values, n_groups, group_len, d_out);
    bioem_launch_end(ctx, KID_LSE_MERGE);
    return bioem_check_cuda(ctx, cudaGetLastError(), "k_group_lse");
}

__global__ void k_ln1m(const float* __restrict__ x, long long n, float* __restrict__ t) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        t[i] = ln1m(x[i]);
}

int bioem_ln1m(bioem_ctx* ctx, const float* d_x, long long n, float* d_t) {
    if (!ctx || n < 0 || (n > 0 && (!d_x || !d_t))) return BIOEM_ERR_INVALID_ARG;
    if (n == 0) return BIOEM_OK;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return bioem_set_error(ctx, BIOEM_ERR_CUDA, "cudaSetDevice");
    const long long blocks = (n + 255) / 256;
    bioem_launch_begin(ctx, KID_LSE_MERGE);
    k_ln1m<<<(unsigned)(blocks < 4096 ? blocks : 4096), 256, 0, ctx->stream>>>(d_x, n, d_t);
    bioem_launch_end(ctx, KID_LSE_MERGE);
    return bioem_check_cuda(ctx, cudaGetLastError(), "k_ln1m");
}

int bioem_acc_logP(bioem_ctx* ctx, const double* d_acc, int n_img, double log_norm, double* d_logP) {
    if (!ctx || (n_img > 0 && (!d_acc || !d_logP)) || n_img < 0) return BIOEM_ERR_INVALID_ARG;
    if (n_img == 0) return BIOEM_OK;
    cudaSetDevice(ctx->device);
    bioem_launch_begin(ctx, KID_FINALIZE);
    k_acc_logP<<<(n_img + 255) / 256, 256, 0, ctx->stream>>>(d_acc, n_img, log_norm, d_logP);
    bioem_launch_end(ctx, KID_FINALIZE);
    return bioem_check_cuda(ctx, cudaGetLastError(), "k_acc_logP");
}

}  // extern "C"
