// Scoring with the column transforms on the fifth-generation tensor cores (128 px images,
// displacements |dx|, |dy| <= 16): the FP32 scoring form's two-stage pruned inverse transform
// (Sec. 3.3, Eqs. 11-12; Sec. 3.9 and Sec. 5 on evaluating only the wanted coefficients), with its
// first stage (along ky, per column kx) written as a matrix product and run by tcgen05 MMAs:
//
//   Q(dy, kx) = sum_ky E(dy, ky) P(ky, kx),   E(dy, ky) = exp(+2 pi i ky dy / N),
//   P(ky, kx) = conj(O(ky, kx)) C(ky, kx)     (the Fourier product of Eq. 11)
//
// as a real product D = A B over K = (ky, re/im) = 256 terms, for the 32 rows dy != 0.  Both
// operands are split into two 16-bit floats (x = hi + lo, FP16 scaled by powers of two), and the
// 128 rows of A stack E_hi and E_lo:
//   row 4 i + 2 h + c:  (dy_i, c = Re / Im, h = 0: E_hi, 1: E_lo),   dy_i = i - 16 (i < 16), i - 15
// Two MMAs per K step, against P_hi and P_lo, give D[.., h = 0] + D[.., h = 1] = all four split
// products E P with FP32 accumulation.  The N = 256 columns are four pairs x 64 columns: kx = 1..63
// and, in column 0, the packed edge columns Z = P(., 0) + i P(., N/2) (both Hermitian in ky, so the
// two real rows of Q(dy, 0) and Q(dy, N/2) come out as the real and imaginary part).
//
// CUDA cores do the rest:
//   * products P (FP32, the image spectrum in shared memory scaled by 2^e, the projection read
//     once from L2) split into hi / lo and written in the tensor cores' K-major layout, 16 ky at a
//     time, into a two-stage ring the MMAs consume; the dy = 0 row Q(0, kx) = sum_ky P is summed
//     by the same threads in FP32;
//   * stage B along kx per row from tensor memory: after the hi / lo halves are exchanged between
//     lane pairs, each lane evaluates one real component c of its row over half of the eight kx
//     sub-sequences kx = b + 8 a,  C(dx) = sum w Re Q cos(2 pi kx dx / N) (even in dx) or
//     S(dx) = sum w Im Q sin(...) (odd), with a real 16-point transform per sub-sequence and the
//     17 wanted outputs dx = 0..16 recombined, so rho(dy, +-dx) = C(dx) -+ S(dx) + (-1)^dx Q(dy, N/2);
//   * the likelihood epilogue (closed form of Eq. 8 integrated over N, mu, lambda) and the per-pair
//     log-sum-exp records (t_min, sum exp, argmin) the float64 reductions of score.cu consume.
//
// Layout: one CTA of 512 threads per SM, persistent over (chunk of parameter sets, image) items in
// index order from a global counter.  Per group of four pairs the threads produce eight K chunks
// (each followed by one barrier, after which thread 0 issues that chunk's four MMAs), then run the
// epilogue of the previous group, whose accumulator (one of two 256-column halves of tensor memory)
// the MMAs finished meanwhile.  Every barrier wait is bounded in time; on expiry the kernel sets a
// status bit, leaves its loops together, waits for its MMAs and frees its tensor memory.
#include <math.h>

#include <cuda_fp16.h>

#include "bioem_internal.cuh"
#include "tc_util.cuh"
#include "rdft16.cuh"

namespace {

namespace tcs {
constexpr int N = 128, NC = 64, H = 65;
constexpr int SMAX = 16, NS = 2 * SMAX + 1;
constexpr int THREADS = 512;
constexpr int PG = 4;              // pairs per group (MMA N = 4 x 64 columns)
constexpr int KCH = 8;             // K chunks of 16 ky per group
constexpr int IMG_LD = 66;         // float2 per image row in shared memory: 64 columns, Nyquist, pad
constexpr float E_SCALE = 1024.f;  // A operand scale (keeps the lo parts normal)
constexpr uint32_t A_CHUNK = 128 * 32 * 2;   // one K chunk of A: 128 rows x 32 K x FP16 = 8 KB
constexpr uint32_t B_TERM = 256 * 32 * 2;    // one term (hi or lo) of a ring stage: 16 KB
constexpr size_t OFF_E = 0;                                   // 8 chunks x 8 KB
constexpr size_t OFF_RING = OFF_E + 8 * A_CHUNK;              // 2 stages x (hi, lo)
constexpr size_t OFF_IMG = OFF_RING + 4 * (size_t)B_TERM;     // [128][66] float2
constexpr size_t OFF_R0P = OFF_IMG + (size_t)N * IMG_LD * 8;  // [4 pairs][4 kg][64 kx] float2
constexpr size_t OFF_R0 = OFF_R0P + 4 * 4 * 64 * 8;           // [2 groups][4 pairs][64 kx] float2
constexpr size_t OFF_P64 = OFF_R0 + 2 * 4 * 64 * 8;           // [4 pairs][128 ky] float2
constexpr size_t OFF_TW = OFF_P64 + 4 * 128 * 8;              // [2 c][8 b][17 dx] float2
constexpr size_t OFF_DY0 = OFF_TW + 2 * 8 * 17 * 8;           // [4 pairs][4 q][2 bsel][2 c][17] float
constexpr size_t OFF_PART = OFF_DY0 + 4 * 4 * 2 * 2 * 17 * 4; // [4 pairs][4 q] parts
constexpr size_t OFF_NYQ0 = OFF_PART + 4 * 4 * 16;            // [4 pairs] float
constexpr size_t SMEM = OFF_NYQ0 + 64;
constexpr int TMEM_COLS = 512;                                 // two 256-column accumulators
static_assert(SMEM <= 227u * 1024u - 1024u, "dynamic shared memory per block");
static_assert(OFF_IMG % 16 == 0 && OFF_R0P % 16 == 0 && OFF_P64 % 16 == 0 && OFF_TW % 16 == 0, "alignment");
}  // namespace tcs

struct TcArgs {
    const float2* img_spec;   // [n_img][128][65]
    const float* img_amax;    // [n_img] largest |coefficient|
    int n_img;
    const float2* ps_spec;    // [n_ps][128][65]
    const float* ps_amax;     // [n_ps]
    int ps_begin, ps_count;   // the wave: sets [ps_begin, ps_begin + ps_count)
    int chunk, n_items, s;
    float c1;                 // (3 - n) / 2
    float* rec_t;             // [n_img][ps_count]
    float* rec_s;
    int* rec_d;
    int* status;
    int* work;
    long long skip_chunk;         // failure-detection test: thread 0 skips this chunk's MMAs (-1: none)
    unsigned long long wait_ns;   // limit of every barrier wait
};

struct TPart {
    float t;   // min ln(1 - rho^2)
    float s;   // sum exp(c1 (t(d) - t))
    int d;     // index of the minimum, (dy + 16) * 33 + (dx + 16)
};

__device__ __forceinline__ TPart tmerge(TPart a, TPart b, float c1) {
    if (b.t > a.t || (b.t == a.t && b.d > a.d)) {
        const TPart x = a;
        a = b;
        b = x;
    }
    if (!(a.t < INFINITY)) return b;
    return TPart{b.t, b.s + a.s * __expf(c1 * (a.t - b.t)), b.d};
}

__device__ __forceinline__ TPart warp_merge(TPart p, float c1) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        TPart o;
        o.t = __shfl_xor_sync(0xffffffffu, p.t, off);
        o.s = __shfl_xor_sync(0xffffffffu, p.s, off);
        o.d = __shfl_xor_sync(0xffffffffu, p.d, off);
        p = tmerge(p, o, c1);   // tmerge orders its operands, so both lanes agree
    }
    return p;
}

__device__ __forceinline__ float tc_loglik(float rho, int* status) {
    float r2 = rho * rho;
    if (r2 >= 1.0f) {
        atomicOr(status, BIOEM_DEV_NUMERIC);
        r2 = 1.0f - 5.9604645e-8f;
    }
    return ln1m(r2);
}

__device__ __forceinline__ uint32_t pack_half2(float a, float b) {
    const __half2 h = __floats2half2_rn(a, b);
    return *reinterpret_cast<const uint32_t*>(&h);
}

// (re, im) -> hi and lo half2 words: hi = round(v), lo = round(v - hi).
__device__ __forceinline__ void split_c(float2 v, uint32_t& hi, uint32_t& lo) {
    const __half2 h = __floats2half2_rn(v.x, v.y);
    const float2 hf = __half22float2(h);
    hi = *reinterpret_cast<const uint32_t*>(&h);
    lo = pack_half2(v.x - hf.x, v.y - hf.y);
}

// OR of a flag over the block at a barrier (every thread must call it).
__device__ __forceinline__ bool block_any(bool f) { return __syncthreads_or(f ? 1 : 0) != 0; }

__device__ __forceinline__ void proxy_fence_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Bounded wait on an mbarrier phase by any number of threads (false on expiry; raises the status bit).
__device__ __forceinline__ bool bwait(uint32_t bar, uint32_t parity, int* status, unsigned long long limit_ns) {
    if (mbar_try(bar, parity)) return true;
    const unsigned long long t0 = globaltimer();
    for (;;) {
        if (mbar_try(bar, parity)) return true;
        if (globaltimer() - t0 > limit_ns) {
            atomicOr(status, BIOEM_DEV_TIMEOUT);
            return false;
        }
    }
}

__global__ void __launch_bounds__(tcs::THREADS, 1) k_score_tc(const TcArgs g) {
    using namespace tcs;
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t bar_empty[2], bar_tfull[2], bar_drain;
    __shared__ uint32_t tmem_slot;
    __shared__ int s_item;
    __shared__ float s_red[THREADS / 32];

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    float2* sImg = reinterpret_cast<float2*>(smem + OFF_IMG);
    float2* sR0P = reinterpret_cast<float2*>(smem + OFF_R0P);
    float2* sR0 = reinterpret_cast<float2*>(smem + OFF_R0);
    float2* sP64 = reinterpret_cast<float2*>(smem + OFF_P64);
    float2* sTw = reinterpret_cast<float2*>(smem + OFF_TW);
    float* sDy0 = reinterpret_cast<float*>(smem + OFF_DY0);
    TPart* sPart = reinterpret_cast<TPart*>(smem + OFF_PART);
    float* sNyq0 = reinterpret_cast<float*>(smem + OFF_NYQ0);
    const uint32_t sbase = smem_u32(smem);

    // ---------------- set-up: barriers, tensor memory, the A operand (E stacked hi / lo), tables
    if (tid == 0) {
        for (int b = 0; b < 2; ++b) {
            mbar_init(smem_u32(&bar_empty[b]), 1);
            mbar_init(smem_u32(&bar_tfull[b]), 1);
        }
        mbar_init(smem_u32(&bar_drain), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    // A[r][k], r = 4 i + 2 h + c, k = 2 ky + part: c = 0 (Re Q): (E_re, -E_im); c = 1 (Im Q): (E_im, E_re),
    // x E_SCALE, split hi (h = 0) / lo (h = 1) in float64; K-major core-matrix layout per 32-K chunk.
    for (int idx = tid; idx < 128 * 256; idx += THREADS) {
        const int r = idx >> 8, k = idx & 255;
        const int i = r >> 2, h = (r >> 1) & 1, c = r & 1;
        const int dy = i < 16 ? i - 16 : i - 15;
        const int ky = k >> 1, part = k & 1;
        const int t = ((ky * dy) % N + N) % N;
        double sn, cs;
        sincospi(2.0 * (double)t / (double)N, &sn, &cs);
        const double v = (double)E_SCALE * (c == 0 ? (part == 0 ? cs : -sn) : (part == 0 ? sn : cs));
        const __half vh = __double2half(v);
        const __half val = h == 0 ? vh : __double2half(v - (double)__half2float(vh));
        const int kc = k >> 5, kk = k & 31;
        const size_t off = OFF_E + (size_t)kc * A_CHUNK + (size_t)(r >> 3) * 512 + (kk >> 3) * 128 + (r & 7) * 16 +
                           (kk & 7) * 2;
        *reinterpret_cast<__half*>(smem + off) = val;
    }
    // stage-B recombination table: (c, b, dx) -> (T1, T2) x 2 (weight of kx != 0) / E_SCALE
    for (int idx = tid; idx < 2 * 8 * 17; idx += THREADS) {
        const int c = idx / (8 * 17), b = (idx / 17) % 8, dx = idx % 17;
        const int u = dx & 15;
        const bool cj = u > 8;
        double sn, cs;
        sincospi(2.0 * (double)((b * dx) % N) / (double)N, &sn, &cs);
        const double f = 2.0 / (double)E_SCALE;
        const double t1 = c == 0 ? cs : sn;
        const double t2 = c == 0 ? (cj ? sn : -sn) : (cj ? -cs : cs);
        sTw[idx] = make_float2((float)(f * t1), (float)(f * t2));
    }
    proxy_fence_async();   // the A operand was written by the generic proxy
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;

    // producer identity: pairs 2 pp, 2 pp + 1 of a group; column kx = b + 8 a (tensor column n = 8 b + a)
    const int pp = tid >> 8;
    const int w8 = (tid & 255) >> 5;
    const int kg = w8 >> 1;                  // 4 consecutive ky at 4 kg within a 16-ky chunk
    const int pa = lane & 7, pb = (lane >> 3) + 4 * (w8 & 1);
    const int pkx = pb + 8 * pa, pn = 8 * pb + pa;
    const bool pz = pkx == 0;                // the packed edge column
    // epilogue identity: warp w reads lane quarter q of pair jj; lane = 4 i' + 2 h + c
    const int eq = warp & 3, ejj = warp >> 2;
    const int eh = (lane >> 1) & 1, ec = lane & 1;
    const int ei = 8 * eq + (lane >> 2);
    const int edy = ei < 16 ? ei - 16 : ei - 15;
    const uint32_t idesc = (1u << 4) | ((uint32_t)(256 >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);

    uint32_t cc = 0;   // K chunks produced (ring position)
    uint32_t gg = 0;   // groups produced (accumulator position)
    bool fail = false;

    for (;;) {
        if (tid == 0) s_item = atomicAdd(g.work, 1);
        __syncthreads();
        const int item = s_item;
        if (item >= g.n_items) break;
        const int ci = item / g.n_img;
        const int w = item - ci * g.n_img;
        const int lo = ci * g.chunk;
        const int hi = min(lo + g.chunk, g.ps_count);
        const int n_groups = (hi - lo + PG - 1) / PG;
        // ---- scale 2^e: |P| <= 2 amax(img) max amax(ps) (x 2 for the packed column) below 2^15
        float m = 0.f;
        for (int p = lo + tid; p < hi; p += THREADS) m = fmaxf(m, __ldg(g.ps_amax + g.ps_begin + p));
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
        if (lane == 0) s_red[warp] = m;
        __syncthreads();
        m = 0.f;
#pragma unroll
        for (int k = 0; k < THREADS / 32; ++k) m = fmaxf(m, s_red[k]);
        const float bound = 2.f * __ldg(g.img_amax + w) * m;
        int ex = 0;
        if (bound > 0.f && isfinite(bound)) {
            frexpf(bound, &ex);
            ex = 15 - ex;
        }
        const float scale = ldexpf(1.f, ex), inv_scale = ldexpf(1.f, -ex);
        // ---- the image spectrum, scaled, columns permuted (kx = b + 8 a at n = 8 b + a; Nyquist at 64)
        const float2* img = g.img_spec + (size_t)w * N * H;
        for (int i = tid; i < N * H; i += THREADS) {
            const int ky = i / H, kx = i - (i / H) * H;
            const int n = kx == NC ? NC : 8 * (kx & 7) + (kx >> 3);
            const float2 v = __ldg(img + i);
            sImg[ky * IMG_LD + n] = make_float2(v.x * scale, v.y * scale);
        }
        // products of the Nyquist column for group 0: P64[j][ky] = conj(O(ky, 64)) C_j(ky, 64)
        {
            const int j = tid >> 7, ky = tid & 127;
            const int p = min(lo + j, hi - 1);
            const float2 cv = __ldg(g.ps_spec + (size_t)(g.ps_begin + p) * N * H + (size_t)ky * H + NC);
            const float2 o = __ldg(img + (size_t)ky * H + NC);
            sP64[j * 128 + ky] = c_mulc(make_float2(o.x * scale, o.y * scale), cv);
        }
        __syncthreads();

        for (int gi = 0; gi <= n_groups && !fail; ++gi) {
            const int p0 = lo + gi * PG;
            if (gi < n_groups) {
                // ================= production of group gi (8 K chunks into the ring)
                const uint32_t buf = gg & 1;
                float2 r0[2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
                const float2* psrc[2];
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    const int p = min(p0 + 2 * pp + q, hi - 1);
                    psrc[q] = g.ps_spec + (size_t)(g.ps_begin + p) * N * H + pkx;
                }
#pragma unroll 1
                for (int c = 0; c < KCH; ++c, ++cc) {
                    const uint32_t s = cc & 1;
                    bool ok = true;
                    if (cc >= 2) ok = bwait(smem_u32(&bar_empty[s]), ((cc >> 1) - 1) & 1, g.status, g.wait_ns);
                    if (ok) {
                        const int ky0 = 16 * c + 4 * kg;
                        float2 o[4];
#pragma unroll
                        for (int t4 = 0; t4 < 4; ++t4) o[t4] = sImg[(ky0 + t4) * IMG_LD + pn];
                        unsigned char* stage = smem + OFF_RING + (size_t)s * 2 * B_TERM;
#pragma unroll
                        for (int q = 0; q < 2; ++q) {
                            const int jj = 2 * pp + q;
                            float2 pv[4];
#pragma unroll
                            for (int t4 = 0; t4 < 4; ++t4) pv[t4] = c_mulc(o[t4], __ldg(psrc[q] + (ky0 + t4) * H));
                            if (pz) {
#pragma unroll
                                for (int t4 = 0; t4 < 4; ++t4) {
                                    const float2 z = sP64[jj * 128 + ky0 + t4];
                                    pv[t4] = make_float2(pv[t4].x - z.y, pv[t4].y + z.x);
                                }
                            }
                            uint4 h4, l4;
                            split_c(pv[0], h4.x, l4.x);
                            split_c(pv[1], h4.y, l4.y);
                            split_c(pv[2], h4.z, l4.z);
                            split_c(pv[3], h4.w, l4.w);
#pragma unroll
                            for (int t4 = 0; t4 < 4; ++t4) r0[q] = __fadd2_rn(r0[q], pv[t4]);
                            const size_t off = (size_t)jj * 4096 + pb * 512 + kg * 128 + pa * 16;
                            *reinterpret_cast<uint4*>(stage + off) = h4;
                            *reinterpret_cast<uint4*>(stage + B_TERM + off) = l4;
                        }
                    }
                    proxy_fence_async();
                    if (block_any(!ok)) {
                        fail = true;
                        break;
                    }
                    if (tid == 0 && (long long)cc != g.skip_chunk) {   // test: skipped chunk, no commit
                        tc_fence_after();
                        const uint32_t d = tmem + buf * 256;
                        const uint32_t a0 = sbase + (uint32_t)OFF_E + c * A_CHUNK;
                        const uint32_t b0 = sbase + (uint32_t)OFF_RING + s * 2 * B_TERM;
#pragma unroll
                        for (int j = 0; j < 2; ++j) {
                            const uint64_t ad = sdesc(a0 + j * 256, 128, 512);
                            umma(d, ad, sdesc(b0 + j * 256, 128, 512), idesc, (c == 0 && j == 0) ? 0u : 1u);
                            umma(d, ad, sdesc(b0 + B_TERM + j * 256, 128, 512), idesc, 1u);
                        }
                        umma_commit(smem_u32(&bar_empty[s]));
                        if (c == KCH - 1) umma_commit(smem_u32(&bar_tfull[buf]));
                    }
                }
                if (fail) break;
                // ---- group end: the dy = 0 row Q(0, kx) = sum_ky P, reduced over kg in a fixed order;
                // the Nyquist products of the next group
#pragma unroll
                for (int q = 0; q < 2; ++q) sR0P[((2 * pp + q) * 4 + kg) * 64 + pkx] = r0[q];
                if (gi + 1 < n_groups) {
                    const int j = tid >> 7, ky = tid & 127;
                    const int p = min(p0 + PG + j, hi - 1);
                    const float2 cv = __ldg(g.ps_spec + (size_t)(g.ps_begin + p) * N * H + (size_t)ky * H + NC);
                    sP64[j * 128 + ky] = c_mulc(sImg[ky * IMG_LD + NC], cv);
                }
                __syncthreads();
                if (tid < 256) {
                    const int j = tid >> 6, kx = tid & 63;
                    float2 v = sR0P[(j * 4 + 0) * 64 + kx];
                    v = __fadd2_rn(v, sR0P[(j * 4 + 1) * 64 + kx]);
                    v = __fadd2_rn(v, sR0P[(j * 4 + 2) * 64 + kx]);
                    v = __fadd2_rn(v, sR0P[(j * 4 + 3) * 64 + kx]);
                    sR0[(buf * 4 + j) * 64 + kx] = v;
                }
                ++gg;
            }
            if (gi == 0) continue;
            // ================= epilogue of group gi - 1 (accumulator buffer eb)
            const uint32_t eg = gg - 1 - (gi < n_groups ? 1 : 0);   // its group number
            const uint32_t eb = eg & 1;
            const int ep0 = lo + (gi - 1) * PG;
            const bool ok = bwait(smem_u32(&bar_tfull[eb]), (eg >> 1) & 1, g.status, g.wait_ns);
            tc_fence_after();
            float qv[32];
            {
                float v0[32], v1[32];
                const uint32_t ta = tmem + ((uint32_t)(32 * eq) << 16) + eb * 256 + ejj * 64;
                tmem_ld32(ta, v0);
                tmem_ld32(ta + 32, v1);
                tc_fence_before();
                // lane h keeps sub-sequences b = 4 h .. 4 h + 3 and adds its partner's (E_lo or E_hi) half
#pragma unroll
                for (int k = 0; k < 32; ++k) {
                    const float send = eh ? v0[k] : v1[k];
                    const float keep = eh ? v1[k] : v0[k];
                    qv[k] = keep + __shfl_xor_sync(0xffffffffu, send, 2);
                }
            }
            // column 0 holds (Q(dy, 0), Q(dy, N/2)): Q(dy, 0) has weight 1 (the table carries 2), the
            // Nyquist part enters as (-1)^dx Q(dy, N/2) below
            const float nyq = __shfl_sync(0xffffffffu, qv[0], (lane & ~3) | 1);
            qv[0] *= eh ? 1.f : (ec ? 0.f : 0.5f);
            float acc[17];
#pragma unroll
            for (int k = 0; k < 17; ++k) acc[k] = 0.f;
#pragma unroll
            for (int bb = 0; bb < 4; ++bb) {
                float x[8], yr[9], yi[9];
#pragma unroll
                for (int a = 0; a < 8; ++a) x[a] = qv[8 * bb + a];
                rdft16(x, yr, yi);
                recombine<17>(acc, yr, yi, sTw + (ec * 8 + 4 * eh + bb) * 17);
            }
            // ---- the dy = 0 row: lanes 0..3 of each warp take (c, b = 2 q + bsel) of pair jj
            if (lane < 4) {
                const int c0 = lane & 1, bs = lane >> 1;
                const int b0 = 2 * eq + bs;
                const float* r0v = reinterpret_cast<const float*>(sR0 + (eb * 4 + ejj) * 64);
                float x[8], yr[9], yi[9], a17[17];
#pragma unroll
                for (int a = 0; a < 8; ++a) x[a] = r0v[2 * (b0 + 8 * a) + c0];
                if (b0 == 0) {
                    if (c0) sNyq0[ejj] = x[0];
                    x[0] *= c0 ? 0.f : 0.5f;
                }
                rdft16(x, yr, yi);
#pragma unroll
                for (int k = 0; k < 17; ++k) a17[k] = 0.f;
                recombine<17>(a17, yr, yi, sTw + (c0 * 8 + b0) * 17);
                float* dst = sDy0 + (((ejj * 4 + eq) * 2 + bs) * 2 + c0) * 17;
#pragma unroll
                for (int k = 0; k < 17; ++k) dst[k] = a17[k];
            }
            // ---- rows dy != 0: h splits the outputs (h = 0: dx 0..8, h = 1: dx 9..16), c the sign of dx
            float mine[9];
#pragma unroll
            for (int k = 0; k < 9; ++k) {
                const float send = eh ? acc[k] : (k + 9 < 17 ? acc[k + 9] : 0.f);
                const float keep = eh ? (k + 9 < 17 ? acc[k + 9] : 0.f) : acc[k];
                mine[k] = keep + __shfl_xor_sync(0xffffffffu, send, 2);
            }
            const float nys = nyq * (1.f / E_SCALE);            // the table carries 1 / E_SCALE for the rest
            const float nq = ec ? 0.f : (eh ? -nys : nys);   // (-1)^dx Q(dy, N/2), dx = 9 h + k
#pragma unroll
            for (int k = 0; k < 9; ++k) mine[k] = fmaf((k & 1) ? -1.f : 1.f, nq, mine[k]);
            const float beta = ec ? 1.f : -1.f;
            const bool row_ok = abs(edy) <= g.s;
            TPart part{INFINITY, 0.f, 0x7fffffff};
            float tv[9];
#pragma unroll
            for (int k = 0; k < 9; ++k) {
                const float rho = fmaf(__shfl_xor_sync(0xffffffffu, mine[k], 1), beta, mine[k]) * inv_scale;
                const int dx = 9 * eh + k;
                const bool okk = row_ok && dx <= g.s && !(ec && dx == 0);
                tv[k] = okk ? tc_loglik(rho, g.status) : INFINITY;
                const int d = (edy + SMAX) * NS + (ec ? SMAX - dx : SMAX + dx);
                if (tv[k] < part.t || (tv[k] == part.t && d < part.d)) {
                    part.t = tv[k];
                    part.d = d;
                }
            }
            float ssum = 0.f;
#pragma unroll
            for (int k = 0; k < 9; ++k) ssum += (tv[k] < INFINITY) ? __expf(g.c1 * (tv[k] - part.t)) : 0.f;
            part.s = part.t < INFINITY ? ssum : 0.f;
            part = warp_merge(part, g.c1);
            if (block_any(!ok)) {   // also orders the dy = 0 partial sums before their readers
                fail = true;
                break;
            }
            // ---- the dy = 0 row's outputs: lane l < 9 of warp (jj, q) takes dx = 9 q + l - 16
            {
                TPart p0p{INFINITY, 0.f, 0x7fffffff};
                const int k = 9 * eq + lane;
                if (lane < 9 && k < NS) {
                    const int dxs = k - SMAX, dxa = abs(dxs);
                    float cs = 0.f, sn = 0.f;
#pragma unroll
                    for (int qq = 0; qq < 4; ++qq) {
#pragma unroll
                        for (int bs = 0; bs < 2; ++bs) {
                            const float* src = sDy0 + (((ejj * 4 + qq) * 2 + bs) * 2) * 17;
                            cs += src[dxa];
                            sn += src[17 + dxa];
                        }
                    }
                    const float ny = sNyq0[ejj];
                    const float rho = fmaf(cs - (dxs > 0 ? sn : -sn), E_SCALE, (dxa & 1) ? -ny : ny) * inv_scale;
                    const bool okk = dxa <= g.s;
                    p0p.t = okk ? tc_loglik(rho, g.status) : INFINITY;
                    p0p.s = okk ? 1.f : 0.f;
                    p0p.d = SMAX * NS + (dxs + SMAX);
                }
                p0p = warp_merge(p0p, g.c1);
                part = tmerge(part, p0p, g.c1);
            }
            if (lane == 0) sPart[ejj * 4 + eq] = part;
            __syncthreads();
            if (tid < PG) {
                const int p = ep0 + tid;
                if (p < hi) {
                    TPart r = sPart[tid * 4];
                    for (int qq = 1; qq < 4; ++qq) r = tmerge(r, sPart[tid * 4 + qq], g.c1);
                    const size_t o = (size_t)w * g.ps_count + p;
                    g.rec_t[o] = r.t;
                    g.rec_s[o] = r.s;
                    g.rec_d[o] = r.d;
                }
            }
        }
        if (fail) break;
    }
    // ---------------- teardown: every MMA issued has completed before tensor memory is released
    if (tid == 0) {
        umma_commit(smem_u32(&bar_drain));
        mbar_drain(smem_u32(&bar_drain), 0, g.wait_ns);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
}

}  // namespace

int bioem_tc_supported(int npix, int max_shift) { return npix == tcs::N && max_shift >= 0 && max_shift <= tcs::SMAX; }

// Records of sets [wbegin, wbegin + wl) of the wave for every image; chunking as the FP32 form's.
int bioem_tc_records(bioem_ctx* ctx, const bioem_images* im, const bioem_projset* ps, int max_shift, int wbegin,
                     int wl, float* rec_t, float* rec_s, int* rec_d) {
    using namespace tcs;
    const int n_img = im->n_img;
    if (wl <= 0 || n_img == 0) return BIOEM_OK;
    if (cudaFuncSetAttribute(k_score_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM) != cudaSuccess)
        return bioem_check_cuda(ctx, cudaGetLastError(), "tensor-core scoring shared memory attribute");
    const int slots = ctx->num_sms;   // one block per SM (shared memory and tensor memory)
    const long long per_img = (4ll * slots + n_img - 1) / n_img;
    long long chunk = (wl + per_img - 1) / per_img;
    chunk = ((chunk + PG - 1) / PG) * PG;
    if (chunk > 512) chunk = 512;
    if (chunk < PG) chunk = PG;
    const long long n_items = ((wl + chunk - 1) / chunk) * n_img;
    if (n_items > 0x7fffffffll) return bioem_set_error(ctx, BIOEM_ERR_UNSUPPORTED_SIZE, "too many work items");
    TcArgs a{};
    a.img_spec = im->d_spec;
    a.img_amax = im->d_amax;
    a.n_img = n_img;
    a.ps_spec = ps->d_spec;
    a.ps_amax = ps->d_amax;
    a.ps_begin = wbegin;
    a.ps_count = wl;
    a.chunk = (int)chunk;
    a.n_items = (int)n_items;
    a.s = max_shift;
    a.c1 = 0.5f * (3.0f - (float)(N * N));
    a.rec_t = rec_t;
    a.rec_s = rec_s;
    a.rec_d = rec_d;
    a.status = ctx->d_status;
    a.work = ctx->d_work;
    a.skip_chunk = ctx->test_skip_chunk;
    a.wait_ns = ctx->test_wait_ns ? ctx->test_wait_ns : kWaitNs;
    ctx->test_skip_chunk = -1;   // armed for one launch
    ctx->test_wait_ns = 0;
    const int grid = (int)(n_items < slots ? n_items : slots);
    bioem_launch_begin(ctx, KID_SCORE_TC);
    if (cudaMemsetAsync(ctx->d_work, 0, sizeof(int), ctx->stream) != cudaSuccess)
        return bioem_check_cuda(ctx, cudaGetLastError(), "work counter");
    k_score_tc<<<grid, THREADS, SMEM, ctx->stream>>>(a);
    bioem_launch_end(ctx, KID_SCORE_TC);
    return bioem_check_cuda(ctx, cudaGetLastError(), "k_score_tc");
}
