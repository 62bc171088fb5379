// Image preparation, model projection and PSF application (sm_103a).
//
//   k_prepare_images  per image: float64 moments C_o, C_oo (Sec. 3: precomputed image constants),
//                     zero-mean real-to-half-complex transform (Sec. 3.3: the observed images'
//                     transforms are precomputed once), unit-norm spectrum (C_oo by Plancherel).
//   k_project         per orientation: rotate the atoms by the quaternion (Sec. 3.1) and integrate
//                     each Gaussian atom over z and over every pixel (Eq. 1) into I0.
//   k_ctf_table       per PSF grid point: CTF(s) Env(s) on the half-spectrum grid (Eq. 4's forms).
//   k_psf_spectra     per orientation: transform I0, multiply by each PSF (Eq. 5), float64 moment
//                     B = n C_cc - C_c^2 (Plancherel), unit-norm spectrum per parameter set.
//   k_psf_real        the synthetic map I1 = F^-1[F(I0) CTF Env] in real space (Sec. 3.8).
//
// The forward transforms here use exp(-2 pi i k x / N).  For a real image this is the complex
// conjugate of Eq. 2's transform; the scoring kernel applies the matching inverse phase, so the
// correlation it evaluates is C_co(d) = sum_r o(r) I1(r + d) with d as in Eq. 7.  These
// transforms run once per image and once per orientation, so they are plain dense DFT sums over
// shared memory; the hot loop is the scoring kernel.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>

#include "bioem_internal.cuh"

namespace {

constexpr int kThreads = 256;

// Deterministic block sum of two doubles (fixed tree order).
__device__ void block_sum2(double& a, double& b, double* red) {
    const int tid = threadIdx.x;
    red[tid] = a;
    red[blockDim.x + tid] = b;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (tid < s) {
            red[tid] += red[tid + s];
            red[blockDim.x + tid] += red[blockDim.x + tid + s];
        }
        __syncthreads();
    }
    a = red[0];
    b = red[blockDim.x];
    __syncthreads();
}

// F[y][kx] = sum_x (img[y][x] - mean) W^(kx x), kx = 0..N/2 (row pass of a real 2-D transform).
template <int N>
__device__ void r2c_rows(const float* __restrict__ img, float mean, float2* F, const float2* tw) {
    constexpr int H = N / 2 + 1;
    for (int o = threadIdx.x; o < N * H; o += blockDim.x) {
        const int y = o / H, kx = o - y * H;
        const float* row = img + y * N;
        float re = 0.f, im = 0.f;
        int idx = 0;
#pragma unroll 8
        for (int x = 0; x < N; ++x) {
            const float v = row[x] - mean;
            const float2 w = tw[idx];
            re = fmaf(v, w.x, re);
            im = fmaf(v, w.y, im);
            idx += kx;
            idx -= (idx >= N) ? N : 0;
        }
        F[o] = make_float2(re, im);
    }
}

// In place over shared memory: F[ky][kx] <- sum_y F[y][kx] W^(ky y) (column pass), or with the
// conjugate twiddle when inverse is true.  Processed in blocks of columns so that every read of
// a column precedes every write to it.
template <int N, bool INVERSE>
__device__ void c2c_columns_inplace(float2* F, const float2* tw) {
    constexpr int H = N / 2 + 1;
    constexpr int CB = 8;                               // columns per block
    constexpr int PER = (N * CB + kThreads - 1) / kThreads;
    for (int c0 = 0; c0 < H; c0 += CB) {
        const int ncol = min(CB, H - c0);
        float2 res[PER];
#pragma unroll
        for (int i = 0; i < PER; ++i) {
            const int o = threadIdx.x + i * kThreads;
            res[i] = make_float2(0.f, 0.f);
            if (o < N * ncol) {
                const int ky = o / ncol, kx = c0 + (o - (o / ncol) * ncol);
                float re = 0.f, im = 0.f;
                int idx = 0;
#pragma unroll 8
                for (int y = 0; y < N; ++y) {
                    const float2 v = F[y * H + kx];
                    float2 w = tw[idx];
                    if (INVERSE) w.y = -w.y;
                    re = fmaf(v.x, w.x, fmaf(-v.y, w.y, re));
                    im = fmaf(v.x, w.y, fmaf(v.y, w.x, im));
                    idx += ky;
                    idx -= (idx >= N) ? N : 0;
                }
                res[i] = make_float2(re, im);
            }
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < PER; ++i) {
            const int o = threadIdx.x + i * kThreads;
            if (o < N * ncol) {
                const int ky = o / ncol, kx = c0 + (o - (o / ncol) * ncol);
                F[ky * H + kx] = res[i];
            }
        }
        __syncthreads();
    }
}

template <int N>
__device__ void load_twiddles(const float2* __restrict__ g_tw, float2* tw) {
    for (int i = threadIdx.x; i < N; i += blockDim.x) tw[i] = g_tw[i];
}

// Write F * T * scale (DC zeroed) to a [N][N/2 + 1] half spectrum; returns (to thread 0) the largest
// |coefficient| written (block reduction over red, which must hold blockDim.x floats).
template <int N>
__device__ float store_half_spectrum(const float2* F, const float* __restrict__ T, float scale,
                                     float2* __restrict__ spec, float* red) {
    constexpr int H = N / 2 + 1;
    float amax = 0.f;
    for (int o = threadIdx.x; o < N * H; o += blockDim.x) {
        float2 v = F[o];
        if (T) v = c_scale(v, T[o]);
        v = c_scale(v, scale);
        if (o == 0) v = make_float2(0.f, 0.f);
        spec[o] = v;
        amax = fmaxf(amax, fmaxf(fabsf(v.x), fabsf(v.y)));
    }
    red[threadIdx.x] = amax;
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if (threadIdx.x < st) red[threadIdx.x] = fmaxf(red[threadIdx.x], red[threadIdx.x + st]);
        __syncthreads();
    }
    const float r = red[0];
    __syncthreads();
    return r;
}

// sum over k != 0 of w_kx |F T|^2 over the full spectrum (w = 1 on the kx = 0 and N/2 columns,
// 2 elsewhere: the Hermitian partners of the half spectrum), in float64.
template <int N>
__device__ double half_spectrum_energy(const float2* F, const float* __restrict__ T, double* red) {
    constexpr int H = N / 2 + 1;
    double e = 0.0, dummy = 0.0;
    for (int o = threadIdx.x; o < N * H; o += blockDim.x) {
        if (o == 0) continue;
        const int kx = o % H;
        float2 v = F[o];
        if (T) v = c_scale(v, T[o]);
        const double m = (double)v.x * v.x + (double)v.y * v.y;
        e += (kx == 0 || kx == N / 2) ? m : 2.0 * m;
    }
    block_sum2(e, dummy, red);
    return e;
}

template <int N>
__global__ void __launch_bounds__(kThreads) k_prepare_images(const float* __restrict__ images,
                                                              const float2* __restrict__ g_tw,
                                                              float2* __restrict__ spec,
                                                              double* __restrict__ kA, float* __restrict__ amax,
                                                              double cn,
                                                              int* __restrict__ status) {
    constexpr int H = N / 2 + 1;
    extern __shared__ __align__(16) unsigned char smem[];
    float2* F = reinterpret_cast<float2*>(smem);
    float2* tw = F + N * H;
    double* red = reinterpret_cast<double*>(tw + N);
    const int w = blockIdx.x;
    const float* img = images + (size_t)w * N * N;
    load_twiddles<N>(g_tw, tw);

    double s1 = 0.0, s2 = 0.0;
    for (int i = threadIdx.x; i < N * N; i += blockDim.x) {
        const double v = img[i];
        s1 += v;
        s2 += v * v;
    }
    block_sum2(s1, s2, red);
    const double n = (double)N * N;
    const double A = n * s2 - s1 * s1;   // n C_oo - C_o^2
    const float mean = (float)(s1 / n);

    r2c_rows<N>(img, mean, F, tw);
    __syncthreads();
    c2c_columns_inplace<N, false>(F, tw);
    const double e = half_spectrum_energy<N>(F, nullptr, red);
    const bool bad = !(A > 0.0) || !(e > 0.0);
    const float scale = bad ? 0.f : (float)(1.0 / sqrt(e));
    const float mx = store_half_spectrum<N>(F, nullptr, scale, spec + (size_t)w * N * H, reinterpret_cast<float*>(red));
    if (threadIdx.x == 0) {
        amax[w] = mx;
        if (bad) {
            atomicOr(status, BIOEM_DEV_NUMERIC);
            kA[w] = -INFINITY;
        } else {
            kA[w] = 0.5 * (3.0 - n) * log(A) + cn;
        }
    }
}

// Pixel integral of a unit Gaussian between two boundaries whose scaled positions are a0 < a1,
// given T = erfc(|a|) and the sign of a at each boundary; written without cancellation in either
// tail: for a0, a1 > 0 it is (T0 - T1) / 2, for a0, a1 < 0 it is (T1 - T0) / 2.
__device__ __forceinline__ float pixel_mass(float t0, bool neg0, float t1, bool neg1) {
    if (!neg0) return 0.5f * (t0 - t1);
    if (neg1) return 0.5f * (t1 - t0);
    return 0.5f * ((1.f - t0) + (1.f - t1));
}

// One orientation per block.  Threads form a 16 x 16 grid, each owning a (N/16) x (N/16) pixel
// tile.  Atoms are processed in chunks: per chunk the x and y pixel integrals are tabulated in
// shared memory, then every thread accumulates w_a gy[a][k] gx[a][j] over the chunk.
template <int N>
struct ProjCfg {
    static constexpr int CH = (2048 / N) < 8 ? 8 : (2048 / N);   // atoms per chunk (shared-memory bound)
    static constexpr int RY = N / 8;                               // rows per warp (8 warps)
    static constexpr int CX = N / 32;                              // columns per lane
    static constexpr int NB = N + 1;                               // pixel boundaries per axis
    static_assert(N % 32 == 0 && kThreads == 256, "8 warps x 32 lanes tile the image");
};

// |u| beyond which erfc(|u|) (about 1.4e-54 at 11) is zero in FP32: table entries past it are set
// to zero without evaluating erfc, and an atom's rows whose two boundaries both lie past it get a
// pixel integral of exactly zero.
constexpr float kErfcZero = 11.f;

template <int TL>
__device__ __forceinline__ void load_row(const float* src, float (&v)[TL]) {
    if constexpr (TL % 4 == 0) {
#pragma unroll
        for (int i = 0; i < TL / 4; ++i) {
            const float4 t = reinterpret_cast<const float4*>(src)[i];
            v[4 * i] = t.x; v[4 * i + 1] = t.y; v[4 * i + 2] = t.z; v[4 * i + 3] = t.w;
        }
    } else if constexpr (TL % 2 == 0) {
#pragma unroll
        for (int i = 0; i < TL / 2; ++i) {
            const float2 t = reinterpret_cast<const float2*>(src)[i];
            v[2 * i] = t.x; v[2 * i + 1] = t.y;
        }
    } else {
#pragma unroll
        for (int i = 0; i < TL; ++i) v[i] = src[i];
    }
}

// One orientation per block.  Warp w owns rows [w N/8, (w + 1) N/8), lane l columns [l N/32,
// (l + 1) N/32).  Atoms are processed in chunks: per chunk the x and y pixel integrals are tabulated
// in shared memory (erfc evaluated only where it is not zero in FP32), then every thread accumulates
// w_a gy[a][k] gx[a][j] over the chunk, a warp skipping the atoms whose y integrals vanish on all of
// its rows (their products are exact zeros, so the sums are unchanged bit for bit).
template <int N>
__global__ void __launch_bounds__(kThreads) k_project(const float4* __restrict__ atoms, int n_atoms,
                                                       const float4* __restrict__ quats, double sigma,
                                                       double pixel, float* __restrict__ out) {
    constexpr int CH = ProjCfg<N>::CH, RY = ProjCfg<N>::RY, CX = ProjCfg<N>::CX, NB = ProjCfg<N>::NB;
    __shared__ double rot[6];
    __shared__ float bx_t[CH][NB], by_t[CH][NB];
    __shared__ __align__(16) float gx[CH][N];
    __shared__ __align__(16) float gy[CH][N];
    // per atom and axis, u_j = (edge_j - a) / (sigma sqrt 2) = j D - A as float pairs (hi + lo), so the
    // table below runs in FP32 (an FMA forms j D_hi - A_hi exactly before rounding) with the accuracy
    // of a float64 evaluation of u rounded to float
    __shared__ float axh[CH], axl[CH], ayh[CH], ayl[CH];
    __shared__ float aw[CH];
    __shared__ int rlo[CH], rhi[CH];   // rows outside [rlo, rhi] have a zero y integral for the atom

    const int q = blockIdx.x;
    if (threadIdx.x == 0) {
        const float4 qq = quats[q];
        double w = qq.x, x = qq.y, y = qq.z, z = qq.w;
        const double nrm = sqrt(w * w + x * x + y * y + z * z);
        w /= nrm; x /= nrm; y /= nrm; z /= nrm;
        rot[0] = 1.0 - 2.0 * (y * y + z * z); rot[1] = 2.0 * (x * y - w * z); rot[2] = 2.0 * (x * z + w * y);
        rot[3] = 2.0 * (x * y + w * z); rot[4] = 1.0 - 2.0 * (x * x + z * z); rot[5] = 2.0 * (y * z - w * x);
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;   // rows [warp RY, +RY), columns [lane CX, +CX)
    float acc[RY][CX];
#pragma unroll
    for (int i = 0; i < RY; ++i)
#pragma unroll
        for (int j = 0; j < CX; ++j) acc[i][j] = 0.f;
    const double inv = 1.0 / (sigma * 1.4142135623730951);
    const double dd = pixel * inv;                 // D: the pixel in units of sigma sqrt 2
    const float d_hi = (float)dd, d_lo = (float)(dd - (double)d_hi);
    const float inv_d = (float)(1.0 / dd);        // for the rows an atom can reach (margins absorb rounding)
    const double a_off = (0.5 * N + 0.5) * pixel;  // edge_j = j pixel - a_off

    for (int a0 = 0; a0 < n_atoms; a0 += CH) {
        const int na = min(CH, n_atoms - a0);
        for (int a = threadIdx.x; a < CH; a += blockDim.x) {
            if (a < na) {
                const float4 p = atoms[a0 + a];
                const double ax = ((rot[0] * p.x + rot[1] * p.y + rot[2] * p.z) + a_off) * inv;
                const double ay = ((rot[3] * p.x + rot[4] * p.y + rot[5] * p.z) + a_off) * inv;
                axh[a] = (float)ax;
                axl[a] = (float)(ax - (double)axh[a]);
                ayh[a] = (float)ay;
                ayl[a] = (float)(ay - (double)ayh[a]);
                aw[a] = p.w;
                // boundary j has |u_j| < kErfcZero for (A - 11) / D < j < (A + 11) / D; row j uses
                // boundaries j and j + 1 (one row of margin each side for rounding)
                rlo[a] = (int)floorf(((float)ay - kErfcZero) * inv_d) - 2;
                rhi[a] = (int)ceilf(((float)ay + kErfcZero) * inv_d) + 1;
            } else {
                axh[a] = 1.0e30f; axl[a] = 0.f; ayh[a] = 1.0e30f; ayl[a] = 0.f; aw[a] = 0.f;
                rlo[a] = 1 << 30; rhi[a] = -(1 << 30);
            }
        }
        __syncthreads();
        // boundary table: erfc(|u|) with the sign of u stored in the sign of the entry
        for (int i = threadIdx.x; i < CH * NB; i += blockDim.x) {
            const int a = i / NB, j = i - (i / NB) * NB;
            const float fj = (float)j;
            const float ux = fmaf(fj, d_hi, -axh[a]) + fmaf(fj, d_lo, -axl[a]);
            const float uy = fmaf(fj, d_hi, -ayh[a]) + fmaf(fj, d_lo, -ayl[a]);
            float ex = 0.f, ey = 0.f;
            if (fabsf(ux) < kErfcZero) ex = erfcf(fabsf(ux));
            if (fabsf(uy) < kErfcZero) ey = erfcf(fabsf(uy));
            // the sign bit carries the sign of u, also when erfc underflows to zero
            bx_t[a][j] = __int_as_float(__float_as_int(ex) | (ux < 0.f ? (int)0x80000000 : 0));
            by_t[a][j] = __int_as_float(__float_as_int(ey) | (uy < 0.f ? (int)0x80000000 : 0));
        }
        __syncthreads();
        for (int i = threadIdx.x; i < CH * N; i += blockDim.x) {
            const int a = i / N, j = i - (i / N) * N;
            const float x0 = bx_t[a][j], x1 = bx_t[a][j + 1];
            const float y0 = by_t[a][j], y1 = by_t[a][j + 1];
            gx[a][j] = pixel_mass(fabsf(x0), __float_as_int(x0) < 0, fabsf(x1), __float_as_int(x1) < 0);
            gy[a][j] = aw[a] * pixel_mass(fabsf(y0), __float_as_int(y0) < 0, fabsf(y1), __float_as_int(y1) < 0);
        }
        __syncthreads();
        for (int a = 0; a < na; ++a) {
            // the warp's rows all have a zero integral for this atom: its products are all +0
            if (rhi[a] < warp * RY || rlo[a] >= (warp + 1) * RY) continue;
            float vy[RY], vx[CX];
            load_row<RY>(&gy[a][warp * RY], vy);
            load_row<CX>(&gx[a][lane * CX], vx);
#pragma unroll
            for (int i = 0; i < RY; ++i)
#pragma unroll
                for (int j = 0; j < CX; ++j) acc[i][j] = fmaf(vy[i], vx[j], acc[i][j]);
        }
        __syncthreads();
    }
    float* o = out + (size_t)q * N * N;
#pragma unroll
    for (int i = 0; i < RY; ++i)
#pragma unroll
        for (int j = 0; j < CX; ++j) o[(warp * RY + i) * N + lane * CX + j] = acc[i][j];
}

// T[c][ky][kx] = CTF(s) Env(s) for PSF c on the half-spectrum grid, evaluated in float64.
// coef[3c..3c+2] = (a, A, b); s = 2 pi (kx~, ky~) / (N pixel) with signed frequency indices.
__global__ void k_ctf_table(const double* __restrict__ coef, int nctf, int N, double pixel,
                            float* __restrict__ T) {
    const int H = N / 2 + 1;
    const int total = nctf * N * H;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        const int c = i / (N * H);
        const int r = i - c * N * H;
        const int ky = r / H, kx = r - (r / H) * H;
        const double fy = (ky <= N / 2) ? ky : ky - N;
        const double f = 2.0 * 3.14159265358979323846 / (N * pixel);
        const double s2 = f * f * ((double)kx * kx + fy * fy);
        const double a = coef[3 * c], A = coef[3 * c + 1], b = coef[3 * c + 2];
        const double ctf = -A * cos(0.5 * a * s2) - sqrt(1.0 - A * A) * sin(0.5 * a * s2);
        T[i] = (float)(ctf * exp(-0.5 * b * s2));
    }
}

template <int N>
__global__ void __launch_bounds__(kThreads) k_psf_spectra(const float* __restrict__ img0,
                                                           const float2* __restrict__ g_tw,
                                                           const float* __restrict__ T, int nctf,
                                                           float2* __restrict__ spec,
                                                           double* __restrict__ kB, float* __restrict__ amax,
                                                           int* __restrict__ status) {
    constexpr int H = N / 2 + 1;
    extern __shared__ __align__(16) unsigned char smem[];
    float2* F = reinterpret_cast<float2*>(smem);
    float2* tw = F + N * H;
    double* red = reinterpret_cast<double*>(tw + N);
    const int q = blockIdx.x;
    load_twiddles<N>(g_tw, tw);
    __syncthreads();
    r2c_rows<N>(img0 + (size_t)q * N * N, 0.f, F, tw);
    __syncthreads();
    c2c_columns_inplace<N, false>(F, tw);
    for (int c = 0; c < nctf; ++c) {
        const float* Tc = T + (size_t)c * N * H;
        const double B = half_spectrum_energy<N>(F, Tc, red);   // n C_cc - C_c^2 (Plancherel)
        const bool bad = !(B > 0.0);
        const size_t p = (size_t)q * nctf + c;
        const float mx = store_half_spectrum<N>(F, Tc, bad ? 0.f : (float)(1.0 / sqrt(B)), spec + p * N * H,
                                                reinterpret_cast<float*>(red));
        if (threadIdx.x == 0) {
            amax[p] = mx;
            if (bad) {
                atomicOr(status, BIOEM_DEV_NUMERIC);
                kB[p] = -INFINITY;
            } else {
                kB[p] = -0.5 * log(B);
            }
        }
    }
}

// Synthetic map for pair i: I1 = Re F^-1[F(I0_i) T_i] with F^-1 normalised by 1/N^2.
template <int N>
__global__ void __launch_bounds__(kThreads) k_psf_real(const float* __restrict__ img0,
                                                        const float2* __restrict__ g_tw,
                                                        const float* __restrict__ T,
                                                        float* __restrict__ out) {
    constexpr int H = N / 2 + 1;
    extern __shared__ __align__(16) unsigned char smem[];
    float2* F = reinterpret_cast<float2*>(smem);
    float2* tw = F + N * H;
    const int i = blockIdx.x;
    load_twiddles<N>(g_tw, tw);
    __syncthreads();
    r2c_rows<N>(img0 + (size_t)i * N * N, 0.f, F, tw);
    __syncthreads();
    c2c_columns_inplace<N, false>(F, tw);
    const float* Ti = T + (size_t)i * N * H;
    for (int o = threadIdx.x; o < N * H; o += blockDim.x) F[o] = c_scale(F[o], Ti[o]);
    __syncthreads();
    c2c_columns_inplace<N, true>(F, tw);
    // rows: I(y, x) = (1/N^2) [G0 + GN (-1)^x + 2 sum_{0<kx<N/2} Re(G(kx) exp(+2 pi i kx x / N))]
    float* o = out + (size_t)i * N * N;
    const float inv = 1.0f / ((float)N * N);
    for (int p = threadIdx.x; p < N * N; p += blockDim.x) {
        const int y = p / N, x = p - (p / N) * N;
        const float2* G = F + y * H;
        float v = G[0].x + ((x & 1) ? -G[N / 2].x : G[N / 2].x);
        float acc = 0.f;
        int idx = x;
        for (int kx = 1; kx < N / 2; ++kx) {
            const float2 w = tw[idx];          // exp(-2 pi i kx x / N); conjugated below
            acc = fmaf(G[kx].x, w.x, fmaf(G[kx].y, w.y, acc));
            idx += x;
            idx -= (idx >= N) ? N : 0;
        }
        o[p] = (v + 2.f * acc) * inv;
    }
}

// Real-space image of a stored unit-norm half spectrum S (Eq. 3, inverse transform):
//   x(r) = Re sum_k w_kx S(k) exp(+2 pi i k.r / N),  w = 1 on kx = 0, N/2 and 2 elsewhere,
// rescaled to unit norm (float64 sum of squares); zero-mean because S(0) = 0.  With the forward
// transforms above this is the zero-mean, unit-norm image whose correlations the scoring kernels
// evaluate: sum_r o'(r) c'(r + d) = rho(d).  Writes x [N][N] and max |x|.
template <int N>
__global__ void __launch_bounds__(kThreads) k_spec_to_real(const float2* __restrict__ spec,
                                                           const float2* __restrict__ g_tw, float* __restrict__ out,
                                                           float* __restrict__ amax) {
    constexpr int H = N / 2 + 1;
    extern __shared__ __align__(16) unsigned char smem[];
    float2* F = reinterpret_cast<float2*>(smem);
    float2* tw = F + N * H;
    double* red = reinterpret_cast<double*>(tw + N);
    const int i = blockIdx.x;
    load_twiddles<N>(g_tw, tw);
    const float2* S = spec + (size_t)i * N * H;
    for (int o = threadIdx.x; o < N * H; o += blockDim.x) F[o] = S[o];
    __syncthreads();
    c2c_columns_inplace<N, true>(F, tw);
    float* xo = out + (size_t)i * N * N;
    double e = 0.0, dummy = 0.0;
    for (int p = threadIdx.x; p < N * N; p += blockDim.x) {
        const int y = p / N, x = p - (p / N) * N;
        const float2* G = F + y * H;
        const float v = G[0].x + ((x & 1) ? -G[N / 2].x : G[N / 2].x);
        float acc = 0.f;
        int idx = x;
        for (int kx = 1; kx < N / 2; ++kx) {
            const float2 w = tw[idx];   // exp(-2 pi i kx x / N); conjugated below
            acc = fmaf(G[kx].x, w.x, fmaf(G[kx].y, w.y, acc));
            idx += x;
            idx -= (idx >= N) ? N : 0;
        }
        const float r = v + 2.f * acc;
        xo[p] = r;
        e += (double)r * r;
    }
    block_sum2(e, dummy, red);
    const float scale = e > 0.0 ? (float)(1.0 / sqrt(e)) : 0.f;
    float mx = 0.f;
    for (int p = threadIdx.x; p < N * N; p += blockDim.x) {   // the same elements this thread wrote
        const float r = xo[p] * scale;
        xo[p] = r;
        mx = fmaxf(mx, fabsf(r));
    }
    float* redf = reinterpret_cast<float*>(red);
    __syncthreads();
    redf[threadIdx.x] = mx;
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if (threadIdx.x < st) redf[threadIdx.x] = fmaxf(redf[threadIdx.x], redf[threadIdx.x + st]);
        __syncthreads();
    }
    if (threadIdx.x == 0) amax[i] = redf[0];
}

template <int N>
size_t fwd_smem() {
    return (size_t)(N * (N / 2 + 1) + N) * sizeof(float2) + 2 * kThreads * sizeof(double);
}

template <int N>
int set_smem(const void* fn, size_t bytes) {
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) == cudaSuccess ? 0 : -1;
}

void ctf_coefficients(const bioem_ctf& c, double* out3) {
    const double v = c.voltage_kV * 1.0e3;
    const double lam = 12.2643 / sqrt(v * (1.0 + 0.97845e-6 * v));
    out3[0] = lam * c.defocus_A / (2.0 * 3.14159265358979323846);
    out3[1] = c.amp_contrast;
    out3[2] = c.bfactor_A2 / (8.0 * 3.14159265358979323846 * 3.14159265358979323846);
}

// Build the CTF table for nctf PSFs into *d_T (allocated here; caller frees).
int build_ctf_table(bioem_ctx* ctx, const bioem_ctf* ctfs, int nctf, int npix, double pixel_A, float** d_T) {
    double* h = (double*)malloc(sizeof(double) * 3 * nctf);
    if (!h) return bioem_set_error(ctx, BIOEM_ERR_OOM, "host allocation failed");
    for (int c = 0; c < nctf; ++c) ctf_coefficients(ctfs[c], h + 3 * c);
    double* d_coef = nullptr;
    cudaError_t e = cudaMallocAsync((void**)&d_coef, sizeof(double) * 3 * nctf, ctx->stream);
    if (e != cudaSuccess) { free(h); return bioem_set_error(ctx, BIOEM_ERR_OOM, "cudaMallocAsync(ctf coef)"); }
    const size_t tsize = (size_t)nctf * npix * (npix / 2 + 1);
    e = cudaMallocAsync((void**)d_T, sizeof(float) * tsize, ctx->stream);
    if (e != cudaSuccess) {
        cudaFreeAsync(d_coef, ctx->stream);
        free(h);
        return bioem_set_error(ctx, BIOEM_ERR_OOM, "cudaMallocAsync(ctf table)");
    }
    e = cudaMemcpyAsync(d_coef, h, sizeof(double) * 3 * nctf, cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) {
        const int blocks = (int)((tsize + 255) / 256 < 4096 ? (tsize + 255) / 256 : 4096);
        bioem_launch_begin(ctx, KID_CTF_TABLE);
        k_ctf_table<<<blocks, 256, 0, ctx->stream>>>(d_coef, nctf, npix, pixel_A, *d_T);
        e = cudaGetLastError();
        bioem_launch_end(ctx, KID_CTF_TABLE);
    }
    // the copy reads h asynchronously from pageable memory: it has completed once the call returns
    cudaFreeAsync(d_coef, ctx->stream);
    free(h);
    if (e != cudaSuccess) {
        cudaFreeAsync(*d_T, ctx->stream);
        *d_T = nullptr;
        return bioem_check_cuda(ctx, e, "ctf table");
    }
    return BIOEM_OK;
}

template <int N>
int launch_prepare_n(bioem_ctx* ctx, const float* d_images, bioem_images* im) {
    const size_t sm = fwd_smem<N>();
    if (set_smem<N>((const void*)k_prepare_images<N>, sm)) return bioem_set_error(ctx, BIOEM_ERR_CUDA, "smem attribute");
    const double cn = bioem_log_norm_constant(N * N);
    bioem_launch_begin(ctx, KID_PREPARE);
    k_prepare_images<N><<<im->n_img, kThreads, sm, ctx->stream>>>(d_images, bioem_twiddles(ctx, N), im->d_spec,
                                                                    im->d_kA, im->d_amax, cn, ctx->d_status);
    bioem_launch_end(ctx, KID_PREPARE);
    return bioem_check_cuda(ctx, cudaGetLastError(), "k_prepare_images");
}

template <int N>
int launch_project_n(bioem_ctx* ctx, const float* d_atoms, int n_atoms, double sigma_A, const float* d_quats,
                     int nq, const bioem_ctf* ctfs, int nctf, bioem_projset* ps) {
    float* d_T = nullptr;
    int rc = build_ctf_table(ctx, ctfs, nctf, N, ps->pixel_A, &d_T);
    if (rc) return rc;
    // orientations in waves bounded to ~1 GiB of I0 scratch
    const int wave = (int)((1ull << 30) / ((size_t)N * N * sizeof(float)));
    const int qw = nq < wave ? nq : wave;
    float* d_I0 = nullptr;
    if (cudaMallocAsync((void**)&d_I0, sizeof(float) * (size_t)qw * N * N, ctx->stream) != cudaSuccess) {
        cudaFreeAsync(d_T, ctx->stream);
        return bioem_set_error(ctx, BIOEM_ERR_OOM, "cudaMallocAsync(projection scratch)");
    }
    const size_t sm = fwd_smem<N>();
    if (set_smem<N>((const void*)k_psf_spectra<N>, sm)) rc = bioem_set_error(ctx, BIOEM_ERR_CUDA, "smem attribute");
    for (int q0 = 0; q0 < nq && rc == BIOEM_OK; q0 += qw) {
        const int nb = nq - q0 < qw ? nq - q0 : qw;
        bioem_launch_begin(ctx, KID_PROJECT);
        k_project<N><<<nb, kThreads, 0, ctx->stream>>>(reinterpret_cast<const float4*>(d_atoms), n_atoms,
                                                        reinterpret_cast<const float4*>(d_quats) + q0, sigma_A,
                                                        ps->pixel_A, d_I0);
        bioem_launch_end(ctx, KID_PROJECT);
        rc = bioem_check_cuda(ctx, cudaGetLastError(), "k_project");
        if (rc) break;
        const size_t p0 = (size_t)q0 * nctf;
        bioem_launch_begin(ctx, KID_PSF_SPECTRA);
        k_psf_spectra<N><<<nb, kThreads, sm, ctx->stream>>>(d_I0, bioem_twiddles(ctx, N), d_T, nctf,
                                                             ps->d_spec + p0 * N * (N / 2 + 1), ps->d_kB + p0,
                                                             ps->d_amax + p0, ctx->d_status);
        bioem_launch_end(ctx, KID_PSF_SPECTRA);
        rc = bioem_check_cuda(ctx, cudaGetLastError(), "k_psf_spectra");
    }
    cudaFreeAsync(d_I0, ctx->stream);
    cudaFreeAsync(d_T, ctx->stream);
    return rc;
}

template <int N>
int launch_synthetic_n(bioem_ctx* ctx, const float* d_atoms, int n_atoms, double sigma_A, const float* d_quats,
                       const bioem_ctf* ctfs, int n, double pixel_A, float* d_out) {
    float* d_T = nullptr;
    int rc = build_ctf_table(ctx, ctfs, n, N, pixel_A, &d_T);
    if (rc) return rc;
    float* d_I0 = nullptr;
    if (cudaMallocAsync((void**)&d_I0, sizeof(float) * (size_t)n * N * N, ctx->stream) != cudaSuccess) {
        cudaFreeAsync(d_T, ctx->stream);
        return bioem_set_error(ctx, BIOEM_ERR_OOM, "cudaMallocAsync(synthetic scratch)");
    }
    bioem_launch_begin(ctx, KID_PROJECT);
    k_project<N><<<n, kThreads, 0, ctx->stream>>>(reinterpret_cast<const float4*>(d_atoms), n_atoms,
                                                   reinterpret_cast<const float4*>(d_quats), sigma_A, pixel_A, d_I0);
    bioem_launch_end(ctx, KID_PROJECT);
    rc = bioem_check_cuda(ctx, cudaGetLastError(), "k_project");
    const size_t sm = fwd_smem<N>();
    if (!rc && set_smem<N>((const void*)k_psf_real<N>, sm)) rc = bioem_set_error(ctx, BIOEM_ERR_CUDA, "smem attribute");
    if (!rc) {
        bioem_launch_begin(ctx, KID_PSF_REAL);
        k_psf_real<N><<<n, kThreads, sm, ctx->stream>>>(d_I0, bioem_twiddles(ctx, N), d_T, d_out);
        bioem_launch_end(ctx, KID_PSF_REAL);
        rc = bioem_check_cuda(ctx, cudaGetLastError(), "k_psf_real");
    }
    cudaFreeAsync(d_I0, ctx->stream);
    cudaFreeAsync(d_T, ctx->stream);
    return rc;
}

template <int N>
int launch_spec_to_real_n(bioem_ctx* ctx, const float2* spec, int count, float* out, float* amax) {
    const size_t sm = fwd_smem<N>();
    if (set_smem<N>((const void*)k_spec_to_real<N>, sm)) return bioem_set_error(ctx, BIOEM_ERR_CUDA, "smem attribute");
    bioem_launch_begin(ctx, KID_GEMM_OPS);
    k_spec_to_real<N><<<count, kThreads, sm, ctx->stream>>>(spec, bioem_twiddles(ctx, N), out, amax);
    bioem_launch_end(ctx, KID_GEMM_OPS);
    return bioem_check_cuda(ctx, cudaGetLastError(), "k_spec_to_real");
}

}  // namespace

double bioem_log_norm_constant(int n) {
    const double nn = n;
    return -log(2.0) + (1.0 - nn / 2.0) * log(2.0 * 3.14159265358979323846) + lgamma((nn - 3.0) / 2.0) +
           (nn - 3.0) / 2.0 * log(2.0 * nn);
}

#define BIOEM_DISPATCH_N(npix, CALL)                                          \
    switch (npix) {                                                           \
        case 32: return CALL(32);                                             \
        case 64: return CALL(64);                                             \
        case 96: return CALL(96);                                             \
        case 128: return CALL(128);                                           \
        case 192: return CALL(192);                                           \
        default: return bioem_set_error(ctx, BIOEM_ERR_UNSUPPORTED_SIZE, "unsupported image size %d", npix); \
    }

int bioem_launch_prepare(bioem_ctx* ctx, const float* d_images, bioem_images* im) {
#define CALL(N) launch_prepare_n<N>(ctx, d_images, im)
    BIOEM_DISPATCH_N(im->nx, CALL)
#undef CALL
}

int bioem_launch_project(bioem_ctx* ctx, const float* d_atoms, int n_atoms, double sigma_A, const float* d_quats,
                         int nq, const bioem_ctf* ctfs, int nctf, bioem_projset* ps) {
#define CALL(N) launch_project_n<N>(ctx, d_atoms, n_atoms, sigma_A, d_quats, nq, ctfs, nctf, ps)
    BIOEM_DISPATCH_N(ps->nx, CALL)
#undef CALL
}

int bioem_launch_spec_to_real(bioem_ctx* ctx, const float2* spec, int count, int npix, float* out, float* amax) {
    if (count <= 0) return BIOEM_OK;
#define CALL(N) launch_spec_to_real_n<N>(ctx, spec, count, out, amax)
    BIOEM_DISPATCH_N(npix, CALL)
#undef CALL
}

int bioem_launch_synthetic(bioem_ctx* ctx, const float* d_atoms, int n_atoms, double sigma_A, const float* d_quats,
                           const bioem_ctf* ctfs, int n, int npix, double pixel_A, float* d_out) {
#define CALL(N) launch_synthetic_n<N>(ctx, d_atoms, n_atoms, sigma_A, d_quats, ctfs, n, pixel_A, d_out)
    BIOEM_DISPATCH_N(npix, CALL)
#undef CALL
}
