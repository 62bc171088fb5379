// Real-input pieces of the pruned inverse transform's second stage (along kx), shared by the
// scoring kernels: for one row dy and one real component c of Q(dy, kx) (c = 0: Re, 1: Im), the
// even function C(dx) = sum_kx w Re Q cos(2 pi kx dx / N) or the odd S(dx) = sum_kx w Im Q sin(...)
// for dx = 0..NOUT-1, from the kx sub-sequences kx = b + R a (a = 0..7, R = N / 16): a real 16-point
// transform per sub-sequence, recombined with W_N^(b dx) for the wanted dx only.  rho(dy, +-dx) is
// then C(dx) -+ S(dx) plus the Nyquist column's (-1)^dx Q(dy, N/2).
#pragma once

#include "bioem_internal.cuh"

namespace {

// Real 16-point transform of eight real inputs (x[8..15] = 0): Y(u) = sum_a x[a] exp(+2 pi i a u / 16)
// for u = 0..8 (Y(16 - u) = conj Y(u)).  Even u from an 8-point transform of x, odd u from an
// 8-point transform of x[a] exp(2 pi i a / 16), each split once more into 4-point transforms.
__device__ __forceinline__ void rdft16(const float (&x)[8], float (&yr)[9], float (&yi)[9]) {
    const float r = 0.70710678118654752f, c1 = 0.92387953251128674f, s1 = 0.38268343236508977f;
    const float e0 = x[0] + x[4], e1 = x[1] + x[5], e2 = x[2] + x[6], e3 = x[3] + x[7];
    const float d0 = x[0] - x[4], d1 = x[1] - x[5], d2 = x[2] - x[6], d3 = x[3] - x[7];
    const float s02 = e0 + e2, s13 = e1 + e3;
    yr[0] = s02 + s13;
    yi[0] = 0.f;
    yr[8] = s02 - s13;
    yi[8] = 0.f;
    yr[4] = e0 - e2;
    yi[4] = e1 - e3;
    const float t1 = d1 - d3, t2 = d1 + d3;
    yr[2] = fmaf(r, t1, d0);
    yi[2] = fmaf(r, t2, d2);
    yr[6] = fmaf(-r, t1, d0);
    yi[6] = fmaf(r, t2, -d2);
    // f[m] = W^m (x_m + i x_{m+4}),  g[m] = W^{3m} (x_m - i x_{m+4}),  W = exp(2 pi i / 16)
    const float f1r = fmaf(c1, x[1], -s1 * x[5]), f1i = fmaf(s1, x[1], c1 * x[5]);
    const float f2r = r * (x[2] - x[6]), f2i = r * (x[2] + x[6]);
    const float f3r = fmaf(s1, x[3], -c1 * x[7]), f3i = fmaf(c1, x[3], s1 * x[7]);
    const float g1r = fmaf(s1, x[1], c1 * x[5]), g1i = fmaf(c1, x[1], -s1 * x[5]);
    const float g3r = fmaf(-c1, x[3], -s1 * x[7]), g3i = fmaf(c1, x[7], -s1 * x[3]);
    // Y1 = sum f, Y5 = sum f i^m; Y3 = sum g, Y7 = sum g i^m  (g0 = (x0, -x4), g2 = (-f2r, f2i))
    const float ar = x[0] + f2r, ai = x[4] + f2i, br = f1r + f3r, bi = f1i + f3i;
    const float cr = x[0] - f2r, ci = x[4] - f2i, dr = f1r - f3r, di = f1i - f3i;
    yr[1] = ar + br;
    yi[1] = ai + bi;
    yr[5] = cr - di;
    yi[5] = ci + dr;
    const float er = x[0] - f2r, ei = f2i - x[4], fr = g1r + g3r, fi = g1i + g3i;
    const float gr = x[0] + f2r, gi = -x[4] - f2i, kr = g1r - g3r, ki = g1i - g3i;
    yr[3] = er + fr;
    yi[3] = ei + fi;
    yr[7] = gr - ki;
    yi[7] = gi + kr;
}

// acc[dx] += the sub-sequence's share of component c, dx = 0..NOUT-1; tw = the (c, b) row of the
// table of (T1, T2) pairs, T = (cos, -+sin) for c = 0 and (sin, +-cos) for c = 1 at angle 2 pi b dx / N,
// the second sign for u = dx mod 16 > 8 (where Y(u) = conj Y(16 - u) is used).
template <int NOUT>
__device__ __forceinline__ void recombine(float (&acc)[NOUT], const float (&yr)[9], const float (&yi)[9],
                                          const float2* __restrict__ tw) {
#pragma unroll
    for (int dx = 0; dx < NOUT; ++dx) {
        const int u = dx & 15;
        const int yidx = u > 8 ? 16 - u : u;
        const float2 t = tw[dx];
        if (yidx == 0 || yidx == 8) acc[dx] = fmaf(t.x, yr[yidx], acc[dx]);
        else acc[dx] = fmaf(t.x, yr[yidx], fmaf(t.y, yi[yidx], acc[dx]));
    }
}

}  // namespace
