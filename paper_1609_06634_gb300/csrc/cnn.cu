// Learned orientation / defocus proposal network: own forward, backward and Adam kernels.
//
// The paper has no learned component; this network proposes where on the orientation x defocus
// grid an image's posterior mass lies, so that only those parameter sets are scored exactly.
//
// Network (input S x S, S = 64 in production: the 128 px image averaged over 2 x 2 pixels and
// standardised per image):
//   conv1 1->C, 3x3, stride 1, pad 1, ReLU       S   x S
//   conv2 C->C, stride 2, ReLU                   S/2
//   conv3 C->C, stride 1, ReLU                   S/2
//   conv4 C->C, stride 2, ReLU                   S/4
//   conv5 C->C, stride 1, ReLU                   S/4
//   conv6 C->C, stride 2, ReLU                   S/8  -> F = C (S/8)^2 features
//   head_q: F -> n_q logits (coarse orientation bins); head_d: F -> n_d logits (defocus bins)
//   loss = mean over the batch of CE(head_q, label_q) + CE(head_d, label_d)
// Parameters are kept in float32 (Adam state and master copy); the forward and backward passes
// read a float16 copy of the weights (rounded after every update).  Activations are float32, NCHW.
// Flat parameter order: for each conv layer W[co][ci][3][3] then b[co]; then Wq[n_q][F], bq[n_q],
// Wd[n_d][F], bd[n_d].
#include <cuda_fp16.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <new>
#include <vector>

#include "bioem_internal.cuh"

namespace {

constexpr int kLayers = 6;
constexpr int kT = 256;

struct Layer {
    int cin, cout, stride, hin, hout;
    size_t w_off, b_off;     // offsets in the flat parameter vector
    size_t in_off, out_off;  // activation offsets (per-sample element counts are cin*hin^2, cout*hout^2)
};

// ------------------------------------------------------------------ input preparation
// out[b][y][x] = standardised 2x2 average of img[b]; per image: zero mean, unit variance over S^2.
__global__ void __launch_bounds__(kT) k_downsample_norm(const float* __restrict__ img, int n_in, int down,
                                                        float* __restrict__ out) {
    const int b = blockIdx.x;
    const int S = n_in / down;
    const float* src = img + (size_t)b * n_in * n_in;
    float* dst = out + (size_t)b * S * S;
    __shared__ double r1[kT], r2[kT];
    double s1 = 0.0, s2 = 0.0;
    for (int i = threadIdx.x; i < S * S; i += blockDim.x) {
        const int y = i / S, x = i - (i / S) * S;
        float v = 0.f;
        for (int dy = 0; dy < down; ++dy)
            for (int dx = 0; dx < down; ++dx) v += src[(y * down + dy) * n_in + x * down + dx];
        v *= 1.0f / (float)(down * down);
        dst[i] = v;
        s1 += v;
        s2 += (double)v * v;
    }
    r1[threadIdx.x] = s1;
    r2[threadIdx.x] = s2;
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if (threadIdx.x < st) {
            r1[threadIdx.x] += r1[threadIdx.x + st];
            r2[threadIdx.x] += r2[threadIdx.x + st];
        }
        __syncthreads();
    }
    const double n = (double)S * S;
    const double mean = r1[0] / n;
    const double var = r2[0] / n - mean * mean;
    const float inv = var > 0.0 ? (float)(1.0 / sqrt(var)) : 0.f;
    const float m = (float)mean;
    for (int i = threadIdx.x; i < S * S; i += blockDim.x) dst[i] = (dst[i] - m) * inv;
}

// ------------------------------------------------------------------ convolution
// out[b][co][y][x] = ReLU(b[co] + sum_ci,ky,kx W[co][ci][ky][kx] in[b][ci][y s + ky - 1][x s + kx - 1])
__global__ void __launch_bounds__(kT) k_conv_fwd(const float* __restrict__ in, const __half* __restrict__ W,
                                                 const __half* __restrict__ bias, int B, int cin, int cout, int hin,
                                                 int hout, int stride, float* __restrict__ out) {
    extern __shared__ float wsm[];   // [cin][9] for this block's output channel
    const int co = blockIdx.y;
    for (int i = threadIdx.x; i < cin * 9; i += blockDim.x) wsm[i] = __half2float(W[(size_t)co * cin * 9 + i]);
    __syncthreads();
    const float bv = __half2float(bias[co]);
    const int per = hout * hout;
    const size_t total = (size_t)B * per;
    for (size_t o = (size_t)blockIdx.x * blockDim.x + threadIdx.x; o < total; o += (size_t)gridDim.x * blockDim.x) {
        const int b = (int)(o / per);
        const int r = (int)(o - (size_t)b * per);
        const int y = r / hout, x = r - (r / hout) * hout;
        float acc = bv;
        const float* ib = in + (size_t)b * cin * hin * hin;
        for (int ci = 0; ci < cin; ++ci) {
            const float* ic = ib + (size_t)ci * hin * hin;
#pragma unroll
            for (int ky = 0; ky < 3; ++ky) {
                const int iy = y * stride + ky - 1;
                if (iy < 0 || iy >= hin) continue;
#pragma unroll
                for (int kx = 0; kx < 3; ++kx) {
                    const int ix = x * stride + kx - 1;
                    if (ix < 0 || ix >= hin) continue;
                    acc = fmaf(wsm[ci * 9 + ky * 3 + kx], __ldg(ic + iy * hin + ix), acc);
                }
            }
        }
        out[((size_t)b * cout + co) * per + r] = acc > 0.f ? acc : 0.f;
    }
}

// g *= (y > 0): back through the ReLU of a layer whose output is y.
__global__ void k_relu_bwd(const float* __restrict__ y, float* __restrict__ g, size_t n) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        if (!(y[i] > 0.f)) g[i] = 0.f;
}

// din[b][ci][iy][ix] = sum over (co, ky, kx) with iy = y s + ky - 1, ix = x s + kx - 1 of
// gout[b][co][y][x] W[co][ci][ky][kx]   (gout already through the ReLU)
__global__ void __launch_bounds__(kT) k_conv_bwd_data(const float* __restrict__ gout, const __half* __restrict__ W,
                                                      int B, int cin, int cout, int hin, int hout, int stride,
                                                      float* __restrict__ din) {
    const int per_in = hin * hin;
    const size_t total = (size_t)B * cin * per_in;
    for (size_t o = (size_t)blockIdx.x * blockDim.x + threadIdx.x; o < total; o += (size_t)gridDim.x * blockDim.x) {
        const int b = (int)(o / ((size_t)cin * per_in));
        const int rem = (int)(o - (size_t)b * cin * per_in);
        const int ci = rem / per_in;
        const int p = rem - ci * per_in;
        const int iy = p / hin, ix = p - (p / hin) * hin;
        float acc = 0.f;
        for (int ky = 0; ky < 3; ++ky) {
            const int ty = iy + 1 - ky;   // = y * stride
            if (ty < 0 || ty % stride) continue;
            const int y = ty / stride;
            if (y >= hout) continue;
            for (int kx = 0; kx < 3; ++kx) {
                const int tx = ix + 1 - kx;
                if (tx < 0 || tx % stride) continue;
                const int x = tx / stride;
                if (x >= hout) continue;
                const float* g = gout + ((size_t)b * cout) * hout * hout + y * hout + x;
                const __half* w = W + (size_t)ci * 9 + ky * 3 + kx;
                for (int co = 0; co < cout; ++co)
                    acc = fmaf(__ldg(g + (size_t)co * hout * hout), __half2float(w[(size_t)co * cin * 9]), acc);
            }
        }
        din[o] = acc;
    }
}

// gW[co][ci][ky][kx] = sum_{b,y,x} gout[b][co][y][x] in[b][ci][y s + ky - 1][x s + kx - 1]; one block
// per (co, ci), fixed-order block reduction; gb[co] = sum_{b,y,x} gout[b][co][y][x] (ci = 0 blocks).
__global__ void __launch_bounds__(kT) k_conv_bwd_weight(const float* __restrict__ gout, const float* __restrict__ in,
                                                        int B, int cin, int cout, int hin, int hout, int stride,
                                                        float* __restrict__ gW, float* __restrict__ gb) {
    const int co = blockIdx.x / cin, ci = blockIdx.x - (blockIdx.x / cin) * cin;
    float acc[10];
#pragma unroll
    for (int k = 0; k < 10; ++k) acc[k] = 0.f;
    const int per = hout * hout;
    const size_t total = (size_t)B * per;
    for (size_t o = threadIdx.x; o < total; o += blockDim.x) {
        const int b = (int)(o / per);
        const int r = (int)(o - (size_t)b * per);
        const int y = r / hout, x = r - (r / hout) * hout;
        const float g = gout[((size_t)b * cout + co) * per + r];
        if (g == 0.f) continue;
        const float* ic = in + ((size_t)b * cin + ci) * hin * hin;
#pragma unroll
        for (int ky = 0; ky < 3; ++ky) {
            const int iy = y * stride + ky - 1;
#pragma unroll
            for (int kx = 0; kx < 3; ++kx) {
                const int ix = x * stride + kx - 1;
                if (iy >= 0 && iy < hin && ix >= 0 && ix < hin) acc[ky * 3 + kx] = fmaf(g, ic[iy * hin + ix], acc[ky * 3 + kx]);
            }
        }
        acc[9] += g;
    }
    __shared__ float red[10][kT];
#pragma unroll
    for (int k = 0; k < 10; ++k) red[k][threadIdx.x] = acc[k];
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if (threadIdx.x < st)
#pragma unroll
            for (int k = 0; k < 10; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + st];
        __syncthreads();
    }
    if (threadIdx.x < 9) gW[((size_t)co * cin + ci) * 9 + threadIdx.x] = red[threadIdx.x][0];
    if (threadIdx.x == 9 && ci == 0) gb[co] = red[9][0];
}

// ------------------------------------------------------------------ dense layers (tiled GEMM)
// C[m][n] (+)= sum_k A(m, k) B(n, k) (+ bias[n]); A(m, k) = A[m sam + k sak], B(n, k) = B[n sbn + k sbk].
// 64 x 64 tiles, 16 of k per step, 4 x 4 outputs per thread.
template <class TB>
__global__ void __launch_bounds__(256) k_gemm(const float* __restrict__ A, long long sam, long long sak,
                                              const TB* __restrict__ Bm, long long sbn, long long sbk,
                                              const TB* __restrict__ bias, float* __restrict__ C, int M, int N, int K,
                                              int ldc, int accumulate) {
    __shared__ float As[16][64 + 4], Bs[16][64 + 4];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
    float acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
    for (int k0 = 0; k0 < K; k0 += 16) {
        for (int i = threadIdx.x; i < 16 * 64; i += 256) {
            const int kk = i / 64, mm = i - (i / 64) * 64;
            const int m = m0 + mm, k = k0 + kk;
            As[kk][mm] = (m < M && k < K) ? A[(long long)m * sam + (long long)k * sak] : 0.f;
            const int n = n0 + mm;
            Bs[kk][mm] = (n < N && k < K) ? (float)Bm[(long long)n * sbn + (long long)k * sbk] : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            float a[4], bv[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
            for (int j = 0; j < 4; ++j) bv[j] = Bs[kk][tx * 4 + j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], bv[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int m = m0 + ty * 4 + i;
        if (m >= M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int n = n0 + tx * 4 + j;
            if (n >= N) continue;
            const float v = acc[i][j] + (bias ? (float)bias[n] : 0.f);
            if (accumulate) C[(long long)m * ldc + n] += v;
            else C[(long long)m * ldc + n] = v;
        }
    }
}

// column sums: out[n] = sum_m G[m][n]   (bias gradients; fixed order)
__global__ void k_colsum(const float* __restrict__ G, int M, int N, float* __restrict__ out) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    float s = 0.f;
    for (int m = 0; m < M; ++m) s += G[(size_t)m * N + n];
    out[n] = s;
}

// ------------------------------------------------------------------ loss
// Per sample: log-softmax of both heads, loss = -lq[label_q] - ld[label_d]; gradients
// (softmax - onehot) / B written over the logits.  loss_out[b] (may be null).
__global__ void __launch_bounds__(kT) k_softmax_ce(float* __restrict__ lq, int nq, float* __restrict__ ld, int nd,
                                                   const int* __restrict__ yq, const int* __restrict__ yd, int B,
                                                   float* __restrict__ loss_out) {
    const int b = blockIdx.x;
    __shared__ float red[kT];
    __shared__ float stat[2];
    float loss = 0.f;
    for (int head = 0; head < 2; ++head) {
        float* l = head == 0 ? lq + (size_t)b * nq : ld + (size_t)b * nd;
        const int n = head == 0 ? nq : nd;
        const int y = head == 0 ? yq[b] : yd[b];
        float m = -INFINITY;
        for (int i = threadIdx.x; i < n; i += blockDim.x) m = fmaxf(m, l[i]);
        red[threadIdx.x] = m;
        __syncthreads();
        for (int st = blockDim.x / 2; st > 0; st >>= 1) {
            if (threadIdx.x < st) red[threadIdx.x] = fmaxf(red[threadIdx.x], red[threadIdx.x + st]);
            __syncthreads();
        }
        m = red[0];
        __syncthreads();
        float s = 0.f;
        for (int i = threadIdx.x; i < n; i += blockDim.x) s += expf(l[i] - m);
        red[threadIdx.x] = s;
        __syncthreads();
        for (int st = blockDim.x / 2; st > 0; st >>= 1) {
            if (threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            stat[0] = m + logf(red[0]);
            stat[1] = l[y];
        }
        __syncthreads();
        const float lse = stat[0];
        loss += lse - stat[1];
        if (yq) {
            for (int i = threadIdx.x; i < n; i += blockDim.x) l[i] = (expf(l[i] - lse) - (i == y ? 1.f : 0.f)) / (float)B;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0 && loss_out) loss_out[b] = loss;
}

// Adam on the flat float32 parameters; the float16 copy is refreshed from the result.
__global__ void k_adam(float* __restrict__ p, __half* __restrict__ p16, const float* __restrict__ g,
                       float* __restrict__ m, float* __restrict__ v, size_t n, float lr, float b1, float b2, float eps,
                       float c1, float c2) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float pi = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
        p[i] = pi;
        p16[i] = __float2half_rn(pi);
    }
}

__global__ void k_to_half(const float* __restrict__ p, __half* __restrict__ p16, size_t n) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        p16[i] = __float2half_rn(p[i]);
}

// Counter-based initialisation (SplitMix64 of the index and seed -> uniform in [-a, a)).
__global__ void k_init_uniform(float* __restrict__ p, size_t n, unsigned long long seed, float a) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        unsigned long long z = seed + (unsigned long long)i * 0x9E3779B97F4A7C15ull;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        const float u = (float)(z >> 40) * (1.0f / 16777216.0f);
        p[i] = (2.f * u - 1.f) * a;
    }
}

// ------------------------------------------------------------------ top-k joint bins
// score(q, d) = log_softmax(lq)[q] + log_softmax(ld)[d]; the k best joint bins q * nd + d of each
// sample, best first; ties to the lower bin.
__global__ void __launch_bounds__(kT) k_topk_joint(const float* __restrict__ lq, int nq, const float* __restrict__ ld,
                                                   int nd, int k, int* __restrict__ bins, float* __restrict__ scores) {
    const int b = blockIdx.x;
    const float* q = lq + (size_t)b * nq;
    const float* d = ld + (size_t)b * nd;
    __shared__ float rv[kT];
    __shared__ int ri[kT];
    __shared__ float lse_q, lse_d;
    __shared__ float dls[64];
    // log-sum-exp of both heads
    for (int head = 0; head < 2; ++head) {
        const float* l = head ? d : q;
        const int n = head ? nd : nq;
        float m = -INFINITY;
        for (int i = threadIdx.x; i < n; i += blockDim.x) m = fmaxf(m, l[i]);
        rv[threadIdx.x] = m;
        __syncthreads();
        for (int st = blockDim.x / 2; st > 0; st >>= 1) {
            if (threadIdx.x < st) rv[threadIdx.x] = fmaxf(rv[threadIdx.x], rv[threadIdx.x + st]);
            __syncthreads();
        }
        m = rv[0];
        __syncthreads();
        float s = 0.f;
        for (int i = threadIdx.x; i < n; i += blockDim.x) s += expf(l[i] - m);
        rv[threadIdx.x] = s;
        __syncthreads();
        for (int st = blockDim.x / 2; st > 0; st >>= 1) {
            if (threadIdx.x < st) rv[threadIdx.x] += rv[threadIdx.x + st];
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            if (head) lse_d = m + logf(rv[0]);
            else lse_q = m + logf(rv[0]);
        }
        __syncthreads();
    }
    for (int i = threadIdx.x; i < nd; i += blockDim.x) dls[i] = d[i] - lse_d;
    __syncthreads();
    const int total = nq * nd;
    int last = -1;
    float last_v = INFINITY;
    for (int r = 0; r < k; ++r) {
        float bv = -INFINITY;
        int bi = 0x7fffffff;
        for (int j = threadIdx.x; j < total; j += blockDim.x) {
            const int qi = j / nd, di = j - (j / nd) * nd;
            const float v = q[qi] - lse_q + dls[di];
            // strictly after the previous pick in (value desc, index asc) order
            const bool after = (v < last_v) || (v == last_v && j > last);
            if (after && (v > bv || (v == bv && j < bi))) {
                bv = v;
                bi = j;
            }
        }
        rv[threadIdx.x] = bv;
        ri[threadIdx.x] = bi;
        __syncthreads();
        for (int st = blockDim.x / 2; st > 0; st >>= 1) {
            if (threadIdx.x < st) {
                const float v2 = rv[threadIdx.x + st];
                const int i2 = ri[threadIdx.x + st];
                if (v2 > rv[threadIdx.x] || (v2 == rv[threadIdx.x] && i2 < ri[threadIdx.x])) {
                    rv[threadIdx.x] = v2;
                    ri[threadIdx.x] = i2;
                }
            }
            __syncthreads();
        }
        last = ri[0];
        last_v = rv[0];
        if (threadIdx.x == 0) {
            bins[(size_t)b * k + r] = last;
            if (scores) scores[(size_t)b * k + r] = last_v;
        }
        __syncthreads();
    }
}

int grid_for(size_t n) {
    size_t g = (n + kT - 1) / kT;
    return (int)(g < 65535 * 4 ? (g < 1 ? 1 : g) : 65535 * 4);
}

}  // namespace

struct bioem_cnn {
    bioem_ctx* ctx;
    int device;            // bioem_cnn_free uses these, never the (possibly destroyed) context
    cudaStream_t stream;
    int S, C, n_q, n_d, max_batch, down, n_in;
    Layer layers[kLayers];
    size_t n_params, F;
    float* d_p;        // float32 master parameters
    __half* d_p16;     // float16 copy used by the passes
    float* d_g;        // gradients
    float* d_m;        // Adam moments
    float* d_v;
    long long step;
    float* d_act;      // activations: x0 (input) then every layer output
    float* d_gact;     // their gradients
    size_t act_per_sample;
    float* d_lq;       // [max_batch][n_q]
    float* d_ld;       // [max_batch][n_d]
    float* d_loss;     // [max_batch]
};

namespace {

template <class T>
int cnn_alloc(bioem_ctx* ctx, T** p, size_t n) {
    if (cudaMalloc((void**)p, sizeof(T) * (n ? n : 1)) != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        return bioem_set_error(ctx, BIOEM_ERR_OOM, "network allocation of %zu bytes", sizeof(T) * n);
    }
    return BIOEM_OK;
}

int check(bioem_ctx* ctx, const char* what) { return bioem_check_cuda(ctx, cudaGetLastError(), what); }

struct HeadOffsets {
    size_t wq, bq, wd, bd;
};

HeadOffsets heads(const bioem_cnn* n) {
    HeadOffsets h;
    h.wq = n->layers[kLayers - 1].b_off + n->C;
    h.bq = h.wq + (size_t)n->n_q * n->F;
    h.wd = h.bq + n->n_q;
    h.bd = h.wd + (size_t)n->n_d * n->F;
    return h;
}

int prepare_input(bioem_cnn* n, const float* d_images, int B) {
    k_downsample_norm<<<B, kT, 0, n->ctx->stream>>>(d_images, n->n_in, n->down, n->d_act);
    n->ctx->n_launches++;
    return check(n->ctx, "cnn input");
}

// Forward from the prepared input (x0 at d_act) of B samples; logits into d_lq, d_ld.
int forward(bioem_cnn* n, int B) {
    bioem_ctx* ctx = n->ctx;
    cudaStream_t st = ctx->stream;
    for (int l = 0; l < kLayers; ++l) {
        const Layer& Ly = n->layers[l];
        const float* in = n->d_act + Ly.in_off * B;
        float* out = n->d_act + Ly.out_off * B;
        const size_t per = (size_t)B * Ly.hout * Ly.hout;
        dim3 grid((unsigned)((per + kT - 1) / kT < 2048 ? (per + kT - 1) / kT : 2048), Ly.cout);
        k_conv_fwd<<<grid, kT, sizeof(float) * Ly.cin * 9, st>>>(in, n->d_p16 + Ly.w_off, n->d_p16 + Ly.b_off, B, Ly.cin,
                                                                Ly.cout, Ly.hin, Ly.hout, Ly.stride, out);
        ctx->n_launches++;
    }
    const float* feat = n->d_act + n->layers[kLayers - 1].out_off * B;
    const HeadOffsets h = heads(n);
    dim3 gq((n->n_q + 63) / 64, (B + 63) / 64), gd((n->n_d + 63) / 64, (B + 63) / 64);
    k_gemm<__half><<<gq, 256, 0, st>>>(feat, (long long)n->F, 1, n->d_p16 + h.wq, (long long)n->F, 1, n->d_p16 + h.bq,
                                       n->d_lq, B, n->n_q, (int)n->F, n->n_q, 0);
    k_gemm<__half><<<gd, 256, 0, st>>>(feat, (long long)n->F, 1, n->d_p16 + h.wd, (long long)n->F, 1, n->d_p16 + h.bd,
                                       n->d_ld, B, n->n_d, (int)n->F, n->n_d, 0);
    ctx->n_launches += 2;
    return check(ctx, "cnn forward");
}

// Loss and every parameter gradient (into d_g) for B labelled samples, after forward().
int backward(bioem_cnn* n, const int* d_yq, const int* d_yd, int B) {
    bioem_ctx* ctx = n->ctx;
    cudaStream_t st = ctx->stream;
    k_softmax_ce<<<B, kT, 0, st>>>(n->d_lq, n->n_q, n->d_ld, n->n_d, d_yq, d_yd, B, n->d_loss);
    const Layer& last = n->layers[kLayers - 1];
    const float* feat = n->d_act + last.out_off * B;
    const HeadOffsets h = heads(n);
    const int F = (int)n->F;
    // head weights gW[o][f] = sum_b glogit[b][o] feat[b][f]; biases: column sums
    dim3 g1((F + 63) / 64, (n->n_q + 63) / 64), g2((F + 63) / 64, (n->n_d + 63) / 64);
    k_gemm<float><<<g1, 256, 0, st>>>(n->d_lq, 1, n->n_q, feat, 1, F, nullptr, n->d_g + h.wq, n->n_q, F, B, F, 0);
    k_gemm<float><<<g2, 256, 0, st>>>(n->d_ld, 1, n->n_d, feat, 1, F, nullptr, n->d_g + h.wd, n->n_d, F, B, F, 0);
    k_colsum<<<(n->n_q + 255) / 256, 256, 0, st>>>(n->d_lq, B, n->n_q, n->d_g + h.bq);
    k_colsum<<<(n->n_d + 255) / 256, 256, 0, st>>>(n->d_ld, B, n->n_d, n->d_g + h.bd);
    // feature gradient gfeat[b][f] = sum_o glq[b][o] Wq[o][f] + sum_o gld[b][o] Wd[o][f]
    float* gfeat = n->d_gact + last.out_off * B;
    dim3 g3((F + 63) / 64, (B + 63) / 64);
    k_gemm<__half><<<g3, 256, 0, st>>>(n->d_lq, n->n_q, 1, n->d_p16 + h.wq, 1, F, nullptr, gfeat, B, F, n->n_q, F, 0);
    k_gemm<__half><<<g3, 256, 0, st>>>(n->d_ld, n->n_d, 1, n->d_p16 + h.wd, 1, F, nullptr, gfeat, B, F, n->n_d, F, 1);
    ctx->n_launches += 7;
    // conv layers, last to first
    for (int l = kLayers - 1; l >= 0; --l) {
        const Layer& Ly = n->layers[l];
        const float* out = n->d_act + Ly.out_off * B;
        float* gout = n->d_gact + Ly.out_off * B;
        const size_t nout = (size_t)B * Ly.cout * Ly.hout * Ly.hout;
        k_relu_bwd<<<grid_for(nout), kT, 0, st>>>(out, gout, nout);
        const float* in = n->d_act + Ly.in_off * B;
        k_conv_bwd_weight<<<Ly.cout * Ly.cin, kT, 0, st>>>(gout, in, B, Ly.cin, Ly.cout, Ly.hin, Ly.hout, Ly.stride,
                                                           n->d_g + Ly.w_off, n->d_g + Ly.b_off);
        ctx->n_launches += 2;
        if (l > 0) {
            const size_t nin = (size_t)B * Ly.cin * Ly.hin * Ly.hin;
            k_conv_bwd_data<<<grid_for(nin), kT, 0, st>>>(gout, n->d_p16 + Ly.w_off, B, Ly.cin, Ly.cout, Ly.hin, Ly.hout,
                                                          Ly.stride, n->d_gact + Ly.in_off * B);
            ctx->n_launches++;
        }
    }
    return check(ctx, "cnn backward");
}

}  // namespace

extern "C" {

int bioem_cnn_create(bioem_ctx* ctx, int image_px, int downsample, int channels, int n_qbins, int n_dbins,
                     int max_batch, unsigned long long seed, bioem_cnn** out) {
    if (!ctx || !out) return BIOEM_ERR_INVALID_ARG;
    *out = nullptr;
    if (downsample < 1 || image_px % downsample || (image_px / downsample) % 8 || image_px / downsample < 8 ||
        channels < 1 || channels > 64 || n_qbins < 1 || n_dbins < 1 || n_dbins > 64 || max_batch < 1)
        return bioem_set_error(ctx, BIOEM_ERR_INVALID_ARG, "cnn_create: bad shape");
    if (cudaSetDevice(ctx->device) != cudaSuccess) return bioem_set_error(ctx, BIOEM_ERR_CUDA, "cudaSetDevice");
    bioem_cnn* n = new (std::nothrow) bioem_cnn();
    if (!n) return BIOEM_ERR_OOM;
    n->ctx = ctx;
    n->device = ctx->device;
    n->stream = ctx->stream;
    n->n_in = image_px;
    n->down = downsample;
    n->S = image_px / downsample;
    n->C = channels;
    n->n_q = n_qbins;
    n->n_d = n_dbins;
    n->max_batch = max_batch;
    const int strides[kLayers] = {1, 2, 1, 2, 1, 2};
    size_t poff = 0, aoff = (size_t)n->S * n->S;   // x0 occupies the first S^2 per sample
    int h = n->S, cin = 1;
    for (int l = 0; l < kLayers; ++l) {
        Layer& Ly = n->layers[l];
        Ly.cin = cin;
        Ly.cout = channels;
        Ly.stride = strides[l];
        Ly.hin = h;
        Ly.hout = h / strides[l];
        Ly.w_off = poff;
        poff += (size_t)channels * cin * 9;
        Ly.b_off = poff;
        poff += channels;
        Ly.in_off = (l == 0) ? 0 : n->layers[l - 1].out_off;
        Ly.out_off = aoff;
        aoff += (size_t)channels * Ly.hout * Ly.hout;
        h = Ly.hout;
        cin = channels;
    }
    n->F = (size_t)channels * h * h;
    n->n_params = poff + (size_t)n_qbins * n->F + n_qbins + (size_t)n_dbins * n->F + n_dbins;
    n->act_per_sample = aoff;
    int rc = cnn_alloc(ctx, &n->d_p, n->n_params);
    if (!rc) rc = cnn_alloc(ctx, &n->d_p16, n->n_params);
    if (!rc) rc = cnn_alloc(ctx, &n->d_g, n->n_params);
    if (!rc) rc = cnn_alloc(ctx, &n->d_m, n->n_params);
    if (!rc) rc = cnn_alloc(ctx, &n->d_v, n->n_params);
    if (!rc) rc = cnn_alloc(ctx, &n->d_act, n->act_per_sample * max_batch);
    if (!rc) rc = cnn_alloc(ctx, &n->d_gact, n->act_per_sample * max_batch);
    if (!rc) rc = cnn_alloc(ctx, &n->d_lq, (size_t)max_batch * n_qbins);
    if (!rc) rc = cnn_alloc(ctx, &n->d_ld, (size_t)max_batch * n_dbins);
    if (!rc) rc = cnn_alloc(ctx, &n->d_loss, (size_t)max_batch);
    if (rc) {
        bioem_cnn_free(n);
        return rc;
    }
    cudaStream_t st = ctx->stream;
    // uniform He-style initialisation per tensor: a = sqrt(6 / fan_in); biases zero
    for (int l = 0; l < kLayers; ++l) {
        const Layer& Ly = n->layers[l];
        const size_t nw = (size_t)Ly.cout * Ly.cin * 9;
        k_init_uniform<<<grid_for(nw), kT, 0, st>>>(n->d_p + Ly.w_off, nw, seed + 1000003ull * l,
                                                    sqrtf(6.f / (9.f * Ly.cin)));
        cudaMemsetAsync(n->d_p + Ly.b_off, 0, sizeof(float) * Ly.cout, st);
    }
    const HeadOffsets hd = heads(n);
    k_init_uniform<<<grid_for((size_t)n_qbins * n->F), kT, 0, st>>>(n->d_p + hd.wq, (size_t)n_qbins * n->F, seed + 77ull,
                                                                     sqrtf(3.f / (float)n->F));
    k_init_uniform<<<grid_for((size_t)n_dbins * n->F), kT, 0, st>>>(n->d_p + hd.wd, (size_t)n_dbins * n->F, seed + 78ull,
                                                                     sqrtf(3.f / (float)n->F));
    cudaMemsetAsync(n->d_p + hd.bq, 0, sizeof(float) * n_qbins, st);
    cudaMemsetAsync(n->d_p + hd.bd, 0, sizeof(float) * n_dbins, st);
    cudaMemsetAsync(n->d_m, 0, sizeof(float) * n->n_params, st);
    cudaMemsetAsync(n->d_v, 0, sizeof(float) * n->n_params, st);
    k_to_half<<<grid_for(n->n_params), kT, 0, st>>>(n->d_p, n->d_p16, n->n_params);
    ctx->n_launches += kLayers + 3;
    rc = check(ctx, "cnn init");
    if (rc) {
        bioem_cnn_free(n);
        return rc;
    }
    *out = n;
    return BIOEM_OK;
}

long long bioem_cnn_num_params(const bioem_cnn* n) { return n ? (long long)n->n_params : -1; }

int bioem_cnn_set_params(bioem_cnn* n, const float* d_params) {
    if (!n || !d_params) return BIOEM_ERR_INVALID_ARG;
    cudaSetDevice(n->ctx->device);
    cudaStream_t st = n->ctx->stream;
    cudaError_t e = cudaMemcpyAsync(n->d_p, d_params, sizeof(float) * n->n_params, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return bioem_check_cuda(n->ctx, e, "set params");
    k_to_half<<<grid_for(n->n_params), kT, 0, st>>>(n->d_p, n->d_p16, n->n_params);
    n->ctx->n_launches++;
    cudaMemsetAsync(n->d_m, 0, sizeof(float) * n->n_params, st);
    cudaMemsetAsync(n->d_v, 0, sizeof(float) * n->n_params, st);
    n->step = 0;
    return check(n->ctx, "set params");
}

int bioem_cnn_get_params(bioem_cnn* n, float* d_params) {
    if (!n || !d_params) return BIOEM_ERR_INVALID_ARG;
    cudaSetDevice(n->ctx->device);
    return bioem_check_cuda(n->ctx, cudaMemcpyAsync(d_params, n->d_p, sizeof(float) * n->n_params,
                                                    cudaMemcpyDeviceToDevice, n->ctx->stream), "get params");
}

int bioem_cnn_forward(bioem_cnn* n, const float* d_images, int B, float* d_logits_q, float* d_logits_d) {
    if (!n || !d_images || B < 1 || B > n->max_batch) return BIOEM_ERR_INVALID_ARG;
    cudaSetDevice(n->ctx->device);
    int rc = prepare_input(n, d_images, B);
    if (!rc) rc = forward(n, B);
    cudaStream_t st = n->ctx->stream;
    if (!rc && d_logits_q)
        rc = bioem_check_cuda(n->ctx, cudaMemcpyAsync(d_logits_q, n->d_lq, sizeof(float) * B * n->n_q,
                                                      cudaMemcpyDeviceToDevice, st), "logits");
    if (!rc && d_logits_d)
        rc = bioem_check_cuda(n->ctx, cudaMemcpyAsync(d_logits_d, n->d_ld, sizeof(float) * B * n->n_d,
                                                      cudaMemcpyDeviceToDevice, st), "logits");
    return rc;
}

int bioem_cnn_gradients(bioem_cnn* n, const float* d_images, const int* d_label_q, const int* d_label_d, int B,
                        float* d_grads, float* d_loss) {
    if (!n || !d_images || !d_label_q || !d_label_d || B < 1 || B > n->max_batch) return BIOEM_ERR_INVALID_ARG;
    cudaSetDevice(n->ctx->device);
    int rc = prepare_input(n, d_images, B);
    if (!rc) rc = forward(n, B);
    if (!rc) rc = backward(n, d_label_q, d_label_d, B);
    cudaStream_t st = n->ctx->stream;
    if (!rc && d_grads)
        rc = bioem_check_cuda(n->ctx, cudaMemcpyAsync(d_grads, n->d_g, sizeof(float) * n->n_params,
                                                      cudaMemcpyDeviceToDevice, st), "gradients");
    if (!rc && d_loss)
        rc = bioem_check_cuda(n->ctx, cudaMemcpyAsync(d_loss, n->d_loss, sizeof(float) * B, cudaMemcpyDeviceToDevice, st),
                              "loss");
    return rc;
}

int bioem_cnn_train_step(bioem_cnn* n, const float* d_images, const int* d_label_q, const int* d_label_d, int B,
                         float lr, float* d_loss) {
    int rc = bioem_cnn_gradients(n, d_images, d_label_q, d_label_d, B, nullptr, d_loss);
    if (rc) return rc;
    n->step++;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - powf(b1, (float)n->step), c2 = 1.f - powf(b2, (float)n->step);
    k_adam<<<grid_for(n->n_params), kT, 0, n->ctx->stream>>>(n->d_p, n->d_p16, n->d_g, n->d_m, n->d_v, n->n_params, lr,
                                                             b1, b2, 1e-8f, c1, c2);
    n->ctx->n_launches++;
    return check(n->ctx, "adam");
}

int bioem_propose(bioem_cnn* n, const float* d_images, int n_img, int k, int* d_bins, float* d_scores) {
    if (!n || !d_images || n_img < 0 || k < 1 || k > n->n_q * n->n_d || !d_bins) return BIOEM_ERR_INVALID_ARG;
    cudaSetDevice(n->ctx->device);
    for (int b0 = 0; b0 < n_img; b0 += n->max_batch) {
        const int B = n_img - b0 < n->max_batch ? n_img - b0 : n->max_batch;
        int rc = prepare_input(n, d_images + (size_t)b0 * n->n_in * n->n_in, B);
        if (!rc) rc = forward(n, B);
        if (rc) return rc;
        k_topk_joint<<<B, kT, 0, n->ctx->stream>>>(n->d_lq, n->n_q, n->d_ld, n->n_d, k, d_bins + (size_t)b0 * k,
                                                   d_scores ? d_scores + (size_t)b0 * k : nullptr);
        n->ctx->n_launches++;
        rc = check(n->ctx, "propose");
        if (rc) return rc;
    }
    return BIOEM_OK;
}

void bioem_cnn_free(bioem_cnn* n) {
    if (!n) return;
    cudaSetDevice(n->device);
    cudaStreamSynchronize(n->stream);
    cudaFree(n->d_p);
    cudaFree(n->d_p16);
    cudaFree(n->d_g);
    cudaFree(n->d_m);
    cudaFree(n->d_v);
    cudaFree(n->d_act);
    cudaFree(n->d_gact);
    cudaFree(n->d_lq);
    cudaFree(n->d_ld);
    cudaFree(n->d_loss);
    cudaGetLastError();
    delete n;
}

}  // extern "C"
