// Learned RFI flagger: a 4-layer 5x5 convolutional network (1 -> 32 -> 32 ->
// 32 -> 1 channels, ReLU, logistic output) over (time x channel) tiles of
// autocorrelation power, trained and run on the GPU, with the MAD rule of
// Eq. 2 (Sec. 7) as the fallback on tiles where the network is not confident.
//
// Every convolution is an im2col product on the tcgen05 GEMM (BF16 operands,
// FP32 accumulation):
//   forward   Z[p][o]   = sum_k A[p][k] Wf[o][k],   A = im2col(X), k = (5u+v) C + c
//   data grad dX[p][c]  = sum_k A'[p][k] Wd[c][k],  A' = im2col of dZ at negated offsets
//   weight    dW^T[k][o] = sum_p A^T[k][p] dZ^T[o][p]  (K = pixels, split over CTAs)
// Activations are NHWC BF16; FP32 master weights with Adam.
#include "corr.h"
#include "corr_internal.h"

#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

namespace corr {
namespace {

constexpr int TH = 64, TW = 256, TPIX = TH * TW;   // tile: 64 rows (time) x 256 channels
constexpr int NL = 4;
constexpr int kChunk = 64;   // tiles per pass through the network (workspace bound)
constexpr int CI[NL] = {1, 32, 32, 32};
constexpr int CO[NL] = {32, 32, 32, 1};

__host__ __device__ inline int kpad(int k) { return (k + 63) / 64 * 64; }
__host__ __device__ inline int npad(int co) { return co < 16 ? 16 : co; }

__device__ __forceinline__ uint16_t f2bf(float x) { return __bfloat16_as_ushort(__float2bfloat16_rn(x)); }
__device__ __forceinline__ float bf2f(uint16_t x) { return __bfloat162float(__ushort_as_bfloat16(x)); }

// A[p][k] = X[n][i+u-2][j+v-2][c] (k = (5u+v) C + c < 25 C, else 0) for
// C = 32: one 16-byte chunk (8 channels of one tap) per thread.  sgn = -1
// gives the negated offsets of the data-gradient product.
__global__ void im2col32_kernel(const uint4* X, int P, int sgn, uint4* A) {
    constexpr int KP = 832, SL = KP / 8, CS = 4;     // 104 chunks per row, 4 per pixel
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)P * SL) return;
    const int p = (int)(idx / SL), s = (int)(idx % SL);
    uint4 v = make_uint4(0, 0, 0, 0);
    if (s < 25 * CS) {
        const int tap = s >> 2, c8 = s & 3, u = tap / 5, w = tap % 5;
        const int n = p / TPIX, ij = p % TPIX, i = ij / TW, j = ij % TW;
        const int ii = i + sgn * (u - 2), jj = j + sgn * (w - 2);
        if (ii >= 0 && ii < TH && jj >= 0 && jj < TW) v = X[((size_t)n * TPIX + ii * TW + jj) * CS + c8];
    }
    A[idx] = v;
}

// The same for C = 1 (K = 25 taps padded to 64): 8 taps per thread.
__global__ void im2col1_kernel(const uint16_t* X, int P, int sgn, uint4* A) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)P * 8) return;
    const int p = (int)(idx >> 3), s = (int)(idx & 7);
    const int n = p / TPIX, ij = p % TPIX, i = ij / TW, j = ij % TW;
    uint32_t w[4] = {0, 0, 0, 0};
#pragma unroll
    for (int e = 0; e < 8; ++e) {
        const int k = s * 8 + e;
        if (k < 25) {
            const int ii = i + sgn * (k / 5 - 2), jj = j + sgn * (k % 5 - 2);
            if (ii >= 0 && ii < TH && jj >= 0 && jj < TW)
                w[e >> 1] |= (uint32_t)X[(size_t)n * TPIX + ii * TW + jj] << (16 * (e & 1));
        }
    }
    A[idx] = make_uint4(w[0], w[1], w[2], w[3]);
}

// AT[k][p] = A[p][k] for C = 32 (the weight-gradient operand, K = pixels):
// one CTA per 64-pixel row segment stages the 5 x 68-pixel neighbourhood in
// shared memory (channel stride padded to 34), then writes each k-row's 64
// pixels as 8 coalesced 16-byte chunks.
constexpr int kSegPix = 64, kHalo = kSegPix + 4, kCPad = 34;
__global__ void __launch_bounds__(256) im2colT32_kernel(const uint16_t* X, int P, uint16_t* AT) {
    __shared__ uint32_t sx[5 * kHalo * kCPad / 2];
    const int p0 = blockIdx.x * kSegPix;
    const int n = p0 / TPIX, i = (p0 % TPIX) / TW, j0 = p0 % TW;
    // stage: (u, jj, c8) chunks of 8 channels
    for (int t = threadIdx.x; t < 5 * kHalo * 4; t += blockDim.x) {
        const int c8 = t & 3, jj = (t >> 2) % kHalo, u = (t >> 2) / kHalo;
        const int ii = i + u - 2, jx = j0 + jj - 2;
        uint4 v = make_uint4(0, 0, 0, 0);
        if (ii >= 0 && ii < TH && jx >= 0 && jx < TW)
            v = reinterpret_cast<const uint4*>(X + ((size_t)n * TPIX + ii * TW + jx) * 32)[c8];
        uint32_t* d = sx + ((u * kHalo + jj) * kCPad + c8 * 8) / 2;
        d[0] = v.x;
        d[1] = v.y;
        d[2] = v.z;
        d[3] = v.w;
    }
    __syncthreads();
    const uint16_t* s16 = reinterpret_cast<const uint16_t*>(sx);
    for (int t = threadIdx.x; t < 832 * 8; t += blockDim.x) {
        const int g = t & 7, k = t >> 3;
        uint32_t w[4] = {0, 0, 0, 0};
        if (k < 800) {
            const int tap = k >> 5, c = k & 31, u = tap / 5, v = tap % 5;
            const uint16_t* src = s16 + (u * kHalo + g * 8 + v) * kCPad + c;
#pragma unroll
            for (int e = 0; e < 8; ++e) w[e >> 1] |= (uint32_t)src[e * kCPad] << (16 * (e & 1));
        }
        *reinterpret_cast<uint4*>(AT + (size_t)k * P + p0 + g * 8) = make_uint4(w[0], w[1], w[2], w[3]);
    }
}

// AT[k][p] for C = 1 (k < 25 taps, rows up to 64 zero): 8 pixels per thread.
__global__ void im2colT1_kernel(const uint16_t* X, int P, uint16_t* AT) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)P * 8) return;
    const int k = (int)(idx / (P / 8)), p = (int)(idx % (P / 8)) * 8;
    const int n = p / TPIX, ij = p % TPIX, i = ij / TW, j = ij % TW;
    uint32_t w[4] = {0, 0, 0, 0};
    if (k < 25) {
        const int ii = i + k / 5 - 2;
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const int jj = j + e + k % 5 - 2;
            if (ii >= 0 && ii < TH && jj >= 0 && jj < TW)
                w[e >> 1] |= (uint32_t)X[(size_t)n * TPIX + ii * TW + jj] << (16 * (e & 1));
        }
    }
    *reinterpret_cast<uint4*>(AT + (size_t)k * P + p) = make_uint4(w[0], w[1], w[2], w[3]);
}

__global__ void input_bf16_kernel(const float* x, int P, uint16_t* X) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < P) X[p] = f2bf(x[p]);
}

// dz = (sigmoid(z) - t) / P_total as FP32 and BF16 (NHWC and transposed),
// plus per-block partial sums of the loss softplus(z) - t z.
__global__ void loss_grad_kernel(const float* z, const uint8_t* t, int P, float inv_total, float* dz32,
                                 uint16_t* dz, uint16_t* dzT, float* loss_part) {
    __shared__ float red[256];
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    float l = 0.f;
    if (p < P) {
        const float zz = z[p], tt = t[p] ? 1.f : 0.f;
        const float s = 1.f / (1.f + expf(-zz));
        const float g = (s - tt) * inv_total;
        dz32[p] = g;
        dz[p] = f2bf(g);
        dzT[p] = f2bf(g);
        l = fmaxf(zz, 0.f) + log1pf(expf(-fabsf(zz))) - tt * zz;
    }
    red[threadIdx.x] = l;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) loss_part[blockIdx.x] = red[0];
}

// dz_prev[p][c] = D[p][c] * (act[p][c] > 0) in FP32, BF16 and transposed BF16.
__global__ void relu_grad_kernel(const float* D, const uint16_t* act, int P, int C, float* dz32, uint16_t* dz,
                                 uint16_t* dzT) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)P * C) return;
    const int p = (int)(idx / C), c = (int)(idx % C);
    const float g = bf2f(act[idx]) > 0.f ? D[(size_t)p * 32 + c] : 0.f;
    dz32[idx] = g;
    dz[idx] = f2bf(g);
    dzT[(size_t)c * P + p] = f2bf(g);
}

// Fixed-order column sums: out[c] = sum_p g[p][c].
__global__ void colsum_kernel(const float* g, int P, int C, float* out) {
    __shared__ float red[256];
    const int c = blockIdx.x;
    float acc = 0.f;
    for (int p = threadIdx.x; p < P; p += blockDim.x) acc += g[(size_t)p * C + c];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[c] = red[0];
}

__global__ void sum_kernel(const float* x, int n, float* out) {
    __shared__ float red[256];
    float acc = 0.f;
    for (int i = threadIdx.x; i < n; i += blockDim.x) acc += x[i];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = red[0];
}

// dW[o][c][u][v] = DW[(5u+v) C + c][o] (the weight-gradient product).
__global__ void gather_dw_kernel(const float* DW, int C, int Co, int Np, float* dw) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= Co * C * 25) return;
    const int o = idx / (C * 25), r = idx % (C * 25), c = r / 25, uv = r % 25;
    dw[idx] = DW[(size_t)(uv * C + c) * Np + o];
}

__global__ void adam_kernel(float* w, const float* g, float* m, float* v, int n, float lr, float b1, float b2,
                            float c1, float c2, float eps) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// Wf[o][(5u+v) C + c] = w[o][c][u][v]; Wd[c][(5u+v) Co + o] = w[o][c][u][v] (BF16).
__global__ void pack_weights_kernel(const float* w, int C, int Co, int Kf, int Kd, uint16_t* wf, uint16_t* wd) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= Co * C * 25) return;
    const int o = idx / (C * 25), r = idx % (C * 25), c = r / 25, uv = r % 25;
    const uint16_t b = f2bf(w[idx]);
    wf[(size_t)o * Kf + uv * C + c] = b;
    if (wd) wd[(size_t)c * Kd + uv * Co + o] = b;
}

// Output layer (32 -> 1 channel) on CUDA cores: one warp per 32
// consecutive pixels of a tile row, lane c holding input channel c.  Each
// lane streams the five input rows once (36 pixels a row, zero outside the
// tile) and forms all 32 outputs' partial sums over its channel with the
// layer's BF16 weights (FP32 sums); a 31-step exchange then leaves the sum
// over the channels of output x0 + l in lane l.  On the tensor cores the one
// output channel filled a sixteenth of each MMA.
__global__ void __launch_bounds__(256) conv_last_kernel(const uint16_t* __restrict__ act, int B,
                                                        const uint16_t* __restrict__ wf,
                                                        const float* __restrict__ bias, float* __restrict__ logit) {
    constexpr int SEG = TW / 32;
    const int lane = (int)threadIdx.x & 31;
    const long long wid = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (wid >= (long long)B * TH * SEG) return;   // uniform over the warp
    const int x0 = (int)(wid % SEG) * 32;
    const int i = (int)((wid / SEG) % TH);
    const int n = (int)(wid / ((long long)TH * SEG));
    float w[25];
#pragma unroll
    for (int t = 0; t < 25; ++t) w[t] = bf2f(wf[t * 32 + lane]);   // k = (5u + v) 32 + c, output row 0
    float acc[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) acc[j] = 0.f;
    const uint16_t* an = act + (size_t)n * TPIX * 32 + lane;
#pragma unroll
    for (int u = 0; u < 5; ++u) {
        const int ii = i + u - 2;
        if (ii < 0 || ii >= TH) continue;         // uniform over the warp
        float a[36];
#pragma unroll
        for (int q = 0; q < 36; ++q) {
            const int xx = x0 - 2 + q;
            a[q] = (xx >= 0 && xx < TW) ? bf2f(an[((size_t)ii * TW + xx) * 32]) : 0.f;
        }
#pragma unroll
        for (int v = 0; v < 5; ++v)
#pragma unroll
            for (int j = 0; j < 32; ++j) acc[j] = fmaf(w[5 * u + v], a[j + v], acc[j]);
    }
    // sum over the lanes: at distance d each lane keeps the half of its
    // outputs on its side of bit d and adds the partner's share of it
#pragma unroll
    for (int d = 16; d >= 1; d >>= 1) {
        const bool up = (lane & d) != 0;
#pragma unroll
        for (int j = 0; j < d; ++j) {
            const float send = up ? acc[j] : acc[j + d];
            const float keep = up ? acc[j + d] : acc[j];
            acc[j] = keep + __shfl_xor_sync(0xffffffffu, send, d);
        }
    }
    logit[(size_t)n * TPIX + (size_t)i * TW + x0 + lane] = acc[0] + __ldg(bias);
}

// Layer 0 (1 -> 32 channels) on CUDA cores in FP32: one thread per pixel
// takes its 5x5 neighbourhood of the FP32 input (zero outside the tile) and
// forms all 32 outputs, then stores BF16 ReLU(z + b) NHWC (64 bytes).  With
// one input channel the layer has 800 multiply-adds per pixel, too few to
// feed the tensor cores through an im2col buffer.
__global__ void __launch_bounds__(256) conv0_kernel(const float* x, int P, const float* w, const float* b,
                                                    uint16_t* act) {
    __shared__ float sw[32 * 25];
    __shared__ float sb[32];
    for (int i = threadIdx.x; i < 32 * 25; i += blockDim.x) sw[i] = w[i];
    if (threadIdx.x < 32) sb[threadIdx.x] = b[threadIdx.x];
    __syncthreads();
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    const int n = p / TPIX, ij = p % TPIX, i = ij / TW, j = ij % TW;
    const float* xt = x + (size_t)n * TPIX;
    float v[25];
#pragma unroll
    for (int u = 0; u < 5; ++u)
#pragma unroll
        for (int q = 0; q < 5; ++q) {
            const int ii = i + u - 2, jj = j + q - 2;
            v[5 * u + q] = (ii >= 0 && ii < TH && jj >= 0 && jj < TW) ? __ldg(xt + ii * TW + jj) : 0.f;
        }
    uint32_t pk[16];
#pragma unroll
    for (int o = 0; o < 32; o += 2) {
        float z0 = sb[o], z1 = sb[o + 1];
#pragma unroll
        for (int t = 0; t < 25; ++t) {
            z0 = fmaf(sw[o * 25 + t], v[t], z0);
            z1 = fmaf(sw[(o + 1) * 25 + t], v[t], z1);
        }
        const __nv_bfloat162 h = __floats2bfloat162_rn(fmaxf(z0, 0.f), fmaxf(z1, 0.f));
        pk[o >> 1] = *reinterpret_cast<const uint32_t*>(&h);
    }
    uint4* o4 = reinterpret_cast<uint4*>(act + (size_t)p * 32);
#pragma unroll
    for (int q = 0; q < 4; ++q) o4[q] = make_uint4(pk[4 * q], pk[4 * q + 1], pk[4 * q + 2], pk[4 * q + 3]);
}

// Order-preserving 32-bit key of a float (larger float, larger key).
__device__ __forceinline__ uint32_t fkey(float f) {
    const uint32_t u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float fkey_inv(uint32_t k) {
    return __uint_as_float((k & 0x80000000u) ? (k & 0x7FFFFFFFu) : ~k);
}

// x = ln(P / median(P)) per tile with the exact median (mean of the order
// statistics of rank 8191 and 8192 of 16384) found by a radix select: four
// passes of 8 bits over the order-preserving keys, each a 256-bin histogram
// of the candidates sharing the prefix found so far.
__global__ void __launch_bounds__(1024) median_normalize_kernel(const float* power, float* x) {
    constexpr int PER = TPIX / 1024;          // 16 values per thread
    __shared__ unsigned int hist[256];
    __shared__ uint32_t s_prefix;
    __shared__ int s_rank;
    __shared__ uint32_t s_next;
    const float* P = power + (size_t)blockIdx.x * TPIX;
    uint32_t key[PER];
#pragma unroll
    for (int e = 0; e < PER; ++e) key[e] = fkey(P[threadIdx.x + e * 1024]);
    if (threadIdx.x == 0) {
        s_prefix = 0;
        s_rank = TPIX / 2 - 1;
        s_next = 0xFFFFFFFFu;
    }
    for (int pass = 0; pass < 4; ++pass) {
        const int shift = 24 - 8 * pass;
        if (threadIdx.x < 256) hist[threadIdx.x] = 0;
        __syncthreads();
        const uint32_t prefix = s_prefix;
        const uint32_t pmask = pass == 0 ? 0u : (0xFFFFFFFFu << (shift + 8));
#pragma unroll
        for (int e = 0; e < PER; ++e)
            if ((key[e] & pmask) == prefix) atomicAdd(&hist[(key[e] >> shift) & 0xFF], 1u);
        __syncthreads();
        if (threadIdx.x == 0) {
            int r = s_rank;
            int d = 0;
            while (r >= (int)hist[d]) {
                r -= (int)hist[d];
                ++d;
            }
            s_rank = r;
            s_prefix = prefix | ((uint32_t)d << shift);
        }
        __syncthreads();
    }
    // s_prefix is the key of rank 8191; the rank-8192 value is the same key
    // when it repeats beyond that rank, else the smallest larger key
    const uint32_t k1 = s_prefix;
    unsigned int cnt_le = 0;
    uint32_t next = 0xFFFFFFFFu;
#pragma unroll
    for (int e = 0; e < PER; ++e) {
        if (key[e] <= k1) ++cnt_le;
        else next = min(next, key[e]);
    }
    if (threadIdx.x == 0) hist[0] = 0;
    __syncthreads();
    atomicAdd(&hist[0], cnt_le);
    atomicMin(&s_next, next);
    __syncthreads();
    const float v1 = fkey_inv(k1);
    const float v2 = hist[0] > (unsigned)(TPIX / 2) ? v1 : fkey_inv(s_next);
    const float med = 0.5f * (v1 + v2);
    const float inv = med > 0.f ? 1.f / med : 1.f;
    for (int i = threadIdx.x; i < TPIX; i += 1024)
        x[(size_t)blockIdx.x * TPIX + i] = logf(fmaxf(P[i] * inv, 1e-30f));
}

// Per tile: confidence = mean |2p - 1|, p = sigmoid(logit).
__global__ void confidence_kernel(const float* logit, float* conf) {
    __shared__ float red[256];
    const float* z = logit + (size_t)blockIdx.x * TPIX;
    float acc = 0.f;
    for (int i = threadIdx.x; i < TPIX; i += blockDim.x) acc += fabsf(2.f / (1.f + expf(-z[i])) - 1.f);
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) conf[blockIdx.x] = red[0] / (float)TPIX;
}

__device__ float warp_median64(const float* v, float* sorted, int lane) {
    for (int c = lane; c < 64; c += 32) {
        const float x = v[c];
        int rank = 0;
        for (int d = 0; d < 64; ++d) {
            const float y = v[d];
            rank += (y < x) || (y == x && d < c);
        }
        sorted[rank] = x;
    }
    __syncwarp();
    const float med = 0.5f * (sorted[31] + sorted[32]);
    __syncwarp();
    return med;
}

// Flags of a tile: the network's (p > 1/2) when conf >= c_min, else Eq. 2
// along each row over aligned windows of 64 channels (always Eq. 2 when
// conf is null).  One warp per (tile, row, window).
__global__ void final_flags_kernel(const float* power, const float* logit, const float* conf, int B, float c_min,
                                   float sigma, uint8_t* flags) {
    __shared__ float sm[4][3][64];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long item = (long long)blockIdx.x * 4 + warp;
    if (item >= (long long)B * TH * (TW / 64)) return;
    const int win = (int)(item % (TW / 64));
    const int r = (int)((item / (TW / 64)) % TH);
    const int t = (int)(item / ((TW / 64) * TH));
    const size_t base = (size_t)t * TPIX + (size_t)r * TW + win * 64;
    if (conf && conf[t] >= c_min) {
        for (int c = lane; c < 64; c += 32) flags[base + c] = logit[base + c] > 0.f ? 1 : 0;
        return;
    }
    float* vA = sm[warp][0];
    float* vS = sm[warp][1];
    float* vD = sm[warp][2];
    for (int c = lane; c < 64; c += 32) vA[c] = power[base + c];
    __syncwarp();
    const float med = warp_median64(vA, vS, lane);
    for (int c = lane; c < 64; c += 32) vD[c] = fabsf(vA[c] - med);
    __syncwarp();
    const float mad = warp_median64(vD, vS, lane);
    const float T = med + sigma * mad * 1.4826f;
    for (int c = lane; c < 64; c += 32) flags[base + c] = vA[c] > T ? 1 : 0;
}

// Eq. 2 along time: per (tile, channel) over the tile's 64 rows; the flags
// are OR-ed into `flags` when `accumulate` is set.  One warp per item.
__global__ void mad_time_kernel(const float* power, int B, float sigma, bool accumulate, uint8_t* flags) {
    __shared__ float sm[4][3][64];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long item = (long long)blockIdx.x * 4 + warp;
    if (item >= (long long)B * TW) return;
    const int k = (int)(item % TW);
    const int t = (int)(item / TW);
    const size_t base = (size_t)t * TPIX + k;
    float* vA = sm[warp][0];
    float* vS = sm[warp][1];
    float* vD = sm[warp][2];
    for (int r = lane; r < TH; r += 32) vA[r] = power[base + (size_t)r * TW];
    __syncwarp();
    const float med = warp_median64(vA, vS, lane);
    for (int r = lane; r < TH; r += 32) vD[r] = fabsf(vA[r] - med);
    __syncwarp();
    const float mad = warp_median64(vD, vS, lane);
    const float T = med + sigma * mad * 1.4826f;
    for (int r = lane; r < TH; r += 32) {
        const uint8_t f = vA[r] > T ? 1 : 0;
        uint8_t* o = flags + base + (size_t)r * TW;
        *o = accumulate ? (uint8_t)(*o | f) : f;
    }
}

}  // namespace

}  // namespace corr

// ---------------------------------------------------------------------------
// C ABI of the flagger

using namespace corr;

struct corr_flagnet_s {
    int dev = 0;
    float* w[NL] = {};
    float* b[NL] = {};
    float* mw[NL] = {};
    float* vw[NL] = {};
    float* mb[NL] = {};
    float* vb[NL] = {};
    float* gw[NL] = {};
    float* gb[NL] = {};
    uint16_t* wf[NL] = {};   // [npad(Co)][kpad(25 Ci)]
    uint16_t* wd[NL] = {};   // [Ci][kpad(25 Co)]
    long long steps = 0;
    long long launches = 0;  // kernels launched by this handle
    int cap = 0;             // tiles the workspace holds
    uint16_t* act[NL + 1] = {};   // act[0] input BF16 [P], act[l] [P][32]
    float* logit = nullptr;
    uint16_t* A = nullptr;   // im2col scratch (largest: P x 832 or 832 x P)
    float* D = nullptr;      // GEMM output / partial sums
    float* D2 = nullptr;
    float* dz32 = nullptr;
    uint16_t* dz = nullptr;
    uint16_t* dzT = nullptr;
    float* loss_part = nullptr;
    float* scalar = nullptr;
    float* norm = nullptr;
    float* conf = nullptr;
    int* status = nullptr;
    std::string err;
};

namespace {

thread_local std::string g_fn_err;

int ffail(corr_flagnet_t n, int code, const std::string& m) {
    if (n) n->err = m;
    else g_fn_err = m;
    corr::set_global_error(m);
    return code;
}

#define FK(call)                                                                                 \
    do {                                                                                         \
        cudaError_t e_ = (call);                                                                 \
        if (e_ != cudaSuccess) return ffail(net, CORR_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

inline unsigned blocks(long long n, int t = 256) { return (unsigned)((n + t - 1) / t); }

int ensure_ws(corr_flagnet_t net, int B) {
    if (B <= net->cap) return CORR_OK;
    auto fr = [](void* p) { if (p) cudaFree(p); };
    for (int l = 0; l <= NL; ++l) fr(net->act[l]);
    fr(net->logit); fr(net->A); fr(net->D); fr(net->D2); fr(net->dz32); fr(net->dz); fr(net->dzT);
    fr(net->loss_part); fr(net->norm); fr(net->conf);
    const size_t P = (size_t)B * TPIX;
    FK(cudaMalloc(&net->act[0], P * 2));
    for (int l = 1; l <= NL; ++l) FK(cudaMalloc(&net->act[l], P * 32 * 2));
    FK(cudaMalloc(&net->logit, P * 4));
    FK(cudaMalloc(&net->A, P * 832 * 2));
    const int splits = 64;
    FK(cudaMalloc(&net->D, std::max(P * 32, (size_t)splits * 896 * 32) * 4));
    FK(cudaMalloc(&net->D2, (size_t)896 * 32 * 4));
    FK(cudaMalloc(&net->dz32, P * 32 * 4));
    FK(cudaMalloc(&net->dz, P * 32 * 2));
    FK(cudaMalloc(&net->dzT, P * 32 * 2));
    FK(cudaMemset(net->dzT, 0, P * 32 * 2));
    FK(cudaMalloc(&net->loss_part, blocks(P) * 4));
    FK(cudaMalloc(&net->norm, P * 4));
    FK(cudaMalloc(&net->conf, (size_t)B * 4));
    net->cap = B;
    return CORR_OK;
}

int repack(corr_flagnet_t net, cudaStream_t st) {
    net->launches += NL;
    for (int l = 0; l < NL; ++l) {
        const int n = CO[l] * CI[l] * 25;
        pack_weights_kernel<<<blocks(n), 256, 0, st>>>(net->w[l], CI[l], CO[l], kpad(25 * CI[l]), kpad(25 * CO[l]),
                                                       net->wf[l], l > 0 ? net->wd[l] : nullptr);
    }
    FK(cudaGetLastError());
    return CORR_OK;
}

// im2col of NHWC BF16 activations with C = 1 or 32 channels.
void im2col(const uint16_t* X, int C, int P, int sgn, uint16_t* A, cudaStream_t st) {
    if (C == 32)
        im2col32_kernel<<<blocks((long long)P * 104), 256, 0, st>>>(reinterpret_cast<const uint4*>(X), P, sgn,
                                                                    reinterpret_cast<uint4*>(A));
    else
        im2col1_kernel<<<blocks((long long)P * 8), 256, 0, st>>>(X, P, sgn, reinterpret_cast<uint4*>(A));
}

int gemm(corr_flagnet_t net, const void* A, const void* Bm, int M, int N, int K, int lda, int ldb, int splits,
         float* D, float* out, cudaStream_t st) {
    GemmArgs g{};
    g.A = A;
    g.B = Bm;
    g.M = M;
    g.N = N;
    g.K = K;
    g.lda = lda;
    g.ldb = ldb;
    g.splits = splits;
    g.k_per_split = ((K + splits - 1) / splits + 63) / 64 * 64;
    g.D = D;
    g.status = net->status;
    const int rc = launch_gemm(g, st);
    if (rc != CORR_OK) return ffail(net, rc, "flagnet GEMM: bad layout");
    FK(cudaGetLastError());
    if (splits > 1) launch_split_sum(D, splits, (long long)M * N, out, st);
    FK(cudaGetLastError());
    return CORR_OK;
}

int conv(corr_flagnet_t net, const uint16_t* X, const uint16_t* W, int B, int bn, int sgn, int mode,
         const float* bias, void* out, cudaStream_t st) {
    ConvArgs c{};
    c.X = X;
    c.W = W;
    c.kp = 832;
    c.n_images = B;
    c.bn = bn;
    c.sgn = sgn;
    c.mode = mode;
    c.bias = bias;
    c.out = out;
    c.status = net->status;
    const int rc = launch_conv(c, st);
    if (rc != CORR_OK) return ffail(net, rc, "flagnet convolution: bad layout");
    ++net->launches;
    FK(cudaGetLastError());
    return CORR_OK;
}

// Forward pass over B normalised tiles x [B][64][256] -> logits.  The
// 1-channel first and last layers run on CUDA cores (conv0_kernel,
// conv_last_kernel); the 32-channel layers are implicit-GEMM convolutions
// on the tensor cores.
int forward(corr_flagnet_t net, const float* x, int B, cudaStream_t st, bool training) {
    const int P = B * TPIX;
    int rc = CORR_OK;
    // the BF16 copy of the input is the weight-gradient operand of layer 0
    if (training) {
        input_bf16_kernel<<<blocks(P), 256, 0, st>>>(x, P, net->act[0]);
        ++net->launches;
    }
    conv0_kernel<<<blocks(P), 256, 0, st>>>(x, P, net->w[0], net->b[0], net->act[1]);
    ++net->launches;
    for (int l = 1; l < NL - 1; ++l) {
        rc = conv(net, net->act[l], net->wf[l], B, 32, 1, 0, net->b[l], net->act[l + 1], st);
        if (rc != CORR_OK) return rc;
    }
    conv_last_kernel<<<blocks((long long)B * TH * (TW / 32) * 32), 256, 0, st>>>(net->act[NL - 1], B, net->wf[NL - 1],
                                                                                net->b[NL - 1], net->logit);
    ++net->launches;
    FK(cudaGetLastError());
    return CORR_OK;
}

// Loss and gradients (into gw/gb) for B tiles; loss summed on the device.
int backward(corr_flagnet_t net, const uint8_t* truth, int B, cudaStream_t st) {
    const int P = B * TPIX;
    net->launches += 2 + NL * 5 + 3 + 2;   // + the implicit convolutions, counted in conv()
    // rows 1..15 of the transposed gradient are the zero padding of the
    // 1-channel output layer's weight-gradient operand
    FK(cudaMemsetAsync(net->dzT + P, 0, (size_t)15 * P * 2, st));
    loss_grad_kernel<<<blocks(P), 256, 0, st>>>(net->logit, truth, P, 1.0f / (float)P, net->dz32, net->dz, net->dzT,
                                                net->loss_part);
    sum_kernel<<<1, 256, 0, st>>>(net->loss_part, (int)blocks(P), net->scalar);
    for (int l = NL - 1; l >= 0; --l) {
        const int C = CI[l], Co = CO[l], Kp = kpad(25 * C), Np = npad(Co);
        // bias gradient
        colsum_kernel<<<Co, 256, 0, st>>>(net->dz32, P, Co, net->gb[l]);
        // weight gradient: DW[Kp][Np] = A^T[Kp][P] . dZ^T[Np][P]
        if (C == 32) im2colT32_kernel<<<P / kSegPix, 256, 0, st>>>(net->act[l], P, net->A);
        else im2colT1_kernel<<<blocks((long long)P * 8), 256, 0, st>>>(net->act[l], P, net->A);
        const int splits = 64;
        int rc = gemm(net, net->A, net->dzT, Kp, Np, P, P * 2, P * 2, splits, net->D, net->D2, st);
        if (rc != CORR_OK) return rc;
        gather_dw_kernel<<<blocks(Co * C * 25), 256, 0, st>>>(net->D2, C, Co, Np, net->gw[l]);
        if (l == 0) break;
        // data gradient: dX[P][C] = sum over taps at negated offsets of dZ . Wd,
        // then the ReLU mask of layer l-1
        const int Kd = kpad(25 * Co);
        if (Co == 32) {
            rc = conv(net, net->dz, net->wd[l], B, 32, -1, 2, nullptr, net->D, st);
        } else {
            im2col(net->dz, Co, P, -1, net->A, st);
            rc = gemm(net, net->A, net->wd[l], P, 32, Kd, Kd * 2, Kd * 2, 1, net->D, nullptr, st);
        }
        if (rc != CORR_OK) return rc;
        relu_grad_kernel<<<blocks((long long)P * C), 256, 0, st>>>(net->D, net->act[l], P, C, net->dz32, net->dz,
                                                                   net->dzT);
    }
    FK(cudaGetLastError());
    return CORR_OK;
}

size_t n_params() {
    size_t n = 0;
    for (int l = 0; l < NL; ++l) n += (size_t)CO[l] * CI[l] * 25 + CO[l];
    return n;
}

}  // namespace

extern "C" {

int corr_flagnet_create(corr_flagnet_t* out) {
    if (!out) return ffail(nullptr, CORR_EINVAL, "out is NULL");
    *out = nullptr;
    corr_flagnet_t net = new corr_flagnet_s();
    cudaGetDevice(&net->dev);
    auto bad = [&](int code, const char* m) {
        corr_flagnet_destroy(net);
        return ffail(nullptr, code, m);
    };
    for (int l = 0; l < NL; ++l) {
        const size_t nw = (size_t)CO[l] * CI[l] * 25;
        float** fs[] = {&net->w[l], &net->mw[l], &net->vw[l], &net->gw[l]};
        for (float** f : fs)
            if (cudaMalloc(f, nw * 4) != cudaSuccess || cudaMemset(*f, 0, nw * 4) != cudaSuccess)
                return bad(CORR_ENOMEM, "flagnet allocation failed");
        float** bs[] = {&net->b[l], &net->mb[l], &net->vb[l], &net->gb[l]};
        for (float** f : bs)
            if (cudaMalloc(f, CO[l] * 4) != cudaSuccess || cudaMemset(*f, 0, CO[l] * 4) != cudaSuccess)
                return bad(CORR_ENOMEM, "flagnet allocation failed");
        const size_t wfb = (size_t)npad(CO[l]) * kpad(25 * CI[l]) * 2;
        if (cudaMalloc(&net->wf[l], wfb) != cudaSuccess || cudaMemset(net->wf[l], 0, wfb) != cudaSuccess)
            return bad(CORR_ENOMEM, "flagnet allocation failed");
        if (l > 0) {
            const size_t wdb = (size_t)32 * kpad(25 * CO[l]) * 2;
            if (cudaMalloc(&net->wd[l], wdb) != cudaSuccess || cudaMemset(net->wd[l], 0, wdb) != cudaSuccess)
                return bad(CORR_ENOMEM, "flagnet allocation failed");
        }
    }
    if (cudaMalloc(&net->scalar, 4) != cudaSuccess || cudaMalloc(&net->status, 4) != cudaSuccess ||
        cudaMemset(net->status, 0, 4) != cudaSuccess)
        return bad(CORR_ENOMEM, "flagnet allocation failed");
    *out = net;
    return CORR_OK;
}

int corr_flagnet_destroy(corr_flagnet_t net) {
    if (!net) return CORR_OK;
    cudaDeviceSynchronize();
    for (int l = 0; l < NL; ++l) {
        void* ps[] = {net->w[l], net->b[l], net->mw[l], net->vw[l], net->mb[l], net->vb[l], net->gw[l], net->gb[l],
                      net->wf[l], net->wd[l]};
        for (void* p : ps)
            if (p) cudaFree(p);
    }
    for (int l = 0; l <= NL; ++l)
        if (net->act[l]) cudaFree(net->act[l]);
    void* ws[] = {net->logit, net->A, net->D, net->D2, net->dz32, net->dz, net->dzT, net->loss_part, net->scalar,
                  net->norm, net->conf, net->status};
    for (void* p : ws)
        if (p) cudaFree(p);
    cudaGetLastError();
    delete net;
    return CORR_OK;
}

int corr_flagnet_num_params(size_t* n) {
    if (!n) return CORR_EINVAL;
    *n = n_params();
    return CORR_OK;
}

int corr_flagnet_set_params(corr_flagnet_t net, const float* params, size_t n) {
    if (!net || !params || n != n_params()) return ffail(net, CORR_EINVAL, "params: wrong size");
    size_t off = 0;
    for (int l = 0; l < NL; ++l) {
        const size_t nw = (size_t)CO[l] * CI[l] * 25;
        FK(cudaMemcpy(net->w[l], params + off, nw * 4, cudaMemcpyHostToDevice));
        off += nw;
        FK(cudaMemcpy(net->b[l], params + off, CO[l] * 4, cudaMemcpyHostToDevice));
        off += CO[l];
        FK(cudaMemset(net->mw[l], 0, nw * 4));
        FK(cudaMemset(net->vw[l], 0, nw * 4));
        FK(cudaMemset(net->mb[l], 0, CO[l] * 4));
        FK(cudaMemset(net->vb[l], 0, CO[l] * 4));
    }
    net->steps = 0;
    return repack(net, nullptr) == CORR_OK ? (cudaDeviceSynchronize() == cudaSuccess ? CORR_OK : CORR_ECUDA)
                                            : CORR_ECUDA;
}

int corr_flagnet_get_params(corr_flagnet_t net, float* params, size_t n) {
    if (!net || !params || n != n_params()) return ffail(net, CORR_EINVAL, "params: wrong size");
    FK(cudaDeviceSynchronize());
    size_t off = 0;
    for (int l = 0; l < NL; ++l) {
        const size_t nw = (size_t)CO[l] * CI[l] * 25;
        FK(cudaMemcpy(params + off, net->w[l], nw * 4, cudaMemcpyDeviceToHost));
        off += nw;
        FK(cudaMemcpy(params + off, net->b[l], CO[l] * 4, cudaMemcpyDeviceToHost));
        off += CO[l];
    }
    return CORR_OK;
}

int corr_flagnet_prepare(corr_flagnet_t net, const float* d_power, int B, float* d_x, void* stream) {
    if (!net || !d_power || !d_x || B < 1) return ffail(net, CORR_EINVAL, "bad argument");
    median_normalize_kernel<<<B, 1024, 0, static_cast<cudaStream_t>(stream)>>>(d_power, d_x);
    ++net->launches;
    FK(cudaGetLastError());
    return CORR_OK;
}

int corr_flagnet_forward(corr_flagnet_t net, const float* d_x, int B, float* d_logits, void* stream) {
    if (!net || !d_x || !d_logits || B < 1) return ffail(net, CORR_EINVAL, "bad argument");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int rc = ensure_ws(net, std::min(B, kChunk));
    if (rc != CORR_OK) return rc;
    for (int t0 = 0; t0 < B; t0 += kChunk) {
        const int n = std::min(kChunk, B - t0);
        rc = forward(net, d_x + (size_t)t0 * TPIX, n, st, false);
        if (rc != CORR_OK) return rc;
        FK(cudaMemcpyAsync(d_logits + (size_t)t0 * TPIX, net->logit, (size_t)n * TPIX * 4, cudaMemcpyDeviceToDevice,
                           st));
    }
    return CORR_OK;
}

int corr_flagnet_loss_grad(corr_flagnet_t net, const float* d_x, const uint8_t* d_truth, int B, float* loss,
                           float* grads, size_t n, void* stream) {
    if (!net || !d_x || !d_truth || B < 1 || B > kChunk) return ffail(net, CORR_EINVAL, "bad argument");
    if (grads && n != n_params()) return ffail(net, CORR_EINVAL, "grads: wrong size");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int rc = ensure_ws(net, B);
    if (rc != CORR_OK) return rc;
    if ((rc = forward(net, d_x, B, st, true)) != CORR_OK) return rc;
    if ((rc = backward(net, d_truth, B, st)) != CORR_OK) return rc;
    FK(cudaStreamSynchronize(st));
    if (loss) {
        float s = 0.f;
        FK(cudaMemcpy(&s, net->scalar, 4, cudaMemcpyDeviceToHost));
        *loss = s / (float)((size_t)B * TPIX);
    }
    if (grads) {
        size_t off = 0;
        for (int l = 0; l < NL; ++l) {
            const size_t nw = (size_t)CO[l] * CI[l] * 25;
            FK(cudaMemcpy(grads + off, net->gw[l], nw * 4, cudaMemcpyDeviceToHost));
            off += nw;
            FK(cudaMemcpy(grads + off, net->gb[l], CO[l] * 4, cudaMemcpyDeviceToHost));
            off += CO[l];
        }
    }
    return CORR_OK;
}

int corr_flagnet_train_step(corr_flagnet_t net, const float* d_x, const uint8_t* d_truth, int B, float lr,
                            float* loss, void* stream) {
    if (!net || !d_x || !d_truth || B < 1 || B > kChunk || !(lr > 0))
        return ffail(net, CORR_EINVAL, "bad argument");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int rc = ensure_ws(net, B);
    if (rc != CORR_OK) return rc;
    if ((rc = forward(net, d_x, B, st, true)) != CORR_OK) return rc;
    if ((rc = backward(net, d_truth, B, st)) != CORR_OK) return rc;
    ++net->steps;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - std::pow(b1, (float)net->steps), c2 = 1.f - std::pow(b2, (float)net->steps);
    for (int l = 0; l < NL; ++l) {
        const int nw = CO[l] * CI[l] * 25;
        adam_kernel<<<blocks(nw), 256, 0, st>>>(net->w[l], net->gw[l], net->mw[l], net->vw[l], nw, lr, b1, b2, c1, c2,
                                                1e-8f);
        adam_kernel<<<blocks(CO[l]), 256, 0, st>>>(net->b[l], net->gb[l], net->mb[l], net->vb[l], CO[l], lr, b1, b2, c1,
                                                   c2, 1e-8f);
    }
    FK(cudaGetLastError());
    net->launches += 2 * NL;
    if ((rc = repack(net, st)) != CORR_OK) return rc;
    if (loss) {
        float s = 0.f;
        FK(cudaMemcpyAsync(&s, net->scalar, 4, cudaMemcpyDeviceToHost, st));
        FK(cudaStreamSynchronize(st));
        *loss = s / (float)((size_t)B * TPIX);
    }
    return CORR_OK;
}

int corr_flagnet_flag(corr_flagnet_t net, const float* d_power, int B, float c_min, float sigma, uint8_t* d_flags,
                      float* d_conf, void* stream) {
    if (!net || !d_power || !d_flags || B < 1) return ffail(net, CORR_EINVAL, "bad argument");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int rc = ensure_ws(net, std::min(B, kChunk));
    if (rc != CORR_OK) return rc;
    for (int t0 = 0; t0 < B; t0 += kChunk) {
        const int n = std::min(kChunk, B - t0);
        const float* pw = d_power + (size_t)t0 * TPIX;
        if ((rc = corr_flagnet_prepare(net, pw, n, net->norm, stream)) != CORR_OK) return rc;
        if ((rc = forward(net, net->norm, n, st, false)) != CORR_OK) return rc;
        confidence_kernel<<<n, 256, 0, st>>>(net->logit, net->conf);
        net->launches += 2;
        const long long items = (long long)n * TH * (TW / 64);
        final_flags_kernel<<<blocks(items, 4), 128, 0, st>>>(pw, net->logit, net->conf, n, c_min, sigma,
                                                              d_flags + (size_t)t0 * TPIX);
        FK(cudaGetLastError());
        if (d_conf) FK(cudaMemcpyAsync(d_conf + t0, net->conf, (size_t)n * 4, cudaMemcpyDeviceToDevice, st));
    }
    return CORR_OK;
}

long long corr_flagnet_kernel_launches(corr_flagnet_t net) { return net ? net->launches : 0; }

int corr_tile_mad_dev(const float* d_power, int n_tiles, float sigma, int axes, uint8_t* d_flags, void* stream) {
    corr_flagnet_t net = nullptr;
    if (!d_power || !d_flags || n_tiles < 1 || axes < 1 || axes > 3 || !(sigma > 0))
        return ffail(nullptr, CORR_EINVAL, "bad argument");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (axes & 1) {
        const long long items = (long long)n_tiles * TH * (TW / 64);
        final_flags_kernel<<<blocks(items, 4), 128, 0, st>>>(d_power, nullptr, nullptr, n_tiles, 0.f, sigma, d_flags);
    }
    if (axes & 2) {
        const long long items = (long long)n_tiles * TW;
        mad_time_kernel<<<blocks(items, 4), 128, 0, st>>>(d_power, n_tiles, sigma, (axes & 1) != 0, d_flags);
    }
    FK(cudaGetLastError());
    return CORR_OK;
}

int corr_flagnet_status(corr_flagnet_t net, int* status) {
    if (!net || !status) return ffail(net, CORR_EINVAL, "bad argument");
    FK(cudaDeviceSynchronize());
    FK(cudaMemcpy(status, net->status, 4, cudaMemcpyDeviceToHost));
    FK(cudaMemset(net->status, 0, 4));
    return CORR_OK;
}

}  // extern "C"
