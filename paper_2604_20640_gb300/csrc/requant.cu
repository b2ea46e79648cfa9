// Requantiser and rescaling around the tensor-core X-engine.
//
// requant_kernel turns a batch of channelised spectra (U = 2Y, unrotated,
// complex64 in the ring [slot][n_chan][n_in_pad]) into the stacked operand
// Q[k][row][t] of gram_kernel: row a holds Re U_a / sigma_a[k], row N + a
// holds Im U_a / sigma_a[k], t the spectrum index inside the integration:
// int8 codes (round half to even, saturate at +-127) carried as BF16, which
// holds them exactly, or e4m3 (satfinite) bytes.  A CTA
// transposes one channel x 64 spectra through shared memory so that both
// the reads (inputs contiguous) and the writes (time contiguous) coalesce.
// The scales are fixed for a whole integration: the first integration of a
// stream takes them from the mean power of its first spectra, later ones
// from the previous integration's autocorrelations.
#include "corr.h"
#include "corr_internal.h"

#include <cuda_bf16.h>
#include <cuda_fp8.h>

namespace corr {

namespace {

constexpr int kTileS = 64;

__device__ __forceinline__ uint8_t q_int8(float x) {
    x = fminf(fmaxf(x, -127.f), 127.f);
    return (uint8_t)(int8_t)__float2int_rn(x);
}

__device__ __forceinline__ uint8_t q_e4m3(float x) {
    return (uint8_t)__nv_cvt_float_to_fp8(x, __NV_SATFINITE, __NV_E4M3);
}

// Int8 code as the bit pattern of the BF16 value with the same magnitude.
__device__ __forceinline__ uint16_t code_bf16(uint8_t q) {
    return __bfloat16_as_ushort(__float2bfloat16_rn((float)(int8_t)q));
}

__global__ void __launch_bounds__(256) requant_kernel(const RequantArgs A) {
    __shared__ __align__(16) uint8_t T[128][kTileS];
    const int k = blockIdx.x;
    const long long s0 = A.s_begin + (long long)blockIdx.y * kTileS;
    int ns = (int)(A.s_end - s0);
    if (ns > kTileS) ns = kTileS;
    const int N = A.n_in;
    for (int idx = threadIdx.x; idx < N * kTileS; idx += blockDim.x) {
        const int a = idx % N, i = idx / N;
        if (i >= ns) continue;
        const long long slot = (s0 + i - A.v_origin) & A.v_mask;
        const float2 u = A.V[((size_t)slot * A.n_chan + k) * A.n_in_pad + a];
        const float inv = 1.0f / A.scale[(size_t)a * A.n_chan + k];
        const float xr = u.x * inv, xi = u.y * inv;
        T[a][i] = A.fp8 ? q_e4m3(xr) : q_int8(xr);
        T[N + a][i] = A.fp8 ? q_e4m3(xi) : q_int8(xi);
    }
    __syncthreads();
    const long long col0 = s0 - A.int_start;
    if (A.fp8) {
        uint8_t* Qk = A.Q + (size_t)k * 128 * A.k_pitch;
        if ((col0 & 15) == 0) {
            const int chunks = (ns + 15) / 16;
            for (int idx = threadIdx.x; idx < 2 * N * chunks; idx += blockDim.x) {
                const int r = idx / chunks, c = idx % chunks;
                uint8_t* dst = Qk + (size_t)r * A.k_pitch + col0 + 16 * c;
                if (16 * c + 16 <= ns) {
                    *reinterpret_cast<uint4*>(dst) = *reinterpret_cast<const uint4*>(&T[r][16 * c]);
                } else {
                    for (int j = 16 * c; j < ns; ++j) Qk[(size_t)r * A.k_pitch + col0 + j] = T[r][j];
                }
            }
        } else {
            for (int idx = threadIdx.x; idx < 2 * N * ns; idx += blockDim.x) {
                const int r = idx / ns, j = idx % ns;
                Qk[(size_t)r * A.k_pitch + col0 + j] = T[r][j];
            }
        }
    } else {
        uint16_t* Qk = reinterpret_cast<uint16_t*>(A.Q + (size_t)k * 128 * A.k_pitch);
        const int pitch = A.k_pitch / 2;
        if ((col0 & 7) == 0) {
            const int chunks = (ns + 7) / 8;
            for (int idx = threadIdx.x; idx < 2 * N * chunks; idx += blockDim.x) {
                const int r = idx / chunks, c = idx % chunks;
                uint16_t* dst = Qk + (size_t)r * pitch + col0 + 8 * c;
                if (8 * c + 8 <= ns) {
                    uint16_t v[8];
#pragma unroll
                    for (int j = 0; j < 8; ++j) v[j] = code_bf16(T[r][8 * c + j]);
                    *reinterpret_cast<uint4*>(dst) = *reinterpret_cast<const uint4*>(v);
                } else {
                    for (int j = 8 * c; j < ns; ++j) Qk[(size_t)r * pitch + col0 + j] = code_bf16(T[r][j]);
                }
            }
        } else {
            for (int idx = threadIdx.x; idx < 2 * N * ns; idx += blockDim.x) {
                const int r = idx / ns, j = idx % ns;
                Qk[(size_t)r * pitch + col0 + j] = code_bf16(T[r][j]);
            }
        }
    }
}

__global__ void scale_ring_kernel(const float2* V, long long v_origin, long long v_mask, long long s0, int n,
                                  int n_in, int n_in_pad, int n_chan, float gain, float* scale) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int a = blockIdx.y;
    if (k >= n_chan || a >= n_in) return;
    float p = 0.f;
    for (int i = 0; i < n; ++i) {
        const long long slot = (s0 + i - v_origin) & v_mask;
        const float2 u = V[((size_t)slot * n_chan + k) * n_in_pad + a];
        p = fmaf(u.x, u.x, fmaf(u.y, u.y, p));
    }
    p /= (float)n;
    float s = sqrtf(0.5f * p) / gain;
    if (!(s > 0.f) || !isfinite(s)) s = 1.f;
    scale[(size_t)a * n_chan + k] = s;
}

__global__ void scale_vis_kernel(const float2* R, int n_in, int n_in_pad, int n_chan, float gain, float* scale) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int a = blockIdx.y;
    if (k >= n_chan || a >= n_in) return;
    const float raa = R[((size_t)k * n_in + a) * n_in + a].x;
    float s = 2.f * sqrtf(0.5f * fmaxf(raa, 0.f)) / gain;
    if (!(s > 0.f) || !isfinite(s)) s = 1.f;
    scale[(size_t)a * n_chan + k] = s;
}

__global__ void finalize_q_kernel(const FinQArgs F) {
    const int k = blockIdx.x;
    const int N = F.n_in;
    const size_t gbase = (size_t)k * 128 * 128;
    for (int idx = threadIdx.x; idx < N * N; idx += blockDim.x) {
        const int a = idx / N, b = idx % N;
        if (a > b) continue;
        const float* G = reinterpret_cast<const float*>(F.G) + gbase;
        const float cre = G[a * 128 + b] + G[(N + a) * 128 + N + b];
        const float cim = G[(N + a) * 128 + b] - G[a * 128 + N + b];
        const float sc = F.scale[(size_t)a * F.n_chan + k] * F.scale[(size_t)b * F.n_chan + k] /
                         (4.0f * (float)F.count);
        float re = cre * sc, im = cim * sc;
        float2* R = F.R + (size_t)k * N * N;
        if (a == b) {
            R[a * N + a] = make_float2(re, 0.f);
            continue;
        }
        if (F.rot) {
            const float2 qa = F.rot[(size_t)a * F.n_chan + k];
            const float2 qb = F.rot[(size_t)b * F.n_chan + k];
            const float pr = qa.x * qb.x + qa.y * qb.y;
            const float pi = qa.y * qb.x - qa.x * qb.y;
            const float r2 = re * pr - im * pi;
            im = re * pi + im * pr;
            re = r2;
        }
        R[a * N + b] = make_float2(re, im);
        R[b * N + a] = make_float2(re, -im);
    }
}

}  // namespace

void launch_requant(const RequantArgs& a, cudaStream_t st) {
    const long long n = a.s_end - a.s_begin;
    if (n <= 0) return;
    dim3 grid((unsigned)a.n_chan, (unsigned)((n + kTileS - 1) / kTileS));
    requant_kernel<<<grid, 256, 0, st>>>(a);
}

void launch_scale_from_ring(const float2* V, long long v_origin, long long v_mask, long long s0, int n, int n_in,
                            int n_in_pad, int n_chan, float gain, float* scale, cudaStream_t st) {
    dim3 grid((unsigned)((n_chan + 127) / 128), (unsigned)n_in);
    scale_ring_kernel<<<grid, 128, 0, st>>>(V, v_origin, v_mask, s0, n, n_in, n_in_pad, n_chan, gain, scale);
}

void launch_scale_from_vis(const float2* R, int n_in, int n_in_pad, int n_chan, float gain, float* scale,
                           cudaStream_t st) {
    dim3 grid((unsigned)((n_chan + 127) / 128), (unsigned)n_in);
    scale_vis_kernel<<<grid, 128, 0, st>>>(R, n_in, n_in_pad, n_chan, gain, scale);
}

void launch_finalize_q(const FinQArgs& a, cudaStream_t st) {
    finalize_q_kernel<<<a.n_chan, 256, 0, st>>>(a);
}

}  // namespace corr
