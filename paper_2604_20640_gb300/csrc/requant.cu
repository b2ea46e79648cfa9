// Requantiser and rescaling around the tensor-core X-engine.
//
// Pipeline: words_from_spectra_kernel turns channelised spectra (U = 2Y,
// unrotated, in the pair-major ring [slot][pair][n_chan] float4) into the
// integration's int8 or e4m3 code words C[t][pair][k] -- the form the fused
// F-engine writes itself once the scales are fixed, and the form
// gram_w_kernel reads.
// Stage calls and channel counts not a multiple of 4: requant_pm_kernel
// turns the spectra, or code words the fused F-engine made from them, into
// the stacked operand Q[k][row][t]: row a holds Re U_a / sigma_a[k], row
// N + a holds Im U_a / sigma_a[k], t the spectrum index inside the
// integration; int8 codes (round half to even, saturate at +-127) as bytes
// or carried as BF16, or e4m3 (satfinite) bytes.  A thread owns one input pair and channel over a run
// of spectra, so reads coalesce across channels and every row gets whole
// 32-byte sectors of codes.
// The scales are fixed for a whole integration: the first integration of a
// stream takes them from the mean power of its first spectra, later ones
// from the previous integration's autocorrelations.
#include "corr.h"
#include "corr_internal.h"

#include "finq.cuh"
#include "quant.cuh"

#include <cuda_bf16.h>

namespace corr {

namespace {

// Int8 code as the bit pattern of the BF16 value with the same magnitude.
__device__ __forceinline__ uint16_t code_bf16(uint8_t q) {
    return __bfloat16_as_ushort(__float2bfloat16_rn((float)(int8_t)q));
}

// Pair-major ring ([slot][pair][n_chan] float4: the pair's two complex
// values): one thread per (input pair, channel), consecutive channels across
// the warp (coalesced 16-byte reads), a run of RUN spectra per thread; the
// pair's four rows (Re a, Re b, Im a, Im b) each get one whole 32-byte sector
// of codes.
// CODE: 0 int8 carried as BF16 (2 bytes), 1 e4m3 byte, 2 int8 byte, 3 the
// F-engine's code words already made ([slot][pair][n_chan] 32-bit words,
// bytes Re a, Im a, Re a+1, Im a+1): a transpose into Q only.
// RUN spectra per thread: 32 / EB, or 64 for the transpose (two whole
// sectors a row).
template <int CODE, int RUN = (CODE == 3 ? 64 : (CODE == 0 ? 16 : 32))>
__global__ void __launch_bounds__(128) requant_pm_kernel(const RequantArgs A) {
    constexpr bool FP8 = CODE == 1;
    constexpr int EB = CODE == 0 ? 2 : 1;
    constexpr int NW = RUN * EB / 4;        // 32-bit words of codes per row
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int pr = blockIdx.y;
    if (k >= A.n_chan) return;
    const int N = A.n_in;
    const int a0 = 2 * pr, a1 = 2 * pr + 1;
    const int n_pairs = A.n_in_pad >> 1;
    const long long sb = A.s_begin + (long long)blockIdx.z * RUN;
    if (sb >= A.s_end) return;
    const int ns = (int)((A.s_end - sb) < RUN ? (A.s_end - sb) : RUN);
    // inverse scales [n_in_pad][n_chan] follow the scales (scale + n_in_pad n_chan)
    const float* inv = A.scale + (size_t)A.n_in_pad * A.n_chan;
    const float inv0 = (CODE != 3 && a0 < N) ? inv[(size_t)a0 * A.n_chan + k] : 0.f;
    const float inv1 = (CODE != 3 && a1 < N) ? inv[(size_t)a1 * A.n_chan + k] : 0.f;
    uint32_t w[4][NW];                // rows Re a0, Im a0, Re a1, Im a1
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int j = 0; j < NW; ++j) w[r][j] = 0u;
    if constexpr (CODE == 3) {
        const uint32_t* C = reinterpret_cast<const uint32_t*>(A.V);
#pragma unroll
        for (int i = 0; i < RUN; ++i) {
            uint32_t c = 0u;
            if (i < ns) {
                const long long slot = (sb + i - A.v_origin) & A.v_mask;
                c = __ldg(C + ((size_t)slot * n_pairs + pr) * A.n_chan + k);
            }
#pragma unroll
            for (int r = 0; r < 4; ++r) w[r][i / 4] |= ((c >> (8 * r)) & 0xFFu) << (8 * (i % 4));
        }
    }
    const float4* V4 = reinterpret_cast<const float4*>(A.V);
#pragma unroll
    for (int i = 0; i < (CODE == 3 ? 0 : RUN); ++i) {
        float4 u = make_float4(0.f, 0.f, 0.f, 0.f);
        if (i < ns) {
            const long long slot = (sb + i - A.v_origin) & A.v_mask;
            u = __ldg(V4 + ((size_t)slot * n_pairs + pr) * A.n_chan + k);
        }
        const float x[4] = {u.x * inv0, u.y * inv0, u.z * inv1, u.w * inv1};
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            if constexpr (FP8) w[r][i / 4] |= (uint32_t)q_e4m3(x[r]) << (8 * (i % 4));
            else if constexpr (CODE == 2) w[r][i / 4] |= (uint32_t)q_int8(x[r]) << (8 * (i % 4));
            else w[r][i / 2] |= (uint32_t)code_bf16(q_int8(x[r])) << (16 * (i % 2));
        }
    }
    const long long col = sb - A.int_start;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int a = (r < 2) ? a0 : a1;
        if (a >= N) continue;                        // padding inputs have no rows
        const int row = (r & 1) ? N + a : a;
        uint8_t* dst = A.Q + ((size_t)k * 128 + row) * A.k_pitch + col * EB;
        if (ns == RUN && ((col * EB) & 15) == 0) {
            uint4* d = reinterpret_cast<uint4*>(dst);
#pragma unroll
            for (int v = 0; v < NW / 4; ++v) d[v] = make_uint4(w[r][4 * v], w[r][4 * v + 1], w[r][4 * v + 2], w[r][4 * v + 3]);
        } else {
            // ragged run: byte by byte, every index of w a compile-time
            // constant (w stays in registers)
#pragma unroll
            for (int j = 0; j < NW; ++j)
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    if (4 * j + e < ns * EB) dst[4 * j + e] = (uint8_t)(w[r][j] >> (8 * e));
        }
    }
}

// Spectra of the pair-major ring into int8 or e4m3 code words C[t][pair][k]
// (bytes Re U_a, Im U_a, Re U_a+1, Im U_a+1; t = s - int_start): the words
// the fused F-engine writes once the scales are fixed, made here from the
// spectra it wrote before (same arithmetic, same codes).  One thread per
// (channel, pair, spectrum).
template <bool FP8>
__global__ void __launch_bounds__(128) words_from_spectra_kernel(const RequantArgs A) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int pr = blockIdx.y;
    const long long s = A.s_begin + blockIdx.z;
    if (k >= A.n_chan || s >= A.s_end) return;
    const int N = A.n_in;
    const int a0 = 2 * pr, a1 = 2 * pr + 1;
    const int n_pairs = A.n_in_pad >> 1;
    const float* inv = A.scale + (size_t)A.n_in_pad * A.n_chan;
    const float inv0 = a0 < N ? inv[(size_t)a0 * A.n_chan + k] : 0.f;
    const float inv1 = a1 < N ? inv[(size_t)a1 * A.n_chan + k] : 0.f;
    const long long slot = (s - A.v_origin) & A.v_mask;
    const float4 u = __ldg(reinterpret_cast<const float4*>(A.V) + ((size_t)slot * n_pairs + pr) * A.n_chan + k);
    const uint32_t w = q_code<FP8>(u.x * inv0) | (q_code<FP8>(u.y * inv0) << 8) |
                       (q_code<FP8>(u.z * inv1) << 16) | (q_code<FP8>(u.w * inv1) << 24);
    A.C[((size_t)(s - A.int_start) * n_pairs + pr) * A.n_chan + k] = w;
}

__global__ void scale_ring_kernel(const float2* V, long long v_origin, long long v_mask, long long s0, int n,
                                  int n_in, int n_in_pad, int n_chan, float gain, float* scale, int pm) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int a = blockIdx.y;
    if (k >= n_chan || a >= n_in) return;
    float p = 0.f;
    for (int i = 0; i < n; ++i) {
        const long long slot = (s0 + i - v_origin) & v_mask;
        // channel-major [slot][k][a], or pair-major [slot][a/2][k][a%2]
        const float2 u = pm ? V[(((size_t)slot * (n_in_pad >> 1) + (a >> 1)) * n_chan + k) * 2 + (a & 1)]
                            : V[((size_t)slot * n_chan + k) * n_in_pad + a];
        p = fmaf(u.x, u.x, fmaf(u.y, u.y, p));
    }
    p /= (float)n;
    // power of one component: half of |U|^2, all of it in the real DC bin
    float s = sqrtf((k == 0 ? 1.f : 0.5f) * p) / gain;
    if (!(s > 0.f) || !isfinite(s)) s = 1.f;
    scale[(size_t)a * n_chan + k] = s;
    scale[((size_t)n_in_pad + a) * n_chan + k] = 1.0f / s;
}

__global__ void scale_vis_kernel(const float2* R, int n_in, int n_in_pad, int n_chan, float gain, float* scale) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int a = blockIdx.y;
    if (k >= n_chan || a >= n_in) return;
    const float raa = R[((size_t)k * n_in + a) * n_in + a].x;
    float s = 2.f * sqrtf((k == 0 ? 1.f : 0.5f) * fmaxf(raa, 0.f)) / gain;
    if (!(s > 0.f) || !isfinite(s)) s = 1.f;
    scale[(size_t)a * n_chan + k] = s;
    scale[((size_t)n_in_pad + a) * n_chan + k] = 1.0f / s;
}

__global__ void finalize_q_kernel(const FinQArgs F) {
    const int k = blockIdx.x;
    const int N = F.n_in;
    const size_t gbase = (size_t)k * 128 * 128;
    const float inv4c = 1.0f / (4.0f * (float)F.count);
    for (int idx = threadIdx.x; idx < N * N; idx += blockDim.x) {
        const int a = idx / N, b = idx % N;
        if (a > b) continue;
        const float* G = reinterpret_cast<const float*>(F.G) + gbase;
        const float2* qa = F.rot ? F.rot + (size_t)a * F.n_chan + k : nullptr;
        const float2* qb = F.rot ? F.rot + (size_t)b * F.n_chan + k : nullptr;
        const float2 v = vis_from_gram(G[a * 128 + b], G[(N + a) * 128 + N + b], G[(N + a) * 128 + b],
                                       G[a * 128 + N + b], F.scale[(size_t)a * F.n_chan + k],
                                       F.scale[(size_t)b * F.n_chan + k], inv4c, a == b, qa, qb);
        float2* R = F.R + (size_t)k * N * N;
        R[a * N + b] = v;
        if (a != b) R[b * N + a] = make_float2(v.x, -v.y);
    }
}

}  // namespace

void launch_requant(const RequantArgs& a, cudaStream_t st) {
    const long long n = a.s_end - a.s_begin;
    if (n <= 0) return;
    if (a.C) {
        dim3 grid((unsigned)((a.n_chan + 127) / 128), (unsigned)(a.n_in_pad / 2), (unsigned)n);
        if (a.fp8) words_from_spectra_kernel<true><<<grid, 128, 0, st>>>(a);
        else words_from_spectra_kernel<false><<<grid, 128, 0, st>>>(a);
        return;
    }
    const int run = a.codes_in ? 64 : (a.fp8 || a.i8b) ? 32 : 16;
    dim3 grid((unsigned)((a.n_chan + 127) / 128), (unsigned)(a.n_in_pad / 2), (unsigned)((n + run - 1) / run));
    if (a.codes_in) requant_pm_kernel<3><<<grid, 128, 0, st>>>(a);
    else if (a.fp8) requant_pm_kernel<1><<<grid, 128, 0, st>>>(a);
    else if (a.i8b) requant_pm_kernel<2><<<grid, 128, 0, st>>>(a);
    else requant_pm_kernel<0><<<grid, 128, 0, st>>>(a);
}

void launch_scale_from_ring(const float2* V, long long v_origin, long long v_mask, long long s0, int n, int n_in,
                            int n_in_pad, int n_chan, float gain, float* scale, int pair_major, cudaStream_t st) {
    dim3 grid((unsigned)((n_chan + 127) / 128), (unsigned)n_in);
    scale_ring_kernel<<<grid, 128, 0, st>>>(V, v_origin, v_mask, s0, n, n_in, n_in_pad, n_chan, gain, scale,
                                            pair_major);
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
