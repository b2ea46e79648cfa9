// Requantiser around the tensor-core X-engine.
//
// words_from_spectra_kernel turns channelised spectra (U = 2Y, unrotated, in
// the pair-major ring [slot][pair][n_chan] float4) into the integration's
// int8 or e4m3 code words C[t][pair][k] (round half to even, saturate at
// +-127; e4m3 satfinite) -- the form the fused F-engine writes itself once
// the scales are fixed, and the form gram_w_kernel reads.  It serves a
// stream's first ring fill, whose spectra precede the scales, and pipelines
// whose F-engine is the two-kernel form.
// The scales are fixed for a whole integration: the first integration of a
// stream takes them from the mean power of its first spectra
// (scale_ring_kernel), later ones from the previous integration's
// autocorrelations (scale_vis_kernel); both store the inverse scales the
// codes are made with after the scales.
#include "corr.h"
#include "corr_internal.h"

#include "quant.cuh"

namespace corr {

namespace {

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

}  // namespace

void launch_requant(const RequantArgs& a, cudaStream_t st) {
    const long long n = a.s_end - a.s_begin;
    if (n <= 0) return;
    dim3 grid((unsigned)((a.n_chan + 127) / 128), (unsigned)(a.n_in_pad / 2), (unsigned)n);
    if (a.fp8) words_from_spectra_kernel<true><<<grid, 128, 0, st>>>(a);
    else words_from_spectra_kernel<false><<<grid, 128, 0, st>>>(a);
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


}  // namespace corr
