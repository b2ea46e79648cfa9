// FP32 arithmetic peak of the device, measured: the ceiling the F-engine's
// floating-point work (PFB FIR, FFT butterflies, X-engine sums) is held to
// when it is not held by HBM.  Every thread runs independent chains of
// dependent fused multiply-adds (enough chains and resident warps to cover
// the FMA latency), scalar (fma.rn.f32, 2 FLOP per lane per instruction) or
// packed (fma.rn.f32x2, 4 FLOP per lane per instruction), and the kernel is
// timed with CUDA events on the caller's stream.
#include "corr.h"
#include "corr_internal.h"

#include <string>

namespace {

constexpr int kChains = 8;
constexpr int kPeakThreads = 512;

__device__ __forceinline__ unsigned long long pk(float2 v) {
    return (unsigned long long)__float_as_uint(v.x) | ((unsigned long long)__float_as_uint(v.y) << 32);
}

template <bool PACKED>
__global__ void __launch_bounds__(kPeakThreads) fma_peak_kernel(float* out, int iters, float a, float b) {
    const float seed = (float)(threadIdx.x & 7) * 1e-3f;
    if constexpr (!PACKED) {
        float x[kChains];
#pragma unroll
        for (int j = 0; j < kChains; ++j) x[j] = seed + (float)j;
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int j = 0; j < kChains; ++j) x[j] = fmaf(x[j], a, b);
        }
        float s = 0.f;
#pragma unroll
        for (int j = 0; j < kChains; ++j) s += x[j];
        if (s == 12345.678f) out[blockIdx.x * blockDim.x + threadIdx.x] = s;   // keeps the chains live
    } else {
        unsigned long long x[kChains];
        const unsigned long long a2 = pk(make_float2(a, a)), b2 = pk(make_float2(b, b));
#pragma unroll
        for (int j = 0; j < kChains; ++j) x[j] = pk(make_float2(seed + (float)j, seed - (float)j));
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int j = 0; j < kChains; ++j)
                asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(x[j]) : "l"(a2), "l"(b2));
        }
        float s = 0.f;
#pragma unroll
        for (int j = 0; j < kChains; ++j)
            s += __uint_as_float((unsigned)x[j]) + __uint_as_float((unsigned)(x[j] >> 32));
        if (s == 12345.678f) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
    }
}

}  // namespace

extern "C" int corr_peak_fp32(int packed, int iters, double* tflops, double* ms, void* stream) {
    if (!tflops || iters < 1 || (packed != 0 && packed != 1)) {
        corr::set_global_error("corr_peak_fp32: bad argument");
        return CORR_EINVAL;
    }
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
        e = packed ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fma_peak_kernel<true>, kPeakThreads, 0)
                   : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fma_peak_kernel<false>, kPeakThreads, 0);
    if (e != cudaSuccess || sms < 1 || per_sm < 1) {
        corr::set_global_error(std::string("corr_peak_fp32: device query: ") + cudaGetErrorString(e));
        return CORR_ECUDA;
    }
    // four waves of full SMs: the tail of the last wave is a small share
    const int blocks = 4 * sms * per_sm;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    float* out = nullptr;   // written only if the chains hit an impossible value
    e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) e = cudaMalloc(&out, sizeof(float) * (size_t)blocks * kPeakThreads);
    if (e == cudaSuccess) {
        // warm-up launch, then the timed one
        for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {
            if (rep == 1) e = cudaEventRecord(e0, st);
            if (packed) fma_peak_kernel<true><<<blocks, kPeakThreads, 0, st>>>(out, iters, 0.999999f, 1e-7f);
            else fma_peak_kernel<false><<<blocks, kPeakThreads, 0, st>>>(out, iters, 0.999999f, 1e-7f);
            if (e == cudaSuccess) e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaEventRecord(e1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    }
    float t = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
    if (out) cudaFree(out);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e != cudaSuccess || !(t > 0.f)) {
        corr::set_global_error(std::string("corr_peak_fp32: ") + cudaGetErrorString(e));
        return CORR_ECUDA;
    }
    const double flop = (double)blocks * kPeakThreads * (double)iters * kChains * (packed ? 4.0 : 2.0);
    *tflops = flop / (t * 1e-3) / 1e12;
    if (ms) *ms = t;
    return CORR_OK;
}
