// Requantisation codes of the reduced-precision X-engine, shared by the
// requantiser kernel and the F-engine epilogue that writes codes directly:
// int8 (round half to even, saturate at +-127) and e4m3 (round to nearest
// even, saturate at +-448).
#pragma once

#include <cuda_fp8.h>
#include <stdint.h>

namespace corr {

__device__ __forceinline__ uint8_t q_int8(float x) {
    x = fminf(fmaxf(x, -127.f), 127.f);
    return (uint8_t)(int8_t)__float2int_rn(x);
}

__device__ __forceinline__ uint8_t q_e4m3(float x) {
    return (uint8_t)__nv_cvt_float_to_fp8(x, __NV_SATFINITE, __NV_E4M3);
}

template <bool FP8>
__device__ __forceinline__ uint32_t q_code(float x) {
    if constexpr (FP8) return q_e4m3(x);
    else return q_int8(x);
}

}  // namespace corr
