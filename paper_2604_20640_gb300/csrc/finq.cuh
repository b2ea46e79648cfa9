// Visibilities from the Gram matrix of requantised voltages: the
// reduced-precision X-engine's finalisation, done in the Gram kernel's own
// epilogue.
#pragma once

#include <cuda_runtime.h>

namespace corr {

// Baseline (a, b), a <= b, of one channel.  With rows Re q at a and Im q at
// N + a of the stacked codes, sum_s q_a conj(q_b) = (G_rr + G_ii) + j (G_ir -
// G_ri); times sigma_a sigma_b / (4 count) it is the integrated
// correlation of U = 2Y (Sec. 4.2, the scaling restored), then rotated by
// qa conj(qb) (the fine-delay and phase correction of Eq. 1) unless qa is
// null.  inv4c = 1 / (4 count), rounded once by the caller.  The
// autocorrelation (a == b) is real and not rotated.  Roundings are spelled
// out, so the result does not hang on how the compiler contracts them.
__device__ __forceinline__ float2 vis_from_gram(float g_rr, float g_ii, float g_ir, float g_ri, float sa, float sb,
                                                float inv4c, bool diag, const float2* qa, const float2* qb) {
    const float sc = __fmul_rn(__fmul_rn(sa, sb), inv4c);
    const float re = __fmul_rn(__fadd_rn(g_rr, g_ii), sc);
    if (diag) return make_float2(re, 0.f);
    const float im = __fmul_rn(__fsub_rn(g_ir, g_ri), sc);
    if (!qa) return make_float2(re, im);
    const float pr = __fmaf_rn(qa->x, qb->x, __fmul_rn(qa->y, qb->y));
    const float pi = __fmaf_rn(qa->y, qb->x, -__fmul_rn(qa->x, qb->y));
    return make_float2(__fmaf_rn(re, pr, -__fmul_rn(im, pi)), __fmaf_rn(re, pi, __fmul_rn(im, pr)));
}

}  // namespace corr
