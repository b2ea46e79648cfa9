// Delay / phase calibration (Sec. 7, Eq. 3) on the visibilities of one
// integration, one CTA per baseline (ref, a):
//   1. coarse group delay: the peak of the delay spectrum
//      |sum_k w_k R_k exp(-j 2 pi k t / M)| over trial delays t = -T .. T in
//      quarter samples (FP32; the phase k t / M is reduced exactly in integers
//      before the sine and cosine);
//   2. fine delay: weighted (|R_k|) linear fit, in FP64, to the phase of
//      z_k = R_k exp(-j 2 pi k t_c / M) unwrapped about the band's mean
//      vector c0 (psi_k = arg c0 + arg(z_k conj c0)); the coarse step leaves
//      at most 1/8 sample, i.e. pi/8 of drift across the band, so there is
//      no 2 pi ambiguity, and a noisy channel stays a single outlier --
//      giving tau = t_c + slope M / (2 pi);
//   3. residual phase: phi = -arg sum_k R_k exp(-j 2 pi k tau / M) (FP64).
// The result (tau, phi) is what corr_set_delays takes to flatten the phases.
#include "corr.h"
#include "corr_internal.h"

#include <cmath>
#include <vector>

namespace corr {
namespace {

constexpr int kCalThreads = 256;
constexpr int kGrid = 4;          // trial delays per sample

__device__ __forceinline__ bool usable(const uint8_t* flags, int n_in, int ref, int a, int k, int k_lo, int k_hi) {
    if (k < k_lo || k >= k_hi) return false;
    return !flags || flags[((size_t)k * n_in + ref) * n_in + a] == 0;
}

__device__ __forceinline__ double2 vis(const float2* V, int n_in, int ref, int a, int k) {
    const float2 v = V[((size_t)k * n_in + ref) * n_in + a];
    return make_double2(v.x, v.y);
}

// Block-wide exclusive scan of one double per thread; returns the total.
__device__ double block_scan(double v, double* sh, double& excl) {
    const int t = threadIdx.x;
    sh[t] = v;
    __syncthreads();
    for (int off = 1; off < kCalThreads; off <<= 1) {
        const double x = t >= off ? sh[t - off] : 0.0;
        __syncthreads();
        sh[t] += x;
        __syncthreads();
    }
    const double incl = sh[t];
    const double total = sh[kCalThreads - 1];
    __syncthreads();
    excl = incl - v;
    return total;
}

__device__ double block_sum(double v, double* sh) {
    double e;
    return block_scan(v, sh, e);
}

__global__ void __launch_bounds__(kCalThreads) calib_kernel(const float2* V, const uint8_t* flags, int n_chan, int n_in,
                                                           int ref, int k_lo, int k_hi, int T, double* out) {
    __shared__ double sd[kCalThreads];
    __shared__ float sv[kCalThreads];
    __shared__ int si[kCalThreads];
    const int a = blockIdx.x;
    const int t = threadIdx.x;
    const int M = 2 * n_chan;
    if (a == ref) {
        if (t == 0) out[2 * a] = out[2 * a + 1] = 0.0;
        return;
    }
    // ---- 1. delay spectrum peak (first maximum on the grid)
    const int n_trials = 2 * T * kGrid + 1;
    float best = -1.f;
    int best_i = 0;
    for (int i = t; i < n_trials; i += kCalThreads) {
        const long long num = (long long)(i - T * kGrid);     // t_i = num / kGrid
        float re = 0.f, im = 0.f;
        for (int k = k_lo; k < k_hi; ++k) {
            if (!usable(flags, n_in, ref, a, k, k_lo, k_hi)) continue;
            // phase 2 pi k t_i / M = pi q / (kGrid M / 2) with q = k num mod (kGrid M)
            long long q = ((long long)k * num) % ((long long)kGrid * M);
            if (q < 0) q += (long long)kGrid * M;
            float s, c;
            sincospif((float)q / (float)(kGrid * M / 2), &s, &c);
            const float2 r = V[((size_t)k * n_in + ref) * n_in + a];
            // r * exp(-j theta) = (r.x c + r.y s, r.y c - r.x s)
            re = fmaf(r.x, c, fmaf(r.y, s, re));
            im = fmaf(r.y, c, fmaf(-r.x, s, im));
        }
        const float d = re * re + im * im;
        if (d > best) {
            best = d;
            best_i = i;
        }
    }
    sv[t] = best;
    si[t] = best_i;
    __syncthreads();
    for (int off = kCalThreads / 2; off > 0; off >>= 1) {
        if (t < off) {
            const float v2 = sv[t + off];
            const int i2 = si[t + off];
            if (v2 > sv[t] || (v2 == sv[t] && i2 < si[t])) {
                sv[t] = v2;
                si[t] = i2;
            }
        }
        __syncthreads();
    }
    const double t_c = (double)(si[0] - T * kGrid) / kGrid;
    __syncthreads();

    // ---- 2. residual phase about the band's mean vector, weighted fit (FP64)
    auto rot = [&](int k) {
        double sn, cs;
        const double fr = fmod((double)k * t_c, (double)M);          // exact for quarter samples
        sincospi(2.0 * fr / (double)M, &sn, &cs);
        const double2 r = vis(V, n_in, ref, a, k);
        return make_double2(r.x * cs + r.y * sn, r.y * cs - r.x * sn);
    };
    double mre = 0.0, mim = 0.0;
    int cnt = 0;
    for (int k = k_lo + t; k < k_hi; k += kCalThreads) {
        if (!usable(flags, n_in, ref, a, k, k_lo, k_hi)) continue;
        const double2 z = rot(k);
        mre += z.x;
        mim += z.y;
        ++cnt;
    }
    mre = block_sum(mre, sd);
    mim = block_sum(mim, sd);
    const double n_use = block_sum((double)cnt, sd);
    if (n_use < 2.0) {
        if (t == 0) out[2 * a] = out[2 * a + 1] = nan("");
        return;
    }
    const double arg0 = atan2(mim, mre);
    double sw = 0, swk = 0, swkk = 0, swp = 0, swkp = 0;
    for (int k = k_lo + t; k < k_hi; k += kCalThreads) {
        if (!usable(flags, n_in, ref, a, k, k_lo, k_hi)) continue;
        const double2 z = rot(k);
        // arg(z conj c0) + arg c0
        const double psi = arg0 + atan2(z.y * mre - z.x * mim, z.x * mre + z.y * mim);
        const double2 r = vis(V, n_in, ref, a, k);
        const double w = sqrt(r.x * r.x + r.y * r.y);
        sw += w;
        swk += w * k;
        swkk += w * (double)k * k;
        swp += w * psi;
        swkp += w * k * psi;
    }
    sw = block_sum(sw, sd);
    swk = block_sum(swk, sd);
    swkk = block_sum(swkk, sd);
    swp = block_sum(swp, sd);
    swkp = block_sum(swkp, sd);
    const double kb = swk / sw, pb = swp / sw;
    const double slope = (swkp - sw * kb * pb) / (swkk - sw * kb * kb);
    const double tau = t_c + slope * M / (2.0 * 3.14159265358979323846);

    // ---- 3. residual phase from the mean complex vector
    double cre = 0.0, cim = 0.0;
    for (int k = k_lo + t; k < k_hi; k += kCalThreads) {
        if (!usable(flags, n_in, ref, a, k, k_lo, k_hi)) continue;
        double s, c;
        const double fr = fmod((double)k * tau, (double)M);
        sincospi(2.0 * fr / (double)M, &s, &c);
        const double2 r = vis(V, n_in, ref, a, k);
        cre += r.x * c + r.y * s;
        cim += r.y * c - r.x * s;
    }
    cre = block_sum(cre, sd);
    cim = block_sum(cim, sd);
    if (t == 0) {
        out[2 * a] = tau;
        out[2 * a + 1] = -atan2(cim, cre);
    }
}

}  // namespace
}  // namespace corr

extern "C" int corr_calibrate_dev(const float* d_vis, const uint8_t* d_flags, int n_chan, int n_in, int ref, int k_lo,
                                  int k_hi, double max_delay, double* tau, double* phi, void* stream) {
    using namespace corr;
    if (!d_vis || !tau || !phi || n_chan < 2 || n_in < 1 || ref < 0 || ref >= n_in || k_lo < 0 || k_hi > n_chan ||
        k_hi - k_lo < 2 || !(max_delay >= 0) || max_delay > 4096)
        return set_global_error("corr_calibrate_dev: bad argument"), CORR_EINVAL;
    const int T = (int)std::ceil(max_delay);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    double* d_out = nullptr;
    if (cudaMallocAsync(reinterpret_cast<void**>(&d_out), sizeof(double) * 2 * n_in, st) != cudaSuccess)
        return set_global_error("corr_calibrate_dev: allocation failed"), CORR_ENOMEM;
    calib_kernel<<<n_in, kCalThreads, 0, st>>>(reinterpret_cast<const float2*>(d_vis), d_flags, n_chan, n_in, ref,
                                               k_lo, k_hi, T, d_out);
    std::vector<double> h(2 * (size_t)n_in);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(h.data(), d_out, sizeof(double) * 2 * n_in, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFreeAsync(d_out, st);
    if (e != cudaSuccess) return set_global_error(std::string("corr_calibrate_dev: ") + cudaGetErrorString(e)), CORR_ECUDA;
    for (int a = 0; a < n_in; ++a) {
        tau[a] = h[2 * a];
        phi[a] = h[2 * a + 1];
    }
    return CORR_OK;
}
