// Internal declarations shared by the kernels and the runtime of libcorr.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

namespace corr {

// Device-resident view of a sample stream for the F-engine.  Input a's
// sample with stream index n lives at x[a * stride + (n - base)] for
// max(0, base) <= n < vhi; every other index reads as zero.
struct StreamView {
    const int8_t* x;
    long long stride;
    long long base;
    long long vhi;
};

// F-engine launch: spectra s in [s_begin, s_end), one CTA per (input pair,
// block of spt spectra).  Spectrum s is written to ring slot
// (s - v_origin) mod v_cap of V [slot][n_chan][n_in_pad] (float2).
struct FArgs {
    StreamView src;
    const float* h;          // [taps][M] polyphase prototype, FP32
    const float2* tw;        // [M] W_M^k = exp(-2 pi j k / M)
    const float2* phasor;    // [n_in_pad][n_chan] delay/phase rotation (pair factors folded in)
    const int* coarse;       // [n_in_pad] coarse advance d_a
    float2* V;
    long long s_begin, s_end;
    long long v_origin;
    int v_cap;
    int n_in, n_in_pad, M, taps, spt;
};

// X-engine launch: groups of spectra, each group summed into one partial
// slot.  Local group g (0 <= g < n_groups) covers spectra
// [int_start + (j0+g) * G, min(that + G, int_end, s_limit)) where all groups
// of one launch lie inside one integration [int_start, int_end).
struct XArgs {
    const float2* V;
    long long v_origin;
    int v_cap;
    int n_chan, n_in_pad, nt;
    long long int_start, int_end, s_limit;
    int G, j0, n_groups;
    float* part;             // [gpi][nt][32][n_chan]
};

// Finalise: R[k][a][b] = (sum over partial slots 0..n_slots-1) * scale.
struct FinArgs {
    const float* part;
    int n_slots, nt, n_chan, n_in;
    float scale;
    float2* R;               // [n_chan][n_in][n_in]
};

void launch_fengine(const FArgs& a, cudaStream_t st);
void launch_xengine(const XArgs& a, cudaStream_t st);
void launch_finalize(const FinArgs& a, cudaStream_t st);
void launch_mad_flags(const float2* R, uint8_t* F, int n_vis, int n_chan, int n_in, int window,
                      float sigma, cudaStream_t st);

int fengine_threads(int M);

// Error text reported by corr_last_error(NULL) (calls without a handle).
void set_global_error(const std::string& msg);
size_t fengine_smem_bytes(int M);

}  // namespace corr
