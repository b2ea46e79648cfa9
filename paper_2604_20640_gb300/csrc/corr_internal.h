// Internal declarations shared by the kernels and the runtime of libcorr.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

namespace corr {

// Device-resident view of a sample stream for the F-engine.  Input a's
// sample with stream index n lives at x[a * stride + (n - base)] for
// max(0, base) <= n < vhi; every other index reads as zero.
struct StreamView {
    const int8_t* x;          // byte address of the [n_in][stride] sample planes
    long long stride;         // samples between input planes
    long long base;
    long long vhi;
    int es;                   // bytes per sample: 1 (int8) or 2 (int16)
};

// Ring slots: spectrum s lives in slot (s - origin) & mask.  Rings that wrap
// have a power-of-two capacity (mask = capacity - 1); a buffer that holds
// exactly the spectra of one call uses origin = first spectrum and an
// all-ones mask.
//
// F-engine, stage 1 (polyphase FIR).  Spectra s in [s_begin, s_end) of
// every input pair (a, a+1) are filtered into the ring Z
// [zslot][n_pairs][M] float2, z[m] = (y_a[m], y_b[m]).  Each thread owns 4
// branches of one pair over `spt` consecutive spectra.
struct FirArgs {
    StreamView src;
    const float* h;          // [taps][M] polyphase prototype, FP32
    const int* coarse;       // [n_in_pad] coarse advance d_a
    float2* Z;
    long long z_origin;
    long long z_mask;
    long long s_begin, s_end;
    int n_in, n_pairs, M, lgM, taps, spt;
    // complex input: samples are interleaved (I, Q) int8 pairs (src.es = 2);
    // "pair" p is input p, z[m] = (y_I[m], y_Q[m]), n_pairs = n_in_pad
    int iq;
};

// F-engine, stage 2 (M-point complex FFT of z, then the two real spectra of
// the pair).  Writes ring V [slot][n_chan][n_in_pad] (float2) with
// U_a = Z[k] + Z*[M-k] (= 2 Y_a) and U_b = -j (Z[k] - Z*[M-k]) (= 2 Y_b),
// or, when `phasor` is set, the rotated V_a = Y_a P_a (fine delay and
// instrument phase folded into P, Eq. 1).
struct FftArgs {
    const float2* Z;
    long long z_origin;
    long long z_mask;
    const float2* tw;        // per-pass twiddles, see fft_twiddle_table()
    const float2* phasor;    // [n_in_pad][n_chan] or nullptr
    float2* V;
    long long v_origin;
    long long v_mask;
    long long s_begin, s_end;
    int n_in_pad, M, spt;
    // power mode (tiles set): instead of V, accumulate mean |Y|^2 over rows
    // of n_row spectra into dynamic-spectrum tiles [n_in][rows/64][n_chan/256]
    // [64][256] (atomic adds; the caller zeroes them)
    float* tiles;
    int n_row, rows, n_in;
    // spectra ring pair-major, [slot][pair][n_chan] of float4 (the pair's
    // two complex values), instead of [slot][n_chan][n_in_pad] complex64:
    // the small-N FP32 pipeline, whose X-engine reads that layout
    int pair_major;
    // complex input: z of input p is its complex FIR output; all M channels
    // of its M-point spectrum Z are stored, channel-major with n_chan = M,
    // as U = 2Z (phasor null) or V = Z P (phasor = the rotation)
    int iq;
    // codes instead of spectra (M = 16384, the size the fused F-engine does
    // not cover): V holds the pair-major code words [slot][pair][n_chan]
    // made with the inverse scales inv [n_in_pad][n_chan], e4m3 when fp8
    const float* inv;
    bool fp8;
};

// Fused F-engine (PFB + FFT in one kernel; the FIR output stays in shared
// memory).  Spectra [f.s_begin, f.s_end) of the stream `src` are filtered
// and transformed into the outputs `f` describes (same modes and layouts as
// the FFT stage; f.Z is not used).  hs: [taps][M/2] FP32, the lower half of
// every polyphase row, hs[p][m] = h[p M + m]; the prototype is symmetric,
// h[p M + M-1-m] = h[(taps-1-p) M + m], so the half gives every branch.
struct FusedArgs {
    FftArgs f;
    StreamView src;
    const float* hs;
    const int* coarse;       // [n_in_pad] coarse advance d_a
    int taps;
    int run;                 // spectra per CTA run (0: one wave of resident CTAs)
    // Requantised codes instead of spectra (modes 6 int8, 7 e4m3): f.V holds
    // a pair-major ring of 32-bit words [slot][pair][n_chan] (bytes Re U_a,
    // Im U_a, Re U_b, Im U_b), from the inverse scales inv[a][k].
    const float* inv;        // [n_in_pad][n_chan]; nullptr: spectra out (modes 0-3)
    bool fp8;                // e4m3 codes (mode 7), else int8 (mode 6)
};

// True when the fused kernel covers this shape (int8 samples, 4 taps,
// transform lengths whose buffers fit one CTA); otherwise the two-kernel
// path (launch_fir + launch_fft) runs.
bool fused_f_supported(int M, int taps, int es, int mode);
// CORR_OK, or CORR_EINVAL for a shape fused_f_supported rejects.
int launch_fused_f(const FusedArgs& a, cudaStream_t st);

// X-engine launch: groups of spectra, each group summed into one partial
// slot.  Local group g (0 <= g < n_groups) covers spectra
// [int_start + (j0+g) * G, min(that + G, int_end, s_limit)) where all groups
// of one launch lie inside one integration [int_start, int_end).
struct XArgs {
    const float2* V;
    long long v_origin;
    long long v_mask;
    int n_chan, n_in_pad, nt;
    long long int_start, int_end, s_limit;
    int G, j0, n_groups;
    float* part;             // [gpi][nt][32][n_chan]
    int pair_major;          // V pair-major, see FftArgs
    int depth;               // n_in_pad <= 8: spectra in flight per thread, 4 or 6 (0: 6)
};

// Finalise: R[k][a][b] = scale * Q_a[k] conj(Q_b[k]) * (sum over partial
// slots 0..n_slots-1), Q = rot (or 1 when rot is null).
struct FinArgs {
    const float* part;
    const float2* rot;       // [n_in_pad][n_chan] or nullptr
    int n_slots, nt, n_chan, n_in;
    float scale;
    float2* R;               // [n_chan][n_in][n_in]
};

// Persistent tail of a group replay (batched sub-array streams): one launch
// finalises the integrations the members' FP32 pipelines deferred and
// computes every member's MAD flags, pulling work items from a device queue
// built when the group's graph is captured.  Items are claimed in queue
// order by an atomic ticket: all finalise items come first, so a flag item
// only ever waits (bounded by %globaltimer) for items already claimed by
// running CTAs that never wait themselves.
struct TailMember {
    FinArgs fin;             // FP32 members: partial sums and R of integration 0
    long long part_stride;   // floats between integrations' partial sums
    long long vis_stride;    // complex values between integrations' R (and flags)
    uint8_t* flags;          // flags of integration 0, or null (no flagging)
    int window;              // MAD window W (a power of two <= 256)
    float sigma;
};
struct TailItem {
    int kind;                // 0: a finalise block (x, y, z); 1: MAD flags of warp items x .. x+63
    int member, integration;
    int x, y, z;
    int dep;                 // dependency counter of (member, integration)
    int need;                // finalise blocks that must be done first (flag items)
};
struct TailArgs {
    const TailMember* members;
    const TailItem* items;
    int n_items;
    int* ticket;             // zero before the launch
    int* done;               // per (member, integration): finalise blocks done; zero before
    unsigned long long wait_ns;
    int* status;             // set to CORR_ETIMEDOUT when a wait expires
    int inject_skip;         // fault injection: this finalise item never counts itself done (-1: none)
};
constexpr int kTailWarpItems = 64;   // MAD warp items per flag item (16 per warp)
void launch_group_tail(const TailArgs& a, int grid, cudaStream_t st);
// CTAs of the tail kernel resident at once (the persistent grid).
int group_tail_grid();

// Tensor-core Gram matrix G[c] = Q[c] Q[c]^T, Q [n_chan][128 rows][k_pitch
// bytes] of BF16 (int8 codes) or e4m3, K valid elements per row (later ones
// read as zero); G [n_chan][128][128] FP32.  status: device word set to
// CORR_ETIMEDOUT if a bounded wait expires (may be null).
struct GramArgs {
    const void* Q;
    int n_chan, K, k_pitch;
    bool fp8;
    void* G;
    int* status;
    unsigned long long wait_ns;   // limit of each bounded wait (0: the 2 s default)
    int inject_stall;             // fault injection: the producer issues no loads
    int i8b;                      // int8 codes stored as bytes (widened to BF16 on chip)
    // int8 or e4m3 code words C[t][pair][k] (Q points at them; K spectra,
    // n_pairs pairs of n_in inputs): Gram straight from the F-engine's words
    int words, n_pairs, n_in;
    // words only: with R set the kernel writes the visibilities R[k][a][b]
    // (the finalisation: scales [n_in_pad][n_chan], count = K, optional
    // rotation phasors) instead of G
    float2* R;
    const float* scale;
    const float2* rot;
};

// Requantise spectra [s_begin, s_end) of the pair-major ring V (U = 2Y,
// unrotated; [slot][pair][n_chan] float4) into the integration's code words
// C[t][pair][n_chan], t = s - int_start: bytes q(Re U_a / sigma_a), q(Im U_a
// / sigma_a), q(Re U_a+1 / sigma_a+1), q(Im U_a+1 / sigma_a+1), sigma =
// scale[a][k]; int8 codes (round to nearest even, saturate +-127) or e4m3
// (satfinite).
struct RequantArgs {
    const float2* V;
    long long v_origin, v_mask;
    const float* scale;      // [2][n_in_pad][n_chan]: scales, then their inverses
    long long s_begin, s_end, int_start;
    int n_in, n_in_pad, n_chan;
    bool fp8;
    uint32_t* C;
};

// Requantisation gains g (sigma = sqrt(component power) / g): int8 codes
// saturate at 127 = 5.3 g / 24 standard deviations, e4m3 at 448 = 7 g / 64.
constexpr float kInt8Gain = 24.f;
constexpr float kFp8Gain = 64.f;

int launch_gram(const GramArgs& a, cudaStream_t st);

// General tensor-core GEMM, D[s][m][n] = sum_{k in split s} A[m][k] B[n][k]:
// A [M rows][lda bytes] and B [N rows][ldb bytes] BF16, K-major; D FP32
// partial sums per K split ([splits][M][N]); N in {16, 32, 64}.
struct GemmArgs {
    const void* A;
    const void* B;
    int M, N, K, lda, ldb;
    int splits, k_per_split;   // k_per_split a multiple of 64
    float* D;
    int* status;
};
int launch_gemm(const GemmArgs& a, cudaStream_t st);
// out[m][n] = sum over splits of D[s][m][n], fixed order
// Implicit-GEMM 5x5 convolution of NHWC BF16 images [n_images][64][256][32]
// (see conv_tc.cu).  W: [bn][kp] BF16 K-major, k = (5u+v) 32 + c, bn = 32.
// mode 0: out = BF16 ReLU(z + bias) [P][32]; mode 2: out = FP32 z [P][32].
// sgn -1 negates the tap offsets.
struct ConvArgs {
    const void* X;
    const void* W;
    int kp, n_images, bn, sgn, mode;
    const float* bias;
    void* out;
    int* status;
};
int launch_conv(const ConvArgs& a, cudaStream_t st);

void launch_split_sum(const float* D, int splits, long long mn, float* out, cudaStream_t st);
size_t gram_smem_bytes();
void launch_requant(const RequantArgs& a, cudaStream_t st);
// scale[a][k] = sqrt(c P) / gain with P the mean |U|^2 over spectra
// [s0, s0 + n) of the ring (first integration of a stream) and c the
// component share of the power: 1/2, or 1 in the real DC channel k = 0.
void launch_scale_from_ring(const float2* V, long long v_origin, long long v_mask, long long s0, int n, int n_in,
                            int n_in_pad, int n_chan, float gain, float* scale, int pair_major, cudaStream_t st);
// scale[a][k] = 2 sqrt(c R_aa[k]) / gain (U = 2V, c as above) from an
// integration's R.
void launch_scale_from_vis(const float2* R, int n_in, int n_in_pad, int n_chan, float gain, float* scale,
                           cudaStream_t st);

void launch_fir(const FirArgs& a, cudaStream_t st);
// The complex-input forms of the two F-engine stages (a.iq set).
void launch_fir_iq(const FirArgs& a, cudaStream_t st);
int launch_fft_iq(const FftArgs& a, cudaStream_t st);
// CORR_OK, or CORR_EINVAL / CORR_ECUDA when the spectra's tensor map cannot
// be made (V not 16-byte aligned, no driver entry point).
int launch_fft(const FftArgs& a, cudaStream_t st);
void launch_xengine(const XArgs& a, cudaStream_t st);
void launch_finalize(const FinArgs& a, cudaStream_t st);
// Finalisation and MAD flags of one integration in one launch (FP32 path,
// n_in <= 8, window <= 64 channels dividing n_chan): the same results as
// launch_finalize followed by launch_mad_flags.
bool fin_flag_small_supported(int n_in, int window);
void launch_fin_flag_small(const FinArgs& a, uint8_t* F, int window, float sigma, cudaStream_t st);
void launch_mad_flags(const float2* R, uint8_t* F, int n_vis, int n_chan, int n_in, int window,
                      float sigma, cudaStream_t st);

// Twiddles of every radix-16 pass of the M-point Stockham FFT, laid out
// [pass][r][k] (k contiguous) with entry W_{16 Ns}^{r k}, r < 16, k < Ns,
// passes in execution order (Ns = first radix, then x16 ...).  Returns the
// table, computed in FP64 and rounded to FP32.
std::vector<float2> fft_twiddle_table(int M);

// Error text reported by corr_last_error(NULL) (calls without a handle).
void set_global_error(const std::string& msg);

}  // namespace corr
