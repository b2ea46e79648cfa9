/*
 * corr.h -- C ABI of the GB300 FX correlator (libcorr.so).
 *
 * The library computes, on one GPU, the hot path of an FX software correlator
 * (arXiv 2604.20640):
 *
 *   F-engine  (Sec. 4.2, "F-engine (PFB and FFT)"): int8 or int16 samples -> P-tap
 *             windowed-sinc polyphase FIR over M = 2*n_chan branches -> M-point
 *             real FFT (channels 0 .. n_chan-1, DC kept, Nyquist dropped),
 *             with the geometric delay of Eq. 1 (Sec. 4.1) removed per input
 *             as a coarse integer advance d = floor(tau + 1/2) plus a fine
 *             phase exp(+j 2 pi k (tau - d) / M), and the instrument phase
 *             removed as exp(-j phi).
 *   X-engine  (Sec. 4.2, "X-engine and integration"; Algorithm 1):
 *             R[k][a][b] = (1/n_int) sum_s V_a,s[k] conj(V_b,s[k]) over each
 *             integration of n_int consecutive spectra, full Hermitian matrix.
 *   Flagging  (Eq. 2, Sec. 7): per integration, baseline (a,b) and aligned
 *             window of `flag_window` channels, A = |R_ab|,
 *             T = median(A) + sigma * 1.4826 * MAD(A), flag = A > T.
 *
 * Conventions
 *   - Every call returns a status (CORR_OK = 0 or a negative CORR_E* code)
 *     and never aborts; corr_last_error() gives a message for the last
 *     failure on that handle (or on handle creation when h is NULL).
 *   - Inputs are n_in = n_ant * n_pol planes of samples (int8, or int16 with
 *     option "sample_bits" = 16), input index a = ant * n_pol + pol; plane a
 *     starts input_stride samples after plane a-1.
 *   - Visibilities are complex64 stored as interleaved float pairs
 *     (re, im), layout [integration][n_chan][n_in][n_in]; flags are uint8
 *     in the same layout (symmetric in a, b).
 *   - Host pointers are owned by the caller and may be reused as soon as a
 *     call returns.  Device pointers (the *_dev calls) are owned by the
 *     caller and must stay valid until the work queued on `stream` finishes.
 *   - The library owns all of its own device memory and streams.  A handle
 *     is not thread-safe: use one host thread per handle.
 *   - `stream` arguments are cudaStream_t values passed as void*; NULL
 *     means the legacy default stream.
 */
#ifndef CORR_H
#define CORR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct corr_s* corr_t;

enum {
    CORR_OK = 0,
    CORR_EINVAL = -1,     /* bad argument or shape */
    CORR_ENOMEM = -2,     /* device or pinned allocation failed */
    CORR_ECUDA = -3,      /* a CUDA runtime call failed */
    CORR_EAGAIN = -4,     /* nothing ready yet (results) */
    CORR_ETIMEDOUT = -5,  /* a bounded device wait expired */
    CORR_ESTATE = -6      /* call not valid in the handle's current state */
};

/* Precision of the X-engine (option "precision"). */
enum { CORR_FP32 = 0, CORR_INT8 = 1, CORR_FP8 = 2 };
/* Code layouts of corr_gram_dev beside CORR_INT8 (int8 carried as BF16) and
 * CORR_FP8 (e4m3 bytes): int8 codes stored as bytes, and the pipeline's code
 * words of int8 or e4m3 codes. */
enum { CORR_INT8_BYTES = 3, CORR_INT8_WORDS = 4, CORR_FP8_WORDS = 5 };

/*
 * corr_create -- allocate a correlator.
 *   n_ant, n_pol >= 1; n_in = n_ant*n_pol <= 256.
 *   n_chan: power of two, 8 <= n_chan <= 8192 (M = 2*n_chan point real FFT;
 *           the "FFT length" runtime parameter of Sec. 4.3).
 *   taps:   PFB taps P, 1 <= P <= 16 (Sec. 4.3 "number of PFB taps").
 *   n_int:  spectra per integration >= 1 (Sec. 4.3 "integration interval").
 * Delays and phases start at zero.  Returns CORR_EINVAL on bad shapes and
 * CORR_ENOMEM / CORR_ECUDA if device set-up fails (*out is then NULL).
 */
int corr_create(corr_t* out, int n_ant, int n_pol, int n_chan, int taps, int n_int);

/* corr_destroy -- wait for queued work, free everything.  NULL is a no-op. */
int corr_destroy(corr_t h);

/* corr_last_error -- message of the last failed call on h (never NULL). */
const char* corr_last_error(corr_t h);

/*
 * corr_set_option -- set a tunable before the first push (CORR_ESTATE after).
 *   "flag_sigma"  (double > 0, default 5)     sigma of Eq. 2
 *   "flag_window" (power of two, default 64)  channels per MAD window
 *                 (min(window, n_chan) is used)
 *   "max_delay"   (samples, default 4096)     bound on |coarse delay|
 *   "chunk"       (samples/input, default 1<<23) largest device batch
 *   "precision"   (CORR_FP32 / CORR_INT8 / CORR_FP8, default FP32): FP32
 *                 CUDA-core X-engine, or channelised voltages requantised to
 *                 int8 (stored as bytes, widened to BF16 on chip) / e4m3 with
 *                 one scale per (input,
 *                 channel) fixed per integration, correlated on tcgen05
 *                 tensor cores (n_in <= 64).  Scales: first integration from
 *                 the mean power of its first min(n_int, 64) spectra
 *                 (sigma = sqrt(P_c)/g with P_c the power of one component:
 *                 P/2, or P in the real DC channel; g = 24 int8, 64 e4m3),
 *                 later ones from the previous integration's
 *                 autocorrelations.
 *   "result_slots" (default 8)               pinned result FIFO depth (grows)
 *   "stage_timing" (0/1, default 0; may change at any time)  per-stage events
 *   "stage_mask"   (bit mask, default 127 = all; may change at any time)
 *                  stages (numbered as in corr_stage_times) that
 *                  stage_timing brackets; fewer events disturb the
 *                  pipeline less
 *   "ring_mb"      (1..4096, default 64)  MiB of each on-device spectrum ring
 *                  (more spectra per launch; see corr_autotune)
 *   "fir_spt"      (0 = automatic, 1..256; may change at any time)
 *                  spectra each F-engine thread runs over: the FIR kernel's
 *                  run, or the fused kernel's run per CTA (automatic: one
 *                  wave of resident CTAs); results do not depend on it
 *   "x_depth"      (6, default, or 4; may change at any time)  spectra each
 *                  thread of the small X-engine (at most 8 inputs) has in
 *                  flight; results do not depend on it
 *   "fused_f"      (1, default, or 0; may change at any time)  run the
 *                  F-engine as one kernel (FIR output kept in shared
 *                  memory) where it covers the shape -- int8 samples, 4
 *                  taps, 1024 <= M <= 8192 for the pipeline's spectra
 *                  rings and the dynamic spectra, M = 8192 for the stage
 *                  call -- else as FIR + FFT; results are bit-identical.
 *                  With reduced precision the fused kernel also makes the
 *                  int8 / e4m3 code words once an integration's scales are
 *                  fixed, straight into the words the tensor-core X-engine
 *                  reads (at M = 16384 the two-kernel FFT does, whatever
 *                  this option); the codes equal the requantiser's
 *   "sample_bits"  (8, default; or 16)  input sample type of every call that
 *                  takes samples: int8 (the 8-bit truncated recorder mode of
 *                  Sec. 3) or little-endian int16 (the 16-bit padded mode,
 *                  14-bit ADC values, Sec. 3); sample pointers are `const
 *                  void*`, counts and strides are in samples.  Before the
 *                  first push.
 *   "sample_format" (0, default: real samples; 1: complex) -- with 1 every
 *                  input is a stream of complex baseband samples, (I, Q)
 *                  int8 pairs interleaved (Sec. 4.2, "converted into complex
 *                  voltage streams"); counts and strides are in complex
 *                  samples.  The transform is an M = n_chan point complex
 *                  FFT that keeps all n_chan channels in FFT order, channel
 *                  k at k/M cycles per sample below M/2 and (k - M)/M above
 *                  (the fine delay phase exp(j 2 pi f_k r) uses these signed
 *                  frequencies).  FP32 path only (CORR_EINVAL with reduced
 *                  precision, 16-bit samples or n_chan < 16); the dynamic
 *                  spectra call is for real input.  Before any buffers exist.
 *   "max_pending"  (0 = no limit, default; may change at any time) a push
 *                  is refused with CORR_EAGAIN, consuming nothing, while this
 *                  many completed integrations wait to be popped (the
 *                  caller's back-pressure on a full result queue)
 *   "inject_alloc_fail" (0, default, or n; may change at any time) fault
 *                  injection: the n-th device allocation the handle makes
 *                  from now fails with CORR_ENOMEM (the failed step leaves
 *                  no half-built buffers; the handle stays usable)
 *   "tc_wait_ms"   (1 .. 60000, default 2000; may change at any time)
 *                  limit of every bounded wait of the tensor-core X-engine
 *                  (producer / MMA / epilogue barriers); on expiry the kernel
 *                  records CORR_ETIMEDOUT (corr_device_status), frees its
 *                  tensor memory and returns, leaving that integration's
 *                  Gram matrices unwritten
 *   "inject_stall" (0, default, or 1; may change at any time) fault
 *                  injection for testing that path: the tensor-core
 *                  X-engine's load producer issues nothing, so the MMA
 *                  issuer's first wait expires after tc_wait_ms
 *   "window"       (0 Hann, default; 1 Kaiser; 2 unit coefficients) taper
 *                  of the prototype filter h = taper x sinc (Sec. 4.2; the
 *                  8-tap Kaiser of Fig. 4); 2 with taps = 1 is the plain
 *                  per-frame DFT.  Rebuilds the filter; before the first push.
 *   "kaiser_beta"  (0..50, default 8)  Kaiser parameter
 */
int corr_set_option(corr_t h, const char* key, double value);

/*
 * corr_set_delays -- total delay per input in samples (FP64) and instrument
 * phase per input in radians (NULL => zeros), Eq. 1.  The library splits
 * tau into d = floor(tau + 1/2) and r = tau - d.  |d| must be <= max_delay.
 * Before the first push the values apply from spectrum 0; afterwards they
 * take effect at the next integration boundary, never mid-integration.
 */
int corr_set_delays(corr_t h, const double* delay_samples, const double* phase_rad);

/*
 * corr_push -- append n_per_input samples to every input from a host buffer
 * (planar, plane a at samples + a*input_stride, input_stride >= n_per_input).
 * The samples are copied to the device before the call returns, so the
 * buffer may be reused at once; page-locked buffers are copied directly by
 * DMA, others through the library's pinned staging.  Every spectrum whose
 * samples are now all present is channelised and correlated; completed
 * integrations are finalised, flagged and queued for corr_get_vis /
 * corr_get_flags.  Any chunking of a stream gives bit-identical results.
 */
int corr_push(corr_t h, const void* samples, size_t n_per_input, size_t input_stride);

/*
 * corr_push_dev -- as corr_push, from device memory d_samples (caller-owned,
 * planar with input_stride), work queued on `stream`.  No host sync.
 */
int corr_push_dev(corr_t h, const void* d_samples, size_t n_per_input,
                  size_t input_stride, void* stream);

/*
 * corr_flush -- end of stream: samples past the end read as zero, the last
 * spectra are processed, and a partial last integration (if any) is
 * finalised with its actual spectrum count.  The handle then accepts no
 * more pushes (CORR_ESTATE) until corr_reset.
 */
int corr_flush(corr_t h);

/* corr_reset -- forget the stream (history, counters, queued results). */
int corr_reset(corr_t h);

/*
 * corr_get_vis / corr_get_flags -- pop up to max_int completed integrations
 * (oldest first) into the caller's host buffer out
 * [max_int][n_chan][n_in][n_in] (vis: complex64 as float pairs; flags: uint8).
 * Visibilities and flags are popped independently, in the same order.
 * Page-locked (pinned) out is filled by DMA straight from device memory;
 * other host memory receives a copy of the library's pinned image.  While
 * the last pop went to pinned memory, integrations finished afterwards get
 * no pinned image (no second device-to-host copy); a pop into other memory
 * makes it then.  Blocks only until the popped integrations' results have
 * landed.
 * *n_got receives the count (0 and CORR_EAGAIN when none is queued).
 */
int corr_get_vis(corr_t h, float* out, int max_int, int* n_got);
int corr_get_flags(corr_t h, uint8_t* out, int max_int, int* n_got);

/* corr_pending -- number of completed integrations not yet popped (vis). */
int corr_pending(corr_t h, int* n);

/*
 * corr_run_dev -- whole-stream, device-resident form of the hot path:
 * d_samples holds an entire stream of n_samples per input (zero history
 * before sample 0, zero after the end), planar with input_stride.  Computes
 * floor(n_samples / M) spectra with the handle's current delays, every
 * complete integration (plus the partial last one if include_partial != 0),
 * into caller-owned device buffers d_vis [n][n_chan][n_in][n_in] complex64
 * and d_flags (same layout, uint8; may be NULL to skip flagging), with
 * n <= max_int (CORR_EINVAL if too small).  *n_out = integrations written.
 * Work is queued on `stream`; the handle's streaming state is untouched.
 */
int corr_run_dev(corr_t h, const void* d_samples, size_t n_samples, size_t input_stride,
                 float* d_vis, uint8_t* d_flags, int max_int, int include_partial,
                 int* n_out, void* stream);

/*
 * Stateless stage entry points (device pointers, queued on `stream`), used
 * to test and time the stages one by one.  They use the handle's shapes,
 * filter, delays, phases and options only.
 *
 * corr_fengine_dev -- channelise spectra s0 .. s0+n_spec-1 of the
 *   device-resident stream (same conventions as corr_run_dev) into
 *   d_V [n_spec][n_chan][n_in_pad] complex64, n_in_pad = n_in rounded up to
 *   a multiple of 4 (padding inputs are written as zeros); d_V must be
 *   16-byte aligned (the FFT writes it with tensor stores; CORR_EINVAL
 *   otherwise).  Sec. 4.2 F-engine with Eq. 1's delay and phase terms.
 * corr_xengine_dev -- R[k][a][b] = (1/n_spec) sum_s V V^* over all n_spec
 *   spectra of d_V (layout as above) into d_vis [n_chan][n_in][n_in]
 *   complex64.  Sec. 4.2 X-engine.  d_V must be 16-byte aligned (it is read
 *   as 16-byte vectors) and d_vis 8-byte aligned, else CORR_EINVAL before
 *   any launch.
 * corr_flag_dev -- MAD flags (Eq. 2) of n_vis integrations d_vis into d_flags.
 */
int corr_fengine_dev(corr_t h, const void* d_samples, size_t n_samples, size_t input_stride,
                     long long s0, int n_spec, float* d_V, void* stream);
int corr_xengine_dev(corr_t h, const float* d_V, int n_spec, float* d_vis, void* stream);
int corr_flag_dev(corr_t h, const float* d_vis, int n_vis, uint8_t* d_flags, void* stream);

/*
 * corr_gram_dev -- tensor-core Gram matrices, the dense form of the X-engine
 * (Sec. 4.2, Algorithm 1) on requantised voltages: for every channel c,
 * G[c] = Q[c] Q[c]^T with Q [n_chan][128 rows][k_pitch bytes] in device
 * memory, K valid elements per row (later elements read as zero).  Rows hold
 * the real parts of the inputs' codes, then the imaginary parts, then zeros,
 * so sum_s q_a conj(q_b) = (G_rr + G_ii) + j (G_ir - G_ri).
 *   dtype CORR_INT8: int8 codes stored as BF16 values (2 bytes each); the
 *                    products are exact, the sums FP32 (exact while every
 *                    partial sum stays below 2^24).
 *   dtype CORR_FP8:  e4m3 bytes; FP32 sums.
 *   dtype CORR_INT8_BYTES: int8 codes as bytes (1 byte each), widened to
 *                    BF16 on chip (exact), then as CORR_INT8.
 *   dtype CORR_INT8_WORDS: the form the int8 pipeline uses (n_chan a
 *                    multiple of 4) -- d_Q holds code words [K][n_pairs]
 *                    [n_chan] uint32, n_pairs = n_in_pad / 2 (the handle's
 *                    n_in rounded up to a multiple of 4; words of pairs
 *                    past the last input are ignored), the bytes of word
 *                    (t, p, c) being the codes of Re V_2p, Im V_2p, Re
 *                    V_2p+1, Im V_2p+1 (low byte first); rows as above (row
 *                    a = Re of input a, row n_in + a = Im); only the leading
 *                    2 n_in x 2 n_in block of each G[c] is written; k_pitch
 *                    is ignored, n_chan must be a multiple of 4 and n_in <=
 *                    64.
 *   dtype CORR_FP8_WORDS: the e4m3 pipeline's form -- code words as for
 *                    CORR_INT8_WORDS holding e4m3 codes; FP32 sums.
 * d_G: [n_chan][128][128] FP32.  k_pitch must be a multiple of 128 and d_Q
 * 16-byte aligned (else CORR_EINVAL).  Runs on tcgen05 tensor cores with
 * TMA-staged operands; a stalled pipeline sets the status word read by
 * corr_device_status to CORR_ETIMEDOUT instead of hanging.
 */
int corr_gram_dev(corr_t h, const void* d_Q, int n_chan, int k_pitch, int K, int dtype, float* d_G,
                  void* stream);

/*
 * corr_device_status -- wait for the device, return the handle's device
 * status word (CORR_OK or CORR_ETIMEDOUT from a bounded wait) and clear it.
 */
int corr_device_status(corr_t h, int* status);

/*
 * Batched sub-array streams.  corr_group_create bundles n (<= 64) existing
 * handles (their shapes may all differ) into a group handle; the members
 * stay owned by the caller and must outlive the group.
 * corr_group_run_dev runs corr_run_dev for every member (stream i:
 * d_samples[i], n_samples[i], strides[i] -> d_vis[i], d_flags[i] (d_flags may
 * be NULL), complete integrations only) as parallel branches of one CUDA
 * graph, launched on `stream`; n_out[i] (may be NULL) receives the
 * integrations written.  The first call (and any call whose pointers or
 * sizes differ from the last capture) runs each member once uncaptured,
 * then captures the graph; later calls replay it.  Do not run members on
 * their own while a group call may still be executing.
 */
int corr_group_create(corr_t* group, const corr_t* members, int n);
int corr_group_run_dev(corr_t group, const void* const* d_samples, const size_t* n_samples,
                       const size_t* strides, float* const* d_vis, uint8_t* const* d_flags,
                       const int* max_int, int* n_out, void* stream);

/*
 * corr_autotune -- pick the ring capacity ("ring_mb" 32/64/128/256, the
 * spectra per launch), the F-engine's work split ("fir_spt" auto/8/16:
 * spectra per thread run of the FIR kernel, or per CTA of the fused
 * kernel) and, for FP32 pipelines of at most 8 inputs, the X-engine's
 * pipeline depth ("x_depth" 4/6: spectra each thread has in flight) of a
 * handle by timing corr_run_dev on up to eight integrations of a device
 * sample (results do not depend on any of the choices; larger rings mean
 * larger launches).  cache_path (may be NULL) is a text file of
 * "gpu n_in n_chan taps n_int precision ring_mb fir_spt x_depth" lines
 * (x_depth may be missing: 6): a matching line is applied without timing,
 * a new choice is appended.  corr_get_tuning reports the current values
 * (any pointer may be NULL).
 */
int corr_autotune(corr_t h, const void* d_samples, size_t n_samples, size_t input_stride,
                  const char* cache_path, void* stream);
int corr_get_tuning(corr_t h, int* ring_mb, int* fir_spt, int* x_depth);

/*
 * corr_spectrogram_dev -- autocorrelation power of every input in tiles of
 * 64 rows x 256 channels (the (time x channel) dynamic spectra of Sec. 5):
 * row r of input a holds mean_{s in [r n_row, (r+1) n_row)} |Y_a,s[k]|^2 from
 * this F-engine (no fine-delay factor: it has unit modulus; the FFT kernel
 * accumulates the powers, no spectra are stored; FP32 sums, so the order of
 * the additions across the F-engine's work split is not fixed), for
 * rows = 64 floor(n_spec / (64 n_row)) rows, n_spec = floor(n_samples / M):
 * whole tiles only, later spectra are not read.  n_chan must be a multiple
 * of 256 and rows >= 64, else CORR_EINVAL.  d_tiles: [n_in][rows/64]
 * [n_chan/256][64][256] FP32 (device, caller-owned, overwritten).
 */
int corr_spectrogram_dev(corr_t h, const void* d_samples, size_t n_samples, size_t input_stride, int n_row,
                         float* d_tiles, void* stream);

/*
 * Learned RFI flagger (the paper has none: it is the build's counterpart of
 * the MAD flagging of Eq. 2, Sec. 7, on the dynamic spectra of Sec. 5).
 * A 5x5 convolutional net, channels 1 -> 32 -> 32 -> 32 -> 1, zero padding
 * 2, ReLU after the hidden layers, a logistic output per pixel (52,897
 * parameters), on tiles of 64 x 256 pixels x = ln(P / median(P)) of
 * autocorrelation power P.  BF16 operands, FP32 accumulation on tcgen05
 * tensor cores; FP32 master weights trained with Adam on the mean binary
 * cross-entropy.  Inference runs any n_tiles in passes of 64 tiles; the
 * handle keeps a workspace of about 2.5 GB for them.  Parameters are flattened layer by layer as w[o][c][u][v]
 * then b[o].
 *   corr_flagnet_prepare    d_power [B][64][256] -> d_x (the network input)
 *   corr_flagnet_forward    d_x -> d_logits [B][64][256]
 *   corr_flagnet_loss_grad  mean loss and (host) gradients, no update
 *   corr_flagnet_train_step one Adam step (lr), returns the loss
 *                           (both: 1 <= n_tiles <= 64, else CORR_EINVAL)
 *   corr_flagnet_flag       flags of B power tiles: the net's (p > 1/2) when
 *                           the tile confidence mean|2p-1| >= c_min, else
 *                           Eq. 2 along each row over 64-channel windows;
 *                           d_conf [B] (may be NULL) receives the confidences
 *   corr_flagnet_status     device status word (CORR_ETIMEDOUT on a stalled
 *                           tensor-core pipeline), cleared on read
 */
typedef struct corr_flagnet_s* corr_flagnet_t;
int corr_flagnet_create(corr_flagnet_t* out);
int corr_flagnet_destroy(corr_flagnet_t net);
int corr_flagnet_num_params(size_t* n);
int corr_flagnet_set_params(corr_flagnet_t net, const float* params, size_t n);
int corr_flagnet_get_params(corr_flagnet_t net, float* params, size_t n);
int corr_flagnet_prepare(corr_flagnet_t net, const float* d_power, int n_tiles, float* d_x, void* stream);
int corr_flagnet_forward(corr_flagnet_t net, const float* d_x, int n_tiles, float* d_logits, void* stream);
int corr_flagnet_loss_grad(corr_flagnet_t net, const float* d_x, const uint8_t* d_truth, int n_tiles, float* loss,
                           float* grads, size_t n, void* stream);
int corr_flagnet_train_step(corr_flagnet_t net, const float* d_x, const uint8_t* d_truth, int n_tiles, float lr,
                            float* loss, void* stream);
int corr_flagnet_flag(corr_flagnet_t net, const float* d_power, int n_tiles, float c_min, float sigma,
                      uint8_t* d_flags, float* d_conf, void* stream);
int corr_flagnet_status(corr_flagnet_t net, int* status);
/* Kernels this handle has launched since it was created. */
long long corr_flagnet_kernel_launches(corr_flagnet_t net);

/*
 * corr_tile_mad_dev -- Eq. 2 (sigma, 1.4826 MAD scale, strict A > T) on
 * (time x channel) power tiles [n_tiles][64][256] (device FP32 in, device
 * uint8 flags out, same layout): axes bit 1 along each row over aligned
 * 64-channel windows (the paper's direction), bit 2 along each channel over
 * the tile's 64 rows (the time direction, where broadband bursts stand
 * out); 3 = the union.  Stateless; CORR_EINVAL on bad arguments.
 */
int corr_tile_mad_dev(const float* d_power, int n_tiles, float sigma, int axes, uint8_t* d_flags, void* stream);

/*
 * corr_calibrate_dev -- delay and phase calibration (Sec. 7, Eq. 3) from the
 * visibilities of one integration d_vis [n_chan][n_in][n_in] (complex64,
 * device, as corr_run_dev writes them), for every baseline (ref, a):
 *   1. coarse delay: the peak of the delay spectrum
 *      |sum_k R_k exp(-j 2 pi k t / M)| over t = -T .. T in quarter samples
 *      (T = ceil(max_delay), M = 2 n_chan);
 *   2. fine delay: weighted (|R_k|) linear fit to the unwrapped phase of the
 *      coarse-corrected visibilities, tau = t + (M / 2 pi) d phase / d k;
 *   3. residual phase: phi = -arg of the mean complex vector after removing
 *      the delay.
 * Channels outside [k_lo, k_hi) or flagged in d_flags (same layout, may be
 * NULL) are left out.  tau[n_in], phi[n_in] (host, caller-owned) receive
 * samples and radians relative to input ref (0 there; NaN for a baseline
 * with no usable channel) in the convention of corr_set_delays, so that
 * applying them flattens the phases.  Synchronous on `stream`.  The paper
 * fits in FP64; steps 2-3 run in FP64, the delay-spectrum search in FP32.
 */
int corr_calibrate_dev(const float* d_vis, const uint8_t* d_flags, int n_chan, int n_in, int ref, int k_lo, int k_hi,
                       double max_delay, double* tau, double* phi, void* stream);

/*
 * corr_peak_fp32 -- measured FP32 arithmetic peak of the current device, the
 * ceiling of the F-engine's floating-point work (its roofline when HBM is not
 * the bound; the paper states no such figure, this is a library facility).
 * Independent chains of dependent fused multiply-adds in every thread of
 * four waves of full SMs, scalar (packed = 0: 2 FLOP per lane per
 * instruction) or packed FP32 pairs (packed = 1: fma.rn.f32x2, 4 FLOP per
 * lane per instruction), `iters` FMAs per chain; one warm-up launch, then
 * one launch timed with CUDA events on `stream`.  *tflops receives the rate
 * (1e12 FLOP/s) and *ms (may be NULL) the timed launch's duration.  The SM
 * clock during the call sets the figure.  Synchronous; CORR_EINVAL on bad
 * arguments, CORR_ECUDA if a CUDA call fails (corr_last_error(NULL)).
 */
int corr_peak_fp32(int packed, int iters, double* tflops, double* ms, void* stream);

/*
 * corr_save_state / corr_load_state -- checkpoint and resume a stream (a
 * library facility; the paper has no counterpart).  corr_save_state waits
 * for the handle's queued work and writes its streaming state into buf
 * (host, caller-owned, cap bytes): the samples still needed by spectra not
 * yet channelised, the channelised spectra not yet summed, the current
 * integration's partial sums (FP32) or scales and codes (reduced precision),
 * the active and pending delays, the counters and every result not yet
 * popped.  With buf NULL it only sets *size to the bytes needed.
 * corr_load_state restores such a state into a new (or reset) handle
 * created with the same shape and options; pushing the rest of the stream
 * then gives results bit-identical to an uninterrupted stream.  CORR_EINVAL
 * for a state of another shape or options, or a truncated one; CORR_ESTATE
 * when the handle has already started.  The format belongs to this library
 * version.
 */
int corr_save_state(corr_t h, void* buf, size_t cap, size_t* size);
int corr_load_state(corr_t h, const void* buf, size_t size);

/* Shapes of a handle: n_in, n_chan, taps, n_int, n_in_pad (any may be NULL). */
int corr_shape(corr_t h, int* n_in, int* n_chan, int* taps, int* n_int, int* n_in_pad);

/* Number of CUDA kernels this handle has launched (instrumentation). */
long long corr_kernel_launches(corr_t h);

/*
 * corr_stage_times -- per-stage GPU time, the correlator's counterpart of
 * the per-stage timings the paper tracks in Sec. 6 (GPU compute, H2D).
 * With option "stage_timing" = 1 every kernel launch is bracketed by CUDA
 * events on its own stream.  This call waits for those events and returns,
 * for stages 0 FIR, 1 FFT (the two F-engine kernels; the fused F-engine
 * kernel counts as stage 1), 2 X-engine,
 * 3 finalise, 4 flagging, 5 requantise, 6 tensor-core Gram (first
 * n_stages entries, at most 7; the dynamic spectra of
 * corr_spectrogram_dev are accumulated by the FFT kernel; with at most 8
 * inputs and flag windows of at most 64 channels the FP32 path makes the
 * flags in the finalisation launch, stage 3; with reduced precision and a
 * channel count that is a multiple of 4 the Gram launch, stage 6, also
 * finalises), the milliseconds and
 * launch counts accumulated since the previous call, then clears them.
 * ms / counts may be NULL.
 */
int corr_stage_times(corr_t h, double* ms, long long* counts, int n_stages);

/*
 * corr_xengine_noalloc -- the X-engine of corr_xengine_dev for callers that
 * cannot allocate device memory: real-time loops where an allocator call
 * (which can synchronise the device) would stall the stream that has to keep
 * up with the samples, and hosts that manage the GPU's memory budget
 * themselves from a plan fixed at start-up.  The paper has no counterpart;
 * it is a library facility.
 *   d_V:    device [n_spec][n_chan][n_in_pad] complex64, n_in_pad = n_in
 *           rounded up to a multiple of 4 (padding entries are ignored);
 *           16-byte aligned.
 *   d_vis:  device [n_chan][n_in][n_in] complex64 output,
 *           R[k][a][b] = (1/n_spec) sum_s V_a V_b^*; 8-byte aligned.
 *   stream: cudaStream_t as void*.
 * Needs no handle and allocates nothing: its partial sums live in one 8 MiB
 * file-scope device array that every GPU loading the library keeps until
 * exit.  Shapes whose per-group scratch ((blocks of 4 inputs, A <= B) * 32 *
 * n_chan floats) exceeds 2^21 floats are rejected with CORR_EINVAL; long
 * streams are summed in fewer, longer groups.  The first call on a device
 * looks up the array's device address (cudaGetSymbolAddress, a synchronous
 * runtime call) and keeps it for the life of the process; do not call it
 * after cudaDeviceReset.  All calls share the
 * array and it keeps the last call's contents (every part a call reads it
 * first writes itself), so calls that overlap on the GPU race: serialise
 * them on one stream.  Misaligned buffers are rejected with CORR_EINVAL, and
 * a CUDA error already pending from earlier work is reported (CORR_ECUDA)
 * without being cleared.  On failure corr_last_error(NULL) describes the
 * error.
 */
int corr_xengine_noalloc(const float* d_V, int n_spec, int n_in, int n_chan, float* d_vis, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* CORR_H */
