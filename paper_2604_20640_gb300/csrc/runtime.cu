// Runtime and C ABI of libcorr: handles, device tables, the streaming state
// (history carry-over between pushes, integration bookkeeping), the pinned
// result FIFO and the whole-stream / per-stage device entry points.
//
// Streaming follows Algorithm 1 of the paper: samples arrive in pushes, are
// copied host -> device on a copy stream, every spectrum whose samples are
// all present is channelised (F-engine) and summed (X-engine) on a compute
// stream, and each completed integration is finalised, flagged (Eq. 2) and
// copied device -> host asynchronously.
#include "corr.h"
#include "corr_internal.h"

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <deque>
#include <string>
#include <vector>

using namespace corr;

namespace {

thread_local std::string g_create_error;

struct Pipe {
    long long s_next = 0;     // next spectrum to channelise
    long long s_xdone = 0;    // first spectrum not yet summed (or requantised)
    float2* V = nullptr;      // ring of channelised spectra
    float2* Z = nullptr;      // ring of FIR outputs (same capacity)
    int v_cap = 0;
    float* part = nullptr;    // [gpi][nt][32][n_chan]
    // partial sums of every integration of a run whose finalisation is
    // deferred to a group's tail kernel: [integration][gpi][nt][32][n_chan]
    float* part_all = nullptr;
    long long part_all_ints = 0;
    // reduced-precision path (tensor-core X-engine)
    float* scale = nullptr;   // [n_in_pad][n_chan], fixed per integration
    bool have_scale = false;  // false until the first integration's pre-pass
    // the integration's int8 or e4m3 code words C[t][pair][n_chan] (bytes
    // Re a, Im a, Re a+1, Im a+1), read by the Gram kernel directly
    uint32_t* C = nullptr;
};

struct Slot {
    float2* d_R = nullptr;
    uint8_t* d_F = nullptr;
    float2* h_R = nullptr;
    uint8_t* h_F = nullptr;
    cudaEvent_t ev = nullptr;
    bool in_vis = false, in_flag = false;
    bool has_image = false;   // h_R / h_F hold the results (or will once ev completes)
};

struct Tables {
    float2* phasor = nullptr;   // [n_in_pad][n_chan] with the pair factors 1/2, 1/2j
    float2* rot = nullptr;      // [n_in_pad][n_chan] exp(j(2 pi k r/M - phi))
    int* coarse = nullptr;      // [n_in_pad]
    int d_max = 0;              // largest coarse advance
};

// Optional CUDA-event brackets around every kernel launch, per stage
// (0 FIR, 1 FFT, 2 X-engine, 3 finalise, 4 flag, 5 requantise, 6 tensor-core
// Gram).
constexpr int kStages = 7;
struct StageTimer {
    bool on = false;
    int mask = (1 << kStages) - 1;   // stages bracketed while on
    std::vector<cudaEvent_t> pool;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> open[kStages];
    double ms[kStages] = {};
    long long n[kStages] = {};
    cudaEvent_t take() {
        if (!pool.empty()) {
            cudaEvent_t e = pool.back();
            pool.pop_back();
            return e;
        }
        cudaEvent_t e = nullptr;
        cudaEventCreate(&e);
        return e;
    }
};

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

}  // namespace

struct corr_s {
    int n_ant = 0, n_pol = 0, n_in = 0, n_in_pad = 0, n_chan = 0, M = 0, taps = 0, n_int = 0;
    int nt = 0;        // 4x4 block-pairs of the Hermitian matrix
    int G = 0;         // spectra per partial slot
    int gpi = 0;       // partial slots per integration
    int dev = 0;
    // options
    double flag_sigma = 5.0;
    int flag_window = 64;
    long long max_delay = 4096;
    long long chunk = 1LL << 23;
    int precision = CORR_FP32;
    int result_slots = 8;
    int ring_mb = 64;            // tunable: ring capacity of Z and V (MiB each)
    int fir_spt = 0;             // tunable: spectra per FIR thread (0 = automatic)
    int x_depth = 6;             // tunable: small X-engine's spectra in flight per thread (4 or 6)
    int window = 0;              // PFB taper: 0 Hann, 1 Kaiser, 2 unit coefficients
    int es = 1;                  // bytes per input sample: 1 (int8), 2 (int16, 16-bit padded mode; or int8 I/Q)
    int iq = 0;                  // complex input: interleaved int8 I/Q, M = n_chan
    double kaiser_beta = 8.0;
    // group of handles run as one captured graph (corr_group_create)
    bool is_group = false;
    std::vector<corr_s*> members;
    std::vector<cudaStream_t> mstreams;
    std::vector<cudaEvent_t> mjoin;
    cudaEvent_t gfork = nullptr;
    cudaStream_t gorigin = nullptr;  // capture / launch stream of a group
    cudaEvent_t gin = nullptr, gout = nullptr;
    long long graph_kernels = 0;     // kernels in one replay of the group graph
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    std::vector<const void*> gkey;   // pointers/sizes the graph was captured with
    // constant tables
    float* d_h = nullptr;
    float* d_hs = nullptr;       // half rows of d_h for the fused F-engine
    float2* d_tw = nullptr;
    int fused_f = 1;             // F-engine as one fused kernel where supported
    bool defer_tail = false;     // inside a group call: finalise / flag in the group's tail kernel
    // group: the tail kernel's work queue (device) and its counters
    TailMember* d_tail_members = nullptr;
    TailItem* d_tail_items = nullptr;
    int* d_tail_counters = nullptr;   // [0] ticket, [1..] per (member, integration) done counts
    int tail_items = 0, tail_deps = 0, tail_grid = 0, tail_fin_items = 0;
    int inject_alloc_fail = 0;   // fault injection: the n-th next device allocation fails
    int max_pending = 0;         // pushes refused (CORR_EAGAIN) while this many results wait (0: no limit)
    std::vector<double> stream_tau, stream_phi;  // delays in the stream tables now
    double tc_wait_ms = 2000.0;  // limit of every bounded tensor-core wait
    int inject_stall = 0;        // fault injection: tensor-core producer issues nothing
    Tables tab_stream, tab_direct;
    std::vector<double> tau, phi;            // latest values set
    std::vector<double> tau_pend, phi_pend;  // waiting for an integration boundary
    bool pending = false;
    // streaming state
    // s_comp runs the kernels, s_copy the input copies and s_out the result
    // copies to the host: a result copy queued behind an input copy on a
    // copy engine then holds up neither the kernels nor the next input.
    // s_get carries copies into pinned buffers the caller pops into.
    cudaStream_t s_comp = nullptr, s_copy = nullptr, s_out = nullptr, s_get = nullptr;
    cudaEvent_t ev_h2d = nullptr, ev_comp = nullptr, ev_fin = nullptr;
    bool started = false, flushed = false, stream_alloc = false;
    // Host pushes land in two staging buffers used in turn: the next chunk is
    // copied (behind the history it needs) into the buffer the F-engine is
    // not reading, so host->device copies overlap the correlation.
    int8_t* d_stage_buf[2] = {nullptr, nullptr};
    int8_t* d_stage = nullptr;           // the current buffer
    int cur_buf = 0;
    cudaEvent_t ev_buf[2] = {nullptr, nullptr};   // after the last kernels that read buffer b
    bool buf_read[2] = {false, false};
    long long stage_cap = 0, stage_base = 0, stage_len = 0;
    int8_t* h_pin = nullptr;
    long long pin_cap = 0;
    long long n_pushed = 0;
    Pipe ps;                 // stream pipe
    Pipe pd;                 // whole-stream device pipe
    float* d_part_x = nullptr;   // scratch of corr_xengine_dev
    long long part_x_slots = 0;
    float2* d_z_f = nullptr;     // scratch of corr_fengine_dev
    long long z_f_spectra = 0;
    std::vector<Slot> slots;
    std::deque<int> q_vis, q_flag;
    // the last pop went to pinned memory: new results get no host image
    bool pop_pinned = false;
    std::string err;
    long long launches = 0;
    StageTimer timer;
    int* d_status = nullptr;     // device error word of bounded waits
};

namespace {

int fail(corr_t h, int code, const std::string& msg) {
    if (h) h->err = msg;
    else g_create_error = msg;
    return code;
}

#define CK(call)                                                                      \
    do {                                                                              \
        cudaError_t e_ = (call);                                                      \
        if (e_ != cudaSuccess)                                                        \
            return fail(h, CORR_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

#define CKRET(expr)              \
    do {                         \
        int r_ = (expr);         \
        if (r_ != CORR_OK) return r_; \
    } while (0)

// Device allocation of a handle, with the fault-injection hook
// "inject_alloc_fail": the n-th allocation after the option is set fails.
cudaError_t dev_malloc(corr_t h, void** ptr, size_t bytes) {
    if (h && h->inject_alloc_fail > 0 && --h->inject_alloc_fail == 0) {
        *ptr = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMalloc(ptr, bytes);
}

template <class T>
cudaError_t dmalloc(corr_t h, T** ptr, size_t bytes) {
    return dev_malloc(h, reinterpret_cast<void**>(ptr), bytes);
}

#define CKA(call)                                                                           \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess)                                                              \
            return fail(h, CORR_ENOMEM, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

// Bracket one launch of `stage` on stream st with events (when enabled).
struct Timed {
    corr_t h;
    int stage;
    cudaStream_t st;
    cudaEvent_t e0 = nullptr;
    Timed(corr_t h_, int stage_, cudaStream_t st_) : h(h_), stage(stage_), st(st_) {
        if (h->timer.on && ((h->timer.mask >> stage) & 1)) {
            e0 = h->timer.take();
            cudaEventRecord(e0, st);
        }
    }
    ~Timed() {
        ++h->launches;
        if (e0) {
            cudaEvent_t e1 = h->timer.take();
            cudaEventRecord(e1, st);
            h->timer.open[stage].push_back({e0, e1});
        }
    }
};

bool is_pow2(long long v) { return v > 0 && (v & (v - 1)) == 0; }

size_t vis_elems(const corr_s* h) { return (size_t)h->n_chan * h->n_in * h->n_in; }

// Polyphase prototype (Sec. 4.2 PFB weighting): symmetric Hann window times
// a sinc with cutoff 1/M centred on the filter, evaluated in FP64.
// I0(x) by its power series sum_k ((x/2)^k / k!)^2, in FP64.
double bessel_i0(double x) {
    const double q = 0.25 * x * x;
    double term = 1.0, sum = 1.0;
    for (int k = 1; k < 500; ++k) {
        term *= q / ((double)k * k);
        sum += term;
        if (term <= 1e-17 * sum) break;
    }
    return sum;
}

// Polyphase prototype (Sec. 4.2 PFB weighting), evaluated in FP64: a
// symmetric taper (Hann, or Kaiser with parameter beta as in Fig. 4) times a
// sinc with cutoff 1/M centred on the filter; window 2 gives unit
// coefficients (with one tap, the plain per-frame DFT).
std::vector<float> make_filter(int M, int P, int window, double beta) {
    const int L = M * P;
    std::vector<float> h(L);
    const double pi = 3.14159265358979323846;
    const double i0b = bessel_i0(beta);
    for (int n = 0; n < L; ++n) {
        if (window == 2) {
            h[n] = 1.0f;
            continue;
        }
        double w = 1.0;
        if (L > 1) {
            if (window == 1) {
                const double r = 2.0 * n / (double)(L - 1) - 1.0;
                w = bessel_i0(beta * std::sqrt(std::max(0.0, 1.0 - r * r))) / i0b;
            } else {
                w = 0.5 - 0.5 * std::cos(2.0 * pi * n / (double)(L - 1));
            }
        }
        const double x = (n - 0.5 * (L - 1)) / (double)M;
        const double sn = (x == 0.0) ? 1.0 : std::sin(pi * x) / (pi * x);
        h[n] = (float)(w * sn);
    }
    // The taper and the sinc are both symmetric about (L-1)/2; the upper half
    // repeats the lower one exactly (the fused F-engine keeps only half).
    for (int n = 0; n < L / 2; ++n) h[L - 1 - n] = h[n];
    return h;
}

// Lower half of every polyphase row, hs[p][m] = h[p M + m] for m < M/2.
std::vector<float> half_rows(const std::vector<float>& h, int M, int P) {
    std::vector<float> hs((size_t)P * (M / 2));
    for (int p = 0; p < P; ++p)
        for (int m = 0; m < M / 2; ++m) hs[(size_t)p * (M / 2) + m] = h[(size_t)p * M + m];
    return hs;
}

int upload_tables(corr_t h, Tables& t, const std::vector<double>& tau, const std::vector<double>& phi,
                  cudaStream_t st) {
    const double pi = 3.14159265358979323846;
    std::vector<float2> ph((size_t)h->n_in_pad * h->n_chan, make_float2(0.f, 0.f));
    std::vector<float2> rt((size_t)h->n_in_pad * h->n_chan, make_float2(0.f, 0.f));
    std::vector<int> co(h->n_in_pad, 0);
    int dmax = -(1 << 30);
    for (int a = 0; a < h->n_in; ++a) {
        const double d = std::floor(tau[a] + 0.5);
        const double r = tau[a] - d;
        co[a] = (int)d;
        if (co[a] > dmax) dmax = co[a];
        // Pair packing: even inputs carry 1/2, odd inputs 1/(2j) = -j/2.
        // Complex input: channel k at k/M cycles per sample below M/2 and
        // (k - M)/M above, no pair factor.
        const bool odd = (a & 1) != 0;
        for (int k = 0; k < h->n_chan; ++k) {
            const double fk = (h->iq && k >= h->M / 2) ? (double)(k - h->M) : (double)k;
            const double ang = 2.0 * pi * fk * r / (double)h->M - phi[a];
            rt[(size_t)a * h->n_chan + k] = make_float2((float)std::cos(ang), (float)std::sin(ang));
            if (h->iq) {
                ph[(size_t)a * h->n_chan + k] = rt[(size_t)a * h->n_chan + k];
                continue;
            }
            double re = 0.5 * std::cos(ang), im = 0.5 * std::sin(ang);
            if (odd) {
                const double t2 = re;
                re = im;
                im = -t2;
            }
            ph[(size_t)a * h->n_chan + k] = make_float2((float)re, (float)im);
        }
    }
    t.d_max = dmax;
    if (&t == &h->tab_stream) {
        h->stream_tau = tau;
        h->stream_phi = phi;
    }
    CK(cudaMemcpyAsync(t.phasor, ph.data(), ph.size() * sizeof(float2), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(t.rot, rt.data(), rt.size() * sizeof(float2), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(t.coarse, co.data(), co.size() * sizeof(int), cudaMemcpyHostToDevice, st));
    CK(cudaStreamSynchronize(st));
    return CORR_OK;
}

int alloc_tables(corr_t h, Tables& t) {
    CK(cudaMalloc(&t.phasor, sizeof(float2) * (size_t)h->n_in_pad * h->n_chan));
    CK(cudaMalloc(&t.rot, sizeof(float2) * (size_t)h->n_in_pad * h->n_chan));
    CK(cudaMalloc(&t.coarse, sizeof(int) * (size_t)h->n_in_pad));
    return CORR_OK;
}

int choose_spt(long long n_spec, int n_pairs) {
    const long long target = 152LL * 4;
    long long spt = (n_spec * n_pairs) / target;
    if (spt < 1) spt = 1;
    if (spt > 8) spt = 8;
    return (int)spt;
}

// Spectra per FIR thread: long runs amortise the P-1 frames of warm-up,
// but keep at least ~2 waves of CTAs on 152 SMs.
int choose_fir_spt(long long n_spec, int n_pairs, int M, int taps) {
    const long long ctas_per_run = (long long)((M / 2 + 255) / 256) * n_pairs;
    long long spt = 16;
    while (spt > 1 && ((n_spec + spt - 1) / spt) * ctas_per_run < 3 * 152) spt /= 2;
    if (spt < 1) spt = 1;
    (void)taps;
    return (int)spt;
}

void free_pipe(Pipe& p);

int alloc_pipe_impl(corr_t h, Pipe& p);

// All of a pipe's buffers or none (a failed allocation leaves no half-built pipe).
int alloc_pipe(corr_t h, Pipe& p) {
    if (p.V) return CORR_OK;
    const int rc = alloc_pipe_impl(h, p);
    if (rc != CORR_OK) free_pipe(p);
    return rc;
}

int alloc_pipe_impl(corr_t h, Pipe& p) {
    const unsigned long long ring_bytes = (unsigned long long)h->ring_mb << 20;
    // Two power-of-two rings (FIR output and channelised spectra) of half of
    // ring_mb each: at the 64 MiB default both stay in L2 between the
    // kernels; larger rings mean fewer, larger launches.
    const size_t per_spec = (size_t)h->n_chan * h->n_in_pad * sizeof(float2);
    long long cap = 1;
    while (cap * 2 * per_spec <= ring_bytes && cap < 4096) cap *= 2;
    while (cap < h->G) cap *= 2;
    // the reduced-precision scale pre-pass reads the first 64 spectra from the ring
    while (h->precision != CORR_FP32 && cap < 64) cap *= 2;
    p.v_cap = (int)cap;
    CKA(dmalloc(h, &p.V, per_spec * (size_t)p.v_cap));
    CKA(dmalloc(h, &p.Z, per_spec * (size_t)p.v_cap));
    if (h->precision != CORR_FP32) {
        // one 32-bit word of four codes per (spectrum, pair, channel) of an
        // integration (n_chan, a power of two >= 8, is a multiple of the Gram
        // kernel's four channels a CTA); the Gram kernel writes the
        // visibilities itself, so no Gram matrices are kept
        const size_t cbytes = sizeof(uint32_t) * (size_t)h->n_int * (h->n_in_pad / 2) * h->n_chan;
        CKA(dmalloc(h, &p.C, cbytes));
        CK(cudaMemset(p.C, 0, cbytes));
        // scales, then their inverses (the requantiser's multipliers)
        CKA(dmalloc(h, &p.scale, 2 * sizeof(float) * (size_t)h->n_in_pad * h->n_chan));
        p.have_scale = false;
    }
    CKA(dmalloc(h, &p.part, sizeof(float) * (size_t)h->gpi * h->nt * 32 * h->n_chan));
    return CORR_OK;
}

// Every real-input pipeline keeps its spectra ring pair-major: one F-engine
// CTA transforms one input pair and writes its channels contiguously, and the
// X-engines and the requantiser read consecutive channels across a warp.
// Complex input keeps the channel-major ring.
bool pair_major_ring(corr_t h) { return !h->iq; }

// Filter, half-row and twiddle tables for the handle's current M, window
// and taps (replaces the device copies; sizes follow M).
int build_filter_tables(corr_t h) {
    const std::vector<float> hf = make_filter(h->M, h->taps, h->window, h->kaiser_beta);
    const std::vector<float> hsf = half_rows(hf, h->M, h->taps);
    const std::vector<float2> tw = corr::fft_twiddle_table(h->M);
    cudaFree(h->d_h);
    cudaFree(h->d_hs);
    cudaFree(h->d_tw);
    h->d_h = nullptr;
    h->d_hs = nullptr;
    h->d_tw = nullptr;
    if (cudaMalloc(&h->d_h, hf.size() * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&h->d_hs, hsf.size() * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&h->d_tw, tw.size() * sizeof(float2)) != cudaSuccess)
        return fail(h, CORR_ENOMEM, "cudaMalloc of filter tables failed");
    CK(cudaMemcpy(h->d_h, hf.data(), hf.size() * sizeof(float), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(h->d_hs, hsf.data(), hsf.size() * sizeof(float), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(h->d_tw, tw.data(), tw.size() * sizeof(float2), cudaMemcpyHostToDevice));
    return CORR_OK;
}

// Requantised codes made by the F-engine itself (reduced precision, once the
// integration's scales are fixed): the inverse scales and the code type.
struct CodeOut {
    const float* inv;
    bool fp8;
};

// The fused F-engine writes the pipeline's codes for this handle.
bool fused_codes(corr_t h, const StreamView& sv) {
    return h->precision != CORR_FP32 && h->fused_f && !h->iq &&
           fused_f_supported(h->M, h->taps, sv.es, h->precision == CORR_FP8 ? 7 : 6);
}

// The F-engine writes them: the fused kernel, or the two-kernel FFT at
// M = 16384 (beyond the fused kernel's shared memory).
bool f_codes(corr_t h, const StreamView& sv) {
    return fused_codes(h, sv) || (h->precision != CORR_FP32 && !h->iq && h->M == 16384);
}

// F-engine over spectra [s_begin, s_end): FIR into the Z ring, FFT into the
// V ring.  `phasor` set -> rotated V (stage call); `codes` set -> V holds
// requantised code words instead of spectra (where f_codes holds); else
// U = 2Y (pipeline).
int launch_f(corr_t h, const StreamView& sv, const Tables& t, float2* Z, long long z_origin, long long z_mask,
             float2* V, long long v_origin, long long v_mask, const float2* phasor, long long s_begin,
             long long s_end, cudaStream_t st, float* tiles = nullptr, int n_row = 0, int rows = 0,
             const CodeOut* codes = nullptr) {
    FirArgs a{};
    a.src = sv;
    a.h = h->d_h;
    a.coarse = t.coarse;
    a.Z = Z;
    a.z_origin = z_origin;
    a.z_mask = z_mask;
    a.s_begin = s_begin;
    a.s_end = s_end;
    a.n_in = h->n_in;
    a.n_pairs = h->iq ? h->n_in_pad : h->n_in_pad / 2;
    a.iq = h->iq;
    a.M = h->M;
    a.lgM = 0;
    while ((1 << a.lgM) < h->M) ++a.lgM;
    a.taps = h->taps;
    a.spt = h->fir_spt > 0 ? h->fir_spt : choose_fir_spt(s_end - s_begin, a.n_pairs, h->M, h->taps);
    FftArgs f{};
    f.Z = Z;
    f.z_origin = z_origin;
    f.z_mask = z_mask;
    f.tw = h->d_tw;
    f.phasor = phasor;
    f.V = V;
    f.v_origin = v_origin;
    f.v_mask = v_mask;
    f.s_begin = s_begin;
    f.s_end = s_end;
    f.n_in_pad = h->n_in_pad;
    f.M = h->M;
    f.spt = choose_spt(s_end - s_begin, h->n_in_pad / 2);
    f.tiles = tiles;
    f.n_row = n_row;
    f.rows = rows;
    f.n_in = h->n_in;
    f.pair_major = phasor == nullptr && tiles == nullptr && pair_major_ring(h);
    f.iq = h->iq;
    const int mode = codes ? (codes->fp8 ? 7 : 6) : tiles ? 2 : phasor ? 1 : f.pair_major ? 3 : 0;
    if (codes && !f_codes(h, sv)) return fail(h, CORR_EINVAL, "codes from the F-engine: not for this shape");
    if (codes) {
        f.inv = codes->inv;
        f.fp8 = codes->fp8;
    }
    if (h->fused_f && !h->iq && fused_f_supported(h->M, h->taps, sv.es, mode)) {
        FusedArgs u{};
        u.f = f;
        u.src = sv;
        u.hs = h->d_hs;
        u.coarse = t.coarse;
        u.taps = h->taps;
        u.run = h->fir_spt;
        if (codes) {
            u.inv = codes->inv;
            u.fp8 = codes->fp8;
        }
        int rc;
        {
            Timed t_(h, 1, st);
            rc = launch_fused_f(u, st);
        }
        if (rc != CORR_OK) return fail(h, rc, "fused F-engine launch failed");
        CK(cudaGetLastError());
        return CORR_OK;
    }
    {
        Timed t_(h, 0, st);
        launch_fir(a, st);
    }
    CK(cudaGetLastError());
    int rc;
    {
        Timed t_(h, 1, st);
        rc = launch_fft(f, st);
    }
    if (rc != CORR_OK) return fail(h, rc, "FFT launch: spectra buffer not 16-byte aligned or no tensor-map encoder");
    CK(cudaGetLastError());
    return CORR_OK;
}

long long ready_spectra(corr_t h, bool final) {
    if (final) return h->n_pushed / h->M;
    const long long r = h->n_pushed - h->tab_stream.d_max;
    if (r < h->M) return 0;
    return r / h->M;
}

using Sink = int (*)(corr_t, void*, const Tables&, long long /*integration*/, int /*count*/, int /*slots*/,
                     cudaStream_t);

// Drive F -> X -> finalise over every spectrum below ready_end.  When
// `final` is set, the stream has ended: a last partial group / integration
// is closed at ready_end.
int drive(corr_t h, Pipe& p, const StreamView& sv, Tables& t, long long ready_end, bool final, bool is_stream,
          Sink sink, void* ctx, cudaStream_t st) {
    const long long n_int = h->n_int;
    for (;;) {
        const long long i = p.s_next / n_int;
        const long long istart = i * n_int, iend = istart + n_int;
        if (is_stream && h->pending && p.s_next == istart && p.s_xdone == istart) {
            CKRET(upload_tables(h, t, h->tau_pend, h->phi_pend, st));
            h->pending = false;
            ready_end = ready_spectra(h, final);
        }
        bool progress = false;
        long long s_end = ready_end;
        if (s_end > iend) s_end = iend;
        // the ring bounds a launch, except where the F-engine writes code
        // words straight into the integration's word buffer (then one launch
        // may cover the rest of the integration)
        const bool to_words = p.have_scale && p.s_xdone == p.s_next && f_codes(h, sv);
        // (the two-kernel path keeps the bound: its FIR fills the z ring)
        if (!(to_words && fused_codes(h, sv)) && s_end > p.s_xdone + p.v_cap) s_end = p.s_xdone + p.v_cap;
        if (s_end > p.s_next) {
            if (to_words) {
                // scales fixed and nothing left in the ring: the F-engine
                // requantises in its epilogue (the requantiser's arithmetic)
                // and writes 4-byte code words instead of 16-byte spectra,
                // straight into the integration's C at t = s - istart, where
                // the Gram kernel reads them
                const CodeOut q{p.scale + (size_t)h->n_in_pad * h->n_chan, h->precision == CORR_FP8};
                CKRET(launch_f(h, sv, t, p.Z, 0, p.v_cap - 1, reinterpret_cast<float2*>(p.C), istart, -1LL,
                               nullptr, p.s_next, s_end, st, nullptr, 0, 0, &q));
                p.s_xdone = s_end;
            } else {
                CKRET(launch_f(h, sv, t, p.Z, 0, p.v_cap - 1, p.V, 0, p.v_cap - 1, nullptr, p.s_next, s_end, st));
            }
            p.s_next = s_end;
            progress = true;
        }
        const bool closing = final && p.s_next == ready_end && p.s_next < iend;
        const long long s_limit = closing ? p.s_next : iend;
        int j_end = 0;
        if (h->precision != CORR_FP32) {
            // Requantise the spectra the ring still holds (a stream's first
            // ring fill, before the scales are known, or every fill when the
            // F-engine is not the fused kernel) into the integration's code
            // words.  The first integration of a stream first fixes its
            // scales from the mean power of its first min(n_int, 64) spectra.
            if (!p.have_scale) {
                const long long want = n_int < 64 ? n_int : 64;
                const long long have = p.s_next - istart;
                if (have >= want || (closing && have > 0)) {
                    const int n = (int)(have < want ? have : want);
                    launch_scale_from_ring(p.V, 0, p.v_cap - 1, istart, n, h->n_in, h->n_in_pad, h->n_chan,
                                           h->precision == CORR_FP8 ? kFp8Gain : kInt8Gain, p.scale,
                                           pair_major_ring(h), st);
                    ++h->launches;
                    CK(cudaGetLastError());
                    p.have_scale = true;
                }
            }
            if (p.have_scale && p.s_next > p.s_xdone) {
                RequantArgs r{};
                r.V = p.V;
                r.v_origin = 0;
                r.v_mask = p.v_cap - 1;
                r.scale = p.scale;
                r.s_begin = p.s_xdone;
                r.s_end = p.s_next;
                r.int_start = istart;
                r.n_in = h->n_in;
                r.n_in_pad = h->n_in_pad;
                r.n_chan = h->n_chan;
                r.fp8 = h->precision == CORR_FP8;
                r.C = p.C;
                {
                    Timed t_(h, 5, st);
                    launch_requant(r, st);
                }
                CK(cudaGetLastError());
                p.s_xdone = p.s_next;
                progress = true;
            }
        } else {
            // Partial slots: group j covers [istart + jG, min(istart + (j+1)G, iend)).
            const int j_begin = (int)((p.s_xdone - istart) / h->G);
            if (p.s_next >= iend) j_end = h->gpi;
            else if (closing) j_end = (int)((p.s_next - istart + h->G - 1) / h->G);
            else j_end = (int)((p.s_next - istart) / h->G);
            if (j_end > j_begin) {
                XArgs x{};
                x.V = p.V;
                x.v_origin = 0;
                x.v_mask = p.v_cap - 1;
                x.n_chan = h->n_chan;
                x.n_in_pad = h->n_in_pad;
                x.nt = h->nt;
                x.int_start = istart;
                x.int_end = iend;
                x.s_limit = s_limit;
                x.G = h->G;
                x.j0 = j_begin;
                x.n_groups = j_end - j_begin;
                // finalisation deferred to a group's tail: each integration
                // keeps its own partial sums
                x.part = h->defer_tail ? p.part_all + (size_t)i * h->gpi * h->nt * 32 * h->n_chan : p.part;
                x.pair_major = pair_major_ring(h);
                x.depth = h->x_depth;
                {
                    Timed t_(h, 2, st);
                    launch_xengine(x, st);
                }
                CK(cudaGetLastError());
                long long nx = istart + (long long)j_end * h->G;
                if (nx > s_limit) nx = s_limit;
                p.s_xdone = nx;
                progress = true;
            }
        }
        if (p.s_next == iend && p.s_xdone == iend) {
            CKRET(sink(h, ctx, t, i, (int)n_int, h->gpi, st));
            progress = true;
            continue;
        }
        if (closing && p.s_xdone == p.s_next && p.s_next > istart) {
            CKRET(sink(h, ctx, t, i, (int)(p.s_next - istart), j_end, st));
            // The partial integration is closed; nothing further can follow.
            p.s_xdone = p.s_next = iend;
            return CORR_OK;
        }
        if (!progress) return CORR_OK;
    }
}

// The pipeline's spectra are U = 2Y without the fine-delay/phase rotation,
// so R = Q_a conj(Q_b) sum U_a U_b^* / (4 count).
int finalize_into(corr_t h, Pipe& p, const Tables& t, float2* R, uint8_t* F, int count, int slots,
                  cudaStream_t st) {
    if (h->precision != CORR_FP32) {
        // Tensor-core Gram of the integration's code words, rescaled and
        // rotated into visibilities in the same kernel's epilogue; the
        // autocorrelations then fix the next integration's scales.
        GramArgs g{};
        g.Q = p.C;
        g.words = 1;
        g.n_pairs = h->n_in_pad / 2;
        g.n_in = h->n_in;
        g.n_chan = h->n_chan;
        g.K = count;
        g.fp8 = h->precision == CORR_FP8;
        g.status = h->d_status;
        g.wait_ns = (unsigned long long)(h->tc_wait_ms * 1e6);
        g.inject_stall = h->inject_stall;
        g.R = R;
        g.scale = p.scale;
        g.rot = t.rot;
        int rc;
        {
            Timed t_(h, 6, st);
            rc = launch_gram(g, st);
        }
        if (rc != CORR_OK) return fail(h, rc, "tensor-core Gram launch failed");
        CK(cudaGetLastError());
        launch_scale_from_vis(R, h->n_in, h->n_in_pad, h->n_chan, g.fp8 ? kFp8Gain : kInt8Gain, p.scale, st);
        ++h->launches;
        CK(cudaGetLastError());
        if (F) {
            const int w = h->flag_window < h->n_chan ? h->flag_window : h->n_chan;
            {
                Timed t_(h, 4, st);
                launch_mad_flags(R, F, 1, h->n_chan, h->n_in, w, (float)h->flag_sigma, st);
            }
            CK(cudaGetLastError());
        }
        return CORR_OK;
    }
    FinArgs f{};
    f.part = p.part;
    f.rot = t.rot;
    f.n_slots = slots;
    f.nt = h->nt;
    f.n_chan = h->n_chan;
    f.n_in = h->n_in;
    f.scale = 0.25f / (float)count;
    f.R = R;
    const int fw = h->flag_window < h->n_chan ? h->flag_window : h->n_chan;
    if (F && fin_flag_small_supported(h->n_in, fw) && h->n_chan % fw == 0) {
        {
            Timed t_(h, 3, st);
            launch_fin_flag_small(f, F, fw, (float)h->flag_sigma, st);
        }
        CK(cudaGetLastError());
        return CORR_OK;
    }
    {
        Timed t_(h, 3, st);
        launch_finalize(f, st);
    }
    CK(cudaGetLastError());
    if (F) {
        const int w = h->flag_window < h->n_chan ? h->flag_window : h->n_chan;
        {
            Timed t_(h, 4, st);
            launch_mad_flags(R, F, 1, h->n_chan, h->n_in, w, (float)h->flag_sigma, st);
        }
        CK(cudaGetLastError());
    }
    return CORR_OK;
}

int add_slot(corr_t h) {
    Slot s;
    const size_t ne = vis_elems(h);
    bool ok = dmalloc(h, &s.d_R, ne * sizeof(float2)) == cudaSuccess && dmalloc(h, &s.d_F, ne) == cudaSuccess &&
              cudaHostAlloc(&s.h_R, ne * sizeof(float2), cudaHostAllocDefault) == cudaSuccess &&
              cudaHostAlloc(&s.h_F, ne, cudaHostAllocDefault) == cudaSuccess &&
              cudaEventCreateWithFlags(&s.ev, cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
        cudaFree(s.d_R);
        cudaFree(s.d_F);
        if (s.h_R) cudaFreeHost(s.h_R);
        if (s.h_F) cudaFreeHost(s.h_F);
        if (s.ev) cudaEventDestroy(s.ev);
        cudaGetLastError();
        return fail(h, CORR_ENOMEM, "result slot allocation failed");
    }
    h->slots.push_back(s);
    return CORR_OK;
}

int new_slot(corr_t h, int* idx) {
    for (size_t i = 0; i < h->slots.size(); ++i) {
        if (!h->slots[i].in_vis && !h->slots[i].in_flag) {
            *idx = (int)i;
            return CORR_OK;
        }
    }
    CKRET(add_slot(h));
    *idx = (int)h->slots.size() - 1;
    return CORR_OK;
}

// Copies a slot's results into its pinned host image behind its kernels (on
// s_out; s.ev then marks the image complete).
int slot_image(corr_t h, Slot& s) {
    const size_t ne = vis_elems(h);
    CK(cudaStreamWaitEvent(h->s_out, s.ev, 0));
    CK(cudaMemcpyAsync(s.h_R, s.d_R, ne * sizeof(float2), cudaMemcpyDeviceToHost, h->s_out));
    CK(cudaMemcpyAsync(s.h_F, s.d_F, ne, cudaMemcpyDeviceToHost, h->s_out));
    CK(cudaEventRecord(s.ev, h->s_out));
    s.has_image = true;
    return CORR_OK;
}

int sink_stream(corr_t h, void*, const Tables& t, long long, int count, int slots, cudaStream_t st) {
    int idx;
    CKRET(new_slot(h, &idx));
    Slot& s = h->slots[idx];
    CKRET(finalize_into(h, h->ps, t, s.d_R, s.d_F, count, slots, st));
    // The slot is rewritten only after the host has taken its results
    // (pop_results waits on s.ev), so the copies may trail the kernels.  A
    // caller that pops into pinned memory takes the results by DMA straight
    // from the slot: while the last pop was such a one, no host image is
    // made (a later pop into other memory, or a checkpoint, makes it).
    CK(cudaEventRecord(s.ev, st));
    s.has_image = false;
    if (!h->pop_pinned) CKRET(slot_image(h, s));
    s.in_vis = s.in_flag = true;
    h->q_vis.push_back(idx);
    h->q_flag.push_back(idx);
    return CORR_OK;
}

struct DirectCtx {
    float2* vis;
    uint8_t* flags;
    int max_int;
    int n_out;
};

int sink_direct(corr_t h, void* vctx, const Tables& t, long long i, int count, int slots, cudaStream_t st) {
    DirectCtx* c = static_cast<DirectCtx*>(vctx);
    if (i >= c->max_int) return fail(h, CORR_EINVAL, "max_int too small for the stream");
    const size_t ne = vis_elems(h);
    if (h->defer_tail) {
        // inside a group: the group's tail kernel finalises FP32
        // integrations and flags every integration; the reduced-precision
        // finalisation stays here (its autocorrelations set the next scales)
        if (h->precision != CORR_FP32)
            CKRET(finalize_into(h, h->pd, t, c->vis + (size_t)i * ne, nullptr, count, slots, st));
        c->n_out = (int)i + 1;
        return CORR_OK;
    }
    CKRET(finalize_into(h, h->pd, t, c->vis + (size_t)i * ne, c->flags ? c->flags + (size_t)i * ne : nullptr,
                        count, slots, st));
    c->n_out = (int)i + 1;
    return CORR_OK;
}

int ensure_stream_alloc(corr_t h) {
    if (h->stream_alloc) return CORR_OK;
    const long long keep = (long long)(h->taps + 1) * h->M + 2 * h->max_delay + 64;
    h->stage_cap = ((h->chunk + keep + 15) / 16) * 16;
    // all or nothing: a failure releases the staging buffers again
    auto undo = [&](int rc) {
        for (int b = 0; b < 2; ++b) {
            cudaFree(h->d_stage_buf[b]);
            h->d_stage_buf[b] = nullptr;
            if (h->ev_buf[b]) cudaEventDestroy(h->ev_buf[b]);
            h->ev_buf[b] = nullptr;
        }
        h->d_stage = nullptr;
        cudaGetLastError();
        return rc;
    };
    for (int b = 0; b < 2; ++b) {
        if (dmalloc(h, &h->d_stage_buf[b], (size_t)h->stage_cap * h->n_in * h->es) != cudaSuccess)
            return undo(fail(h, CORR_ENOMEM, "staging buffer allocation failed"));
        if (cudaMemset(h->d_stage_buf[b], 0, (size_t)h->stage_cap * h->n_in * h->es) != cudaSuccess ||
            cudaEventCreateWithFlags(&h->ev_buf[b], cudaEventDisableTiming) != cudaSuccess)
            return undo(fail(h, CORR_ECUDA, "staging buffer set-up failed"));
        h->buf_read[b] = false;
    }
    h->cur_buf = 0;
    h->d_stage = h->d_stage_buf[0];
    int rc = alloc_pipe(h, h->ps);
    if (rc != CORR_OK) return undo(rc);
    while ((int)h->slots.size() < h->result_slots) {
        rc = add_slot(h);
        if (rc != CORR_OK) {
            free_pipe(h->ps);
            return undo(rc);
        }
    }
    h->stream_alloc = true;
    return CORR_OK;
}

// Make room for `need` more samples: when the current staging buffer is
// full, switch to the other one, with the samples still needed by
// unprocessed spectra copied to its front.  The other buffer is reused only
// after the kernels that last read it have finished (ev_buf); the history
// copy itself runs on the copy stream behind the copies that wrote it.
int make_room(corr_t h, long long need) {
    if (h->stage_len + need <= h->stage_cap) return CORR_OK;
    long long keep_lo = (h->ps.s_next - h->taps + 1) * (long long)h->M - h->max_delay;
    if (keep_lo < h->stage_base) keep_lo = h->stage_base;
    const long long off = keep_lo - h->stage_base;
    const long long keep = h->stage_len - off;
    if (keep + need > h->stage_cap) return fail(h, CORR_EINVAL, "internal: staging buffer too small");
    const int nb = 1 - h->cur_buf;
    if (h->buf_read[nb]) CK(cudaStreamWaitEvent(h->s_copy, h->ev_buf[nb], 0));
    if (keep > 0)
        CK(cudaMemcpy2DAsync(h->d_stage_buf[nb], h->stage_cap * h->es, h->d_stage + off * h->es, h->stage_cap * h->es,
                             keep * h->es, h->n_in, cudaMemcpyDeviceToDevice, h->s_copy));
    h->cur_buf = nb;
    h->d_stage = h->d_stage_buf[nb];
    h->stage_base = keep_lo;
    h->stage_len = keep;
    return CORR_OK;
}

int process_stream(corr_t h, bool final) {
    StreamView sv;
    sv.x = h->d_stage;
    sv.stride = h->stage_cap;
    sv.base = h->stage_base;
    sv.vhi = h->n_pushed;
    sv.es = h->es;
    CKRET(drive(h, h->ps, sv, h->tab_stream, ready_spectra(h, final), final, true, sink_stream, nullptr,
                h->s_comp));
    CK(cudaEventRecord(h->ev_buf[h->cur_buf], h->s_comp));
    h->buf_read[h->cur_buf] = true;
    return CORR_OK;
}

int push_common(corr_t h, const int8_t* src, size_t n, size_t stride, bool on_device, cudaStream_t ust) {
    const size_t es = (size_t)h->es;   // src is a byte address; n, stride count samples
    if (h->flushed) return fail(h, CORR_ESTATE, "stream already flushed; call corr_reset");
    if (n == 0) return CORR_OK;
    if (h->max_pending > 0 && (int)h->q_vis.size() >= h->max_pending)
        return fail(h, CORR_EAGAIN, "result queue full (max_pending): pop results before pushing");
    if (!src) return fail(h, CORR_EINVAL, "samples is NULL");
    if (stride < n) return fail(h, CORR_EINVAL, "input_stride < n_per_input");
    CKRET(ensure_stream_alloc(h));
    bool pinned = false;
    if (!on_device) {
        cudaPointerAttributes attr;
        if (cudaPointerGetAttributes(&attr, src) == cudaSuccess && attr.type == cudaMemoryTypeHost)
            pinned = true;
        cudaGetLastError();
    } else {
        CK(cudaEventRecord(h->ev_comp, ust));
        CK(cudaStreamWaitEvent(h->s_copy, h->ev_comp, 0));
    }
    h->started = true;
    size_t done = 0;
    while (done < n) {
        const long long piece = (long long)std::min<size_t>(n - done, (size_t)h->chunk);
        CKRET(make_room(h, piece));
        const int8_t* s = src + done * es;
        size_t spitch = stride * es;
        cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
        if (!on_device && !pinned) {
            if (h->pin_cap < piece * h->n_in * (long long)es) {
                if (h->h_pin) cudaFreeHost(h->h_pin);
                h->h_pin = nullptr;
                CK(cudaHostAlloc(&h->h_pin, (size_t)piece * h->n_in * es, cudaHostAllocDefault));
                h->pin_cap = piece * h->n_in * (long long)es;
            }
            for (int a = 0; a < h->n_in; ++a)
                std::memcpy(h->h_pin + (size_t)a * piece * es, src + ((size_t)a * stride + done) * es,
                            (size_t)piece * es);
            s = h->h_pin;
            spitch = (size_t)piece * es;
        }
        CK(cudaMemcpy2DAsync(h->d_stage + h->stage_len * (long long)es, h->stage_cap * es, s, spitch,
                             (size_t)piece * es, h->n_in, kind, h->s_copy));
        CK(cudaEventRecord(h->ev_h2d, h->s_copy));
        CK(cudaStreamWaitEvent(h->s_comp, h->ev_h2d, 0));
        h->stage_len += piece;
        h->n_pushed += piece;
        CKRET(process_stream(h, false));
        if (!on_device) CK(cudaEventSynchronize(h->ev_h2d));
        done += (size_t)piece;
    }
    if (on_device) {
        // The caller's buffer may be reused once its stream passes this point.
        CK(cudaEventRecord(h->ev_h2d, h->s_copy));
        CK(cudaStreamWaitEvent(ust, h->ev_h2d, 0));
    }
    return CORR_OK;
}

int pop_results(corr_t h, std::deque<int>& q, bool vis, void* out, int max_int, int* n_got) {
    if (n_got) *n_got = 0;
    if (max_int < 0) return fail(h, CORR_EINVAL, "max_int < 0");
    if (max_int > 0 && !out) return fail(h, CORR_EINVAL, "out is NULL");
    // A pinned destination takes the results straight from the device slots
    // by DMA (on s_get, behind each slot's own event only); any other host
    // memory gets a copy of the slot's pinned image.
    bool pinned = false;
    if (max_int > 0 && !q.empty()) {
        cudaPointerAttributes attr;
        pinned = cudaPointerGetAttributes(&attr, out) == cudaSuccess && attr.type == cudaMemoryTypeHost;
        cudaGetLastError();
    }
    const size_t ne = vis_elems(h);
    const size_t bytes = vis ? ne * sizeof(float2) : ne;
    int got = 0;
    std::vector<int> taken;
    int rc = CORR_OK;
    while (got < max_int && !q.empty()) {
        const int idx = q.front();
        Slot& s = h->slots[idx];
        char* dst = static_cast<char*>(out) + (size_t)got * bytes;
        cudaError_t e;
        if (pinned) {
            e = cudaStreamWaitEvent(h->s_get, s.ev, 0);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(dst, vis ? static_cast<const void*>(s.d_R) : static_cast<const void*>(s.d_F),
                                    bytes, cudaMemcpyDeviceToHost, h->s_get);
        } else {
            if (!s.has_image && (rc = slot_image(h, s)) != CORR_OK) break;
            e = cudaEventSynchronize(s.ev);
            if (e == cudaSuccess)
                std::memcpy(dst, vis ? static_cast<const void*>(s.h_R) : static_cast<const void*>(s.h_F), bytes);
        }
        if (e != cudaSuccess) {
            rc = fail(h, CORR_ECUDA, std::string("result copy: ") + cudaGetErrorString(e));
            break;
        }
        taken.push_back(idx);
        q.pop_front();
        ++got;
    }
    if (!taken.empty()) h->pop_pinned = pinned;
    if (pinned && !taken.empty()) {
        const cudaError_t e = cudaStreamSynchronize(h->s_get);
        if (e != cudaSuccess && rc == CORR_OK) rc = fail(h, CORR_ECUDA, std::string("result copy: ") + cudaGetErrorString(e));
    }
    for (int idx : taken) (vis ? h->slots[idx].in_vis : h->slots[idx].in_flag) = false;
    if (rc != CORR_OK) return rc;
    if (n_got) *n_got = got;
    return got == 0 && max_int > 0 ? CORR_EAGAIN : CORR_OK;
}

void free_pipe(Pipe& p) {
    if (p.V) cudaFree(p.V);
    if (p.Z) cudaFree(p.Z);
    if (p.C) cudaFree(p.C);
    if (p.scale) cudaFree(p.scale);
    if (p.part) cudaFree(p.part);
    if (p.part_all) cudaFree(p.part_all);
    p = Pipe{};
}

}  // namespace

void corr::set_global_error(const std::string& msg) { g_create_error = msg; }

extern "C" {

int corr_create(corr_t* out, int n_ant, int n_pol, int n_chan, int taps, int n_int) {
    if (!out) return fail(nullptr, CORR_EINVAL, "out is NULL");
    *out = nullptr;
    if (n_ant < 1 || n_pol < 1 || n_ant * n_pol > 256)
        return fail(nullptr, CORR_EINVAL, "need n_ant, n_pol >= 1 and n_ant*n_pol <= 256");
    if (!is_pow2(n_chan) || n_chan < 8 || n_chan > 8192)
        return fail(nullptr, CORR_EINVAL, "n_chan must be a power of two in [8, 8192]");
    if (taps < 1 || taps > 16) return fail(nullptr, CORR_EINVAL, "taps must be in [1, 16]");
    if (n_int < 1) return fail(nullptr, CORR_EINVAL, "n_int must be >= 1");
    corr_t h = new corr_s();
    h->n_ant = n_ant;
    h->n_pol = n_pol;
    h->n_in = n_ant * n_pol;
    h->n_in_pad = (h->n_in + 3) & ~3;
    h->n_chan = n_chan;
    h->M = 2 * n_chan;
    h->taps = taps;
    h->n_int = n_int;
    const int nb = h->n_in_pad / 4;
    h->nt = nb * (nb + 1) / 2;
    int G = n_int < 64 ? n_int : 64;
    if (n_int / G > 16) G = (int)(((n_int + 15) / 16 + 63) / 64 * 64);
    h->G = G;
    h->gpi = (n_int + G - 1) / G;
    h->tau.assign(h->n_in, 0.0);
    h->phi.assign(h->n_in, 0.0);
    cudaError_t e = cudaGetDevice(&h->dev);
    auto bail = [&](int code, const std::string& m) {
        corr_destroy(h);
        return fail(nullptr, code, m);
    };
    if (e != cudaSuccess) return bail(CORR_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    const std::vector<float> hf = make_filter(h->M, taps, h->window, h->kaiser_beta);
    const std::vector<float2> tw = corr::fft_twiddle_table(h->M);
    if (cudaStreamCreateWithFlags(&h->s_comp, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&h->s_copy, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&h->s_out, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&h->s_get, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->ev_h2d, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->ev_comp, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->ev_fin, cudaEventDisableTiming) != cudaSuccess)
        return bail(CORR_ECUDA, "stream/event creation failed");
    const std::vector<float> hsf = half_rows(hf, h->M, taps);
    if (cudaMalloc(&h->d_h, hf.size() * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&h->d_hs, hsf.size() * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&h->d_tw, tw.size() * sizeof(float2)) != cudaSuccess)
        return bail(CORR_ENOMEM, "cudaMalloc of filter tables failed");
    if (cudaMemcpy(h->d_h, hf.data(), hf.size() * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(h->d_hs, hsf.data(), hsf.size() * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(h->d_tw, tw.data(), tw.size() * sizeof(float2), cudaMemcpyHostToDevice) != cudaSuccess)
        return bail(CORR_ECUDA, "upload of filter tables failed");
    if (alloc_tables(h, h->tab_stream) != CORR_OK || alloc_tables(h, h->tab_direct) != CORR_OK)
        return bail(CORR_ENOMEM, "cudaMalloc of delay tables failed");
    if (cudaMalloc(&h->d_status, sizeof(int)) != cudaSuccess || cudaMemset(h->d_status, 0, sizeof(int)) != cudaSuccess)
        return bail(CORR_ENOMEM, "cudaMalloc of the status word failed");
    if (upload_tables(h, h->tab_stream, h->tau, h->phi, h->s_comp) != CORR_OK ||
        upload_tables(h, h->tab_direct, h->tau, h->phi, h->s_comp) != CORR_OK)
        return bail(CORR_ECUDA, "upload of delay tables failed");
    *out = h;
    return CORR_OK;
}

int corr_destroy(corr_t h) {
    if (!h) return CORR_OK;
    DeviceGuard g(h->dev);
    if (h->is_group) {
        for (cudaStream_t s : h->mstreams) {
            cudaStreamSynchronize(s);
            cudaStreamDestroy(s);
        }
        for (cudaEvent_t e : h->mjoin) cudaEventDestroy(e);
        if (h->gfork) cudaEventDestroy(h->gfork);
        if (h->gorigin) {
            cudaStreamSynchronize(h->gorigin);
            cudaStreamDestroy(h->gorigin);
        }
        if (h->gin) cudaEventDestroy(h->gin);
        if (h->gout) cudaEventDestroy(h->gout);
        if (h->gexec) cudaGraphExecDestroy(h->gexec);
        if (h->graph) cudaGraphDestroy(h->graph);
        cudaFree(h->d_tail_members);
        cudaFree(h->d_tail_items);
        cudaFree(h->d_tail_counters);
        cudaFree(h->d_status);
        cudaGetLastError();
        delete h;
        return CORR_OK;
    }
    if (h->s_comp) cudaStreamSynchronize(h->s_comp);
    if (h->s_copy) cudaStreamSynchronize(h->s_copy);
    if (h->s_out) cudaStreamSynchronize(h->s_out);
    for (Slot& s : h->slots) {
        cudaFree(s.d_R);
        cudaFree(s.d_F);
        cudaFreeHost(s.h_R);
        cudaFreeHost(s.h_F);
        if (s.ev) cudaEventDestroy(s.ev);
    }
    for (cudaEvent_t e : h->timer.pool) cudaEventDestroy(e);
    for (int i = 0; i < kStages; ++i)
        for (auto& pr : h->timer.open[i]) {
            cudaEventDestroy(pr.first);
            cudaEventDestroy(pr.second);
        }
    free_pipe(h->ps);
    free_pipe(h->pd);
    cudaFree(h->d_part_x);
    cudaFree(h->d_h);
    cudaFree(h->d_hs);
    cudaFree(h->d_tw);
    cudaFree(h->tab_stream.phasor);
    cudaFree(h->tab_stream.rot);
    cudaFree(h->tab_stream.coarse);
    cudaFree(h->tab_direct.phasor);
    cudaFree(h->tab_direct.rot);
    cudaFree(h->tab_direct.coarse);
    cudaFree(h->d_z_f);
    cudaFree(h->d_status);
    for (int b = 0; b < 2; ++b) {
        cudaFree(h->d_stage_buf[b]);
        if (h->ev_buf[b]) cudaEventDestroy(h->ev_buf[b]);
    }
    if (h->h_pin) cudaFreeHost(h->h_pin);
    if (h->ev_h2d) cudaEventDestroy(h->ev_h2d);
    if (h->ev_comp) cudaEventDestroy(h->ev_comp);
    if (h->ev_fin) cudaEventDestroy(h->ev_fin);
    if (h->s_comp) cudaStreamDestroy(h->s_comp);
    if (h->s_copy) cudaStreamDestroy(h->s_copy);
    if (h->s_out) cudaStreamDestroy(h->s_out);
    if (h->s_get) cudaStreamDestroy(h->s_get);
    cudaGetLastError();
    delete h;
    return CORR_OK;
}

const char* corr_last_error(corr_t h) {
    if (!h) return g_create_error.c_str();
    return h->err.c_str();
}

int corr_set_option(corr_t h, const char* key, double v) {
    if (!h || !key) return fail(h, CORR_EINVAL, "NULL argument");
    const std::string k(key);
    if (h->started && k != "stage_timing" && k != "stage_mask" && k != "fir_spt" && k != "x_depth" &&
        k != "fused_f" &&
        k != "tc_wait_ms" && k != "inject_stall" && k != "inject_alloc_fail" && k != "max_pending")
        return fail(h, CORR_ESTATE, "options must be set before the first push");
    if (k == "flag_sigma") {
        if (!(v > 0)) return fail(h, CORR_EINVAL, "flag_sigma must be > 0");
        h->flag_sigma = v;
    } else if (k == "flag_window") {
        if (!is_pow2((long long)v) || v > 256 || v < 2) return fail(h, CORR_EINVAL, "flag_window: power of two in [2, 256]");
        h->flag_window = (int)v;
    } else if (k == "max_delay") {
        if (v < 0 || v > (1 << 24)) return fail(h, CORR_EINVAL, "max_delay out of range");
        if (h->stream_alloc) return fail(h, CORR_ESTATE, "max_delay must be set before buffers exist");
        h->max_delay = (long long)v;
    } else if (k == "chunk") {
        if (v < 1 || v > (double)(1LL << 32)) return fail(h, CORR_EINVAL, "chunk out of range");
        if (h->stream_alloc) return fail(h, CORR_ESTATE, "chunk must be set before buffers exist");
        h->chunk = (long long)v;
    } else if (k == "sample_format") {
        if (v != 0 && v != 1) return fail(h, CORR_EINVAL, "sample_format: 0 real, 1 complex (interleaved int8 I/Q)");
        if (h->stream_alloc || h->pd.V) return fail(h, CORR_ESTATE, "sample_format must be set before buffers exist");
        if (v == 1 && h->precision != CORR_FP32) return fail(h, CORR_EINVAL, "complex input runs the FP32 path");
        if (v == 1 && h->es != 1 && !h->iq) return fail(h, CORR_EINVAL, "complex input takes int8 I/Q samples");
        if (v == 1 && h->n_chan < 16) return fail(h, CORR_EINVAL, "complex input needs n_chan >= 16");
        if ((int)v == h->iq) return CORR_OK;
        h->iq = (int)v;
        h->M = h->iq ? h->n_chan : 2 * h->n_chan;
        h->es = h->iq ? 2 : 1;
        CKRET(build_filter_tables(h));
        CKRET(upload_tables(h, h->tab_direct, h->tau, h->phi, h->s_comp));
        CKRET(upload_tables(h, h->tab_stream, h->tau, h->phi, h->s_comp));
    } else if (k == "precision") {
        if (v != CORR_FP32 && v != CORR_INT8 && v != CORR_FP8) return fail(h, CORR_EINVAL, "precision: 0, 1 or 2");
        if (v != CORR_FP32 && h->iq) return fail(h, CORR_EINVAL, "complex input runs the FP32 path");
        if (v != CORR_FP32 && h->n_in > 64) return fail(h, CORR_EINVAL, "reduced precision needs n_in <= 64");
        if (h->stream_alloc || h->pd.V) return fail(h, CORR_ESTATE, "precision must be set before buffers exist");
        h->precision = (int)v;
    } else if (k == "ring_mb") {
        if (v < 1 || v > 4096) return fail(h, CORR_EINVAL, "ring_mb out of range");
        if (h->stream_alloc) return fail(h, CORR_ESTATE, "ring_mb must be set before the first push");
        h->ring_mb = (int)v;
        free_pipe(h->pd);
    } else if (k == "inject_alloc_fail") {
        if (v < 0 || v > 1000 || v != (double)(int)v) return fail(h, CORR_EINVAL, "inject_alloc_fail: 0 .. 1000");
        h->inject_alloc_fail = (int)v;
        return CORR_OK;
    } else if (k == "max_pending") {
        if (v < 0 || v > 1e6 || v != (double)(long long)v) return fail(h, CORR_EINVAL, "max_pending: 0 .. 1e6");
        h->max_pending = (int)v;
        return CORR_OK;
    } else if (k == "tc_wait_ms") {
        if (!(v >= 1.0 && v <= 60000.0)) return fail(h, CORR_EINVAL, "tc_wait_ms: 1 .. 60000");
        h->tc_wait_ms = v;
        return CORR_OK;
    } else if (k == "inject_stall") {
        if (v != 0 && v != 1) return fail(h, CORR_EINVAL, "inject_stall: 0 or 1");
        h->inject_stall = (int)v;
        return CORR_OK;
    } else if (k == "fused_f") {
        if (v != 0 && v != 1) return fail(h, CORR_EINVAL, "fused_f: 0 or 1");
        h->fused_f = (int)v;
        return CORR_OK;
    } else if (k == "fir_spt") {
        if (v < 0 || v > 256) return fail(h, CORR_EINVAL, "fir_spt out of range");
        h->fir_spt = (int)v;
        return CORR_OK;
    } else if (k == "x_depth") {
        if (v != 4 && v != 6) return fail(h, CORR_EINVAL, "x_depth: 4 or 6");
        h->x_depth = (int)v;
        return CORR_OK;
    } else if (k == "stage_timing") {
        h->timer.on = v != 0;
        return CORR_OK;
    } else if (k == "stage_mask") {
        if (v < 0 || v >= (double)(1 << kStages) || v != (double)(long long)v)
            return fail(h, CORR_EINVAL, "stage_mask: bit mask of stages 0..6");
        h->timer.mask = (int)v;
        return CORR_OK;
    } else if (k == "sample_bits") {
        if (v != 8 && v != 16) return fail(h, CORR_EINVAL, "sample_bits: 8 or 16");
        if (h->iq && v != 8) return fail(h, CORR_EINVAL, "complex input takes int8 I/Q samples");
        if (h->iq) return CORR_OK;
        if (h->stream_alloc) return fail(h, CORR_ESTATE, "sample_bits must be set before the first push");
        h->es = v == 16 ? 2 : 1;
    } else if (k == "window" || k == "kaiser_beta") {
        if (k == "window" && v != 0 && v != 1 && v != 2) return fail(h, CORR_EINVAL, "window: 0 Hann, 1 Kaiser, 2 none");
        if (k == "kaiser_beta" && !(v >= 0 && v <= 50)) return fail(h, CORR_EINVAL, "kaiser_beta out of range");
        if (k == "window") h->window = (int)v;
        else h->kaiser_beta = v;
        CKRET(build_filter_tables(h));
    } else if (k == "result_slots") {
        if (v < 1 || v > 4096) return fail(h, CORR_EINVAL, "result_slots out of range");
        h->result_slots = (int)v;
    } else {
        return fail(h, CORR_EINVAL, "unknown option " + k);
    }
    return CORR_OK;
}

int corr_set_delays(corr_t h, const double* tau, const double* phi) {
    if (!h || !tau) return fail(h, CORR_EINVAL, "NULL argument");
    DeviceGuard g(h->dev);
    std::vector<double> t(tau, tau + h->n_in), p(h->n_in, 0.0);
    if (phi) p.assign(phi, phi + h->n_in);
    for (int a = 0; a < h->n_in; ++a) {
        if (!std::isfinite(t[a]) || !std::isfinite(p[a])) return fail(h, CORR_EINVAL, "non-finite delay/phase");
        if (std::fabs(std::floor(t[a] + 0.5)) > (double)h->max_delay)
            return fail(h, CORR_EINVAL, "coarse delay exceeds max_delay");
    }
    h->tau = t;
    h->phi = p;
    CKRET(upload_tables(h, h->tab_direct, t, p, h->s_comp));
    if (!h->started) {
        CKRET(upload_tables(h, h->tab_stream, t, p, h->s_comp));
        h->pending = false;
    } else {
        h->tau_pend = t;
        h->phi_pend = p;
        h->pending = true;
    }
    return CORR_OK;
}

int corr_push(corr_t h, const void* samples, size_t n, size_t stride) {
    if (!h) return fail(h, CORR_EINVAL, "NULL handle");
    DeviceGuard g(h->dev);
    return push_common(h, static_cast<const int8_t*>(samples), n, stride, false, nullptr);
}

int corr_push_dev(corr_t h, const void* d_samples, size_t n, size_t stride, void* stream) {
    if (!h) return fail(h, CORR_EINVAL, "NULL handle");
    DeviceGuard g(h->dev);
    return push_common(h, static_cast<const int8_t*>(d_samples), n, stride, true, static_cast<cudaStream_t>(stream));
}

int corr_flush(corr_t h) {
    if (!h) return fail(h, CORR_EINVAL, "NULL handle");
    DeviceGuard g(h->dev);
    if (h->flushed) return fail(h, CORR_ESTATE, "already flushed");
    if (!h->started) {
        h->flushed = true;
        return CORR_OK;
    }
    CKRET(process_stream(h, true));
    h->flushed = true;
    return CORR_OK;
}

int corr_reset(corr_t h) {
    if (!h) return fail(h, CORR_EINVAL, "NULL handle");
    DeviceGuard g(h->dev);
    if (h->s_comp) CK(cudaStreamSynchronize(h->s_comp));
    if (h->s_copy) CK(cudaStreamSynchronize(h->s_copy));
    if (h->s_out) CK(cudaStreamSynchronize(h->s_out));
    h->started = h->flushed = false;
    h->stage_base = h->stage_len = 0;
    h->cur_buf = 0;
    h->d_stage = h->d_stage_buf[0];
    h->buf_read[0] = h->buf_read[1] = false;
    h->n_pushed = 0;
    h->ps.s_next = h->ps.s_xdone = 0;
    h->ps.have_scale = false;
    h->q_vis.clear();
    h->q_flag.clear();
    for (Slot& s : h->slots) s.in_vis = s.in_flag = false;
    if (h->pending) {
        CKRET(upload_tables(h, h->tab_stream, h->tau_pend, h->phi_pend, h->s_comp));
        h->pending = false;
    } else {
        CKRET(upload_tables(h, h->tab_stream, h->tau, h->phi, h->s_comp));
    }
    return CORR_OK;
}

int corr_get_vis(corr_t h, float* out, int max_int, int* n_got) {
    if (!h) return fail(h, CORR_EINVAL, "NULL handle");
    DeviceGuard g(h->dev);
    return pop_results(h, h->q_vis, true, out, max_int, n_got);
}

int corr_get_flags(corr_t h, uint8_t* out, int max_int, int* n_got) {
    if (!h) return fail(h, CORR_EINVAL, "NULL handle");
    DeviceGuard g(h->dev);
    return pop_results(h, h->q_flag, false, out, max_int, n_got);
}

int corr_pending(corr_t h, int* n) {
    if (!h || !n) return fail(h, CORR_EINVAL, "NULL argument");
    *n = (int)h->q_vis.size();
    return CORR_OK;
}

int corr_run_dev(corr_t h, const void* d_samples, size_t n_samples, size_t stride, float* d_vis,
                 uint8_t* d_flags, int max_int, int include_partial, int* n_out, void* stream) {
    if (!h) return fail(h, CORR_EINVAL, "NULL handle");
    if (h->is_group) return fail(h, CORR_EINVAL, "use corr_group_run_dev on a group");
    DeviceGuard g(h->dev);
    if (n_out) *n_out = 0;
    if (!d_samples || !d_vis) return fail(h, CORR_EINVAL, "NULL buffer");
    if (stride < n_samples) return fail(h, CORR_EINVAL, "input_stride < n_samples");
    const long long n_spec = (long long)(n_samples / (size_t)h->M);
    long long need = n_spec / h->n_int + ((include_partial && n_spec % h->n_int) ? 1 : 0);
    if (need > max_int) return fail(h, CORR_EINVAL, "max_int too small for the stream");
    CKRET(alloc_pipe(h, h->pd));
    if (h->defer_tail && h->precision == CORR_FP32 && h->pd.part_all_ints < need) {
        cudaFree(h->pd.part_all);
        h->pd.part_all = nullptr;
        CKA(dmalloc(h, &h->pd.part_all, sizeof(float) * (size_t)need * h->gpi * h->nt * 32 * h->n_chan));
        h->pd.part_all_ints = need;
    }
    h->pd.s_next = h->pd.s_xdone = 0;
    h->pd.have_scale = false;
    StreamView sv;
    sv.x = static_cast<const int8_t*>(d_samples);
    sv.es = h->es;
    sv.stride = (long long)stride;
    sv.base = 0;
    sv.vhi = (long long)n_samples;
    DirectCtx c{reinterpret_cast<float2*>(d_vis), d_flags, max_int, 0};
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    CKRET(drive(h, h->pd, sv, h->tab_direct, n_spec, include_partial != 0, false, sink_direct, &c, st));
    if (n_out) *n_out = c.n_out;
    return CORR_OK;
}

int corr_fengine_dev(corr_t h, const void* d_samples, size_t n_samples, size_t stride, long long s0,
                     int n_spec, float* d_V, void* stream) {
    if (!h) return fail(h, CORR_EINVAL, "NULL handle");
    DeviceGuard g(h->dev);
    if (!d_samples || !d_V || n_spec < 0 || s0 < 0) return fail(h, CORR_EINVAL, "bad argument");
    if (stride < n_samples) return fail(h, CORR_EINVAL, "input_stride < n_samples");
    if (n_spec == 0) return CORR_OK;
    if (n_spec > h->z_f_spectra) {
        cudaFree(h->d_z_f);
        h->d_z_f = nullptr;
        CKA(dmalloc(h, &h->d_z_f, sizeof(float2) * (size_t)n_spec * h->n_in_pad * h->n_chan));
        h->z_f_spectra = n_spec;
    }
    StreamView sv{static_cast<const int8_t*>(d_samples), (long long)stride, 0, (long long)n_samples, h->es};
    CKRET(launch_f(h, sv, h->tab_direct, h->d_z_f, s0, -1LL, reinterpret_cast<float2*>(d_V), s0, -1LL,
                   h->tab_direct.phasor, s0, s0 + n_spec, static_cast<cudaStream_t>(stream)));
    return CORR_OK;
}

int corr_xengine_dev(corr_t h, const float* d_V, int n_spec, float* d_vis, void* stream) {
    if (!h) return fail(h, CORR_EINVAL, "NULL handle");
    DeviceGuard g(h->dev);
    if (!d_V || !d_vis || n_spec < 1) return fail(h, CORR_EINVAL, "bad argument");
    // V is read as 16-byte vectors and R written as complex64.
    if ((reinterpret_cast<uintptr_t>(d_V) & 15) != 0 || (reinterpret_cast<uintptr_t>(d_vis) & 7) != 0)
        return fail(h, CORR_EINVAL, "d_V must be 16-byte and d_vis 8-byte aligned");
    // One partial slot per group of G spectra; the groups are a grid
    // dimension of the X-engine launch, so at most 65535 of them.
    long long G = 64;
    if ((n_spec + G - 1) / G > 65535) G = (n_spec + 65534) / 65535;
    const long long slots = (n_spec + G - 1) / G;
    if (slots > h->part_x_slots) {
        cudaFree(h->d_part_x);
        h->d_part_x = nullptr;
        CKA(dmalloc(h, &h->d_part_x, sizeof(float) * (size_t)slots * h->nt * 32 * h->n_chan));
        h->part_x_slots = slots;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    XArgs x{};
    x.V = reinterpret_cast<const float2*>(d_V);
    x.v_origin = 0;
    x.v_mask = -1LL;
    x.n_chan = h->n_chan;
    x.n_in_pad = h->n_in_pad;
    x.nt = h->nt;
    x.int_start = 0;
    x.int_end = n_spec;
    x.s_limit = n_spec;
    x.G = (int)G;
    x.j0 = 0;
    x.n_groups = (int)slots;
    x.part = h->d_part_x;
    {
        Timed t_(h, 2, st);
        launch_xengine(x, st);
    }
    CK(cudaGetLastError());
    FinArgs f{};
    f.part = h->d_part_x;
    f.n_slots = (int)slots;
    f.nt = h->nt;
    f.n_chan = h->n_chan;
    f.n_in = h->n_in;
    f.scale = 1.0f / (float)n_spec;
    f.R = reinterpret_cast<float2*>(d_vis);
    {
        Timed t_(h, 3, st);
        launch_finalize(f, st);
    }
    CK(cudaGetLastError());
    return CORR_OK;
}

int corr_flag_dev(corr_t h, const float* d_vis, int n_vis, uint8_t* d_flags, void* stream) {
    if (!h) return fail(h, CORR_EINVAL, "NULL handle");
    DeviceGuard g(h->dev);
    if (!d_vis || !d_flags || n_vis < 0) return fail(h, CORR_EINVAL, "bad argument");
    const int w = h->flag_window < h->n_chan ? h->flag_window : h->n_chan;
    {
        Timed t_(h, 4, static_cast<cudaStream_t>(stream));
        launch_mad_flags(reinterpret_cast<const float2*>(d_vis), d_flags, n_vis, h->n_chan, h->n_in, w,
                         (float)h->flag_sigma, static_cast<cudaStream_t>(stream));
    }
    CK(cudaGetLastError());
    return CORR_OK;
}

int corr_shape(corr_t h, int* n_in, int* n_chan, int* taps, int* n_int, int* n_in_pad) {
    if (!h) return fail(h, CORR_EINVAL, "NULL handle");
    if (n_in) *n_in = h->n_in;
    if (n_chan) *n_chan = h->n_chan;
    if (taps) *taps = h->taps;
    if (n_int) *n_int = h->n_int;
    if (n_in_pad) *n_in_pad = h->n_in_pad;
    return CORR_OK;
}

long long corr_kernel_launches(corr_t h) { return h ? h->launches : 0; }

int corr_gram_dev(corr_t h, const void* d_Q, int n_chan, int k_pitch, int K, int dtype, float* d_G, void* stream) {
    if (!h) return fail(h, CORR_EINVAL, "NULL handle");
    DeviceGuard g(h->dev);
    if (!d_Q || !d_G || n_chan < 1 || K < 1 ||
        (dtype != CORR_INT8 && dtype != CORR_FP8 && dtype != CORR_INT8_BYTES && dtype != CORR_INT8_WORDS &&
         dtype != CORR_FP8_WORDS))
        return fail(h, CORR_EINVAL, "bad argument");
    GramArgs a{};
    a.Q = d_Q;
    a.n_chan = n_chan;
    a.K = K;
    a.k_pitch = k_pitch;
    a.fp8 = dtype == CORR_FP8 || dtype == CORR_FP8_WORDS;
    a.i8b = dtype == CORR_INT8_BYTES;
    a.words = dtype == CORR_INT8_WORDS || dtype == CORR_FP8_WORDS;
    a.n_pairs = h->n_in_pad / 2;
    a.n_in = h->n_in;
    a.G = d_G;
    a.status = h->d_status;
    a.wait_ns = (unsigned long long)(h->tc_wait_ms * 1e6);
    a.inject_stall = h->inject_stall;
    int rc;
    {
        Timed t_(h, 2, static_cast<cudaStream_t>(stream));
        rc = launch_gram(a, static_cast<cudaStream_t>(stream));
    }
    if (rc != CORR_OK)
        return fail(h, rc, "gram: bad layout (k_pitch multiple of 128 bytes, 16-byte aligned Q; words: n_chan "
                           "multiple of 4, n_in <= 64)");
    CK(cudaGetLastError());
    return CORR_OK;
}

// ---- batched sub-array streams: one captured graph --------------------------

namespace {

// The work queue of a group's tail kernel for one capture: every FP32
// member's integrations as finalise blocks (the blocks finalize_kernel would
// run), then every member's MAD flags in items of kTailWarpItems warp items,
// each depending on its integration's finalise blocks; uploaded before the
// capture so that the capture records only the counter reset and the launch.
int build_group_tail(corr_t g, const size_t* n_samples, float* const* d_vis, uint8_t* const* d_flags) {
    corr_t h = g;
    const int n = (int)g->members.size();
    std::vector<TailMember> mem(n);
    std::vector<TailItem> fin, flg;
    int deps = 0;
    for (int m = 0; m < n; ++m) {
        corr_t c = g->members[m];
        TailMember& tm = mem[m];
        tm = TailMember{};
        const long long n_out = (long long)(n_samples[m] / (size_t)c->M) / c->n_int;
        tm.fin.part = c->pd.part_all;
        tm.fin.rot = c->tab_direct.rot;
        tm.fin.n_slots = c->gpi;
        tm.fin.nt = c->nt;
        tm.fin.n_chan = c->n_chan;
        tm.fin.n_in = c->n_in;
        tm.fin.scale = 0.25f / (float)c->n_int;
        tm.fin.R = reinterpret_cast<float2*>(d_vis[m]);
        tm.part_stride = (long long)c->gpi * c->nt * 32 * c->n_chan;
        tm.vis_stride = (long long)vis_elems(c);
        tm.flags = d_flags ? d_flags[m] : nullptr;
        tm.window = c->flag_window < c->n_chan ? c->flag_window : c->n_chan;
        tm.sigma = (float)c->flag_sigma;
        const bool fp32 = c->precision == CORR_FP32;
        if (fp32 && !c->pd.part_all && n_out > 0) return fail(g, CORR_ESTATE, "member partial sums missing");
        for (long long i = 0; i < n_out; ++i) {
            const int dep = deps++;
            int need = 0;
            if (fp32) {
                for (int bx = 0; bx < (c->n_chan + 127) / 128; ++bx)
                    for (int t = 0; t < c->nt; ++t)
                        for (int z = 0; z < 16; ++z, ++need)
                            fin.push_back(TailItem{0, m, (int)i, bx, t, z, dep, 0});
            }
            if (tm.flags) {
                const long long n_wi = (long long)(c->n_chan / tm.window) * (c->n_in * (c->n_in + 1) / 2);
                for (long long x = 0; x < n_wi; x += kTailWarpItems)
                    flg.push_back(TailItem{1, m, (int)i, (int)x, 0, 0, dep, need});
            }
        }
    }
    std::vector<TailItem> items(fin);
    items.insert(items.end(), flg.begin(), flg.end());
    cudaFree(g->d_tail_members);
    cudaFree(g->d_tail_items);
    cudaFree(g->d_tail_counters);
    g->d_tail_members = nullptr;
    g->d_tail_items = nullptr;
    g->d_tail_counters = nullptr;
    g->tail_items = (int)items.size();
    g->tail_fin_items = (int)fin.size();
    g->tail_deps = deps;
    if (items.empty()) return CORR_OK;
    CK(cudaMalloc(&g->d_tail_members, sizeof(TailMember) * mem.size()));
    CK(cudaMalloc(&g->d_tail_items, sizeof(TailItem) * items.size()));
    CK(cudaMalloc(&g->d_tail_counters, sizeof(int) * (size_t)(1 + deps)));
    CK(cudaMemcpy(g->d_tail_members, mem.data(), sizeof(TailMember) * mem.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(g->d_tail_items, items.data(), sizeof(TailItem) * items.size(), cudaMemcpyHostToDevice));
    if (!g->tail_grid) g->tail_grid = group_tail_grid();
    return CORR_OK;
}

}  // namespace


int corr_group_create(corr_t* out, const corr_t* members, int n) {
    if (!out || !members || n < 1 || n > 64) return fail(nullptr, CORR_EINVAL, "bad group arguments");
    *out = nullptr;
    for (int i = 0; i < n; ++i) {
        if (!members[i] || members[i]->is_group) return fail(nullptr, CORR_EINVAL, "group members must be handles");
        for (int j = 0; j < i; ++j)
            if (members[j] == members[i]) return fail(nullptr, CORR_EINVAL, "duplicate group member");
        if (members[i]->dev != members[0]->dev) return fail(nullptr, CORR_EINVAL, "members on different devices");
    }
    corr_t g = new corr_s();
    g->is_group = true;
    g->dev = members[0]->dev;
    DeviceGuard dg(g->dev);
    g->members.assign(members, members + n);
    g->mstreams.resize(n, nullptr);
    g->mjoin.resize(n, nullptr);
    bool ok = cudaEventCreateWithFlags(&g->gfork, cudaEventDisableTiming) == cudaSuccess &&
              cudaEventCreateWithFlags(&g->gin, cudaEventDisableTiming) == cudaSuccess &&
              cudaEventCreateWithFlags(&g->gout, cudaEventDisableTiming) == cudaSuccess &&
              cudaStreamCreateWithFlags(&g->gorigin, cudaStreamNonBlocking) == cudaSuccess;
    for (int i = 0; i < n && ok; ++i)
        ok = cudaStreamCreateWithFlags(&g->mstreams[i], cudaStreamNonBlocking) == cudaSuccess &&
             cudaEventCreateWithFlags(&g->mjoin[i], cudaEventDisableTiming) == cudaSuccess;
    if (ok) ok = cudaMalloc(&g->d_status, sizeof(int)) == cudaSuccess &&
                 cudaMemset(g->d_status, 0, sizeof(int)) == cudaSuccess;
    if (!ok) {
        corr_destroy(g);
        return fail(nullptr, CORR_ECUDA, "group stream/event creation failed");
    }
    *out = g;
    return CORR_OK;
}

int corr_group_run_dev(corr_t g, const void* const* d_samples, const size_t* n_samples, const size_t* strides,
                       float* const* d_vis, uint8_t* const* d_flags, const int* max_int, int* n_out, void* stream) {
    if (!g || !g->is_group) return fail(g, CORR_EINVAL, "not a group");
    if (!d_samples || !n_samples || !strides || !d_vis || !max_int) return fail(g, CORR_EINVAL, "NULL argument");
    corr_t h = g;   // error reporting target of the CK macro
    DeviceGuard dg(g->dev);
    const int n = (int)g->members.size();
    // Work is captured and launched on the group's own stream, ordered after
    // the caller's stream and before its later work.
    cudaStream_t user = static_cast<cudaStream_t>(stream);
    cudaStream_t origin = g->gorigin;
    CK(cudaEventRecord(g->gin, user));
    CK(cudaStreamWaitEvent(origin, g->gin, 0));
    // The graph replays fixed pointers and sizes: capture again if they change.
    std::vector<const void*> key;
    for (int i = 0; i < n; ++i) {
        key.push_back(d_samples[i]);
        key.push_back(reinterpret_cast<const void*>(n_samples[i]));
        key.push_back(reinterpret_cast<const void*>(strides[i]));
        key.push_back(d_vis[i]);
        key.push_back(d_flags ? d_flags[i] : nullptr);
        key.push_back(reinterpret_cast<const void*>((size_t)max_int[i]));
    }
    // the tail kernel's wait limit and fault injection are captured values too
    key.push_back(reinterpret_cast<const void*>((size_t)(g->tc_wait_ms * 1e3)));
    key.push_back(reinterpret_cast<const void*>((size_t)g->inject_stall));
    if (!g->gexec || key != g->gkey) {
        // Members defer finalisation (FP32) and flagging to the group's tail
        // kernel while the group runs them.
        struct DeferGuard {
            corr_s* g;
            explicit DeferGuard(corr_s* g_) : g(g_) {
                for (corr_s* m : g->members) m->defer_tail = true;
            }
            ~DeferGuard() {
                for (corr_s* m : g->members) m->defer_tail = false;
            }
        } defer(g);
        if (g->gexec) {
            cudaGraphExecDestroy(g->gexec);
            g->gexec = nullptr;
        }
        if (g->graph) {
            cudaGraphDestroy(g->graph);
            g->graph = nullptr;
        }
        // Uncaptured run first: allocates every member's buffers and
        // configures its kernels, so the capture records launches only.
        for (int i = 0; i < n; ++i) {
            int got = 0;
            corr_t m = g->members[i];
            const bool timing = m->timer.on;
            m->timer.on = false;
            const int rc = corr_run_dev(m, d_samples[i], n_samples[i], strides[i], d_vis[i],
                                        d_flags ? d_flags[i] : nullptr, max_int[i], 0, &got, origin);
            m->timer.on = timing;
            if (rc != CORR_OK) return fail(g, rc, std::string("member ") + std::to_string(i) + ": " + m->err);
        }
        CK(cudaStreamSynchronize(origin));
        CKRET(build_group_tail(g, n_samples, d_vis, d_flags));
        CK(cudaStreamBeginCapture(origin, cudaStreamCaptureModeThreadLocal));
        long long k0 = 0;
        for (int i = 0; i < n; ++i) k0 += g->members[i]->launches;
        int rc = CORR_OK;
        if (cudaEventRecord(g->gfork, origin) != cudaSuccess) rc = CORR_ECUDA;
        for (int i = 0; i < n && rc == CORR_OK; ++i) {
            corr_t m = g->members[i];
            if (cudaStreamWaitEvent(g->mstreams[i], g->gfork, 0) != cudaSuccess) {
                rc = CORR_ECUDA;
                break;
            }
            const bool timing = m->timer.on;
            m->timer.on = false;
            int got = 0;
            rc = corr_run_dev(m, d_samples[i], n_samples[i], strides[i], d_vis[i], d_flags ? d_flags[i] : nullptr,
                              max_int[i], 0, &got, g->mstreams[i]);
            m->timer.on = timing;
            if (rc == CORR_OK && (cudaEventRecord(g->mjoin[i], g->mstreams[i]) != cudaSuccess ||
                                  cudaStreamWaitEvent(origin, g->mjoin[i], 0) != cudaSuccess))
                rc = CORR_ECUDA;
        }
        // the persistent tail over every member: finalise + flags
        if (rc == CORR_OK && g->tail_items > 0) {
            if (cudaMemsetAsync(g->d_tail_counters, 0, sizeof(int) * (size_t)(1 + g->tail_deps), origin) !=
                cudaSuccess)
                rc = CORR_ECUDA;
            TailArgs ta{};
            ta.members = g->d_tail_members;
            ta.items = g->d_tail_items;
            ta.n_items = g->tail_items;
            ta.ticket = g->d_tail_counters;
            ta.done = g->d_tail_counters + 1;
            ta.wait_ns = (unsigned long long)(g->tc_wait_ms * 1e6);
            ta.status = g->d_status;
            ta.inject_skip = (g->inject_stall && g->tail_fin_items > 0) ? 0 : -1;
            launch_group_tail(ta, g->tail_grid, origin);
            if (cudaGetLastError() != cudaSuccess) rc = CORR_ECUDA;
        }
        cudaGraph_t graph = nullptr;
        const cudaError_t ec = cudaStreamEndCapture(origin, &graph);
        if (rc != CORR_OK || ec != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            cudaGetLastError();
            return fail(g, rc != CORR_OK ? rc : CORR_ECUDA, "graph capture of the group failed");
        }
        g->graph = graph;
        long long k1 = 0;
        for (int i = 0; i < n; ++i) k1 += g->members[i]->launches;
        g->graph_kernels = k1 - k0 + (g->tail_items > 0 ? 1 : 0);
        CK(cudaGraphInstantiate(&g->gexec, g->graph, 0));
        g->gkey = key;
    }
    CK(cudaGraphLaunch(g->gexec, origin));
    CK(cudaEventRecord(g->gout, origin));
    CK(cudaStreamWaitEvent(user, g->gout, 0));
    for (int i = 0; i < n; ++i) {
        if (n_out) {
            const long long n_spec = (long long)(n_samples[i] / (size_t)g->members[i]->M);
            n_out[i] = (int)(n_spec / g->members[i]->n_int);
        }
    }
    g->launches += g->graph_kernels;
    return CORR_OK;
}

// ---- autotuner ------------------------------------------------------------

namespace {

std::string tune_key(corr_t h) {
    cudaDeviceProp prop;
    std::string name = "gpu";
    if (cudaGetDeviceProperties(&prop, h->dev) == cudaSuccess) name = prop.name;
    for (char& c : name)
        if (c == ' ') c = '_';
    char buf[256];
    std::snprintf(buf, sizeof(buf), "%s %d %d %d %d %d", name.c_str(), h->n_in, h->n_chan, h->taps, h->n_int,
                  h->precision);
    return buf;
}

bool tune_lookup(const char* path, const std::string& key, int* ring_mb, int* fir_spt, int* x_depth) {
    if (!path) return false;
    FILE* f = std::fopen(path, "r");
    if (!f) return false;
    char line[512];
    bool found = false;
    while (std::fgets(line, sizeof(line), f)) {
        std::string l(line);
        if (l.compare(0, key.size(), key) == 0 && l.size() > key.size() && l[key.size()] == ' ') {
            int r = 0, sp = 0, d = 6;
            if (std::sscanf(l.c_str() + key.size(), "%d %d %d", &r, &sp, &d) >= 2) {
                *ring_mb = r;
                *fir_spt = sp;
                *x_depth = (d == 4) ? 4 : 6;
                found = true;
            }
        }
    }
    std::fclose(f);
    return found;
}

}  // namespace

int corr_autotune(corr_t h, const void* d_samples, size_t n_samples, size_t stride, const char* cache_path,
                  void* stream) {
    if (!h || h->is_group) return fail(h, CORR_EINVAL, "autotune needs a correlator handle");
    if (!d_samples || stride < n_samples) return fail(h, CORR_EINVAL, "bad sample buffer");
    DeviceGuard dg(h->dev);
    const std::string key = tune_key(h);
    int ring = 0, spt = 0, depth = 6;
    if (tune_lookup(cache_path, key, &ring, &spt, &depth)) {
        if (ring != h->ring_mb) {
            h->ring_mb = ring;
            free_pipe(h->pd);
        }
        h->fir_spt = spt;
        h->x_depth = depth;
        return CORR_OK;
    }
    // Time every candidate on (at most) eight integrations of the sample:
    // several fills of the largest ring.
    size_t n_use = (size_t)h->M * (size_t)h->n_int * 8;
    if (n_use > n_samples) n_use = n_samples;
    const long long n_spec = (long long)(n_use / (size_t)h->M);
    const int n_out = (int)(n_spec / h->n_int) > 0 ? (int)(n_spec / h->n_int) : 1;
    float2* vis = nullptr;
    uint8_t* flags = nullptr;
    CK(cudaMalloc(&vis, sizeof(float2) * vis_elems(h) * n_out));
    CK(cudaMalloc(&flags, vis_elems(h) * n_out));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    const int rings[] = {32, 64, 128, 256};
    const int spts[] = {0, 8, 16};
    // the small X-engine's pipeline depth (FP32 pipelines of at most 8 inputs)
    const bool small_x = h->precision == CORR_FP32 && h->n_in_pad <= 8;
    const int depths[] = {6, 4};
    const int n_depths = small_x ? 2 : 1;
    float best = 1e30f;
    int best_ring = h->ring_mb, best_spt = h->fir_spt, best_depth = h->x_depth;
    int rc = CORR_OK;
    for (int r : rings) {
        for (int sp : spts) {
          for (int di = 0; di < n_depths; ++di) {
            if (r != h->ring_mb) {
                h->ring_mb = r;
                free_pipe(h->pd);
            }
            h->fir_spt = sp;
            if (small_x) h->x_depth = depths[di];
            int got = 0;
            rc = corr_run_dev(h, d_samples, n_use, stride, reinterpret_cast<float*>(vis), flags, n_out, 0, &got,
                              stream);
            if (rc != CORR_OK) break;
            cudaEventRecord(e0, st);
            for (int rep = 0; rep < 2 && rc == CORR_OK; ++rep)
                rc = corr_run_dev(h, d_samples, n_use, stride, reinterpret_cast<float*>(vis), flags, n_out, 0, &got,
                                  stream);
            cudaEventRecord(e1, st);
            cudaEventSynchronize(e1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rc == CORR_OK && ms < best) {
                best = ms;
                best_ring = r;
                best_spt = sp;
                best_depth = h->x_depth;
            }
            if (rc != CORR_OK) break;
          }
          if (rc != CORR_OK) break;
        }
        if (rc != CORR_OK) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(vis);
    cudaFree(flags);
    if (rc != CORR_OK) return rc;
    if (best_ring != h->ring_mb) {
        h->ring_mb = best_ring;
        free_pipe(h->pd);
    }
    h->fir_spt = best_spt;
    h->x_depth = best_depth;
    if (cache_path) {
        FILE* f = std::fopen(cache_path, "a");
        if (f) {
            std::fprintf(f, "%s %d %d %d\n", key.c_str(), best_ring, best_spt, best_depth);
            std::fclose(f);
        }
    }
    return CORR_OK;
}

int corr_get_tuning(corr_t h, int* ring_mb, int* fir_spt, int* x_depth) {
    if (!h) return fail(h, CORR_EINVAL, "NULL handle");
    if (ring_mb) *ring_mb = h->ring_mb;
    if (fir_spt) *fir_spt = h->fir_spt;
    if (x_depth) *x_depth = h->x_depth;
    return CORR_OK;
}

int corr_spectrogram_dev(corr_t h, const void* d_samples, size_t n_samples, size_t stride, int n_row,
                         float* d_tiles, void* stream) {
    if (!h || h->is_group) return fail(h, CORR_EINVAL, "NULL handle");
    DeviceGuard dg(h->dev);
    if (!d_samples || !d_tiles || n_row < 1 || stride < n_samples) return fail(h, CORR_EINVAL, "bad argument");
    const long long n_spec = (long long)(n_samples / (size_t)h->M);
    const long long rows = n_spec / n_row / 64 * 64;
    if (rows < 64 || h->n_chan % 256) return fail(h, CORR_EINVAL, "need >= 64 rows and n_chan % 256 == 0");
    if (h->iq) return fail(h, CORR_EINVAL, "dynamic spectra are built for real input");
    CKRET(alloc_pipe(h, h->pd));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    CK(cudaMemsetAsync(d_tiles, 0, sizeof(float) * (size_t)h->n_in * rows * h->n_chan, st));
    StreamView sv{static_cast<const int8_t*>(d_samples), (long long)stride, 0, (long long)n_samples, h->es};
    const long long s_total = rows * n_row;
    // the fused F-engine accumulates the tiles with no ring at all: one
    // launch; the two-kernel path passes its FIR output through the ring
    const bool no_ring = h->fused_f && fused_f_supported(h->M, h->taps, h->es, 2);
    const long long step = no_ring ? s_total : h->pd.v_cap;
    for (long long s0 = 0; s0 < s_total; s0 += step) {
        long long s1 = s0 + step;
        if (s1 > s_total) s1 = s_total;
        // the FFT accumulates the tiles directly (no spectra ring traffic)
        CKRET(launch_f(h, sv, h->tab_direct, h->pd.Z, 0, h->pd.v_cap - 1, h->pd.V, 0, h->pd.v_cap - 1, nullptr, s0, s1,
                       st, d_tiles, n_row, (int)rows));
        CK(cudaGetLastError());
    }
    return CORR_OK;
}

// ---- checkpoint / resume ----------------------------------------------------

namespace {

struct StateHeader {
    char magic[8];
    int32_t version;
    int32_t n_in, n_chan, taps, n_int, precision, es, iq, window, flag_window, ring_mb;
    int32_t v_cap, gpi, nt, G, code_words, n_in_pad;
    int32_t started, flushed, stream_alloc, have_scale, pending, n_vis_q, n_flag_q, reserved;
    double kaiser_beta, flag_sigma;
    int64_t max_delay, chunk, stage_cap, n_pushed, stage_base, stage_len, s_next, s_xdone, q_cols;
};
constexpr char kStateMagic[8] = {'C', 'O', 'R', 'R', 'S', 'T', '0', '1'};

struct StateWriter {
    uint8_t* p;
    size_t cap, n;
    void put(const void* src, size_t b) {
        if (p && n + b <= cap) std::memcpy(p + n, src, b);
        n += b;
    }
};

}  // namespace

int corr_save_state(corr_t h, void* buf, size_t cap, size_t* size) {
    if (!h || h->is_group || !size) return fail(h, CORR_EINVAL, "bad argument");
    DeviceGuard dg(h->dev);
    if (h->s_comp) CK(cudaStreamSynchronize(h->s_comp));
    if (h->s_copy) CK(cudaStreamSynchronize(h->s_copy));
    if (h->s_out) CK(cudaStreamSynchronize(h->s_out));
    StateHeader H{};
    std::memcpy(H.magic, kStateMagic, 8);
    H.version = 2;
    H.n_in = h->n_in; H.n_chan = h->n_chan; H.taps = h->taps; H.n_int = h->n_int; H.precision = h->precision;
    H.es = h->es; H.iq = h->iq; H.window = h->window; H.flag_window = h->flag_window; H.ring_mb = h->ring_mb;
    H.v_cap = h->ps.v_cap; H.gpi = h->gpi; H.nt = h->nt; H.G = h->G; H.code_words = h->precision != CORR_FP32; H.n_in_pad = h->n_in_pad;
    H.started = h->started; H.flushed = h->flushed; H.stream_alloc = h->stream_alloc;
    H.have_scale = h->ps.have_scale; H.pending = h->pending;
    H.n_vis_q = (int32_t)h->q_vis.size(); H.n_flag_q = (int32_t)h->q_flag.size();
    H.kaiser_beta = h->kaiser_beta; H.flag_sigma = h->flag_sigma;
    H.max_delay = h->max_delay; H.chunk = h->chunk; H.stage_cap = h->stage_cap; H.n_pushed = h->n_pushed;
    H.stage_base = h->stage_base; H.stage_len = h->stage_len; H.s_next = h->ps.s_next; H.s_xdone = h->ps.s_xdone;
    const long long istart = (h->ps.s_xdone / h->n_int) * h->n_int;
    H.q_cols = h->precision != CORR_FP32 ? (h->ps.s_xdone - istart) : 0;
    StateWriter w{static_cast<uint8_t*>(buf), buf ? cap : 0, 0};
    w.put(&H, sizeof(H));
    auto put_vec = [&](const std::vector<double>& v) {
        std::vector<double> z(h->n_in, 0.0);
        for (int a = 0; a < h->n_in && a < (int)v.size(); ++a) z[a] = v[a];
        w.put(z.data(), sizeof(double) * z.size());
    };
    put_vec(h->stream_tau);
    put_vec(h->stream_phi);
    put_vec(h->tau);
    put_vec(h->phi);
    put_vec(h->tau_pend);
    put_vec(h->phi_pend);
    const size_t ne = vis_elems(h);
    const size_t per_spec = (size_t)h->n_chan * h->n_in_pad * sizeof(float2);
    std::vector<uint8_t> tmp;
    auto put_dev = [&](const void* src, size_t b) -> int {
        if (buf) {
            tmp.resize(b);
            CK(cudaMemcpy(tmp.data(), src, b, cudaMemcpyDeviceToHost));
            w.put(tmp.data(), b);
        } else {
            w.n += b;
        }
        return CORR_OK;
    };
    if (h->stream_alloc) {
        for (int a = 0; a < h->n_in; ++a)
            CKRET(put_dev(h->d_stage + (size_t)a * h->stage_cap * h->es, (size_t)h->stage_len * h->es));
        for (long long sp = h->ps.s_xdone; sp < h->ps.s_next; ++sp)
            CKRET(put_dev(reinterpret_cast<const uint8_t*>(h->ps.V) + (size_t)(sp & (h->ps.v_cap - 1)) * per_spec,
                          per_spec));
        if (h->precision == CORR_FP32) {
            CKRET(put_dev(h->ps.part, sizeof(float) * (size_t)h->gpi * h->nt * 32 * h->n_chan));
        } else {
            CKRET(put_dev(h->ps.scale, 2 * sizeof(float) * (size_t)h->n_in_pad * h->n_chan));
            if (H.q_cols > 0)
                CKRET(put_dev(h->ps.C, sizeof(uint32_t) * (size_t)H.q_cols * (h->n_in_pad / 2) * h->n_chan));
        }
    }
    // queued results without a host image get one first
    bool imaged = false;
    for (const std::deque<int>* q : {&h->q_vis, &h->q_flag})
        for (int idx : *q)
            if (!h->slots[idx].has_image) {
                CKRET(slot_image(h, h->slots[idx]));
                imaged = true;
            }
    if (imaged) CK(cudaStreamSynchronize(h->s_out));
    for (int idx : h->q_vis) w.put(h->slots[idx].h_R, ne * sizeof(float2));
    for (int idx : h->q_flag) w.put(h->slots[idx].h_F, ne);
    if (buf && w.n > cap) return fail(h, CORR_EINVAL, "state buffer too small (" + std::to_string(w.n) + " bytes needed)");
    *size = w.n;
    return CORR_OK;
}

int corr_load_state(corr_t h, const void* buf, size_t size) {
    if (!h || h->is_group || !buf) return fail(h, CORR_EINVAL, "bad argument");
    if (h->started) return fail(h, CORR_ESTATE, "load a state into a new or reset handle");
    DeviceGuard dg(h->dev);
    const uint8_t* p = static_cast<const uint8_t*>(buf);
    size_t n = 0;
    auto get = [&](void* dst, size_t b) {
        if (n + b > size) return false;
        std::memcpy(dst, p + n, b);
        n += b;
        return true;
    };
    StateHeader H{};
    if (!get(&H, sizeof(H)) || std::memcmp(H.magic, kStateMagic, 8) != 0 || H.version != 2)
        return fail(h, CORR_EINVAL, "not a correlator state of this version");
    if (H.n_in != h->n_in || H.n_chan != h->n_chan || H.taps != h->taps || H.n_int != h->n_int ||
        H.precision != h->precision || H.es != h->es || H.iq != h->iq || H.window != h->window ||
        H.flag_window != h->flag_window || H.ring_mb != h->ring_mb || H.kaiser_beta != h->kaiser_beta ||
        H.flag_sigma != h->flag_sigma || H.max_delay != h->max_delay || H.chunk != h->chunk)
        return fail(h, CORR_EINVAL, "state of a correlator with another shape or other options");
    std::vector<double> v[6];
    for (auto& x : v) {
        x.assign(h->n_in, 0.0);
        if (!get(x.data(), sizeof(double) * h->n_in)) return fail(h, CORR_EINVAL, "truncated state");
    }
    h->tau = v[2];
    h->phi = v[3];
    h->tau_pend = v[4];
    h->phi_pend = v[5];
    h->pending = H.pending != 0;
    CKRET(upload_tables(h, h->tab_direct, h->tau, h->phi, h->s_comp));
    CKRET(upload_tables(h, h->tab_stream, v[0], v[1], h->s_comp));
    const size_t ne = vis_elems(h);
    const size_t per_spec = (size_t)h->n_chan * h->n_in_pad * sizeof(float2);
    if (H.stream_alloc) {
        CKRET(ensure_stream_alloc(h));
        if (H.v_cap != h->ps.v_cap || H.gpi != h->gpi || H.code_words != (h->precision != CORR_FP32) ||
            H.stage_cap != h->stage_cap ||
            H.stage_len > h->stage_cap)
            return fail(h, CORR_EINVAL, "state buffers do not match this handle's");
        auto get_dev = [&](void* dst, size_t b) -> int {
            if (n + b > size) return fail(h, CORR_EINVAL, "truncated state");
            CK(cudaMemcpy(dst, p + n, b, cudaMemcpyHostToDevice));
            n += b;
            return CORR_OK;
        };
        h->cur_buf = 0;
        h->d_stage = h->d_stage_buf[0];
        h->buf_read[0] = h->buf_read[1] = false;
        for (int a = 0; a < h->n_in; ++a)
            CKRET(get_dev(h->d_stage + (size_t)a * h->stage_cap * h->es, (size_t)H.stage_len * h->es));
        for (long long sp = H.s_xdone; sp < H.s_next; ++sp)
            CKRET(get_dev(reinterpret_cast<uint8_t*>(h->ps.V) + (size_t)(sp & (h->ps.v_cap - 1)) * per_spec, per_spec));
        if (h->precision == CORR_FP32) {
            CKRET(get_dev(h->ps.part, sizeof(float) * (size_t)h->gpi * h->nt * 32 * h->n_chan));
        } else {
            CKRET(get_dev(h->ps.scale, 2 * sizeof(float) * (size_t)h->n_in_pad * h->n_chan));
            if (H.q_cols > 0)
                CKRET(get_dev(h->ps.C, sizeof(uint32_t) * (size_t)H.q_cols * (h->n_in_pad / 2) * h->n_chan));
        }
        h->stage_base = H.stage_base;
        h->stage_len = H.stage_len;
        h->n_pushed = H.n_pushed;
        h->ps.s_next = H.s_next;
        h->ps.s_xdone = H.s_xdone;
        h->ps.have_scale = H.have_scale != 0;
    }
    // results not yet popped: the last max(n_vis_q, n_flag_q) integrations
    const int nq = H.n_vis_q > H.n_flag_q ? H.n_vis_q : H.n_flag_q;
    std::vector<std::vector<uint8_t>> vis(H.n_vis_q), fl(H.n_flag_q);
    for (auto& x : vis) {
        x.resize(ne * sizeof(float2));
        if (!get(x.data(), x.size())) return fail(h, CORR_EINVAL, "truncated state");
    }
    for (auto& x : fl) {
        x.resize(ne);
        if (!get(x.data(), x.size())) return fail(h, CORR_EINVAL, "truncated state");
    }
    if (nq > 0) CKRET(ensure_stream_alloc(h));
    for (int j = 0; j < nq; ++j) {
        int idx;
        CKRET(new_slot(h, &idx));
        Slot& sl = h->slots[idx];
        const int jv = j - (nq - H.n_vis_q), jf = j - (nq - H.n_flag_q);
        if (jv >= 0) {
            std::memcpy(sl.h_R, vis[jv].data(), vis[jv].size());
            CK(cudaMemcpy(sl.d_R, sl.h_R, vis[jv].size(), cudaMemcpyHostToDevice));
            sl.in_vis = true;
            h->q_vis.push_back(idx);
        }
        if (jf >= 0) {
            std::memcpy(sl.h_F, fl[jf].data(), fl[jf].size());
            CK(cudaMemcpy(sl.d_F, sl.h_F, fl[jf].size(), cudaMemcpyHostToDevice));
            sl.in_flag = true;
            h->q_flag.push_back(idx);
        }
        CK(cudaEventRecord(sl.ev, h->s_out));
        sl.has_image = true;
    }
    h->started = H.started != 0;
    h->flushed = H.flushed != 0;
    return CORR_OK;
}

int corr_device_status(corr_t h, int* status) {
    if (!h || !status) return fail(h, CORR_EINVAL, "NULL argument");
    DeviceGuard g(h->dev);
    CK(cudaDeviceSynchronize());
    CK(cudaMemcpy(status, h->d_status, sizeof(int), cudaMemcpyDeviceToHost));
    CK(cudaMemset(h->d_status, 0, sizeof(int)));
    return CORR_OK;
}

int corr_stage_times(corr_t h, double* ms, long long* counts, int n_stages) {
    if (!h) return fail(h, CORR_EINVAL, "NULL handle");
    DeviceGuard g(h->dev);
    for (int i = 0; i < kStages; ++i) {
        for (auto& pr : h->timer.open[i]) {
            CK(cudaEventSynchronize(pr.second));
            float t = 0.f;
            CK(cudaEventElapsedTime(&t, pr.first, pr.second));
            h->timer.ms[i] += t;
            ++h->timer.n[i];
            h->timer.pool.push_back(pr.first);
            h->timer.pool.push_back(pr.second);
        }
        h->timer.open[i].clear();
    }
    for (int i = 0; i < n_stages && i < kStages; ++i) {
        if (ms) ms[i] = h->timer.ms[i];
        if (counts) counts[i] = h->timer.n[i];
    }
    for (int i = 0; i < kStages; ++i) {
        h->timer.ms[i] = 0;
        h->timer.n[i] = 0;
    }
    return CORR_OK;
}

}  // extern "C"
