// Device code of the F-engine shared by its translation units (internal):
// the two-kernel path (fir_kernel, fft_kernel), the fused PFB + FFT kernel
// and the complex-input variants.
//
// F-engine (Sec. 4.2 "F-engine (PFB and FFT)"): int8 load with the coarse
// delay of Eq. 1 -> P-tap polyphase FIR -> M-point FFT.
//
// Two kernels.  fir_kernel streams the samples: a thread owns four branches
// m of one input pair over a run of consecutive spectra, converts every int8
// sample once, keeps the last P frames and its P x 4 filter taps in
// registers, and writes z[m] = y_a[m] + j y_b[m] (the pair's two real FIR
// outputs packed as one complex sequence).  fft_kernel transforms z with one
// M-point complex FFT and separates the two real spectra,
// Y_a[k] = (Z[k] + Z*[M-k]) / 2 and Y_b[k] = (Z[k] - Z*[M-k]) / 2j.
//
// The FFT is a Stockham autosort transform: the first pass reads z straight
// from global memory, later passes go through shared memory padded by one
// float2 every 16 (conflict-free strided passes); radix-16 passes plus one
// smaller first pass, 16 points per thread.  The fine-delay and phase
// rotation of Eq. 1 is constant within an integration, so the streaming
// pipeline applies it to the integrated visibilities (finalize_kernel) and
// fft_kernel stores U = 2Y; the stage entry point can still rotate here.
#pragma once

#include "corr.h"
#include "corr_internal.h"
#include "quant.cuh"
#include "tc_common.cuh"

#include <cudaTypedefs.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>


namespace corr {

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder();

namespace {

__device__ __forceinline__ int pidx(int i) { return i + (i >> 4); }

// Packed FP32 pairs (sm_100+): one add.rn.f32x2 / sub.rn.f32x2 per complex
// addition, the same IEEE result per lane as two scalar operations.
__device__ __forceinline__ unsigned long long f2u(float2 v) {
    return (unsigned long long)__float_as_uint(v.x) | ((unsigned long long)__float_as_uint(v.y) << 32);
}
__device__ __forceinline__ float2 u2f(unsigned long long u) {
    return make_float2(__uint_as_float((unsigned)u), __uint_as_float((unsigned)(u >> 32)));
}
__device__ __forceinline__ float2 add2(float2 a, float2 b) {
    unsigned long long r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(f2u(a)), "l"(f2u(b)));
    return u2f(r);
}
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
    unsigned long long r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(f2u(a)), "l"(f2u(b)));
    return u2f(r);
}

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

// v * W_R^K with W_R = exp(-2 pi j / R), R dividing 16; trivial factors free.
template <int K, int R>
__device__ __forceinline__ float2 twc(float2 v) {
    constexpr int q = (K * (16 / R)) % 16;
    constexpr float h = 0.70710678118654752f;
    constexpr float c1 = 0.92387953251128676f, s1 = 0.38268343236508977f;
    if constexpr (q == 0) return v;
    else if constexpr (q == 4) return make_float2(v.y, -v.x);
    else if constexpr (q == 8) return make_float2(-v.x, -v.y);
    else if constexpr (q == 12) return make_float2(-v.y, v.x);
    else if constexpr (q == 2) return make_float2((v.x + v.y) * h, (v.y - v.x) * h);
    else if constexpr (q == 6) return make_float2((v.y - v.x) * h, -(v.x + v.y) * h);
    else if constexpr (q == 10) return make_float2(-(v.x + v.y) * h, (v.x - v.y) * h);
    else if constexpr (q == 14) return make_float2((v.x - v.y) * h, (v.x + v.y) * h);
    else {
        // exp(-2 pi j q / 16) = c - j s
        constexpr float c = (q == 1 || q == 15) ? c1 : (q == 3 || q == 13) ? s1
                          : (q == 5 || q == 11) ? -s1 : -c1;
        constexpr float s = (q == 1 || q == 7) ? s1 : (q == 3 || q == 5) ? c1
                          : (q == 9 || q == 15) ? -s1 : -c1;
        return make_float2(fmaf(v.x, c, v.y * s), fmaf(v.y, c, -v.x * s));
    }
}

// In-register R-point DFT by radix-2 decimation in frequency; on return
// v[bitrev(q)] holds X[q] = sum_r v_in[r] W_R^{rq}.  Written as template
// recursion so every index is a compile-time constant (registers only).
template <int R, int H, int BI>
struct DifButterfly {
    static __device__ __forceinline__ void run(float2 (&v)[R]) {
        constexpr int blk = BI / H;
        constexpr int j = BI % H;
        constexpr int i0 = blk * 2 * H + j;
        constexpr int i1 = i0 + H;
        const float2 u = v[i0], w = v[i1];
        v[i0] = make_float2(u.x + w.x, u.y + w.y);
        v[i1] = twc<j, 2 * H>(make_float2(u.x - w.x, u.y - w.y));
        if constexpr (BI + 1 < R / 2) DifButterfly<R, H, BI + 1>::run(v);
    }
};

template <int R, int H>
struct DifStage {
    static __device__ __forceinline__ void run(float2 (&v)[R]) {
        DifButterfly<R, H, 0>::run(v);
        if constexpr (H > 1) DifStage<R, H / 2>::run(v);
    }
};

template <int R>
__device__ __forceinline__ void dft_dif(float2 (&v)[R]) {
    DifStage<R, R / 2>::run(v);
}

template <int R>
__host__ __device__ constexpr int bitrev(int q) {
    int r = 0;
    for (int b = 1, t = R >> 1; b < R; b <<= 1, t >>= 1)
        if (q & b) r |= t;
    return r;
}

// z[pidx(o + q Ns)] = X[q] = v[bitrev(q)] for q = Q .. R-1.  When Ns is a
// multiple of 16 the padded index is linear in q (one base register).
template <int R, int NS, int Q>
struct StoreBitrev {
    static __device__ __forceinline__ void run(float2* z, const float2 (&v)[R], int o, int po) {
        if constexpr (NS % 16 == 0) z[po + Q * (NS + NS / 16)] = v[bitrev<R>(Q)];
        else z[pidx(o + Q * NS)] = v[bitrev<R>(Q)];
        if constexpr (Q + 1 < R) StoreBitrev<R, NS, Q + 1>::run(z, v, o, po);
    }
};

// One Stockham pass of radix R over M points: butterfly j reads
// x[j + r M/R], multiplies by W_{Ns R}^{r (j mod Ns)}, transforms, and
// writes z[(j - j mod Ns) R + j mod Ns + r Ns] (padded shared buffer).  Each
// of the M/16 active threads owns 16 / R butterflies (16 points).  With
// GLOBAL_IN the inputs come from the unpadded global array `gin`.
__host__ __device__ constexpr int first_radix(int M) {
    int l = 0;
    while ((1 << l) < M) ++l;
    return (l % 4) == 0 ? 16 : (1 << (l % 4));
}

// Offset of the radix-16 pass with stride NS in the twiddle table: the sum
// of 16 * Ns' over the earlier radix-16 passes.
__host__ __device__ constexpr int tw_offset(int M, int NS) {
    int off = 0;
    int ns = first_radix(M) == 16 ? 1 : first_radix(M);
    if (first_radix(M) == 16 && NS == 1) return 0;
    if (first_radix(M) == 16) {
        off += 16 * 1;
        ns = 16;
    }
    while (ns < NS) {
        off += 16 * ns;
        ns *= 16;
    }
    return off;
}

// Twiddle sources of a Stockham pass.
enum { TW_NONE = 0, TW_SMEM = 1, TW_REG = 2, TW_GLOBAL = 3 };

// Butterflies of one Stockham pass of radix R on the 16 points v a thread
// holds: butterfly j = tid + b NACT multiplies input r by W_{16 Ns}^{r k}
// (k = j mod Ns), transforms, and writes z[(j - k) R + k + q Ns] (padded).
// Twiddles come from the shared table `tws` ([r][k], offset TWO) or, for
// the last pass, from the thread's registers `twr` (k = tid there).
template <int M, int R, int NS, int TWM>
__device__ __forceinline__ void pass_compute_store(float2* z, const float2 (&v)[16], const float2* tws,
                                                   const float2 (&twr)[15], int tid,
                                                   const float2* __restrict__ gtw = nullptr) {
    constexpr int B = 16 / R;
    constexpr int NACT = M / 16;
    constexpr int TWO = tw_offset(M, NS);
#pragma unroll
    for (int b = 0; b < B; ++b) {
        const int j = tid + b * NACT;
        const int k = j & (NS - 1);
        float2 u[R];
#pragma unroll
        for (int r = 0; r < R; ++r) u[r] = v[b * R + r];
        if constexpr (TWM == TW_SMEM) {
            static_assert(R == 16, "twiddled passes are radix 16");
#pragma unroll
            for (int r = 1; r < R; ++r) u[r] = cmul(u[r], tws[TWO + r * NS + k]);
        } else if constexpr (TWM == TW_REG) {
            static_assert(R == 16 && B == 1, "register twiddles: last radix-16 pass");
#pragma unroll
            for (int r = 1; r < R; ++r) u[r] = cmul(u[r], twr[r - 1]);
        } else if constexpr (TWM == TW_GLOBAL) {
            static_assert(R == 16, "twiddled passes are radix 16");
#pragma unroll
            for (int r = 1; r < R; ++r) u[r] = cmul(u[r], __ldg(gtw + TWO + r * NS + k));
        }
        dft_dif<R>(u);
        const int o = (j - k) * R + k;
        StoreBitrev<R, NS, 0>::run(z, u, o, pidx(o));
    }
}

// First-pass inputs of a thread: x[tid + b NACT + r M/R0] from global memory.
template <int M>
__device__ __forceinline__ void load_first(float2 (&v)[16], const float2* __restrict__ gin, int tid) {
    constexpr int R = first_radix(M);
    constexpr int B = 16 / R;
    constexpr int NACT = M / 16;
    constexpr int NR = M / R;
    if (tid < NACT) {
#pragma unroll
        for (int b = 0; b < B; ++b)
#pragma unroll
            for (int r = 0; r < R; ++r) v[b * R + r] = __ldg(gin + tid + b * NACT + r * NR);
    }
}

// Inputs of a later (radix-16) pass from the padded shared buffer.
template <int M>
__device__ __forceinline__ void load_smem(float2 (&v)[16], const float2* z, int tid) {
    constexpr int NR = M / 16;
    if constexpr (M >= 256) {
        // tid + r NR with NR a multiple of 16.
        const int pb = pidx(tid);
#pragma unroll
        for (int r = 0; r < 16; ++r) v[r] = z[pb + r * NR / 16 * 17];
    } else {
#pragma unroll
        for (int r = 0; r < 16; ++r) v[r] = z[pidx(tid + r * NR)];
    }
}

// Radix-16 passes from shared memory, Ns = NS .. M/16.  The last one takes
// its twiddles from registers (REGTW) or from the global table, the others
// from the shared copy of the table.
template <int M, int NS, bool REGTW>
__device__ __forceinline__ void later_passes(float2* z, const float2* tws, const float2 (&twr)[15], int tid,
                                             const float2* __restrict__ gtw) {
    if constexpr (NS < M) {
        constexpr bool last = (NS * 16 == M);
        float2 v[16];
        if (tid < M / 16) load_smem<M>(v, z, tid);
        __syncthreads();
        if (tid < M / 16) {
            if constexpr (last && REGTW) pass_compute_store<M, 16, NS, TW_REG>(z, v, tws, twr, tid);
            else if constexpr (last) pass_compute_store<M, 16, NS, TW_GLOBAL>(z, v, tws, twr, tid, gtw);
            else pass_compute_store<M, 16, NS, TW_SMEM>(z, v, tws, twr, tid);
        }
        __syncthreads();
        later_passes<M, NS * 16, REGTW>(z, tws, twr, tid, gtw);
    }
}

// The same passes between two padded buffers (ping-pong): each pass loads
// from zin and stores to zout, so one barrier per pass suffices.  Returns
// the buffer that holds the result.
// With STG, thread 0 waits before the last barrier until the bulk stores
// issued from the staging buffer have read it (the epilogue rewrites it).
template <int M, int NS, bool REGTW, bool STG>
__device__ __forceinline__ float2* later_passes_pp(float2* zin, float2* zout, const float2* tws,
                                                   const float2 (&twr)[15], int tid,
                                                   const float2* __restrict__ gtw) {
    if constexpr (NS < M) {
        constexpr bool last = (NS * 16 == M);
        if (tid < M / 16) {
            float2 v[16];
            load_smem<M>(v, zin, tid);
            if constexpr (last && REGTW) pass_compute_store<M, 16, NS, TW_REG>(zout, v, tws, twr, tid);
            else if constexpr (last) pass_compute_store<M, 16, NS, TW_GLOBAL>(zout, v, tws, twr, tid, gtw);
            else pass_compute_store<M, 16, NS, TW_SMEM>(zout, v, tws, twr, tid);
        }
        if constexpr (STG && last) {
            if (tid == 0) tc::bulk_wait_read_all();
        }
        __syncthreads();
        return later_passes_pp<M, NS * 16, REGTW, STG>(zout, zin, tws, twr, tid, gtw);
    } else {
        return zin;
    }
}

// Radix-16 passes after a first pass of radix R0.
__host__ __device__ constexpr int n_later_passes(int M, int R0) {
    int n = 0;
    for (int ns = R0; ns < M; ns *= 16) ++n;
    return n;
}

// Entries of the twiddle table kept in shared memory: every pass but the
// last (whose twiddles are in registers or read from global memory).
template <int M>
__host__ __device__ constexpr int tw_smem_entries() {
    return M <= 16 ? 16 : tw_offset(M, M / 16);
}

constexpr int kFirThreads = 256;

// Per-input state of one FIR thread: an aligned word pointer at frame 0 for
// branches m0..m0+3 shifted by the coarse delay, the bit offset inside the
// word, and the frames [f_lo, f_hi] whose words lie inside the valid window
// (no bounds checks needed there).  Four samples are one 32-bit raw word for
// int8 input (two words read) and a pair of words for int16 (three read).
struct FirInput {
    const uint32_t* q;
    int sh;
    long long f_lo, f_hi;
    long long n0;             // stream index of branch m0 at frame 0 (with delay)
    int in;
    bool has;
};

template <int ES>
struct Raw4;
template <>
struct Raw4<1> {
    using T = uint32_t;
};
template <>
struct Raw4<2> {
    using T = uint2;
};

template <int ES>
__device__ __forceinline__ FirInput fir_input(const FirArgs& A, int in, bool has, int m0, int d) {
    constexpr int kWords = ES == 1 ? 2 : 3;          // words a raw value reads
    FirInput r;
    r.in = in;
    r.has = has;
    r.n0 = (long long)m0 + d;
    const long long lo = A.src.base > 0 ? A.src.base : 0;
    const int8_t* p0 = A.src.x + ((long long)in * A.src.stride - A.src.base + r.n0) * ES;   // frame 0
    const int c = (int)(reinterpret_cast<uintptr_t>(p0) & 3);
    r.q = reinterpret_cast<const uint32_t*>(p0 - c);
    r.sh = 8 * c;
    // frame f is safe when its words, bytes (n0 + f M) ES - c .. + 4 kWords,
    // lie in [lo ES, vhi ES); M ES = 2^(lgM + ES - 1), so ceil / floor
    // division are arithmetic shifts.
    const int lg = A.lgM + (ES - 1);
    const long long a_lo = lo * ES - r.n0 * ES + c;
    const long long a_hi = A.src.vhi * ES - 4 * kWords - r.n0 * ES + c;
    r.f_lo = (a_lo + ((long long)A.M * ES) - 1) >> lg;
    r.f_hi = a_hi >> lg;
    if (!has) {
        r.f_lo = -(1LL << 62);
        r.f_hi = 1LL << 62;
    }
    return r;
}

// Four samples of one input row from stream index n, each read only inside
// [lo, vhi) (zero elsewhere), packed as the raw value of the fast path.  Out
// of line: only the first and last frames of a stream take this path.
__device__ __noinline__ uint32_t load4_checked8(const int8_t* row, long long lo, long long vhi, long long n) {
    uint32_t v = 0;
    for (int b = 0; b < 4; ++b) {
        const long long i = n + b;
        if (i >= lo && i < vhi) v |= (uint32_t)(uint8_t)row[i] << (8 * b);
    }
    return v;
}

__device__ __noinline__ uint2 load4_checked16(const int16_t* row, long long lo, long long vhi, long long n) {
    uint32_t v[2] = {0u, 0u};
    for (int b = 0; b < 4; ++b) {
        const long long i = n + b;
        if (i >= lo && i < vhi) v[b >> 1] |= (uint32_t)(uint16_t)row[i] << (16 * (b & 1));
    }
    return make_uint2(v[0], v[1]);
}

// Raw value (4 branches) of frame f of one input; zero before the stream.
template <int ES>
__device__ __forceinline__ typename Raw4<ES>::T fir_word(const FirArgs& A, const FirInput& I, long long f) {
    using R = typename Raw4<ES>::T;
    R w{};
    if (I.has && f >= 0) {
        const long long lo = A.src.base > 0 ? A.src.base : 0;
        const long long n = f * A.M + I.n0;
        if (f >= I.f_lo && f <= I.f_hi) {
            const uint32_t* q = I.q + ((f * A.M * ES) >> 2);
            if constexpr (ES == 1) {
                w = __funnelshift_r(__ldg(q), __ldg(q + 1), I.sh);
            } else {
                const uint32_t a = __ldg(q), b = __ldg(q + 1), c = __ldg(q + 2);
                w = make_uint2(__funnelshift_r(a, b, I.sh), __funnelshift_r(b, c, I.sh));
            }
        } else if constexpr (ES == 1) {
            w = load4_checked8(A.src.x + (long long)I.in * A.src.stride - A.src.base, lo, A.src.vhi, n);
        } else {
            w = load4_checked16(reinterpret_cast<const int16_t*>(A.src.x) + (long long)I.in * A.src.stride -
                                    A.src.base,
                                lo, A.src.vhi, n);
        }
    }
    return w;
}

// Packed FP32 fused multiply-add: two lanes of one 64-bit register.
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {
    unsigned long long r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(f2u(a)), "l"(f2u(b)), "l"(f2u(c)));
    return u2f(r);
}

// Exact int8 -> float for four packed samples as two float pairs: flip each
// byte's sign bit, place it in the low mantissa bits of 2^23, and subtract
// 2^23 + 128 with one packed subtraction per pair.
__device__ __forceinline__ void unpack4x2(uint32_t w, float2& lo, float2& hi) {
    const uint32_t f = w ^ 0x80808080u;
    const float2 bias = make_float2(8388736.0f, 8388736.0f);
    lo = sub2(make_float2(__int_as_float((int)__byte_perm(f, 0x4B000000u, 0x7440)),
                          __int_as_float((int)__byte_perm(f, 0x4B000000u, 0x7441))), bias);
    hi = sub2(make_float2(__int_as_float((int)__byte_perm(f, 0x4B000000u, 0x7442)),
                          __int_as_float((int)__byte_perm(f, 0x4B000000u, 0x7443))), bias);
}

// Exact int16 -> float for two packed samples: flip each sample's sign bit,
// place it in the low 16 mantissa bits of 2^23, subtract 2^23 + 32768.
__device__ __forceinline__ float2 unpack2x16(uint32_t w) {
    const uint32_t f = w ^ 0x80008000u;
    return sub2(make_float2(__int_as_float((int)__byte_perm(f, 0x4B000000u, 0x7610)),
                            __int_as_float((int)__byte_perm(f, 0x4B000000u, 0x7632))),
                make_float2(8421376.0f, 8421376.0f));
}

// Complex int8 samples, (I, Q) bytes interleaved: the I (c = 0) or Q (c = 1)
// parts of the four complex samples held in w, exact (see unpack4x2).
__device__ __forceinline__ void unpack_iq(uint2 w, int c, float2& lo, float2& hi) {
    const uint32_t f = w.x ^ 0x80808080u, g = w.y ^ 0x80808080u;
    const uint32_t s0 = 0x7440u + (uint32_t)c, s1 = 0x7442u + (uint32_t)c;
    const float2 bias = make_float2(8388736.0f, 8388736.0f);
    lo = sub2(make_float2(__int_as_float((int)__byte_perm(f, 0x4B000000u, s0)),
                          __int_as_float((int)__byte_perm(f, 0x4B000000u, s1))), bias);
    hi = sub2(make_float2(__int_as_float((int)__byte_perm(g, 0x4B000000u, s0)),
                          __int_as_float((int)__byte_perm(g, 0x4B000000u, s1))), bias);
}

__device__ __forceinline__ void unpack_raw(uint32_t w, float2& lo, float2& hi) { unpack4x2(w, lo, hi); }
__device__ __forceinline__ void unpack_raw(uint2 w, float2& lo, float2& hi) {
    lo = unpack2x16(w.x);
    hi = unpack2x16(w.y);
}

// y_s[m] = sum_p h[pM + m] x'[(s - P + 1 + p) M + m] for 4 branches of one
// input over spectra [s_lo, s_hi).  Lanes 2q and 2q+1 of a warp take the
// same branches of the two inputs of a pair and swap half their outputs with
// one shuffle each, so that every lane stores two packed points
// z[m] = (y_a[m], y_b[m]) as one 16-byte word.  The window holds frames
// s-P+1 .. s in a circular register array indexed at compile time: spectra
// are processed in blocks of P so frame f always sits in slot (f - base) mod
// P.  Inside the frames whose words are in bounds for this thread the block
// loop runs without checks; ring slots advance in 32-bit arithmetic.
// IQ: complex input (ES = 2 bytes per complex int8 sample); lanes 2q and
// 2q+1 take the I and the Q parts of the same input, so z = y_I + j y_Q.
template <int P, int ES, bool IQ = false>
__global__ void __launch_bounds__(kFirThreads, P <= 4 ? 3 : (P <= 8 ? 2 : 1)) fir_kernel(const FirArgs A) {
    static_assert(!IQ || ES == 2, "complex int8 samples are two bytes");
    using R = typename Raw4<ES>::T;
    const int M = A.M;
    const int t = blockIdx.x * kFirThreads + threadIdx.x;   // (branch group, input of pair)
    if (t >= (M >> 1)) return;
    const int odd = t & 1;
    const int m0 = 4 * (t >> 1);
    const int pair = blockIdx.y;
    const int in = IQ ? pair : 2 * pair + odd;
    const long long s_lo = A.s_begin + (long long)blockIdx.z * A.spt;
    long long s_hi = s_lo + A.spt;
    if (s_hi > A.s_end) s_hi = A.s_end;
    if (s_lo >= s_hi) return;   // uniform over the CTA
    const bool has = in < A.n_in;
    const FirInput I = fir_input<ES>(A, in, has, m0, has ? A.coarse[in] : 0);

    float2 h[P][2];
#pragma unroll
    for (int p = 0; p < P; ++p) {
        const float4 v = __ldg(reinterpret_cast<const float4*>(A.h + (size_t)p * M + m0));
        h[p][0] = make_float2(v.x, v.y);
        h[p][1] = make_float2(v.z, v.w);
    }
    float2 w[P][2];
    const long long base_f = s_lo - (P - 1);
#pragma unroll
    for (int q = 0; q < P - 1; ++q) {
        if constexpr (IQ) unpack_iq(fir_word<ES>(A, I, base_f + q), odd, w[q][0], w[q][1]);
        else unpack_raw(fir_word<ES>(A, I, base_f + q), w[q][0], w[q][1]);
    }
    // even lanes store branches m0, m0+1; odd lanes m0+2, m0+3
    float2* const zp = A.Z + (size_t)pair * M + m0 + 2 * odd;
    const unsigned zstride = (unsigned)(A.n_pairs * M);
    const unsigned zmask = (unsigned)A.z_mask;
    unsigned slot = (unsigned)((s_lo - A.z_origin) & A.z_mask);
    const int step = (M * ES) >> 2;                 // words per frame
    // frames s0 .. s0+P-1 are unchecked when all lie in [f_safe_lo, f_safe_hi]
    const long long f_safe_lo = I.f_lo < 0 ? 0 : I.f_lo;
    long long s_fast_end = I.f_hi - (P - 1) + 1;        // blocks starting below this are safe
    if (s_fast_end > s_hi - (P - 1)) s_fast_end = s_hi - (P - 1);

    auto emit = [&](int q, R word) {
        if constexpr (IQ) unpack_iq(word, odd, w[(q + P - 1) % P][0], w[(q + P - 1) % P][1]);
        else unpack_raw(word, w[(q + P - 1) % P][0], w[(q + P - 1) % P][1]);
        float2 y0 = make_float2(0.f, 0.f), y1 = make_float2(0.f, 0.f);
#pragma unroll
        for (int p = 0; p < P; ++p) {
            const int sl = (q + p) % P;            // frame s - P + 1 + p
            y0 = fma2(h[p][0], w[sl][0], y0);
            y1 = fma2(h[p][1], w[sl][1], y1);
        }
        const float x0 = __shfl_xor_sync(0xffffffffu, odd ? y0.x : y1.x, 1);
        const float x1 = __shfl_xor_sync(0xffffffffu, odd ? y0.y : y1.y, 1);
        const float4 o = odd ? make_float4(x0, y1.x, x1, y1.y) : make_float4(y0.x, x0, y0.y, x1);
        *reinterpret_cast<float4*>(zp + (size_t)slot * zstride) = o;
        slot = (slot + 1) & zmask;
    };

    long long s0 = s_lo;
    if (has && s0 >= f_safe_lo) {
        const uint32_t* qp = I.q + ((s0 * M * ES) >> 2);
        for (; s0 < s_fast_end; s0 += P) {
            R r[P];
#pragma unroll
            for (int q = 0; q < P; ++q) {
                if constexpr (ES == 1) {
                    r[q] = __funnelshift_r(__ldg(qp + q * step), __ldg(qp + q * step + 1), I.sh);
                } else {
                    const uint32_t a = __ldg(qp + q * step), b = __ldg(qp + q * step + 1), c = __ldg(qp + q * step + 2);
                    r[q] = make_uint2(__funnelshift_r(a, b, I.sh), __funnelshift_r(b, c, I.sh));
                }
            }
            qp += P * step;
#pragma unroll
            for (int q = 0; q < P; ++q) emit(q, r[q]);
        }
    }
    for (; s0 < s_hi; s0 += P) {
        R r[P];
#pragma unroll
        for (int q = 0; q < P; ++q) r[q] = (s0 + q < s_hi) ? fir_word<ES>(A, I, s0 + q) : R{};
#pragma unroll
        for (int q = 0; q < P; ++q)
            if (s0 + q < s_hi) emit(q, r[q]);   // uniform over the CTA
    }
}

template <int M>
struct FftCfg {
    static constexpr int NACT = M / 16;
    static constexpr int THREADS = NACT < 32 ? 32 : NACT;
    // With at most 512 threads the last pass's 15 twiddles (fixed per thread)
    // stay in registers and the next spectrum's first-pass input is
    // prefetched; one CTA per SM then has up to 128 registers per thread.
    static constexpr bool REGTW = (M >= 32) && NACT <= 512;
    static constexpr int TWS = tw_smem_entries<M>();
    static constexpr int ZB = M + M / 16 + 1;                 // padded buffer entries
    // Two buffers (one barrier per pass) while they fit with the table.
    static constexpr bool PP = M <= 8192;
    // With an odd number of radix-16 passes the result lands in the second
    // buffer, which the next spectrum's first pass does not write: no barrier
    // is needed between one spectrum's epilogue and the next first pass.
    static constexpr bool RES_ALT = PP && (n_later_passes(M, first_radix(M)) % 2 == 1);
    // 512 <= M <= 4096, spectra out (modes 0, 1): two input pairs per CTA,
    // one transform per THREADS-thread group, whose spectra leave through a
    // shared staging buffer [n_chan][2] of float4 by 2D bulk tensor stores of
    // BOXR channels -- 32 contiguous bytes (a whole sector) per channel.
    // Elsewhere one pair per CTA stores its 16 bytes per channel directly.
    static constexpr bool TMA_OUT = PP && M >= 512 && M <= 4096;
    static constexpr int BOXR = (M / 2) < 256 ? (M / 2) : 256;
    __host__ __device__ static constexpr int pairs(int mode) { return (TMA_OUT && mode <= 1) ? 2 : 1; }
    __host__ __device__ static constexpr int threads(int mode) { return THREADS * pairs(mode); }
    // CTAs per SM the register budget is held to (128 registers a thread)
    __host__ __device__ static constexpr int minb(int mode) { return threads(mode) >= 512 ? 1 : 65536 / 128 / threads(mode); }
    __host__ __device__ static constexpr size_t smem_bytes(int mode) {
        return sizeof(float2) * (size_t)(pairs(mode) * (PP ? 2 : 1) * ZB + TWS) +
               ((TMA_OUT && mode <= 1) ? (size_t)(M / 2) * 16 * pairs(mode) + 128 : 0);
    }
};

template <int M>
__device__ __forceinline__ const float2* fft_input(const FftArgs& A, long long s, int pair, int n_pairs) {
    const long long zs = (s - A.z_origin) & A.z_mask;
    return A.Z + ((size_t)zs * n_pairs + pair) * M;
}

// MODE 0: store U = 2Y; 1: store the rotated V; 2: accumulate power tiles;
// 3: store U = 2Y pair-major ([slot][pair][n_chan] float4); 4 / 5: complex
// input; 6 / 7: int8 / e4m3 code words of U (pair-major, as the fused
// kernel writes them).
template <int M, int MODE>
__global__ void __launch_bounds__(FftCfg<M>::threads(MODE), FftCfg<M>::minb(MODE))
    fft_kernel(const FftArgs A, const __grid_constant__ CUtensorMap vmap) {
    using C = FftCfg<M>;
    constexpr bool STG = C::TMA_OUT && MODE <= 1;
    constexpr int P = C::pairs(MODE);                 // input pairs (transforms) per CTA
    extern __shared__ float2 smem[];
    // group g of THREADS threads transforms pair blockIdx.y * P + g
    const int g = P > 1 ? (int)threadIdx.x / C::THREADS : 0;
    const int tid = (int)threadIdx.x - g * C::THREADS;
    float2* zbuf = smem + (size_t)g * (C::PP ? 2 : 1) * C::ZB;
    float2* zalt = zbuf + C::ZB;                      // second buffer (C::PP)
    float2* tws = smem + (size_t)P * (C::PP ? 2 : 1) * C::ZB;
    // staging buffer of one spectrum's output [n_chan][P], 128-byte aligned (STG)
    float4* stg = nullptr;
    if constexpr (STG) {
        char* p = reinterpret_cast<char*>(tws + C::TWS);
        const uint32_t b = tc::smem_u32(p);
        stg = reinterpret_cast<float4*>(p + (((b + 127u) & ~127u) - b));
    }
    constexpr int n_chan = M >> 1;
    constexpr int R0 = first_radix(M);
    const int pair = (int)blockIdx.y * P + g;
    const int n_pairs = (int)gridDim.y * P;
    const int a = 2 * pair;
    const long long s_lo = A.s_begin + (long long)blockIdx.x * A.spt;
    long long s_hi = s_lo + A.spt;
    if (s_hi > A.s_end) s_hi = A.s_end;
    if (s_lo >= s_hi) return;

    for (int i = (int)threadIdx.x; i < C::TWS; i += blockDim.x) tws[i] = __ldg(A.tw + i);
    float2 twr[15];
    if constexpr (C::REGTW) {
        constexpr int NSL = M / 16;
        constexpr int TWL = tw_offset(M, NSL);
        if (tid < C::NACT) {
#pragma unroll
            for (int r = 1; r < 16; ++r) twr[r - 1] = __ldg(A.tw + TWL + r * NSL + tid);
        }
    }
    __syncthreads();

    // power mode: channels tid + i blockDim per thread
    constexpr int PCH = MODE == 2 ? ((n_chan + C::THREADS - 1) / C::THREADS) : 1;
    float pa[PCH], pb[PCH];
#pragma unroll
    for (int i = 0; i < PCH; ++i) pa[i] = pb[i] = 0.f;
    // Bulk stores of the staged spectrum in slot `sl` (thread 0, after a
    // barrier that follows every thread's staging writes and proxy fence).
    auto store_staged = [&](long long sl) {
        for (int b = 0; b < n_chan / C::BOXR; ++b)
            tc::tma_store_2d(&vmap, stg + b * C::BOXR * P, 4 * P * (int)blockIdx.y, (int)(sl * n_chan + b * C::BOXR));
        tc::bulk_commit();
    };
    long long prev_slot = -1;

    float2 cur[16];
    load_first<M>(cur, fft_input<M>(A, s_lo, pair, n_pairs), tid);
    for (long long s = s_lo; s < s_hi; ++s) {
        float2 nxt[16];
        if constexpr (C::REGTW) {
            if (s + 1 < s_hi) load_first<M>(nxt, fft_input<M>(A, s + 1, pair, n_pairs), tid);
        }
        // first pass (Ns = 1, no twiddles) straight from the global input
        if (tid < C::NACT) pass_compute_store<M, R0, 1, TW_NONE>(zbuf, cur, tws, twr, tid);
        __syncthreads();
        if constexpr (STG) {
            // the previous spectrum is staged and fenced by every thread
            if (threadIdx.x == 0 && prev_slot >= 0) store_staged(prev_slot);
        }
        const float2* zres = zbuf;
        if constexpr (C::PP) {
            zres = later_passes_pp<M, R0, C::REGTW, STG>(zbuf, zalt, tws, twr, tid, A.tw);
        } else {
            later_passes<M, R0, C::REGTW>(zbuf, tws, twr, tid, A.tw);
        }
        if constexpr (MODE == 2) {
            // |Y_a|^2 = |S|^2 / 4, |Y_b|^2 = |D|^2 / 4, summed over the row
#pragma unroll
            for (int i = 0; i < PCH; ++i) {
                const int k = tid + i * (int)blockDim.x;
                if (k < n_chan) {
                    const float2 zk = zres[pidx(k)];
                    const float2 zm = zres[pidx((M - k) & (M - 1))];
                    const float sx = zk.x + zm.x, sy = zk.y - zm.y;
                    const float dx = zk.x - zm.x, dy = zk.y + zm.y;
                    pa[i] = fmaf(sx, sx, fmaf(sy, sy, pa[i]));
                    pb[i] = fmaf(dx, dx, fmaf(dy, dy, pb[i]));
                }
            }
            const long long row = s / A.n_row;
            if (s + 1 == s_hi || (s + 1) % A.n_row == 0) {
                const float sc = 0.25f / (float)A.n_row;
                const int n_cb = n_chan / 256, n_rb = A.rows / 64;
#pragma unroll
                for (int i = 0; i < PCH; ++i) {
                    const int k = tid + i * (int)blockDim.x;
                    if (k < n_chan) {
                        const size_t px = (size_t)(row % 64) * 256 + (k % 256);
                        if (a < A.n_in) {
                            const size_t ta = ((size_t)a * n_rb + row / 64) * n_cb + k / 256;
                            atomicAdd(A.tiles + ta * 16384 + px, pa[i] * sc);
                        }
                        if (a + 1 < A.n_in) {
                            const size_t tb = ((size_t)(a + 1) * n_rb + row / 64) * n_cb + k / 256;
                            atomicAdd(A.tiles + tb * 16384 + px, pb[i] * sc);
                        }
                    }
                    pa[i] = 0.f;
                    pb[i] = 0.f;
                }
            }
        } else if constexpr (MODE >= 6) {
            // codes (6 int8, 7 e4m3): the fused F-engine's epilogue -- the
            // requantiser's arithmetic on U = 2Y, one word of the pair's four
            // codes per channel, consecutive channels across the threads
            constexpr bool FP8 = MODE == 7;
            const long long slot = (s - A.v_origin) & A.v_mask;
            uint32_t* const Cout = reinterpret_cast<uint32_t*>(A.V) + ((size_t)slot * n_pairs + pair) * n_chan;
            const float* const inv0 = A.inv + (size_t)a * n_chan;
            const float* const inv1 = inv0 + n_chan;
            const bool has0 = a < A.n_in, has1 = a + 1 < A.n_in;
            for (int k = tid; k < n_chan; k += C::THREADS) {
                const float2 zk = zres[pidx(k)];
                const float2 zm = zres[pidx((M - k) & (M - 1))];
                const float ia = has0 ? __ldg(inv0 + k) : 0.f;
                const float ib = has1 ? __ldg(inv1 + k) : 0.f;
                const float sx = zk.x + zm.x, sy = zk.y - zm.y;
                const float dx = zk.x - zm.x, dy = zk.y + zm.y;
                Cout[k] = q_code<FP8>(sx * ia) | (q_code<FP8>(sy * ia) << 8) | (q_code<FP8>(dy * ib) << 16) |
                          (q_code<FP8>(-dx * ib) << 24);
            }
        } else if constexpr (MODE >= 4) {
            // complex input: all M channels of input `pair`, channel-major
            // (n_chan = M), U = 2Z (4) or the rotated V = Z P (5)
            const long long slot = (s - A.v_origin) & A.v_mask;
            float2* Vout = A.V + (size_t)slot * M * A.n_in_pad + pair;
            for (int k = tid; k < M; k += C::THREADS) {
                const float2 zk = zres[pidx(k)];
                float2 out;
                if constexpr (MODE == 5) out = cmul(zk, __ldg(A.phasor + (size_t)pair * M + k));
                else out = make_float2(2.f * zk.x, 2.f * zk.y);
                Vout[(size_t)k * A.n_in_pad] = out;
            }
        } else {
            const long long slot = (s - A.v_origin) & A.v_mask;
            // channel k of the pair at Vout[k * vstride]
            float4* Vout;
            size_t vstride;
            if constexpr (MODE == 3) {
                Vout = reinterpret_cast<float4*>(A.V) + ((size_t)slot * n_pairs + pair) * n_chan;
                vstride = 1;
            } else {
                Vout = reinterpret_cast<float4*>(A.V + (size_t)slot * n_chan * A.n_in_pad + a);
                vstride = (size_t)(A.n_in_pad >> 1);
            }
            for (int k = tid; k < n_chan; k += C::THREADS) {
                const float2 zk = zres[pidx(k)];
                const float2 zm = zres[pidx((M - k) & (M - 1))];
                const float2 S = make_float2(zk.x + zm.x, zk.y - zm.y);
                const float2 D = make_float2(zk.x - zm.x, zk.y + zm.y);
                float4 out;
                if constexpr (MODE == 1) {
                    const float2 va = cmul(S, __ldg(A.phasor + (size_t)a * n_chan + k));
                    const float2 vb = cmul(D, __ldg(A.phasor + (size_t)(a + 1) * n_chan + k));
                    out = make_float4(va.x, va.y, vb.x, vb.y);
                } else {
                    out = make_float4(S.x, S.y, D.y, -D.x);
                }
                if constexpr (STG) stg[k * P + g] = out;
                else Vout[(size_t)k * vstride] = out;
            }
            if constexpr (STG) {
                tc::fence_proxy_async_smem();
                prev_slot = slot;
            }
        }
        if constexpr (!C::RES_ALT) __syncthreads();
        if constexpr (C::REGTW) {
#pragma unroll
            for (int i = 0; i < 16; ++i) cur[i] = nxt[i];
        } else {
            if (s + 1 < s_hi) load_first<M>(cur, fft_input<M>(A, s + 1, pair, n_pairs), tid);
        }
    }
    if constexpr (STG) {
        __syncthreads();
        if (threadIdx.x == 0) {
            store_staged(prev_slot);
            tc::bulk_wait_all();
        }
    }
}

// ---- fused PFB + FFT --------------------------------------------------------
//
// One kernel per F-engine launch.  A CTA owns one input pair and a run of
// consecutive spectra; for each spectrum it filters the pair's newest frame
// in shared memory and transforms it, so the FIR output (z) never leaves the
// SM and each input sample is read from HBM once.
//
// Thread t owns the branch groups 4t .. 4t+3 and B .. B+3 (B = 4t + M/2 at
// M = 8192, 4t + M/4 below) and their mirrors.  The prototype is symmetric,
// h[pM + M-1-m] = h[(P-1-p)M + m], so the lower half of each polyphase row,
// hs[p][m] (m < M/2, in shared memory), gives the coefficients of both.  The last P-1 frames of the thread's 16 branches of
// both inputs stay in registers as raw int8 words (sign bits flipped, ready to
// unpack).  The newest frame arrives in a shared staging buffer by cp.async:
// bytes [A, A + M + 32) of each input's row, A the 16-byte aligned address at
// or below the frame's first sample, so branch m sits at staging byte o + m
// with o = A's offset, fixed per input.  Frames that reach outside the valid
// samples are staged by checked byte loads instead (zero outside).
//
// The FIR writes z into one of the FFT's two padded buffers and the first
// radix pass reads it from there.  Every FMA keeps the order of fir_kernel,
// and the passes are fft_kernel's, so the spectra are bit-identical to the
// two-kernel path's.

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src) {
    const size_t g = __cvta_generic_to_global(src);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(g) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

template <int M>
struct FusedCfg {
    static constexpr int SB = M + 32;                        // staged bytes per input
    static constexpr int ZB = FftCfg<M>::ZB;
    static constexpr int TWS = FftCfg<M>::TWS;
    static constexpr size_t off_tws = sizeof(float2) * 2 * (size_t)ZB;
    static constexpr size_t off_hs = (off_tws + sizeof(float2) * TWS + 15) / 16 * 16;
    static constexpr size_t off_stg(int P) { return off_hs + sizeof(float) * (size_t)P * (M / 2); }
    static constexpr size_t smem_bytes(int P) { return off_stg(P) + 2 * (size_t)SB; }
};

// Stage the samples of one frame of one input (first sample n0 = f M + d)
// into stg: staging byte i holds sample n0 - o + i (zero outside [lo, vhi)).
template <int M>
__device__ __forceinline__ void stage_frame(const StreamView& sv, const int8_t* row, bool has, long long n0, int o,
                                            uint8_t* stg, int tid, int nthr) {
    constexpr int SB = FusedCfg<M>::SB;
    const long long nA = n0 - o;
    const long long lo = sv.base > 0 ? sv.base : 0;
    if (has && nA >= lo && nA + SB <= sv.vhi) {
        const uint32_t s0 = tc::smem_u32(stg);
        for (int c = tid; c < SB / 16; c += nthr) cp_async16(s0 + 16 * c, row + nA + 16 * c);
    } else {
        for (int i = tid; i < SB; i += nthr) {
            const long long n = nA + i;
            stg[i] = (has && n >= lo && n < sv.vhi) ? (uint8_t)row[n] : (uint8_t)0;
        }
    }
}

// Eight staged bytes from byte offset off (any alignment), sign bits flipped.
__device__ __forceinline__ uint2 staged8(const uint8_t* stg, int off) {
    const uint32_t* w = reinterpret_cast<const uint32_t*>(stg) + (off >> 2);
    const int sh = 8 * (off & 3);
    const uint32_t a = w[0], b = w[1], c = w[2];
    return make_uint2(__funnelshift_r(a, b, sh) ^ 0x80808080u, __funnelshift_r(b, c, sh) ^ 0x80808080u);
}

// Samples n .. n+7 of a row straight from global memory, zero outside
// [lo, vhi) and for frames before the stream; sign bits flipped.  Used for
// the P-1 frames a CTA's run starts with.
__device__ __noinline__ uint2 global8_checked(const int8_t* row, bool has, long long n, long long lo, long long vhi) {
    uint32_t w0 = 0, w1 = 0;
    for (int b = 0; b < 8; ++b) {
        const long long i = n + b;
        const uint32_t v = (has && i >= lo && i < vhi) ? (uint32_t)(uint8_t)row[i] : 0u;
        if (b < 4) w0 |= v << (8 * b);
        else w1 |= v << (8 * (b - 4));
    }
    return make_uint2(w0 ^ 0x80808080u, w1 ^ 0x80808080u);
}

// (x_a, x_b) of byte C of two sign-flipped words, exact (see unpack4x2).
template <int C>
__device__ __forceinline__ float2 unpack_pair(uint32_t fa, uint32_t fb) {
    constexpr uint32_t sel = 0x7440u + C;
    return sub2(make_float2(__int_as_float((int)__byte_perm(fa, 0x4B000000u, sel)),
                            __int_as_float((int)__byte_perm(fb, 0x4B000000u, sel))),
                make_float2(8388736.0f, 8388736.0f));
}

// The first (radix R0, Ns = 1) pass's inputs from the padded shared buffer.
template <int M>
__device__ __forceinline__ void load_first_smem(float2 (&v)[16], const float2* z, int tid) {
    constexpr int R = first_radix(M);
    constexpr int B = 16 / R;
    constexpr int NACT = M / 16;
    constexpr int NR = M / R;
#pragma unroll
    for (int b = 0; b < B; ++b)
#pragma unroll
        for (int r = 0; r < R; ++r) v[b * R + r] = z[pidx(tid + b * NACT + r * NR)];
}

// later_passes_pp with the cp.async copies of the next frame completed
// before the last pass's barrier (so the staging buffer is ready after it).
template <int M, int NS, bool REGTW>
__device__ __forceinline__ float2* later_passes_cp(float2* zin, float2* zout, const float2* tws,
                                                  const float2 (&twr)[15], int tid,
                                                  const float2* __restrict__ gtw) {
    if constexpr (NS < M) {
        constexpr bool last = (NS * 16 == M);
        if (tid < M / 16) {
            float2 v[16];
            load_smem<M>(v, zin, tid);
            if constexpr (last && REGTW) pass_compute_store<M, 16, NS, TW_REG>(zout, v, tws, twr, tid);
            else if constexpr (last) pass_compute_store<M, 16, NS, TW_GLOBAL>(zout, v, tws, twr, tid, gtw);
            else pass_compute_store<M, 16, NS, TW_SMEM>(zout, v, tws, twr, tid);
        }
        if constexpr (last) cp_async_wait_all();
        __syncthreads();
        return later_passes_cp<M, NS * 16, REGTW>(zout, zin, tws, twr, tid, gtw);
    } else {
        return zin;
    }
}

__device__ __forceinline__ float2 unpack_pair(uint32_t fa, uint32_t fb, int c) {
    const uint32_t sel = 0x7440u + (uint32_t)c;
    return sub2(make_float2(__int_as_float((int)__byte_perm(fa, 0x4B000000u, sel)),
                            __int_as_float((int)__byte_perm(fb, 0x4B000000u, sel))),
                make_float2(8388736.0f, 8388736.0f));
}

// MODE as in fft_kernel (0 U = 2Y channel-major, 1 rotated V, 2 power
// tiles, 3 U pair-major), or 6 / 7: U requantised to int8 / e4m3 codes, the
// pair's four codes of a channel (Re U_a, Im U_a, Re U_b, Im U_b, low byte
// first) as one 32-bit word of pair-major words [slot][pair][n_chan] (an
// integration's word buffer, slot = s - int_start); one input pair per CTA;
// P taps.
template <int M, int MODE, int P>
__global__ void __launch_bounds__(M / 16, FftCfg<M>::minb(3)) pfb_fft_kernel(const FusedArgs A) {
    using C = FftCfg<M>;
    using FC = FusedCfg<M>;
    static_assert(C::pairs(MODE) == 1, "fused kernel: one input pair per CTA");
    static_assert(M >= 512 && C::THREADS == M / 16, "fused kernel: every thread owns 16 branches");
    static_assert(P >= 2 && P <= 4, "fused kernel: 2 to 4 taps");
    constexpr int NACT = M / 16;
    constexpr int n_chan = M >> 1;
    constexpr int R0 = first_radix(M);
    // FIR + radix passes: with an even count the result lands in the buffer
    // the FIR wrote, so consecutive spectra alternate between the buffers
    // R0 = 2: the thread's branches are closed under the first pass's
    // butterflies (j, j + M/2), so the FIR outputs go through that pass in
    // registers and the FIR writes its results (FP2)
    constexpr bool FP2 = R0 == 2;
    constexpr bool ALT = (((FP2 ? 0 : 1) + n_later_passes(M, R0)) % 2) == 0;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* const buf0 = reinterpret_cast<float2*>(smem_raw);
    float2* const buf1 = buf0 + FC::ZB;
    float2* const tws = reinterpret_cast<float2*>(smem_raw + FC::off_tws);
    float* const hsm = reinterpret_cast<float*>(smem_raw + FC::off_hs);
    uint8_t* const stg0 = smem_raw + FC::off_stg(P);
    uint8_t* const stg1 = stg0 + FC::SB;
    const FftArgs& F = A.f;
    const int tid = (int)threadIdx.x;
    const int pair = (int)blockIdx.y;
    const int n_pairs = (int)gridDim.y;
    const int a = 2 * pair;
    const long long s_lo = F.s_begin + (long long)blockIdx.x * F.spt;
    long long s_hi = s_lo + F.spt;
    if (s_hi > F.s_end) s_hi = F.s_end;
    if (s_lo >= s_hi) return;   // uniform over the CTA

    for (int i = tid; i < C::TWS; i += NACT) tws[i] = __ldg(F.tw + i);
    {
        const float4* src = reinterpret_cast<const float4*>(A.hs);
        float4* dst = reinterpret_cast<float4*>(hsm);
        for (int i = tid; i < P * M / 8; i += NACT) dst[i] = __ldg(src + i);
    }
    float2 twr[15];
    if constexpr (C::REGTW) {
        constexpr int NSL = M / 16;
        constexpr int TWL = tw_offset(M, NSL);
#pragma unroll
        for (int r = 1; r < 16; ++r) twr[r - 1] = __ldg(F.tw + TWL + r * NSL + tid);
    }

    // the pair's two input rows: row[n] = sample n, valid in [lo, vhi)
    const StreamView& sv = A.src;
    const long long lo = sv.base > 0 ? sv.base : 0;
    const bool has0 = a < F.n_in, has1 = a + 1 < F.n_in;
    const int d0 = has0 ? A.coarse[a] : 0, d1 = has1 ? A.coarse[a + 1] : 0;
    const int8_t* const row0 = sv.x + (long long)a * sv.stride - sv.base;
    const int8_t* const row1 = row0 + sv.stride;
    const int o0 = has0 ? (int)(reinterpret_cast<uintptr_t>(row0 + d0) & 15) : 0;
    const int o1 = has1 ? (int)(reinterpret_cast<uintptr_t>(row1 + d1) & 15) : 0;
    // four words of four branches each: groups A = 4t and B, and their
    // mirrors B' and A' (branch m's mirror M-1-m shares its coefficients).
    // FP2: B = 4t + M/2, the first radix-2 pass's partner of A, so that pass
    // stays in the thread; else B = 4t + M/4.  Consecutive threads take
    // consecutive groups: the coefficient rows and the FIR's stores are read
    // and written without bank conflicts.
    const int wo[4] = {4 * tid, FP2 ? 4 * tid + M / 2 : 4 * tid + M / 4,
                       FP2 ? M / 2 - 4 - 4 * tid : 3 * (M / 4) - 4 - 4 * tid, M - 4 - 4 * tid};

    // W[q][k][w]: frame q of the window (q = P-1 the newest), input k, word w
    // (the four branches from wo[w])
    uint32_t W[P][2][4];
#pragma unroll
    for (int q = 0; q < P - 1; ++q) {
        const long long f = s_lo - (P - 1) + q;
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            uint2 x = make_uint2(0x80808080u, 0x80808080u), y = x;   // zero samples
            if (f >= 0) {
                const int8_t* row = k ? row1 : row0;
                const bool has = k ? has1 : has0;
                const long long n = f * M + (k ? d1 : d0);
                x = make_uint2(global8_checked(row, has, n + wo[0], lo, sv.vhi).x,
                               global8_checked(row, has, n + wo[1], lo, sv.vhi).x);
                y = make_uint2(global8_checked(row, has, n + wo[2], lo, sv.vhi).x,
                               global8_checked(row, has, n + wo[3], lo, sv.vhi).x);
            }
            W[q][k][0] = x.x;
            W[q][k][1] = x.y;
            W[q][k][2] = y.x;
            W[q][k][3] = y.y;
        }
    }
    stage_frame<M>(sv, row0, has0, s_lo * M + d0, o0, stg0, tid, NACT);
    stage_frame<M>(sv, row1, has1, s_lo * M + d1, o1, stg1, tid, NACT);
    cp_async_commit();
    cp_async_wait_all();
    __syncthreads();

    constexpr int PCH = MODE == 2 ? ((n_chan + NACT - 1) / NACT) : 1;
    float pa[PCH], pb[PCH];
#pragma unroll
    for (int i = 0; i < PCH; ++i) pa[i] = pb[i] = 0.f;
    const float4* const hs4 = reinterpret_cast<const float4*>(hsm);

    for (long long s = s_lo; s < s_hi; ++s) {
        const int it = (int)(s - s_lo);
        float2* const X = (ALT && (it & 1)) ? buf1 : buf0;
        float2* const Y = (X == buf0) ? buf1 : buf0;
#pragma unroll
        for (int w = 0; w < 4; ++w) {
            W[P - 1][0][w] = staged8(stg0, o0 + wo[w]).x;
            W[P - 1][1][w] = staged8(stg1, o1 + wo[w]).x;
        }
        if constexpr (FP2) {
            // FIR of branch groups A = 4t + i, B = 4t + i + M/2 (first-pass
            // partner of A), C = M/2 - 1 - 4t - i (mirror of B) and
            // D = M - 1 - 4t - i (mirror of A, partner of C); coefficients
            // from the half rows h1 = hs[.][4t ..], h2 = hs[.][M/2 - 4 - 4t ..]
            // (h[pM + m] = hs[P-1-p][M-1-m] above M/2), taps p = 0 .. P-1
            float2 zA[4], zB[4], zC[4], zD[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) zA[i] = zB[i] = zC[i] = zD[i] = make_float2(0.f, 0.f);
            // two halves, each with one coefficient set live: (A, D) then (B, C)
#pragma unroll
            for (int half = 0; half < 2; ++half) {
                float4 hh[P];
#pragma unroll
                for (int p = 0; p < P; ++p) hh[p] = hs4[(p * (M / 2) + wo[half ? 2 : 0]) >> 2];
#pragma unroll
                for (int p = 0; p < P; ++p) {
                    const float ha[4] = {hh[p].x, hh[p].y, hh[p].z, hh[p].w};
                    const float hb[4] = {hh[P - 1 - p].x, hh[P - 1 - p].y, hh[P - 1 - p].z, hh[P - 1 - p].w};
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        if (half == 0) {
                            zA[i] = fma2(make_float2(ha[i], ha[i]), unpack_pair(W[p][0][0], W[p][1][0], i), zA[i]);
                            zD[i] = fma2(make_float2(hb[i], hb[i]),
                                         unpack_pair(W[p][0][3], W[p][1][3], 3 - i), zD[i]);
                        } else {
                            zB[i] = fma2(make_float2(hb[3 - i], hb[3 - i]),
                                         unpack_pair(W[p][0][1], W[p][1][1], i), zB[i]);
                            zC[i] = fma2(make_float2(ha[3 - i], ha[3 - i]),
                                         unpack_pair(W[p][0][2], W[p][1][2], 3 - i), zC[i]);
                        }
                    }
                }
            }
            // first radix-2 pass (Ns = 1): butterfly j -> positions 2j, 2j + 1
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int j = wo[0] + i, jc = M / 2 - 1 - wo[0] - i;
                X[pidx(2 * j)] = make_float2(zA[i].x + zB[i].x, zA[i].y + zB[i].y);
                X[pidx(2 * j + 1)] = make_float2(zA[i].x - zB[i].x, zA[i].y - zB[i].y);
                X[pidx(2 * jc)] = make_float2(zC[i].x + zD[i].x, zC[i].y + zD[i].y);
                X[pidx(2 * jc + 1)] = make_float2(zC[i].x - zD[i].x, zC[i].y - zD[i].y);
            }
        } else {
        // FIR: y_s[m] = sum_p h[pM + m] x[(s-P+1+p)M + m] for both inputs at
        // once (lanes a, b of a packed pair), taps in order p = 0 .. P-1.
        // Branch wo[j] + c (j = 0: A, 1: B, both below M/2) is byte c of
        // word j; its mirror M-1-(wo[j] + c) = wo[3-j] + 3 - c is byte 3-c
        // of word 3-j and takes h[(P-1-p)M + wo[j] + c] at tap p.
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            float4 hq[P];
#pragma unroll
            for (int p = 0; p < P; ++p) hq[p] = hs4[(p * (M / 2) + wo[j]) >> 2];
            float2 ylo[4], ymi[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) ylo[c] = ymi[c] = make_float2(0.f, 0.f);
#pragma unroll
            for (int p = 0; p < P; ++p) {
                const float hl[4] = {hq[p].x, hq[p].y, hq[p].z, hq[p].w};
                const float hm[4] = {hq[P - 1 - p].x, hq[P - 1 - p].y, hq[P - 1 - p].z, hq[P - 1 - p].w};
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    ylo[c] = fma2(make_float2(hl[c], hl[c]), unpack_pair(W[p][0][j], W[p][1][j], c), ylo[c]);
                    ymi[c] = fma2(make_float2(hm[c], hm[c]),
                                  unpack_pair(W[p][0][3 - j], W[p][1][3 - j], 3 - c), ymi[c]);
                }
            }
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                X[pidx(wo[j] + c)] = ylo[c];
                X[pidx(M - 1 - wo[j] - c)] = ymi[c];
            }
        }
        }
#pragma unroll
        for (int q = 0; q < P - 1; ++q)
#pragma unroll
            for (int k = 0; k < 2; ++k)
#pragma unroll
                for (int w = 0; w < 4; ++w) W[q][k][w] = W[q + 1][k][w];
        __syncthreads();   // z complete; the staging buffer is free
        if (s + 1 < s_hi) {
            stage_frame<M>(sv, row0, has0, (s + 1) * M + d0, o0, stg0, tid, NACT);
            stage_frame<M>(sv, row1, has1, (s + 1) * M + d1, o1, stg1, tid, NACT);
            cp_async_commit();
        }
        const float2* zres;
        if constexpr (FP2) {
            zres = later_passes_cp<M, R0, C::REGTW>(X, Y, tws, twr, tid, F.tw);
        } else {
            {
                float2 v[16];
                load_first_smem<M>(v, X, tid);
                pass_compute_store<M, R0, 1, TW_NONE>(Y, v, tws, twr, tid);
            }
            __syncthreads();
            zres = later_passes_cp<M, R0, C::REGTW>(Y, X, tws, twr, tid, F.tw);
        }

        if constexpr (MODE == 2) {
            // |Y_a|^2 = |S|^2 / 4, |Y_b|^2 = |D|^2 / 4, summed over the row
#pragma unroll
            for (int i = 0; i < PCH; ++i) {
                const int k = tid + i * NACT;
                if (k < n_chan) {
                    const float2 zk = zres[pidx(k)];
                    const float2 zm = zres[pidx((M - k) & (M - 1))];
                    const float sx = zk.x + zm.x, sy = zk.y - zm.y;
                    const float dx = zk.x - zm.x, dy = zk.y + zm.y;
                    pa[i] = fmaf(sx, sx, fmaf(sy, sy, pa[i]));
                    pb[i] = fmaf(dx, dx, fmaf(dy, dy, pb[i]));
                }
            }
            const long long row = s / F.n_row;
            if (s + 1 == s_hi || (s + 1) % F.n_row == 0) {
                const float sc = 0.25f / (float)F.n_row;
                const int n_cb = n_chan / 256, n_rb = F.rows / 64;
#pragma unroll
                for (int i = 0; i < PCH; ++i) {
                    const int k = tid + i * NACT;
                    if (k < n_chan) {
                        const size_t px = (size_t)(row % 64) * 256 + (k % 256);
                        if (has0) {
                            const size_t ta = ((size_t)a * n_rb + row / 64) * n_cb + k / 256;
                            atomicAdd(F.tiles + ta * 16384 + px, pa[i] * sc);
                        }
                        if (has1) {
                            const size_t tb = ((size_t)(a + 1) * n_rb + row / 64) * n_cb + k / 256;
                            atomicAdd(F.tiles + tb * 16384 + px, pb[i] * sc);
                        }
                    }
                    pa[i] = 0.f;
                    pb[i] = 0.f;
                }
            }
        } else if constexpr (MODE >= 6) {
            // the requantiser's arithmetic on the same U = 2Y values: code of
            // U * (1 / sigma) per component; consecutive channels across the
            // warp, so each store instruction writes whole lines
            constexpr bool FP8 = MODE == 7;
            const long long slot = (s - F.v_origin) & F.v_mask;
            uint32_t* const Cout = reinterpret_cast<uint32_t*>(F.V) + ((size_t)slot * n_pairs + pair) * n_chan;
            const float* const inv0 = A.inv + (size_t)a * n_chan;
            const float* const inv1 = inv0 + n_chan;
            for (int k = tid; k < n_chan; k += NACT) {
                const float2 zk = zres[pidx(k)];
                const float2 zm = zres[pidx((M - k) & (M - 1))];
                const float ia = has0 ? __ldg(inv0 + k) : 0.f;
                const float ib = has1 ? __ldg(inv1 + k) : 0.f;
                const float sx = zk.x + zm.x, sy = zk.y - zm.y;
                const float dx = zk.x - zm.x, dy = zk.y + zm.y;
                Cout[k] = q_code<FP8>(sx * ia) | (q_code<FP8>(sy * ia) << 8) | (q_code<FP8>(dy * ib) << 16) |
                          (q_code<FP8>(-dx * ib) << 24);
            }
        } else {
            const long long slot = (s - F.v_origin) & F.v_mask;
            float4* Vout;
            size_t vstride;
            if constexpr (MODE == 3) {
                Vout = reinterpret_cast<float4*>(F.V) + ((size_t)slot * n_pairs + pair) * n_chan;
                vstride = 1;
            } else {
                Vout = reinterpret_cast<float4*>(F.V + (size_t)slot * n_chan * F.n_in_pad + a);
                vstride = (size_t)(F.n_in_pad >> 1);
            }
            for (int k = tid; k < n_chan; k += NACT) {
                const float2 zk = zres[pidx(k)];
                const float2 zm = zres[pidx((M - k) & (M - 1))];
                const float2 S = make_float2(zk.x + zm.x, zk.y - zm.y);
                const float2 D = make_float2(zk.x - zm.x, zk.y + zm.y);
                float4 out;
                if constexpr (MODE == 1) {
                    const float2 va = cmul(S, __ldg(F.phasor + (size_t)a * n_chan + k));
                    const float2 vb = cmul(D, __ldg(F.phasor + (size_t)(a + 1) * n_chan + k));
                    out = make_float4(va.x, va.y, vb.x, vb.y);
                } else {
                    out = make_float4(S.x, S.y, D.y, -D.x);
                }
                Vout[(size_t)k * vstride] = out;
            }
        }
    }
}

// Launch of fft_kernel<M, MODE> (one wave of resident CTAs).
template <int M, int MODE>
int launch_fft_m(const FftArgs& a, cudaStream_t st) {
    using C = FftCfg<M>;
    constexpr bool STG = C::TMA_OUT && MODE <= 1;     // the modes whose spectra leave by tensor stores
    static int resident = 0;     // CTAs per SM at this kernel's registers and shared memory
    static int sms = 0;
    const size_t smem = C::smem_bytes(MODE);
    if (!resident) {
        cudaFuncSetAttribute(fft_kernel<M, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident, fft_kernel<M, MODE>, C::threads(MODE), smem);
        if (resident < 1) resident = 1;
        if (sms < 1) sms = 152;
    }
    CUtensorMap vmap;
    std::memset(&vmap, 0, sizeof(vmap));
    if constexpr (STG) {
        // V as rows of n_in_pad complex64 (2 n_in_pad floats, 8 n_in_pad
        // bytes apart); one row per (slot, channel).  A pair writes the 16
        // bytes at float 4 * pair of each row.
        PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
        if (!enc) return CORR_ECUDA;
        if ((reinterpret_cast<uintptr_t>(a.V) & 15) != 0) return CORR_EINVAL;
        const long long slots = a.v_mask == -1LL ? a.s_end - a.v_origin : a.v_mask + 1;
        cuuint64_t dims[2] = {(cuuint64_t)a.n_in_pad * 2, (cuuint64_t)slots * (M / 2)};
        cuuint64_t strides[1] = {(cuuint64_t)a.n_in_pad * 8};
        cuuint32_t box[2] = {(cuuint32_t)(4 * C::pairs(MODE)), (cuuint32_t)C::BOXR};
        cuuint32_t estr[2] = {1, 1};
        const CUresult r = enc(&vmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, a.V, dims, strides, box, estr,
                               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                               CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return CORR_EINVAL;
    }
    // One wave of resident CTAs, each looping over a run of spectra of one
    // pair: runs x pairs never exceeds the resident slots (rounding up would
    // leave a few CTAs for a second, nearly empty wave as long as the first).
    const long long n = a.s_end - a.s_begin;
    // transforms per spectrum: one per input pair, or one per input (complex
    // input); n_in_pad is a multiple of 4
    const int n_groups = (MODE == 4 || MODE == 5 ? a.n_in_pad : a.n_in_pad / 2) / C::pairs(MODE);
    long long runs = (long long)sms * resident / n_groups;
    if (runs > n) runs = n;
    if (runs < 1) runs = 1;
    FftArgs b = a;
    b.spt = (int)((n + runs - 1) / runs);
    dim3 grid((unsigned)((n + b.spt - 1) / b.spt), (unsigned)n_groups);
    fft_kernel<M, MODE><<<grid, C::threads(MODE), smem, st>>>(b, vmap);
    return CORR_OK;
}

}  // namespace

}  // namespace corr
