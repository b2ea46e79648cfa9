// F-engine: int8 load with coarse delay -> P-tap polyphase FIR -> M-point
// FFT -> fine-delay / instrument-phase rotation (Sec. 4.2 "F-engine (PFB and
// FFT)", with the delay compensation of Eq. 1 applied per input).
//
// One CTA channelises one pair of inputs (a, a+1) for a block of consecutive
// spectra.  The two real FIR outputs of the pair are packed as one complex
// sequence z[m] = y_a[m] + j y_b[m]; a single M-point complex FFT then gives
// both spectra: Y_a[k] = (Z[k] + Z*[M-k]) / 2 and Y_b[k] = (Z[k] - Z*[M-k]) / 2j.
// The 1/2 and 1/2j factors are folded into the per-input phasor table.
//
// The FFT is a Stockham autosort transform held in shared memory (padded by
// one float2 every 16 to keep the strided passes free of bank conflicts),
// radix-16 passes while they fit and one smaller pass for the remainder; each
// thread keeps 16 points in registers per pass.
#include "corr_internal.h"


namespace corr {

namespace {

__device__ __forceinline__ int pidx(int i) { return i + (i >> 4); }

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

// One Stockham pass of radix R over the padded shared buffer z (M points):
// butterfly j reads z[j + r M/R], multiplies by W_{Ns R}^{r (j mod Ns)},
// transforms, and writes z[(j - j mod Ns) R + j mod Ns + r Ns].  Each of the
// M/16 active threads owns 16/R butterflies (16 points).
template <int M, int R, int NS>
__device__ __forceinline__ void stockham_pass(float2* z, const float2* __restrict__ tw, int tid) {
    constexpr int B = 16 / R;
    constexpr int NACT = M / 16;
    constexpr int NR = M / R;
    constexpr int TSTEP = M / (NS * R);
    float2 v[16];
    const bool act = tid < NACT;
    if (act) {
        if constexpr (M >= 256) {
            // tid + b NACT + r NR with both strides multiples of 16.
            const int pb = pidx(tid);
#pragma unroll
            for (int b = 0; b < B; ++b)
#pragma unroll
                for (int r = 0; r < R; ++r) v[b * R + r] = z[pb + (b * NACT + r * NR) / 16 * 17];
        } else {
#pragma unroll
            for (int b = 0; b < B; ++b)
#pragma unroll
                for (int r = 0; r < R; ++r) v[b * R + r] = z[pidx(tid + b * NACT + r * NR)];
        }
    }
    __syncthreads();
    if (act) {
#pragma unroll
        for (int b = 0; b < B; ++b) {
            const int j = tid + b * NACT;
            const int k = j & (NS - 1);
            float2 u[R];
#pragma unroll
            for (int r = 0; r < R; ++r) u[r] = v[b * R + r];
            if constexpr (NS > 1) {
#pragma unroll
                for (int r = 1; r < R; ++r) u[r] = cmul(u[r], __ldg(tw + r * k * TSTEP));
            }
            dft_dif<R>(u);
            const int o = (j - k) * R + k;
            StoreBitrev<R, NS, 0>::run(z, u, o, pidx(o));
        }
    }
    __syncthreads();
}

__host__ __device__ constexpr int first_radix(int M) {
    int l = 0;
    while ((1 << l) < M) ++l;
    return (l % 4) == 0 ? 16 : (1 << (l % 4));
}

// Passes: one small-radix pass (radix M / 16^n) at Ns = 1 if needed, then
// radix-16 passes.
template <int M, int NS>
__device__ __forceinline__ void fft_passes(float2* z, const float2* __restrict__ tw, int tid) {
    if constexpr (NS < M) {
        constexpr int R = NS == 1 ? first_radix(M) : 16;
        stockham_pass<M, R, NS>(z, tw, tid);
        fft_passes<M, NS * R>(z, tw, tid);
    }
}

// Sixteen consecutive int8 samples of one input starting at stream index n0,
// returned as four little-endian words; zero outside the valid window.
__device__ __forceinline__ void load16(const StreamView& sv, int a, long long n0, uint32_t w[4]) {
    const long long lo = sv.base > 0 ? sv.base : 0;
    const int8_t* row = sv.x + (long long)a * sv.stride - sv.base;  // stream index 0
    const uintptr_t addr = reinterpret_cast<uintptr_t>(row + n0);
    const int c = (int)(addr & 15);
    // Fast path: both aligned 16-byte blocks lie inside the valid window.
    if (n0 - c >= lo && n0 - c + 32 <= sv.vhi) {
        const uint4* q = reinterpret_cast<const uint4*>(addr - c);
        const uint4 A = __ldg(q);
        uint4 Bv = make_uint4(0, 0, 0, 0);
        if (c) Bv = __ldg(q + 1);
        const uint32_t W8[8] = {A.x, A.y, A.z, A.w, Bv.x, Bv.y, Bv.z, Bv.w};
        const int qw = c >> 2, sh = (c & 3) * 8;
        // qw is uniform across the CTA (it depends on the input and the
        // buffer alignment only), so this switch does not diverge.
        switch (qw) {
#define CORR_SEL(Q)                                                        \
    case Q:                                                                \
        w[0] = __funnelshift_r(W8[Q + 0], W8[Q + 1], sh);                 \
        w[1] = __funnelshift_r(W8[Q + 1], W8[Q + 2], sh);                 \
        w[2] = __funnelshift_r(W8[Q + 2], W8[Q + 3], sh);                 \
        w[3] = __funnelshift_r(W8[Q + 3], W8[Q + 4], sh);                 \
        break;
            CORR_SEL(0)
            CORR_SEL(1)
            CORR_SEL(2)
            CORR_SEL(3)
#undef CORR_SEL
        }
        return;
    }
    // Edge path: byte loads with bounds checks.
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        uint32_t v = 0;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const long long n = n0 + i * 4 + b;
            uint32_t byte = 0;
            if (n >= lo && n < sv.vhi) byte = (uint8_t)row[n];
            v |= byte << (8 * b);
        }
        w[i] = v;
    }
}

// Exact int8 -> float: flip the sign bit, place the byte in the mantissa of
// 2^23, subtract 2^23 + 128.
__device__ __forceinline__ float b2f(uint32_t wflip, int sel) {
    return __int_as_float((int)__byte_perm(wflip, 0x4B000000u, sel)) - 8388736.0f;
}

__device__ __forceinline__ void fir_accum(float* y, const uint32_t w[4], const float* hv) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const uint32_t f = w[i] ^ 0x80808080u;
        y[4 * i + 0] = fmaf(hv[4 * i + 0], b2f(f, 0x7440), y[4 * i + 0]);
        y[4 * i + 1] = fmaf(hv[4 * i + 1], b2f(f, 0x7441), y[4 * i + 1]);
        y[4 * i + 2] = fmaf(hv[4 * i + 2], b2f(f, 0x7442), y[4 * i + 2]);
        y[4 * i + 3] = fmaf(hv[4 * i + 3], b2f(f, 0x7443), y[4 * i + 3]);
    }
}

template <int M>
__global__ void __launch_bounds__(M / 16 < 32 ? 32 : M / 16) fengine_kernel(const FArgs A) {
    extern __shared__ float2 zbuf[];
    const int tid = threadIdx.x;
    constexpr int n_chan = M >> 1;
    constexpr int nact = M >> 4;
    const int a = 2 * blockIdx.y, b = a + 1;
    const bool has_a = a < A.n_in, has_b = b < A.n_in;
    const int da = A.coarse[a], db = A.coarse[b];
    const long long s_lo = A.s_begin + (long long)blockIdx.x * A.spt;
    long long s_hi = s_lo + A.spt;
    if (s_hi > A.s_end) s_hi = A.s_end;

    for (long long s = s_lo; s < s_hi; ++s) {
        // ---- polyphase FIR, 16 consecutive branches per thread, one input
        //      of the pair at a time (re part: input a, im part: input b) ----
        if (tid < nact) {
            const int m0 = tid * 16;
            float* zf = reinterpret_cast<float*>(zbuf);
#pragma unroll 1
            for (int half = 0; half < 2; ++half) {
                const int in = half ? b : a;
                const bool has = half ? has_b : has_a;
                const int d = half ? db : da;
                float y[16];
#pragma unroll
                for (int i = 0; i < 16; ++i) y[i] = 0.f;
                if (has) {
                    for (int p = 0; p < A.taps; ++p) {
                        const long long f = s - A.taps + 1 + p;
                        if (f < 0) continue;
                        uint32_t w[4];
                        load16(A.src, in, f * M + m0 + d, w);
                        float hv[16];
                        const float4* hp = reinterpret_cast<const float4*>(A.h + (size_t)p * M + m0);
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            const float4 t = __ldg(hp + i);
                            hv[4 * i] = t.x; hv[4 * i + 1] = t.y; hv[4 * i + 2] = t.z; hv[4 * i + 3] = t.w;
                        }
                        fir_accum(y, w, hv);
                    }
                }
#pragma unroll
                for (int i = 0; i < 16; ++i) zf[2 * pidx(m0 + i) + half] = y[i];
            }
        }
        __syncthreads();
        fft_passes<M, 1>(zbuf, A.tw, tid);
        // ---- unpack the two real spectra, rotate, store V[slot][k][a..a+1] ----
        long long slot = (s - A.v_origin) % A.v_cap;
        if (slot < 0) slot += A.v_cap;
        float4* Vout = reinterpret_cast<float4*>(A.V + (size_t)slot * n_chan * A.n_in_pad + a);
        const float2* pa = A.phasor + (size_t)a * n_chan;
        const float2* pb = A.phasor + (size_t)b * n_chan;
        for (int k = tid; k < n_chan; k += blockDim.x) {
            const float2 zk = zbuf[pidx(k)];
            const float2 zm = zbuf[pidx((M - k) & (M - 1))];
            const float2 S = make_float2(zk.x + zm.x, zk.y - zm.y);
            const float2 D = make_float2(zk.x - zm.x, zk.y + zm.y);
            const float2 va = cmul(S, __ldg(pa + k));
            const float2 vb = cmul(D, __ldg(pb + k));
            Vout[(size_t)k * (A.n_in_pad >> 1)] = make_float4(va.x, va.y, vb.x, vb.y);
        }
        __syncthreads();
    }
}

}  // namespace

int fengine_threads(int M) {
    int nt = M / 16;
    if (nt < 32) nt = 32;
    return nt;
}

size_t fengine_smem_bytes(int M) { return sizeof(float2) * (size_t)(M + M / 16 + 1); }

template <int M>
static void launch_m(const FArgs& a, dim3 grid, cudaStream_t st) {
    static bool attr_set = false;
    const size_t smem = fengine_smem_bytes(M);
    if (!attr_set) {
        cudaFuncSetAttribute(fengine_kernel<M>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        attr_set = true;
    }
    fengine_kernel<M><<<grid, fengine_threads(M), smem, st>>>(a);
}

void launch_fengine(const FArgs& a, cudaStream_t st) {
    const long long n = a.s_end - a.s_begin;
    if (n <= 0) return;
    dim3 grid((unsigned)((n + a.spt - 1) / a.spt), (unsigned)(a.n_in_pad / 2));
    switch (a.M) {
        case 16: launch_m<16>(a, grid, st); break;
        case 32: launch_m<32>(a, grid, st); break;
        case 64: launch_m<64>(a, grid, st); break;
        case 128: launch_m<128>(a, grid, st); break;
        case 256: launch_m<256>(a, grid, st); break;
        case 512: launch_m<512>(a, grid, st); break;
        case 1024: launch_m<1024>(a, grid, st); break;
        case 2048: launch_m<2048>(a, grid, st); break;
        case 4096: launch_m<4096>(a, grid, st); break;
        case 8192: launch_m<8192>(a, grid, st); break;
        case 16384: launch_m<16384>(a, grid, st); break;
        default: break;
    }
}

}  // namespace corr
