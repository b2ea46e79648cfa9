// X-engine and integration (Sec. 4.2 "X-engine and integration",
// Algorithm 1): R[k][a][b] = (1/count) sum_s V_a,s[k] conj(V_b,s[k]).
//
// CUDA-core form.  Inputs are taken in blocks of four; one thread owns one
// channel and one 4x4 block-pair (A <= B) of the Hermitian matrix and keeps
// its 16 complex sums in registers over a group of spectra.  Each group's
// sums go to their own partial slot; the finaliser adds the slots of an
// integration in a fixed order, so the result does not depend on how a
// stream was split into pushes (no atomics anywhere).
#include "corr.h"
#include "corr_internal.h"
#include "tc_common.cuh"

namespace corr {

namespace {

__device__ __forceinline__ void tile_decode(int t, int nb, int& A, int& B) {
    // t enumerates (A, B), A <= B < nb, row by row.
    int r = 0, rem = t;
    while (rem >= nb - r) { rem -= nb - r; ++r; }
    A = r;
    B = r + rem;
}

// PM: spectra pair-major ([slot][pair][n_chan] float4), else channel-major.
template <bool PM>
__global__ void __launch_bounds__(128) xengine_kernel(const XArgs X) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int t = blockIdx.y;
    const int g = blockIdx.z;
    if (k >= X.n_chan) return;
    int A, B;
    tile_decode(t, X.n_in_pad >> 2, A, B);
    long long s0 = X.int_start + (long long)(X.j0 + g) * X.G;
    long long s1 = s0 + X.G;
    if (s1 > X.int_end) s1 = X.int_end;
    if (s1 > X.s_limit) s1 = X.s_limit;

    float acc[32];
#pragma unroll
    for (int e = 0; e < 32; ++e) acc[e] = 0.f;
    const int q4 = X.n_in_pad >> 1;   // float4 (input pairs) per (slot, channel)
    for (long long s = s0; s < s1; ++s) {
        const long long slot = (s - X.v_origin) & X.v_mask;
        float4 a01, a23, b01, b23;
        if constexpr (PM) {
            // pair p of this slot at [(slot * q4 + p) * n_chan + k]
            const float4* vp = reinterpret_cast<const float4*>(X.V) + (size_t)slot * q4 * X.n_chan + k;
            a01 = __ldg(vp + (size_t)(2 * A) * X.n_chan);
            a23 = __ldg(vp + (size_t)(2 * A + 1) * X.n_chan);
            b01 = __ldg(vp + (size_t)(2 * B) * X.n_chan);
            b23 = __ldg(vp + (size_t)(2 * B + 1) * X.n_chan);
        } else {
            const float4* vp = reinterpret_cast<const float4*>(X.V) + ((size_t)slot * X.n_chan + k) * q4;
            a01 = __ldg(vp + 2 * A);
            a23 = __ldg(vp + 2 * A + 1);
            b01 = __ldg(vp + 2 * B);
            b23 = __ldg(vp + 2 * B + 1);
        }
        const float ar[4] = {a01.x, a01.z, a23.x, a23.z}, ai[4] = {a01.y, a01.w, a23.y, a23.w};
        const float br[4] = {b01.x, b01.z, b23.x, b23.z}, bi[4] = {b01.y, b01.w, b23.y, b23.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                float& re = acc[(i * 4 + j) * 2];
                float& im = acc[(i * 4 + j) * 2 + 1];
                re = fmaf(ar[i], br[j], re);
                re = fmaf(ai[i], bi[j], re);
                im = fmaf(ai[i], br[j], im);
                im = fmaf(-ar[i], bi[j], im);
            }
        }
    }
    float* out = X.part + (((size_t)(X.j0 + g) * X.nt + t) * 32) * X.n_chan + k;
#pragma unroll
    for (int e = 0; e < 32; ++e) out[(size_t)e * X.n_chan] = acc[e];
}

// n_in_pad <= 8: one thread keeps the whole Hermitian triangle (a <= b) of
// one channel.  A warp covers 16 consecutive channels x 2 sub-groups;
// sub-group q sums spectra q, q+2, q+4, ... of the group (one pair's 16
// channels are 256 contiguous bytes of the pair-major ring), the two partial
// sums are added by one xor-shuffle, then written in the 4x4 block layout.
// PM: spectra pair-major ([slot][pair][n_chan] float4), else channel-major.
// Each thread streams its spectra through DEPTH stages of shared memory
// with cp.async (16-byte copies of its own chunks, so no barrier is needed):
// DEPTH spectra in flight a thread instead of one.  DEPTH (4 or 6; 48 KiB a
// CTA at n_in 8 and 6) is a tile shape the autotuner picks; it does not
// change the result.
constexpr int kXsChan = 16;       // channels per warp
constexpr int kXsSub = 2;         // sub-groups per channel

__device__ __forceinline__ void xs_cp16(float4* dst, const float4* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(tc::smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void xs_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void xs_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

template <int NB, int DEPTH>
constexpr size_t xs_smem_bytes() { return sizeof(float4) * DEPTH * (2 * NB) * 128; }

template <int NB, bool PM, int DEPTH>
__global__ void __launch_bounds__(128, 5) xengine_small_kernel(const XArgs X) {
    constexpr int NI = 4 * NB;
    constexpr int NC = NI * (NI - 1) / 2;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int q = lane / kXsChan;
    const int k = (blockIdx.x * (blockDim.x >> 5) + warp) * kXsChan + (lane % kXsChan);
    const int g = blockIdx.y;
    const bool valid = k < X.n_chan;
    const int kk = valid ? k : X.n_chan - 1;
    long long s0 = X.int_start + (long long)(X.j0 + g) * X.G;
    long long s1 = s0 + X.G;
    if (s1 > X.int_end) s1 = X.int_end;
    if (s1 > X.s_limit) s1 = X.s_limit;
    float au[NI], cr[NC], ci[NC];
#pragma unroll
    for (int i = 0; i < NI; ++i) au[i] = 0.f;
#pragma unroll
    for (int i = 0; i < NC; ++i) { cr[i] = 0.f; ci[i] = 0.f; }
    // stage buffer [depth][pair][thread]: thread-private chunks
    extern __shared__ float4 xs_buf[];
    const size_t vs = PM ? (size_t)X.n_chan : 1;          // float4 between pairs
    auto fetch = [&](long long s, int stage) {
        if (s < s1) {
            const long long slot = (s - X.v_origin) & X.v_mask;
            const float4* vp = PM ? reinterpret_cast<const float4*>(X.V) + (size_t)slot * (NI / 2) * X.n_chan + kk
                                  : reinterpret_cast<const float4*>(X.V) + ((size_t)slot * X.n_chan + kk) * (NI / 2);
#pragma unroll
            for (int i = 0; i < NI / 2; ++i)
                xs_cp16(xs_buf + ((size_t)stage * (NI / 2) + i) * 128 + threadIdx.x, vp + i * vs);
        }
        xs_commit();   // one group per stage, empty past the end
    };
#pragma unroll
    for (int d = 0; d < DEPTH; ++d) fetch(s0 + q + (long long)d * kXsSub, d);
    int stage = 0;
    for (long long s = s0 + q; s < s1; s += kXsSub) {
        xs_wait<DEPTH - 1>();      // this thread's copies of spectrum s have landed
        float xr[NI], xi[NI];
#pragma unroll
        for (int i = 0; i < NI / 2; ++i) {
            const float4 t = xs_buf[((size_t)stage * (NI / 2) + i) * 128 + threadIdx.x];
            xr[2 * i] = t.x; xi[2 * i] = t.y; xr[2 * i + 1] = t.z; xi[2 * i + 1] = t.w;
        }
#pragma unroll
        for (int a = 0; a < NI; ++a) au[a] = fmaf(xr[a], xr[a], fmaf(xi[a], xi[a], au[a]));
        int c = 0;
#pragma unroll
        for (int a = 0; a < NI; ++a) {
#pragma unroll
            for (int b = a + 1; b < NI; ++b, ++c) {
                cr[c] = fmaf(xr[a], xr[b], fmaf(xi[a], xi[b], cr[c]));
                ci[c] = fmaf(xi[a], xr[b], fmaf(-xr[a], xi[b], ci[c]));
            }
        }
        // this stage's values are used: refill it DEPTH spectra ahead
        fetch(s + (long long)DEPTH * kXsSub, stage);
        stage = stage + 1 == DEPTH ? 0 : stage + 1;
    }
#pragma unroll
    for (int m = kXsChan; m < 32; m <<= 1) {
#pragma unroll
        for (int i = 0; i < NI; ++i) au[i] += __shfl_xor_sync(0xffffffffu, au[i], m);
#pragma unroll
        for (int i = 0; i < NC; ++i) {
            cr[i] += __shfl_xor_sync(0xffffffffu, cr[i], m);
            ci[i] += __shfl_xor_sync(0xffffffffu, ci[i], m);
        }
    }
    if (q != 0 || !valid) return;
#pragma unroll
    for (int A = 0; A < NB; ++A) {
#pragma unroll
        for (int B = A; B < NB; ++B) {
            const int t = A * NB - A * (A - 1) / 2 + (B - A);
            float* out = X.part + (((size_t)(X.j0 + g) * X.nt + t) * 32) * X.n_chan + k;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int a = 4 * A + i, b = 4 * B + j;
                    float re = 0.f, im = 0.f;
                    if (a == b) {
                        re = au[a];
                    } else if (a < b) {
                        const int c = a * NI - a * (a + 1) / 2 + (b - a - 1);
                        re = cr[c];
                        im = ci[c];
                    }
                    out[(size_t)((i * 4 + j) * 2) * X.n_chan] = re;
                    out[(size_t)((i * 4 + j) * 2 + 1) * X.n_chan] = im;
                }
            }
        }
    }
}

// One thread per (channel, 4x4 block, entry): sums the entry's partial
// slots in slot order, scales, rotates and writes R_ab and its mirror.
// (bx, t, z): the block's channel block, 4x4 block pair and entry.
// Visibility (a, b), a <= b, of channel k from element z of tile t: the
// partial slots summed in order, scaled, rotated by Q_a conj(Q_b) off the
// diagonal.  False where the element is padding or below the diagonal.
__device__ __forceinline__ bool fin_value(const FinArgs& F, int k, int t, int z, int& a, int& b, float& re,
                                          float& im) {
    const int i = z >> 2, j = z & 3;
    const int n_in_pad = (F.n_in + 3) & ~3;
    int A, B;
    tile_decode(t, n_in_pad >> 2, A, B);
    a = 4 * A + i;
    b = 4 * B + j;
    if (a >= F.n_in || b >= F.n_in) return false;
    if (A == B && i > j) return false;
    const int e = (i * 4 + j) * 2;
    re = 0.f;
    im = 0.f;
    // slots summed in order; their loads issued 16 at a time
    const float* p = F.part + ((size_t)t * 32 + e) * F.n_chan + k;
    const size_t ss = (size_t)F.nt * 32 * F.n_chan;
    int s = 0;
    for (; s + 16 <= F.n_slots; s += 16) {
        float vr[16], vi[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            vr[q] = __ldcg(p + (size_t)(s + q) * ss);
            vi[q] = __ldcg(p + (size_t)(s + q) * ss + F.n_chan);
        }
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            re += vr[q];
            im += vi[q];
        }
    }
    if (s < F.n_slots) {
        // the last n_slots mod 16 slots, loaded together as well
        const int rem = F.n_slots - s;
        float vr[16], vi[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            vr[q] = q < rem ? __ldcg(p + (size_t)(s + q) * ss) : 0.f;
            vi[q] = q < rem ? __ldcg(p + (size_t)(s + q) * ss + F.n_chan) : 0.f;
        }
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            if (q < rem) {
                re += vr[q];
                im += vi[q];
            }
        }
    }
    re *= F.scale;
    im *= F.scale;
    if (a == b) {
        im = 0.f;
        return true;
    }
    if (F.rot) {
        // R_ab = Q_a conj(Q_b) * sum U_a U_b^*
        const float2 qa = F.rot[(size_t)a * F.n_chan + k];
        const float2 qb = F.rot[(size_t)b * F.n_chan + k];
        const float pr = qa.x * qb.x + qa.y * qb.y;
        const float pi = qa.y * qb.x - qa.x * qb.y;
        const float r2 = re * pr - im * pi;
        im = re * pi + im * pr;
        re = r2;
    }
    return true;
}

__device__ __forceinline__ void fin_store(const FinArgs& F, int k, int a, int b, float re, float im) {
    float2* R = F.R + (size_t)k * F.n_in * F.n_in;
    R[a * F.n_in + b] = make_float2(re, im);
    if (a != b) R[b * F.n_in + a] = make_float2(re, -im);
}

__device__ __forceinline__ void finalize_block(const FinArgs& F, int bx, int t, int z) {
    const int k = bx * 128 + (int)threadIdx.x;
    if (k >= F.n_chan) return;
    int a, b;
    float re, im;
    if (fin_value(F, k, t, z, a, b, re, im)) fin_store(F, k, a, b, re, im);
}

__global__ void __launch_bounds__(128) finalize_kernel(const FinArgs F) {
    finalize_block(F, (int)blockIdx.x, (int)blockIdx.y, (int)blockIdx.z);
}

// ---- MAD flagging, Eq. 2 ------------------------------------------------
// An item is one (integration, window, baseline a <= b).  Its W values are
// spread over a group of L lanes (L a power of two dividing 32; E values a
// lane, element i = (lane mod L) E + e, padding +inf) and sorted exactly by
// a bitonic network -- exchanges between registers below distance E, by
// shuffles inside the group above -- the median read from the sorted order
// (even count: mean of the two middle values), then |A - med| sorted the
// same way for the MAD.  L = 32 (a warp an item) where a call has few items;
// L = 4 where it has many (more items a warp, fewer shuffles).  Every form
// gives the same order statistics and the same threshold bits.
constexpr int kFlagWarps = 4;

template <int E, int L>
__device__ __forceinline__ void group_bitonic_stage(float (&v)[E], int lane, int k) {
    // merge step of size k: element i pairs with i ^ j, ascending where i & k == 0
    const int gl = lane & (L - 1);
#pragma unroll
    for (int j = k >> 1; j > 0; j >>= 1) {
        if (j < E) {
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int ep = e ^ j;
                if (ep > e) {
                    const int i = gl * E + e;
                    const bool asc = (i & k) == 0;
                    const float lo = fminf(v[e], v[ep]), hi = fmaxf(v[e], v[ep]);
                    v[e] = asc ? lo : hi;
                    v[ep] = asc ? hi : lo;
                }
            }
        } else {
            const int lm = j / E;                  // partner lane distance (< L: inside the group)
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const float o = __shfl_xor_sync(0xffffffffu, v[e], lm);
                const int i = gl * E + e;
                const bool keep_min = ((i & j) == 0) == ((i & k) == 0);
                v[e] = keep_min ? fminf(v[e], o) : fmaxf(v[e], o);
            }
        }
    }
}

template <int E, int L>
__device__ __forceinline__ void group_bitonic_sort(float (&v)[E], int lane) {
#pragma unroll
    for (int k = 2; k <= L * E; k <<= 1) group_bitonic_stage<E, L>(v, lane, k);
}

// Sort a bitonic sequence (non-increasing, then non-decreasing) ascending:
// the last merge step of the sort alone.
template <int E, int L>
__device__ __forceinline__ void group_bitonic_merge(float (&v)[E], int lane) {
    group_bitonic_stage<E, L>(v, lane, L * E);
}

// Element i of a group's sorted array (i the same in every lane).
template <int E, int L>
__device__ __forceinline__ float group_sorted_at(const float (&v)[E], int i, int lane) {
    const int src = (lane & ~(L - 1)) + i / E, e = i % E;
    float x = v[0];
#pragma unroll
    for (int q = 1; q < E; ++q)
        if (q == e) x = v[q];
    return __shfl_sync(0xffffffffu, x, src);
}

template <int E, int L>
__device__ __forceinline__ float group_sorted_median(const float (&v)[E], int W, int lane) {
    return (W & 1) ? group_sorted_at<E, L>(v, W >> 1, lane)
                   : __fmul_rn(0.5f, __fadd_rn(group_sorted_at<E, L>(v, (W >> 1) - 1, lane),
                                               group_sorted_at<E, L>(v, W >> 1, lane)));
}

__device__ __forceinline__ float vis_abs(float2 r) { return sqrtf(r.x * r.x + r.y * r.y); }

// Eq. 2's threshold median + sigma 1.4826 MAD over the group's W values A
// (element (lane mod L) E + e; +inf past W); the roundings spelled out.
template <int E, int L = 32>
__device__ __forceinline__ float group_mad_threshold(const float (&A)[E], int W, float sigma, int lane) {
    float v[E];
#pragma unroll
    for (int e = 0; e < E; ++e) v[e] = A[e];
    group_bitonic_sort<E, L>(v, lane);
    const float med = group_sorted_median<E, L>(v, W, lane);
    // |A - med| in the sorted order falls to the median and rises after it
    // (the +inf padding stays last): a bitonic sequence, which one merge
    // sorts -- the same values as sorting |A - med| from scratch
#pragma unroll
    for (int e = 0; e < E; ++e) v[e] = fabsf(v[e] - med);
    group_bitonic_merge<E, L>(v, lane);
    const float mad = group_sorted_median<E, L>(v, W, lane);
    return __fmaf_rn(__fmul_rn(sigma, mad), 1.4826f, med);
}

// Baseline index bl (upper triangle, row by row) -> (a, b), a <= b.
__device__ __forceinline__ void baseline_decode(int bl, int n_in, int& a, int& b) {
    int aa = 0, rem = bl;
    while (rem >= n_in - aa) {
        rem -= n_in - aa;
        ++aa;
    }
    a = aa;
    b = aa + rem;
}

// The flags of item `item` = (integration, window, baseline) of R, by the
// group of L lanes that holds it (store = false: compute only).
template <int E, int L>
__device__ __forceinline__ void mad_flag_item(const float2* R, uint8_t* F, int n_chan, int n_in, int W, float sigma,
                                              long long item, int lane, bool store = true) {
    const int n_bl = n_in * (n_in + 1) / 2;
    const int n_win = n_chan / W;
    const int bl = (int)(item % n_bl);
    const int w = (int)((item / n_bl) % n_win);
    const int i = (int)(item / ((long long)n_bl * n_win));
    int a, b;
    baseline_decode(bl, n_in, a, b);
    const size_t cs = (size_t)n_in * n_in;
    const size_t base = (size_t)i * n_chan * cs + (size_t)w * W * cs;
    const int c0 = (lane & (L - 1)) * E;
    // every load issued before the first magnitude
    float2 u[E];
#pragma unroll
    for (int e = 0; e < E; ++e)
        u[e] = c0 + e < W ? __ldcg(R + base + (size_t)(c0 + e) * cs + (size_t)a * n_in + b) : make_float2(0.f, 0.f);
    float A[E];
#pragma unroll
    for (int e = 0; e < E; ++e) A[e] = c0 + e < W ? vis_abs(u[e]) : __int_as_float(0x7f800000);   // +inf last
    const float T = group_mad_threshold<E, L>(A, W, sigma, lane);
    if (!store) return;
#pragma unroll
    for (int e = 0; e < E; ++e) {
        if (c0 + e < W) {
            const uint8_t f = A[e] > T ? 1 : 0;
            F[base + (size_t)(c0 + e) * cs + (size_t)a * n_in + b] = f;
            F[base + (size_t)(c0 + e) * cs + (size_t)b * n_in + a] = f;
        }
    }
}

template <int E>
__global__ void __launch_bounds__(32 * kFlagWarps) mad_flag_kernel(const float2* R, uint8_t* F, int n_vis,
                                                                   int n_chan, int n_in, int W, float sigma) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long item = (long long)blockIdx.x * kFlagWarps + warp;
    const long long n_items = (long long)n_vis * (n_chan / W) * (n_in * (n_in + 1) / 2);
    if (item >= n_items) return;   // uniform over the warp
    mad_flag_item<E, 32>(R, F, n_chan, n_in, W, sigma, item, lane);
}

// Many items (large arrays): groups of 4 lanes, 32 / 4 items a warp.  A
// group past the last item computes the last item again without storing, so
// that every lane of the warp takes part in the shuffles.
constexpr long long kGroupFlagItems = 16384;
constexpr int kFlagGroup = 4;

template <int E>
__global__ void __launch_bounds__(128) mad_flag_group_kernel(const float2* R, uint8_t* F, int n_vis, int n_chan,
                                                             int n_in, int W, float sigma) {
    const int lane = threadIdx.x & 31;
    const long long n_items = (long long)n_vis * (n_chan / W) * (n_in * (n_in + 1) / 2);
    long long item = ((long long)blockIdx.x * blockDim.x + threadIdx.x) / kFlagGroup;
    const bool valid = item < n_items;
    if (!valid) item = n_items - 1;
    mad_flag_item<E, kFlagGroup>(R, F, n_chan, n_in, W, sigma, item, lane, valid);
}

// Finalisation and MAD flags in one kernel for small arrays (n_in <= 8,
// windows of at most 64 channels): one CTA per (channel window, 4 x 4 tile).
// Its threads finalise the tile's elements for the window's channels (the
// arithmetic of finalize_kernel; consecutive threads take consecutive
// channels, so the partial-slot reads coalesce) and keep |R| of each
// baseline in shared memory; then one warp per baseline derives Eq. 2's
// threshold from them exactly as mad_flag_kernel does from R, and writes
// the flags.  One launch instead of two, and R is not read back.
constexpr int kFinFlagW = 64;
__global__ void __launch_bounds__(512) fin_flag_small_kernel(const FinArgs F, uint8_t* Fl, int W, float sigma) {
    __shared__ float mag[16][kFinFlagW];
    const int w = blockIdx.x, t = blockIdx.y;
    for (int it = (int)threadIdx.x; it < 16 * W; it += (int)blockDim.x) {
        const int z = it / W, c = it % W;
        const int k = w * W + c;
        int a, b;
        float re, im;
        if (fin_value(F, k, t, z, a, b, re, im)) {
            fin_store(F, k, a, b, re, im);
            mag[z][c] = vis_abs(make_float2(re, im));
        }
    }
    __syncthreads();
    const int warp = (int)threadIdx.x >> 5, lane = (int)threadIdx.x & 31;
    const int n_in_pad = (F.n_in + 3) & ~3;
    int A, B;
    tile_decode(t, n_in_pad >> 2, A, B);
    for (int z = warp; z < 16; z += (int)(blockDim.x >> 5)) {
        const int i = z >> 2, j = z & 3;
        const int a = 4 * A + i, b = 4 * B + j;
        if (a >= F.n_in || b >= F.n_in || (A == B && i > j)) continue;   // uniform over the warp
        float v[2];
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const int c = lane * 2 + e;
            v[e] = c < W ? mag[z][c] : __int_as_float(0x7f800000);
        }
        const float T = group_mad_threshold<2>(v, W, sigma, lane);
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const int c = lane * 2 + e;
            if (c < W) {
                const int k = w * W + c;
                const uint8_t f = v[e] > T ? 1 : 0;
                Fl[((size_t)k * F.n_in + a) * F.n_in + b] = f;
                Fl[((size_t)k * F.n_in + b) * F.n_in + a] = f;
            }
        }
    }
}

template <int E>
__device__ __forceinline__ void tail_flags(const TailMember& m, const TailItem& it, int warp, int lane) {
    const int n_bl = m.fin.n_in * (m.fin.n_in + 1) / 2;
    const long long n_wi = (long long)(m.fin.n_chan / m.window) * n_bl;
    const float2* R = m.fin.R + (size_t)it.integration * m.vis_stride;
    uint8_t* F = m.flags + (size_t)it.integration * m.vis_stride;
    for (int q = warp; q < kTailWarpItems; q += kFlagWarps) {
        const long long wi = (long long)it.x + q;
        if (wi < n_wi) mad_flag_item<E, 32>(R, F, m.fin.n_chan, m.fin.n_in, m.window, m.sigma, wi, lane);
    }
}

__global__ void __launch_bounds__(128) group_tail_kernel(const TailArgs T) {
    __shared__ int tk, ok;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (;;) {
        if (threadIdx.x == 0) tk = atomicAdd(T.ticket, 1);
        __syncthreads();
        const int t = tk;
        __syncthreads();                 // every thread has t before tk is rewritten
        if (t >= T.n_items) return;      // uniform over the CTA
        const TailItem it = T.items[t];
        const TailMember& m = T.members[it.member];
        if (it.kind == 0) {
            FinArgs f = m.fin;
            f.part += (size_t)it.integration * m.part_stride;
            f.R += (size_t)it.integration * m.vis_stride;
            finalize_block(f, it.x, it.y, it.z);
            __syncthreads();             // the block's R values are written
            if (threadIdx.x == 0) {
                __threadfence();
                if (t != T.inject_skip) atomicAdd(T.done + it.dep, 1);
            }
        } else {
            if (threadIdx.x == 0) {
                int good = 1;
                if (it.need > 0) {
                    const volatile int* d = T.done + it.dep;
                    if (*d < it.need) {
                        const unsigned long long t0 = tc::globaltimer();
                        while (*d < it.need) {
                            if (tc::globaltimer() - t0 > T.wait_ns) {
                                good = 0;
                                break;
                            }
                        }
                    }
                    __threadfence();
                }
                if (!good && T.status) atomicExch(T.status, CORR_ETIMEDOUT);
                ok = good;
            }
            __syncthreads();
            if (ok) {
                if (m.window <= 32) tail_flags<1>(m, it, warp, lane);
                else if (m.window <= 64) tail_flags<2>(m, it, warp, lane);
                else if (m.window <= 128) tail_flags<4>(m, it, warp, lane);
                else tail_flags<8>(m, it, warp, lane);
            }
        }
    }
}

}  // namespace

void launch_group_tail(const TailArgs& a, int grid, cudaStream_t st) {
    if (a.n_items <= 0) return;
    group_tail_kernel<<<grid, 128, 0, st>>>(a);
}

int group_tail_grid() {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, group_tail_kernel, 128, 0);
    if (sms < 1) sms = 152;
    if (per < 1) per = 1;
    return sms * per;
}

void launch_xengine(const XArgs& a, cudaStream_t st) {
    if (a.n_groups <= 0) return;
    if (a.n_in_pad <= 8) {
        constexpr int per_cta = 4 * kXsChan;          // 4 warps of 16 channels
        dim3 grid((a.n_chan + per_cta - 1) / per_cta, a.n_groups);
        const bool d4 = a.depth == 4;                 // else 6 (the default)
#define CORR_XS(NB, PM, D) xengine_small_kernel<NB, PM, D><<<grid, 128, xs_smem_bytes<NB, D>(), st>>>(a)
        if (a.pair_major) {
            if (a.n_in_pad == 4) { if (d4) CORR_XS(1, true, 4); else CORR_XS(1, true, 6); }
            else { if (d4) CORR_XS(2, true, 4); else CORR_XS(2, true, 6); }
        } else {
            if (a.n_in_pad == 4) { if (d4) CORR_XS(1, false, 4); else CORR_XS(1, false, 6); }
            else { if (d4) CORR_XS(2, false, 4); else CORR_XS(2, false, 6); }
        }
#undef CORR_XS
        return;
    }
    dim3 grid((a.n_chan + 127) / 128, a.nt, a.n_groups);
    if (a.pair_major) xengine_kernel<true><<<grid, 128, 0, st>>>(a);
    else xengine_kernel<false><<<grid, 128, 0, st>>>(a);
}

void launch_finalize(const FinArgs& a, cudaStream_t st) {
    dim3 grid((a.n_chan + 127) / 128, a.nt, 16);
    finalize_kernel<<<grid, 128, 0, st>>>(a);
}

bool fin_flag_small_supported(int n_in, int window) { return n_in <= 8 && window <= kFinFlagW; }

void launch_fin_flag_small(const FinArgs& a, uint8_t* F, int window, float sigma, cudaStream_t st) {
    dim3 grid((unsigned)(a.n_chan / window), (unsigned)a.nt);
    fin_flag_small_kernel<<<grid, 512, 0, st>>>(a, F, window, sigma);
}

void launch_mad_flags(const float2* R, uint8_t* F, int n_vis, int n_chan, int n_in, int window,
                      float sigma, cudaStream_t st) {
    const long long items = (long long)n_vis * (n_chan / window) * (n_in * (n_in + 1) / 2);
    if (items <= 0) return;
    if (window <= 64 && items >= kGroupFlagItems) {
        const unsigned tb = (unsigned)((items * kFlagGroup + 127) / 128);
        constexpr int G = kFlagGroup;
        if (window <= 16) mad_flag_group_kernel<16 / G><<<tb, 128, 0, st>>>(R, F, n_vis, n_chan, n_in, window, sigma);
        else if (window <= 32) mad_flag_group_kernel<32 / G><<<tb, 128, 0, st>>>(R, F, n_vis, n_chan, n_in, window, sigma);
        else mad_flag_group_kernel<64 / G><<<tb, 128, 0, st>>>(R, F, n_vis, n_chan, n_in, window, sigma);
        return;
    }
    const unsigned blocks = (unsigned)((items + kFlagWarps - 1) / kFlagWarps);
    if (window <= 32) mad_flag_kernel<1><<<blocks, 32 * kFlagWarps, 0, st>>>(R, F, n_vis, n_chan, n_in, window, sigma);
    else if (window <= 64) mad_flag_kernel<2><<<blocks, 32 * kFlagWarps, 0, st>>>(R, F, n_vis, n_chan, n_in, window, sigma);
    else if (window <= 128) mad_flag_kernel<4><<<blocks, 32 * kFlagWarps, 0, st>>>(R, F, n_vis, n_chan, n_in, window, sigma);
    else mad_flag_kernel<8><<<blocks, 32 * kFlagWarps, 0, st>>>(R, F, n_vis, n_chan, n_in, window, sigma);
}

}  // namespace corr
