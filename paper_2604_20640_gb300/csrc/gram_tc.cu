// Tensor-core X-engine: per channel, the Gram matrix G = Q Q^T of the
// requantised voltages stacked as Q = [Q_re; Q_im] (2N <= 128 rows, K = time),
// so that
//   sum_s q_a conj(q_b) = (G_rr + G_ii)[a][b] + j (G_ir - G_ri)[a][b]
// (the X-engine of Sec. 4.2 / Algorithm 1 as a dense contraction).
//
// sm_103a has no integer tcgen05 MMA, so int8 codes travel as BF16 (exact
// for |q| <= 127; every product is exact) through tcgen05.mma.kind::f16, and
// e4m3 codes through kind::f8f6f4; both accumulate in FP32.  Either way one
// MMA consumes 32 bytes of K per row.
//
// One CTA per channel, 128 threads.  Warp 0 lane 0 streams 128-row x 128-byte
// K-tiles of Q through a ring of shared-memory stages with TMA (128-byte
// swizzle); warp 1 lane 0 issues tcgen05.mma (M = N = 128, the same shared
// tile as A and B operand) into a 128-column FP32 TMEM accumulator; all four
// warps then read their 32 TMEM lanes with tcgen05.ld and store G.  Every
// mbarrier wait is bounded by %globaltimer; on expiry the CTA records
// CORR_ETIMEDOUT in the status word, frees its TMEM and returns.
#include "corr.h"
#include "corr_internal.h"

#include <cuda.h>
#include <cudaTypedefs.h>

#include "finq.cuh"
#include "tc_common.cuh"

#include <cstdio>

namespace corr {

namespace {

using namespace tc;

constexpr int kRows = 128;
constexpr int kKTile = 128;                      // bytes of K per stage
constexpr int kStages = 6;
constexpr int kStageBytes = kRows * kKTile;      // 16 KiB
constexpr uint32_t kTmemCols = 128;
struct __align__(8) GramShared {
    uint64_t full[kStages];
    uint64_t empty[kStages];
    uint64_t accum;
    uint32_t tmem_addr;
    int abort;
};

// Instruction descriptor: dense, K-major A and B, M = N = 128, FP32
// accumulator; A/B format BF16 (kind::f16) or E4M3 (kind::f8f6f4).
__host__ __device__ constexpr uint32_t idesc(bool fp8) {
    return (1u << 4)                                 // FP32 accumulator
           | (fp8 ? 0u : (1u << 7))                  // A: E4M3 (0) / BF16 (1)
           | (fp8 ? 0u : (1u << 10))                 // B: E4M3 (0) / BF16 (1)
           | ((uint32_t)(kRows >> 3) << 17)          // N >> 3
           | ((uint32_t)(kRows >> 4) << 24);         // M >> 4
}

template <bool FP8>
__device__ __forceinline__ void mma(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t acc) {
    if constexpr (FP8) {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
            "l"(a), "l"(b), "r"(idesc(true)), "r"(acc)
            : "memory");
    } else {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
            "l"(a), "l"(b), "r"(idesc(false)), "r"(acc)
            : "memory");
    }
}

template <bool FP8>
__global__ void __launch_bounds__(128, 1) gram_kernel(const __grid_constant__ CUtensorMap tmap, GramArgs A) {
    extern __shared__ __align__(1024) uint8_t gsm_raw[];
    // stage buffers first (1024-byte aligned), then the barriers
    uint8_t* stages = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(gsm_raw) + 1023) & ~uintptr_t(1023));
    GramShared* sh = reinterpret_cast<GramShared*>(stages + kStages * kStageBytes);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ch = blockIdx.x;
    const int kt_elems = FP8 ? kKTile : kKTile / 2;
    const int num_k = (A.K + kt_elems - 1) / kt_elems;
    const unsigned long long lim = A.wait_ns ? A.wait_ns : kWaitNs;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&sh->full[s], 1);
            mbar_init(&sh->empty[s], 1);
        }
        mbar_init(&sh->accum, 1);
        sh->abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&sh->tmem_addr)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = sh->tmem_addr;
    int issued = 0;   // TMA loads issued (producer thread)

    if (warp == 0 && lane == 0) {
        // TMA producer (with inject_stall it issues nothing: the MMA issuer's
        // first wait on a full barrier then expires -- the test of this path)
        for (int it = 0; it < (A.inject_stall ? 0 : num_k); ++it) {
            const int s = it % kStages;
            const uint32_t ph = (uint32_t)(it / kStages) & 1u;
            if (!mbar_wait(&sh->empty[s], ph ^ 1u, lim)) {
                sh->abort = 1;
                break;
            }
            mbar_expect_tx(&sh->full[s], kStageBytes);
            // inner coordinate in elements: 128 bytes = 128 e4m3 or 64 BF16
            tma_load_2d(stages + s * kStageBytes, &tmap, &sh->full[s], it * (FP8 ? kKTile : kKTile / 2),
                        ch * kRows);
            issued = it + 1;
        }
    } else if (warp == 1 && lane == 0) {
        // MMA issuer
        bool ok = true;
        for (int it = 0; it < num_k && ok; ++it) {
            const int s = it % kStages;
            const uint32_t ph = (uint32_t)(it / kStages) & 1u;
            if (!mbar_wait(&sh->full[s], ph, lim)) {
                ok = false;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint64_t d0 = sdesc(smem_u32(stages + s * kStageBytes));
#pragma unroll
            for (int kk = 0; kk < kKTile / 32; ++kk) {
                const uint64_t d = d0 + (uint64_t)((kk * 32) >> 4);
                mma<FP8>(tmem, d, d, (it | kk) != 0 ? 1u : 0u);
            }
            mma_commit(&sh->empty[s]);
        }
        if (!ok) sh->abort = 1;
        mma_commit(&sh->accum);
    }
    __syncwarp();
    // Epilogue: warp w owns TMEM lanes (rows) 32w .. 32w+31.
    if (!mbar_wait(&sh->accum, 0, lim)) sh->abort = 1;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    __syncthreads();
    if (sh->abort) {
        if (threadIdx.x == 0 && A.status) atomicExch(A.status, CORR_ETIMEDOUT);
        if (warp == 0 && lane == 0) drain_loads(sh->full, kStages, issued, lim);
    } else {
        const int row = warp * 32 + lane;
        uint32_t* G = reinterpret_cast<uint32_t*>(A.G) + ((size_t)ch * kRows + row) * kRows;
#pragma unroll
        for (int c0 = 0; c0 < kRows; c0 += 32) {
            uint32_t r[32];
            tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, r);
            uint4* o = reinterpret_cast<uint4*>(G + c0);
#pragma unroll
            for (int i = 0; i < 8; ++i) o[i] = make_uint4(r[4 * i], r[4 * i + 1], r[4 * i + 2], r[4 * i + 3]);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols)
                     : "memory");
    }
}

// ---- int8 codes stored as bytes ---------------------------------------------
// The same Gram matrix with the codes in HBM as int8 bytes (half the bytes of
// the BF16-carried form).  There is no integer tcgen05 MMA on sm_103a, so the
// codes are widened on chip: 256 threads; warp 0 lane 0 streams raw
// 128-row x 128-byte int8 tiles by TMA (128-byte swizzle, so a converter
// warp's row reads spread over all banks); warps 4-11 (half a row per
// thread) widen each tile to two BF16 operand tiles of 64 K-elements in the
// 128-byte-swizzled K-major layout the MMA descriptors describe (16-byte
// chunk q of row r at r * 128 + ((q ^ (r & 7)) << 4)), make them visible to
// the async proxy and signal the MMA issuer (warp 1 lane 0); warps 0-3 read
// the accumulator.  Every wait is bounded; the converters decide each step
// together (barrier with an AND reduction), so no converter can be left
// alone at a named barrier.
// 4 raw + 3 converted stages, one CTA per SM (a 3 + 2 form with two CTAs
// per SM measured slower)
constexpr int kRawStages = 4;
constexpr int kConvStages = 3;
constexpr int kRawBytes = kRows * 128;           // 128 int8 codes per row
constexpr int kConvBytes = 2 * kRows * 128;      // two BF16 tiles of 64 codes per row
struct __align__(8) GramI8Shared {
    uint64_t raw_full[kRawStages];
    uint64_t raw_empty[kRawStages];
    uint64_t conv_full[kConvStages];
    uint64_t conv_empty[kConvStages];
    uint64_t accum;
    uint32_t tmem_addr;
    int abort;
};

constexpr int kConvThreads = 256;   // warps 4-11: two threads a row

// AND of p over the converter threads (named barrier 1).
__device__ __forceinline__ bool converters_all(bool p) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred a, b;\n\tsetp.ne.u32 a, %1, 0;\n\t"
        "bar.red.and.pred b, 1, %2, a;\n\tselp.u32 %0, 1, 0, b;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)p), "n"(kConvThreads)
        : "memory");
    return r != 0;
}

__device__ __forceinline__ void converters_sync() {
    asm volatile("bar.sync 1, %0;" ::"n"(kConvThreads) : "memory");
}

// Two BF16 values (low: byte c of w, high: byte c+1) of sign-flipped int8
// bytes, exact: the float of each code, then its upper half (the lower half
// of a float holding an 8-bit integer is zero).
__device__ __forceinline__ uint32_t bf16x2_of_codes(uint32_t f, int c) {
    const uint32_t s0 = 0x7440u + (uint32_t)c, s1 = 0x7440u + (uint32_t)(c + 1);
    const float x0 = __int_as_float((int)__byte_perm(f, 0x4B000000u, s0)) - 8388736.0f;
    const float x1 = __int_as_float((int)__byte_perm(f, 0x4B000000u, s1)) - 8388736.0f;
    return __byte_perm(__float_as_uint(x0), __float_as_uint(x1), 0x7632);
}

__global__ void __launch_bounds__(128 + kConvThreads, 1) gram_i8_kernel(const __grid_constant__ CUtensorMap tmap,
                                                                        GramArgs A) {
    extern __shared__ __align__(1024) uint8_t gsm_raw[];
    uint8_t* conv = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(gsm_raw) + 1023) & ~uintptr_t(1023));
    uint8_t* raw = conv + kConvStages * kConvBytes;
    GramI8Shared* sh = reinterpret_cast<GramI8Shared*>(raw + kRawStages * kRawBytes);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ch = blockIdx.x;
    const int num_k = (A.K + 127) / 128;
    const unsigned long long lim = A.wait_ns ? A.wait_ns : kWaitNs;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kRawStages; ++s) {
            mbar_init(&sh->raw_full[s], 1);
            mbar_init(&sh->raw_empty[s], 1);
        }
        for (int c = 0; c < kConvStages; ++c) {
            mbar_init(&sh->conv_full[c], 1);
            mbar_init(&sh->conv_empty[c], 1);
        }
        mbar_init(&sh->accum, 1);
        sh->abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&sh->tmem_addr)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = sh->tmem_addr;
    int issued = 0;   // TMA loads issued (producer thread)

    if (warp == 0 && lane == 0) {
        // TMA producer of raw int8 tiles (with inject_stall it issues nothing)
        for (int it = 0; it < (A.inject_stall ? 0 : num_k); ++it) {
            const int s = it % kRawStages;
            const uint32_t ph = (uint32_t)(it / kRawStages) & 1u;
            if (!mbar_wait(&sh->raw_empty[s], ph ^ 1u, lim)) {
                sh->abort = 1;
                break;
            }
            mbar_expect_tx(&sh->raw_full[s], kRawBytes);
            tma_load_2d(raw + s * kRawBytes, &tmap, &sh->raw_full[s], it * 128, ch * kRows);
            issued = it + 1;
        }
    } else if (warp == 1 && lane == 0) {
        // MMA issuer: two BF16 tiles of 64 codes per converted stage
        bool ok = true;
        for (int it = 0; it < num_k && ok; ++it) {
            const int c = it % kConvStages;
            const uint32_t ph = (uint32_t)(it / kConvStages) & 1u;
            if (!mbar_wait(&sh->conv_full[c], ph, lim)) {
                ok = false;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
            for (int hf = 0; hf < 2; ++hf) {
                const uint64_t d0 = sdesc(smem_u32(conv + c * kConvBytes + hf * kRows * 128));
#pragma unroll
                for (int kk = 0; kk < 4; ++kk) {
                    const uint64_t d = d0 + (uint64_t)((kk * 32) >> 4);
                    mma<false>(tmem, d, d, (it | hf | kk) != 0 ? 1u : 0u);
                }
            }
            mma_commit(&sh->conv_empty[c]);
        }
        if (!ok) sh->abort = 1;
        mma_commit(&sh->accum);
    } else if (warp >= 4) {
        // converters: threads 2r and 2r + 1 widen the two halves of row r of
        // each raw tile (16-byte chunks 0-3 and 4-7; the second half visits
        // its chunks rotated by two, so the halves of a row never share a
        // bank in the same step)
        const int cv = (int)threadIdx.x - 128;
        const int r = cv >> 1, hf = cv & 1;
        for (int it = 0; it < num_k; ++it) {
            const int s = it % kRawStages, c = it % kConvStages;
            bool ok = mbar_wait(&sh->raw_full[s], (uint32_t)(it / kRawStages) & 1u, lim);
            ok = ok && mbar_wait(&sh->conv_empty[c], ((uint32_t)(it / kConvStages) & 1u) ^ 1u, lim);
            if (!converters_all(ok)) {
                if (cv == 0) sh->abort = 1;
                break;
            }
            const uint4* src = reinterpret_cast<const uint4*>(raw + s * kRawBytes + r * 128);
            uint8_t* drow = conv + c * kConvBytes + r * 128;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int c16 = 4 * hf + ((j + 2 * hf) & 3);
                const uint4 v = src[c16 ^ (r & 7)];   // the raw tile is 128-byte swizzled too
                const uint32_t w[4] = {v.x ^ 0x80808080u, v.y ^ 0x80808080u, v.z ^ 0x80808080u,
                                       v.w ^ 0x80808080u};
                const uint4 lo = make_uint4(bf16x2_of_codes(w[0], 0), bf16x2_of_codes(w[0], 2),
                                            bf16x2_of_codes(w[1], 0), bf16x2_of_codes(w[1], 2));
                const uint4 hi = make_uint4(bf16x2_of_codes(w[2], 0), bf16x2_of_codes(w[2], 2),
                                            bf16x2_of_codes(w[3], 0), bf16x2_of_codes(w[3], 2));
                // codes 16 c16 .. +15 -> tile c16 / 4, BF16 chunks q0, q0 + 1 of that row
                uint8_t* t = drow + (c16 >> 2) * (kRows * 128);
                const int q0 = 2 * (c16 & 3);
                *reinterpret_cast<uint4*>(t + ((q0 ^ (r & 7)) << 4)) = lo;
                *reinterpret_cast<uint4*>(t + (((q0 + 1) ^ (r & 7)) << 4)) = hi;
            }
            fence_proxy_async_smem();
            converters_sync();
            if (cv == 0) {
                mbar_arrive(&sh->conv_full[c]);
                mbar_arrive(&sh->raw_empty[s]);
            }
        }
    }
    __syncwarp();
    if (!mbar_wait(&sh->accum, 0, lim)) sh->abort = 1;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    __syncthreads();
    if (sh->abort) {
        if (threadIdx.x == 0 && A.status) atomicExch(A.status, CORR_ETIMEDOUT);
        if (warp == 0 && lane == 0) drain_loads(sh->raw_full, kRawStages, issued, lim);
    } else if (warp < 4) {
        const int row = warp * 32 + lane;
        uint32_t* G = reinterpret_cast<uint32_t*>(A.G) + ((size_t)ch * kRows + row) * kRows;
#pragma unroll
        for (int c0 = 0; c0 < kRows; c0 += 32) {
            uint32_t rr[32];
            tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, rr);
            uint4* o = reinterpret_cast<uint4*>(G + c0);
#pragma unroll
            for (int i = 0; i < 8; ++i) o[i] = make_uint4(rr[4 * i], rr[4 * i + 1], rr[4 * i + 2], rr[4 * i + 3]);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols)
                     : "memory");
    }
}

// ---- codes as the F-engine's code words -------------------------------------
// The Gram matrices of an integration straight from the pair-major code
// words C[t][pair][k] (bytes Re U_a, Im U_a, Re U_a+1, Im U_a+1 of input
// pair (a, a+1), a = 2 pair), with no transpose into row-major codes first.
// One CTA per four channels (their four 128 x 128 FP32 accumulators fill
// TMEM's 512 columns), 384 threads: warp 0 lane 0 loads raw boxes of 4
// channels x 32 pairs x 64 spectra (16 contiguous bytes per pair and
// spectrum; pairs past the last, and spectra past K, read as zero) by 3D
// TMA; warps 4-11 turn them into each channel's operand tile (Re of input a
// at row a, Im at row N + a; 128 bytes of K per swizzled row, chunk q of row
// r at (q ^ (r & 7)) x 16) and signal the MMA issuer (warp 1 lane 0); warps
// 0-3 read the accumulators out.  int8 codes are widened to BF16 (exact), 64
// spectra a tile; e4m3 codes are regrouped bytewise, 128 spectra a tile (two
// raw boxes, kind::f8f6f4).  Rows from 2N up are never written: they meet
// only Gram entries no visibility uses.  The epilogue stores the 2N x 2N
// block of each G, or (the pipeline) finalises it into visibilities.
constexpr int kWRawStages = 3;
constexpr int kWConvStages = 2;
constexpr int kWChan = 4;                                   // channels per CTA
constexpr int kWK = 64;                                     // spectra per stage
constexpr int kWPairs = 32;                                 // pairs per box
constexpr int kWRawBytes = kWK * kWPairs * kWChan * 4;      // 32 KiB
constexpr int kWTileBytes = kRows * 128;                    // one channel's operand tile, 16 KiB
constexpr int kWConvBytes = kWChan * kWTileBytes;           // 64 KiB
constexpr uint32_t kWTmemCols = kWChan * 128;               // 512
struct __align__(8) GramWShared {
    uint64_t raw_full[kWRawStages];
    uint64_t raw_empty[kWRawStages];
    uint64_t conv_full[kWConvStages];
    uint64_t conv_empty[kWConvStages];
    uint64_t accum;
    uint32_t tmem_addr;
    int abort;
};

// Byte b of each of w0..w3 gathered into word b (byte m of it from w_m).
__device__ __forceinline__ void bytes_transpose4(uint32_t w0, uint32_t w1, uint32_t w2, uint32_t w3, uint32_t& o0,
                                                 uint32_t& o1, uint32_t& o2, uint32_t& o3) {
    const uint32_t t0 = __byte_perm(w0, w1, 0x5140u), t1 = __byte_perm(w0, w1, 0x7362u);
    const uint32_t t2 = __byte_perm(w2, w3, 0x5140u), t3 = __byte_perm(w2, w3, 0x7362u);
    o0 = __byte_perm(t0, t2, 0x5410u);
    o1 = __byte_perm(t0, t2, 0x7632u);
    o2 = __byte_perm(t1, t3, 0x5410u);
    o3 = __byte_perm(t1, t3, 0x7632u);
}

template <bool FP8>
__global__ void __launch_bounds__(128 + kConvThreads, 1) gram_w_kernel(const __grid_constant__ CUtensorMap tmap,
                                                                       GramArgs A) {
    extern __shared__ __align__(1024) uint8_t gsm_raw[];
    uint8_t* conv = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(gsm_raw) + 1023) & ~uintptr_t(1023));
    uint8_t* raw = conv + kWConvStages * kWConvBytes;
    GramWShared* sh = reinterpret_cast<GramWShared*>(raw + kWRawStages * kWRawBytes);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int quad = blockIdx.x;
    // raw boxes per operand tile: 64 spectra of BF16 or 128 of e4m3 fill a
    // tile's 128-byte rows (a last box wholly past K reads as zeros)
    constexpr int kRawPerConv = FP8 ? 2 : 1;
    const int num_conv = (A.K + kRawPerConv * kWK - 1) / (kRawPerConv * kWK);
    const int num_raw = num_conv * kRawPerConv;
    const unsigned long long lim = A.wait_ns ? A.wait_ns : kWaitNs;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kWRawStages; ++s) {
            mbar_init(&sh->raw_full[s], 1);
            mbar_init(&sh->raw_empty[s], 1);
        }
        for (int c = 0; c < kWConvStages; ++c) {
            mbar_init(&sh->conv_full[c], 1);
            mbar_init(&sh->conv_empty[c], 1);
        }
        mbar_init(&sh->accum, 1);
        sh->abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&sh->tmem_addr)),
                     "r"(kWTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = sh->tmem_addr;
    int issued = 0;   // TMA loads issued (producer thread)

    if (warp == 0 && lane == 0) {
        // TMA producer of raw code-word boxes (with inject_stall it issues nothing)
        for (int it = 0; it < (A.inject_stall ? 0 : num_raw); ++it) {
            const int s = it % kWRawStages;
            const uint32_t ph = (uint32_t)(it / kWRawStages) & 1u;
            if (!mbar_wait(&sh->raw_empty[s], ph ^ 1u, lim)) {
                sh->abort = 1;
                break;
            }
            if (it * kWK >= A.K) {
                // the e4m3 tile's second box wholly past K: nothing to load,
                // the converters write zeros
                mbar_arrive(&sh->raw_full[s]);
            } else {
                mbar_expect_tx(&sh->raw_full[s], kWRawBytes);
                // x: channel 4 quad (16-byte aligned), y: pair 0, z: spectrum
                tma_load_3d(raw + s * kWRawBytes, &tmap, &sh->raw_full[s], kWChan * quad, 0, it * kWK);
            }
            issued = it + 1;
        }
    } else if (warp == 1 && lane == 0) {
        // MMA issuer: per tile and channel, four MMAs of 32 bytes of K
        bool ok = true;
        for (int it = 0; it < num_conv && ok; ++it) {
            const int c = it % kWConvStages;
            const uint32_t ph = (uint32_t)(it / kWConvStages) & 1u;
            if (!mbar_wait(&sh->conv_full[c], ph, lim)) {
                ok = false;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
            for (int ch = 0; ch < kWChan; ++ch) {
                const uint64_t d0 = sdesc(smem_u32(conv + c * kWConvBytes + ch * kWTileBytes));
#pragma unroll
                for (int kk = 0; kk < 4; ++kk) {
                    const uint64_t d = d0 + (uint64_t)((kk * 32) >> 4);
                    mma<FP8>(tmem + (uint32_t)(ch * 128), d, d, (it | kk) != 0 ? 1u : 0u);
                }
            }
            mma_commit(&sh->conv_empty[c]);
        }
        if (!ok) sh->abort = 1;
        mma_commit(&sh->accum);
    } else if (warp >= 4) {
        // converters: thread (ch, p, half) fills the four rows of input pair
        // p in channel ch for the spectrum blocks of its parity (8 spectra a
        // block as BF16, 16 as e4m3), visited in an order rotated by channel
        // so lanes of one store phase write different chunks
        const int cv = (int)threadIdx.x - 128;
        const int ch = cv & 3, p = (cv >> 2) & 31, tb0 = cv >> 7;
        const int N = A.n_in;
        int row[4];
        bool has[4];
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int a = 2 * p + (b >> 1);
            has[b] = a < N;
            row[b] = (b & 1) ? N + a : a;
        }
        for (int it = 0; it < num_raw; ++it) {
            // raw box it fills half h of tile ct (all of it for BF16)
            const int ct = it / kRawPerConv, h = it % kRawPerConv;
            const int s = it % kWRawStages, c = ct % kWConvStages;
            bool ok = mbar_wait(&sh->raw_full[s], (uint32_t)(it / kWRawStages) & 1u, lim);
            ok = ok && mbar_wait(&sh->conv_empty[c], ((uint32_t)(ct / kWConvStages) & 1u) ^ 1u, lim);
            if (!converters_all(ok)) {
                if (cv == 0) sh->abort = 1;
                break;
            }
            const uint32_t* rw = reinterpret_cast<const uint32_t*>(raw + s * kWRawBytes);
            uint8_t* tile = conv + c * kWConvBytes + ch * kWTileBytes;
            if constexpr (FP8) {
                // e4m3 bytes as they are: 16 spectra of one row per 16-byte
                // chunk, in spectrum order; chunk 4h + j of the row
                const bool past = it * kWK >= A.K;
#pragma unroll
                for (int k = 0; k < 2; ++k) {
                    const int j = (tb0 + 2 * k + ch) & 3;
                    uint32_t w[16];
#pragma unroll
                    for (int i = 0; i < 16; ++i) w[i] = past ? 0u : rw[((j * 16 + i) * kWPairs + p) * kWChan + ch];
                    uint32_t o[4][4];
#pragma unroll
                    for (int g = 0; g < 4; ++g)
                        bytes_transpose4(w[4 * g], w[4 * g + 1], w[4 * g + 2], w[4 * g + 3], o[0][g], o[1][g],
                                         o[2][g], o[3][g]);
                    const int q = 4 * h + j;
#pragma unroll
                    for (int b = 0; b < 4; ++b) {
                        if (!has[b]) continue;
                        *reinterpret_cast<uint4*>(tile + row[b] * 128 + ((q ^ (row[b] & 7)) << 4)) =
                            make_uint4(o[b][0], o[b][1], o[b][2], o[b][3]);
                    }
                }
            } else {
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const int tb = (tb0 + 2 * k + 2 * ch) & 7;
                    uint32_t w[8];
#pragma unroll
                    for (int i = 0; i < 8; ++i) w[i] = rw[((tb * 8 + i) * kWPairs + p) * kWChan + ch];
#pragma unroll
                    for (int b = 0; b < 4; ++b) {
                        if (!has[b]) continue;
                        uint32_t o[4];
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            // byte b of spectra 2q and 2q + 1 -> low, high BF16
                            const uint32_t x = __byte_perm(w[2 * q], w[2 * q + 1], (uint32_t)(b | ((4 + b) << 4)));
                            o[q] = bf16x2_of_codes(x ^ 0x80808080u, 0);
                        }
                        *reinterpret_cast<uint4*>(tile + row[b] * 128 + ((tb ^ (row[b] & 7)) << 4)) =
                            make_uint4(o[0], o[1], o[2], o[3]);
                    }
                }
            }
            fence_proxy_async_smem();
            converters_sync();
            if (cv == 0) {
                if (h == kRawPerConv - 1) mbar_arrive(&sh->conv_full[c]);
                mbar_arrive(&sh->raw_empty[s]);
            }
        }
    }
    __syncwarp();
    if (!mbar_wait(&sh->accum, 0, lim)) sh->abort = 1;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    __syncthreads();
    if (sh->abort) {
        if (threadIdx.x == 0 && A.status) atomicExch(A.status, CORR_ETIMEDOUT);
        if (warp == 0 && lane == 0) drain_loads(sh->raw_full, kWRawStages, issued, lim);
    } else if (A.R) {
        // the finalisation in place, a channel at a time: the 2N x 2N block
        // goes to shared memory (row pitch 2N + 1: conflict-free by rows and
        // by columns; the operand stages are free now) -- warps w, w + 4,
        // w + 8 share TMEM lane quarter w and split its 32-column chunks --
        // with the channel's scales and phasors; then every thread makes
        // visibilities, output (a, b) from the entries of (min, max) so that
        // both triangles are stored in order
        float* __restrict__ Gs = reinterpret_cast<float*>(conv);
        float* __restrict__ sS = Gs + kRows * (kRows + 1);
        float2* __restrict__ sQ = reinterpret_cast<float2*>(sS + 64);
        const int N = A.n_in, n2 = 2 * N, pitch = n2 + 1;
        const float inv4c = 1.0f / (4.0f * (float)A.K);
        const int lq = warp & 3, part = warp >> 2;
#pragma unroll 1
        for (int ch = 0; ch < kWChan; ++ch) {
            const int k = kWChan * quad + ch;
            if (lq * 32 < n2) {
                const int r = lq * 32 + lane;
#pragma unroll 1
                for (int c0 = part * 32; c0 < n2; c0 += 96) {
                    uint32_t rr[32];
                    tmem_ld32(tmem + ((uint32_t)(lq * 32) << 16) + (uint32_t)(ch * 128 + c0), rr);
                    if (r < n2) {
#pragma unroll
                        for (int i = 0; i < 32; ++i)
                            if (c0 + i < n2) Gs[r * pitch + c0 + i] = __uint_as_float(rr[i]);
                    }
                }
            }
            for (int a = (int)threadIdx.x; a < N; a += (int)blockDim.x) {
                sS[a] = __ldg(A.scale + (size_t)a * A.n_chan + k);
                if (A.rot) sQ[a] = __ldg(A.rot + (size_t)a * A.n_chan + k);
            }
            __syncthreads();
            float2* __restrict__ R = A.R + (size_t)k * N * N;
#pragma unroll 4
            for (int idx = (int)threadIdx.x; idx < N * N; idx += (int)blockDim.x) {
                const int a = idx / N, b = idx - a * N;
                const int lo = a < b ? a : b, hi = a < b ? b : a;
                const float2 v = vis_from_gram(Gs[lo * pitch + hi], Gs[(N + lo) * pitch + N + hi],
                                               Gs[(N + lo) * pitch + hi], Gs[lo * pitch + N + hi], sS[lo], sS[hi],
                                               inv4c, lo == hi, A.rot ? sQ + lo : nullptr, sQ + hi);
                R[idx] = a <= b ? v : make_float2(v.x, -v.y);
            }
            __syncthreads();
        }
    } else if (warp < 4 && warp * 32 < 2 * A.n_in) {
        // only the 2N x 2N block the visibilities use is written (in 32-column
        // pieces); the TMEM loads are warp-wide, the stores per row
        const int r = warp * 32 + lane;
        const int n2 = 2 * A.n_in;
#pragma unroll 1
        for (int ch = 0; ch < kWChan; ++ch) {
            uint32_t* G = reinterpret_cast<uint32_t*>(A.G) + ((size_t)(kWChan * quad + ch) * kRows + r) * kRows;
#pragma unroll 1
            for (int c0 = 0; c0 < n2; c0 += 32) {
                uint32_t rr[32];
                tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(ch * 128 + c0), rr);
                if (r < n2) {
                    uint4* o = reinterpret_cast<uint4*>(G + c0);
#pragma unroll
                    for (int i = 0; i < 8; ++i)
                        o[i] = make_uint4(rr[4 * i], rr[4 * i + 1], rr[4 * i + 2], rr[4 * i + 3]);
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kWTmemCols)
                     : "memory");
    }
}

}  // namespace

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

size_t gram_smem_bytes() { return (size_t)kStages * kStageBytes + sizeof(GramShared) + 1024; }

size_t gram_w_smem_bytes() {
    return (size_t)kWConvStages * kWConvBytes + (size_t)kWRawStages * kWRawBytes + sizeof(GramWShared) + 1024;
}

size_t gram_i8_smem_bytes() {
    return (size_t)kConvStages * kConvBytes + (size_t)kRawStages * kRawBytes + sizeof(GramI8Shared) + 1024;
}

int launch_gram(const GramArgs& a, cudaStream_t st) {
    if (a.n_chan <= 0 || a.K <= 0) return CORR_OK;
    if (a.words) {
        // code words C[t][pair][k]: 3D map (k, pair, t) of 32-bit words
        if ((a.n_chan % kWChan) != 0 || a.n_pairs < 1 || a.n_pairs > kWPairs || a.n_in < 1 ||
            a.n_in > 2 * a.n_pairs)
            return CORR_EINVAL;
        if ((reinterpret_cast<uintptr_t>(a.Q) & 15) != 0) return CORR_EINVAL;
        PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
        if (!enc) return CORR_ECUDA;
        CUtensorMap map;
        cuuint64_t dims[3] = {(cuuint64_t)a.n_chan, (cuuint64_t)a.n_pairs, (cuuint64_t)a.K};
        cuuint64_t strides[2] = {(cuuint64_t)a.n_chan * 4, (cuuint64_t)a.n_pairs * a.n_chan * 4};
        cuuint32_t box[3] = {(cuuint32_t)kWChan, (cuuint32_t)kWPairs, (cuuint32_t)kWK};
        cuuint32_t estr[3] = {1, 1, 1};
        CUresult r = enc(&map, CU_TENSOR_MAP_DATA_TYPE_UINT32, 3, const_cast<void*>(a.Q), dims, strides, box, estr,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return CORR_EINVAL;
        const size_t smem = gram_w_smem_bytes();
        static bool attrw[2] = {false, false};
        if (!attrw[a.fp8]) {
            const void* fn = a.fp8 ? reinterpret_cast<const void*>(gram_w_kernel<true>)
                                   : reinterpret_cast<const void*>(gram_w_kernel<false>);
            if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
                return CORR_ECUDA;
            attrw[a.fp8] = true;
        }
        if (a.fp8) gram_w_kernel<true><<<a.n_chan / kWChan, 128 + kConvThreads, smem, st>>>(map, a);
        else gram_w_kernel<false><<<a.n_chan / kWChan, 128 + kConvThreads, smem, st>>>(map, a);
        return CORR_OK;
    }
    if (a.i8b) {
        // int8 codes as bytes: raw tiles of 128 codes x 128 rows, 128-byte
        // swizzle (16-byte chunk q of row r at r * 128 + ((q ^ (r & 7)) << 4)),
        // so the converters' row reads are free of bank conflicts
        if (a.fp8 || a.k_pitch % 128 != 0 || a.K > a.k_pitch) return CORR_EINVAL;
        if ((reinterpret_cast<uintptr_t>(a.Q) & 15) != 0) return CORR_EINVAL;
        PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
        if (!enc) return CORR_ECUDA;
        CUtensorMap map;
        cuuint64_t dims[2] = {(cuuint64_t)a.K, (cuuint64_t)a.n_chan * kRows};
        cuuint64_t strides[1] = {(cuuint64_t)a.k_pitch};
        cuuint32_t box[2] = {128u, (cuuint32_t)kRows};
        cuuint32_t estr[2] = {1, 1};
        CUresult r = enc(&map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<void*>(a.Q), dims, strides, box, estr,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return CORR_EINVAL;
        const size_t smem = gram_i8_smem_bytes();
        static bool attr8 = false;
        if (!attr8) {
            if (cudaFuncSetAttribute(gram_i8_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
                cudaSuccess)
                return CORR_ECUDA;
            attr8 = true;
        }
        gram_i8_kernel<<<a.n_chan, 128 + kConvThreads, smem, st>>>(map, a);
        return CORR_OK;
    }
    const int eb = a.fp8 ? 1 : 2;
    if (a.k_pitch % 128 != 0 || (long long)a.K * eb > a.k_pitch) return CORR_EINVAL;
    if ((reinterpret_cast<uintptr_t>(a.Q) & 15) != 0) return CORR_EINVAL;
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return CORR_ECUDA;
    CUtensorMap map;
    // dim 0: K columns (elements, only the valid ones: later columns read as
    // 0); dim 1: n_chan * 128 rows, k_pitch bytes apart.
    cuuint64_t dims[2] = {(cuuint64_t)a.K, (cuuint64_t)a.n_chan * kRows};
    cuuint64_t strides[1] = {(cuuint64_t)a.k_pitch};
    cuuint32_t box[2] = {(cuuint32_t)(kKTile / eb), (cuuint32_t)kRows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(&map, a.fp8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                     const_cast<void*>(a.Q), dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return CORR_EINVAL;
    const size_t smem = gram_smem_bytes();
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(gram_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaFuncSetAttribute(gram_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        attr = true;
    }
    if (a.fp8) gram_kernel<true><<<a.n_chan, 128, smem, st>>>(map, a);
    else gram_kernel<false><<<a.n_chan, 128, smem, st>>>(map, a);
    return CORR_OK;
}

}  // namespace corr
