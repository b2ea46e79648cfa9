// Implicit-GEMM 5x5 convolution on tcgen05 for the learned flagger's
// 32-channel layers (no im2col buffer):
//   Z[p][o] = sum_{u,v} sum_c X[n][i + s(u-2)][j + s(v-2)][c] W[o][(5u+v) 32 + c]
// with s = +1 (forward) or -1 (the data gradient, whose operand is the
// output gradient and whose weights are the transposed layout).
//
// X is NHWC BF16 [n][64][256][32].  One M tile is 128 pixels of one image
// row.  For each of the five kernel rows u the producer loads the halo row
// segment X[n][i + s(u-2)][j0-2 .. j0+129][0..31] once, with a 5D TMA box
// that lays it out as the K-major no-swizzle operand format: core matrices
// of 8 consecutive pixels x 8 channels (16 bytes) stored contiguously,
// [channel group][pixel][8 channels].  The A operand of tap (u, v) is then
// the same buffer with its start moved by 2 + s(v-2) pixels (16 bytes each):
// five taps per load, 42 KiB of operand traffic per M tile instead of 200.
// Pixels outside the image come back as zeros from the TMA's out-of-bounds
// fill, which is exactly the convolution's zero padding.  All 25 taps'
// weights (BN x 32 each, 64-byte swizzle) stay resident in shared memory.
// K per M tile = 25 taps x 32 channels = 50 MMAs of K = 16.
//
// Warp roles (192 threads): warp 0 lane 0 issues TMA into a ring of A
// stages, warp 1 lane 0 issues tcgen05.mma into one of two TMEM accumulators
// (M = 128, N = BN = 32), warps 2-5 drain the other accumulator (bias, ReLU,
// BF16 NHWC store; or raw FP32).  CTAs are persistent over M
// tiles.  Every wait is bounded by %globaltimer; on expiry the CTA records
// CORR_ETIMEDOUT, stops issuing, frees its TMEM and returns.
#include "corr.h"
#include "corr_internal.h"

#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include "tc_common.cuh"

namespace corr {

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder();

namespace {

using namespace tc;

constexpr int kImgH = 64, kImgW = 256, kCh = 32;
constexpr int kTaps = 25;
constexpr int kAStages = 6;
constexpr int kHalo = 132;                   // 128 pixels + 2 on each side
constexpr int kGroupBytes = kHalo * 16;      // one 8-channel group of the halo row: 2112 bytes
constexpr int kATile = 4 * kGroupBytes;      // 8448 bytes: 132 pixels x 32 channels BF16
constexpr int kConvThreads = 192;

struct __align__(8) ConvShared {
    uint64_t full[kAStages];
    uint64_t empty[kAStages];
    uint64_t wfull;
    uint64_t acc_full[2];
    uint64_t acc_empty[2];
    uint64_t mma_done;       // every MMA the issuer started has completed
    uint32_t tmem_addr;
    int abort;
};

template <int BN>
__host__ __device__ constexpr uint32_t conv_idesc() {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

template <int BN>
__host__ __device__ constexpr size_t conv_smem() {
    // 1024-byte alignment slack twice, A ring, resident weights, 8 KiB guard, barriers
    return 2048 + (size_t)kAStages * kATile + (size_t)kTaps * BN * 64 + 8192 + sizeof(ConvShared);
}

template <int BN>
__device__ __forceinline__ void conv_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
        "l"(a), "l"(b), "r"(conv_idesc<BN>()), "r"(acc)
        : "memory");
}

__device__ __forceinline__ bool aborted(ConvShared* sh) { return *(volatile int*)&sh->abort != 0; }

template <int BN>
__global__ void __launch_bounds__(kConvThreads, 1)
    conv_kernel(const __grid_constant__ CUtensorMap tx, const __grid_constant__ CUtensorMap tw, ConvArgs A) {
    constexpr int kWTile = BN * 64;
    constexpr uint32_t kCols = 2 * BN < 32 ? 32 : 2 * BN;
    extern __shared__ __align__(1024) uint8_t csm_raw[];
    uint8_t* a_st = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(csm_raw) + 1023) & ~uintptr_t(1023));
    uint8_t* w_st = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(a_st + kAStages * kATile) + 1023) &
                                               ~uintptr_t(1023));
    ConvShared* sh = reinterpret_cast<ConvShared*>(w_st + kTaps * kWTile + 8192);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n_mt = A.n_images * kImgH * 2;
    const int my_count = (int)blockIdx.x < n_mt ? (n_mt - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x : 0;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kAStages; ++s) {
            mbar_init(&sh->full[s], 1);
            mbar_init(&sh->empty[s], 1);
        }
        mbar_init(&sh->wfull, 1);
        for (int b = 0; b < 2; ++b) {
            mbar_init(&sh->acc_full[b], 1);
            mbar_init(&sh->acc_empty[b], 4);
        }
        mbar_init(&sh->mma_done, 1);
        sh->abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&sh->tmem_addr)),
                     "r"(kCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = sh->tmem_addr;
    int issued = 0;   // A-ring loads issued (producer thread)

    if (warp == 0 && lane == 0) {
        // ---- TMA producer: resident weights, then the A ring
        mbar_expect_tx(&sh->wfull, kTaps * kWTile);
        for (int t = 0; t < kTaps; ++t) tma_load_2d(w_st + t * kWTile, &tw, &sh->wfull, t * kCh, 0);
        int it = 0;
        for (int lt = 0; lt < my_count && !aborted(sh); ++lt) {
            const int mt = (int)blockIdx.x + lt * (int)gridDim.x;
            const int n = mt / (kImgH * 2), rem = mt % (kImgH * 2);
            const int i = rem >> 1, j0 = (rem & 1) * 128;
            for (int u = 0; u < 5; ++u, ++it) {
                const int s = it % kAStages;
                const uint32_t ph = (uint32_t)(it / kAStages) & 1u;
                if (!mbar_wait(&sh->empty[s], ph ^ 1u)) {
                    sh->abort = 1;
                    break;
                }
                mbar_expect_tx(&sh->full[s], kATile);
                // box {8 channels, 132 pixels, 4 channel groups, 1 row, 1 image}
                tma_load_5d(a_st + s * kATile, &tx, &sh->full[s], 0, j0 - 2, 0, i + A.sgn * (u - 2), n);
                issued = it + 1;
            }
        }
    } else if (warp == 1 && lane == 0) {
        // ---- MMA issuer
        if (!mbar_wait(&sh->wfull, 0)) sh->abort = 1;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        int it = 0;
        for (int lt = 0; lt < my_count && !aborted(sh); ++lt) {
            const int b = lt & 1;
            const uint32_t use = (uint32_t)(lt >> 1);
            if (!mbar_wait(&sh->acc_empty[b], (use & 1u) ^ 1u)) {
                sh->abort = 1;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t d = tmem + (uint32_t)(b * BN);
            bool ok = true;
            for (int u = 0; u < 5; ++u, ++it) {
                const int s = it % kAStages;
                const uint32_t ph = (uint32_t)(it / kAStages) & 1u;
                if (!mbar_wait(&sh->full[s], ph)) {
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t a0 = smem_u32(a_st + s * kATile);
#pragma unroll
                for (int v = 0; v < 5; ++v) {
                    const int tap = 5 * u + v;
                    // tap (u, v) reads pixels j0 + s(v-2) .. : 2 + s(v-2) rows into the halo
                    const uint32_t off = (uint32_t)(2 + A.sgn * (v - 2)) * 16u;
                    const uint64_t da = sdesc_plain(a0 + off, kGroupBytes, 128);
                    const uint64_t db = sdesc64(smem_u32(w_st + tap * kWTile));
                    conv_mma<BN>(d, da, db, tap != 0 ? 1u : 0u);
                    // channels 16..31: two 8-channel groups further in K, +32 bytes in the weights
                    conv_mma<BN>(d, sdesc_plain(a0 + off + 2 * kGroupBytes, kGroupBytes, 128), db + 2, 1u);
                }
                mma_commit(&sh->empty[s]);
            }
            if (!ok) {
                sh->abort = 1;
                break;
            }
            mma_commit(&sh->acc_full[b]);
        }
        mma_commit(&sh->mma_done);
    } else if (warp >= 2) {
        // ---- epilogue: warp w reads TMEM lanes 32 (w % 4) .. +31
        const int q = warp & 3;
        const int row = q * 32 + lane;
        for (int lt = 0; lt < my_count; ++lt) {
            const int b = lt & 1;
            const uint32_t use = (uint32_t)(lt >> 1);
            bool ready = !aborted(sh) && mbar_wait(&sh->acc_full[b], use & 1u);
            ready = __all_sync(0xffffffffu, ready);
            if (!ready) {
                if (lane == 0) sh->abort = 1;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            uint32_t r[32];
            const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(b * BN);
            tmem_ld32(taddr, r);
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(&sh->acc_empty[b]);
            const int mt = (int)blockIdx.x + lt * (int)gridDim.x;
            const int n = mt / (kImgH * 2), rem = mt % (kImgH * 2);
            const size_t p = (size_t)n * (kImgH * kImgW) + (size_t)(rem >> 1) * kImgW + (rem & 1) * 128 + row;
            if (A.mode == 0) {
                // hidden layer: BF16 ReLU(z + b), 32 channels = 64 bytes
                uint32_t pk[16];
#pragma unroll
                for (int c = 0; c < 16; ++c) {
                    const float z0 = fmaxf(__uint_as_float(r[2 * c]) + __ldg(A.bias + 2 * c), 0.f);
                    const float z1 = fmaxf(__uint_as_float(r[2 * c + 1]) + __ldg(A.bias + 2 * c + 1), 0.f);
                    const __nv_bfloat162 h = __floats2bfloat162_rn(z0, z1);
                    pk[c] = *reinterpret_cast<const uint32_t*>(&h);
                }
                uint4* o = reinterpret_cast<uint4*>(reinterpret_cast<uint16_t*>(A.out) + p * kCh);
#pragma unroll
                for (int v = 0; v < 4; ++v) o[v] = make_uint4(pk[4 * v], pk[4 * v + 1], pk[4 * v + 2], pk[4 * v + 3]);
            } else {
                float4* o = reinterpret_cast<float4*>(reinterpret_cast<float*>(A.out) + p * BN);
#pragma unroll
                for (int v = 0; v < BN / 4; ++v)
                    o[v] = make_float4(__uint_as_float(r[4 * v]), __uint_as_float(r[4 * v + 1]),
                                       __uint_as_float(r[4 * v + 2]), __uint_as_float(r[4 * v + 3]));
            }
        }
    }
    __syncwarp();
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (sh->abort) {   // uniform: written before the barrier above only
        // wait (bounded) for the copies and MMAs still in flight before the
        // shared memory and TMEM are given back
        if (threadIdx.x == 0 && A.status) atomicExch(A.status, CORR_ETIMEDOUT);
        if (warp == 0 && lane == 0) {
            drain_loads(sh->full, kAStages, issued, kWaitNs);
            mbar_wait(&sh->wfull, 0);
        }
        if (warp == 1 && lane == 0) mbar_wait(&sh->mma_done, 0);
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
    }
    if (warp == 0) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kCols) : "memory");
    }
}

bool encode(CUtensorMap* map, CUtensorMapDataType dt, cuuint32_t rank, const void* base, const cuuint64_t* dims,
            const cuuint64_t* strides, const cuuint32_t* box, CUtensorMapSwizzle swz) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return false;
    cuuint32_t estr[5] = {1, 1, 1, 1, 1};
    return enc(map, dt, rank, const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, swz,
               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int BN>
int launch_bn(const ConvArgs& a, cudaStream_t st) {
    CUtensorMap tx, tw;
    // X viewed as [n][row][channel group g][pixel][8 channels]: dims (fastest
    // first) 8 channels, 256 pixels (64 B apart), 4 groups (16 B apart), 64
    // rows, n images
    const cuuint64_t xd[5] = {8, (cuuint64_t)kImgW, 4, (cuuint64_t)kImgH, (cuuint64_t)a.n_images};
    const cuuint64_t xs[4] = {(cuuint64_t)kCh * 2, 16, (cuuint64_t)kCh * 2 * kImgW, (cuuint64_t)kCh * 2 * kImgW * kImgH};
    const cuuint32_t xb[5] = {8, (cuuint32_t)kHalo, 4, 1, 1};
    const cuuint64_t wd[2] = {(cuuint64_t)a.kp, (cuuint64_t)BN};
    const cuuint64_t ws[1] = {(cuuint64_t)a.kp * 2};
    const cuuint32_t wb[2] = {(cuuint32_t)kCh, (cuuint32_t)BN};
    if (!encode(&tx, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, a.X, xd, xs, xb, CU_TENSOR_MAP_SWIZZLE_NONE) ||
        !encode(&tw, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, a.W, wd, ws, wb, CU_TENSOR_MAP_SWIZZLE_64B))
        return CORR_EINVAL;
    static int resident = 0, sms = 0;
    const size_t smem = conv_smem<BN>();
    if (!resident) {
        cudaFuncSetAttribute(conv_kernel<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaFuncSetAttribute(conv_kernel<BN>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared);
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident, conv_kernel<BN>, kConvThreads, smem);
        // the occupancy query can assume a smaller shared-memory carveout
        // than the one requested; take the device's own limits as well
        int smem_sm = 0, reserved = 0;
        cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
        cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
        cudaFuncAttributes fa{};
        cudaFuncGetAttributes(&fa, conv_kernel<BN>);
        int by_smem = smem_sm / (int)(smem + (size_t)reserved);
        int by_regs = fa.numRegs > 0 ? 65536 / (fa.numRegs * kConvThreads) : 1;
        int by_tmem = 512 / (int)(2 * BN < 32 ? 32 : 2 * BN);
        int fit = by_smem < by_regs ? by_smem : by_regs;
        if (by_tmem < fit) fit = by_tmem;
        if (fit > resident) resident = fit;
        if (resident < 1) resident = 1;
        if (sms < 1) sms = 152;
    }
    const int n_mt = a.n_images * kImgH * 2;
    int grid = sms * resident;
    if (grid > n_mt) grid = n_mt;
    conv_kernel<BN><<<grid, kConvThreads, smem, st>>>(tx, tw, a);
    return CORR_OK;
}

}  // namespace

int launch_conv(const ConvArgs& a, cudaStream_t st) {
    if (a.n_images <= 0) return CORR_OK;
    if (!a.X || !a.W || !a.out || (a.sgn != 1 && a.sgn != -1) || a.kp < kTaps * kCh || a.kp % 8) return CORR_EINVAL;
    if ((reinterpret_cast<uintptr_t>(a.X) & 15) || (reinterpret_cast<uintptr_t>(a.W) & 15)) return CORR_EINVAL;
    if (a.bn == 32 && (a.mode == 0 || a.mode == 2)) return launch_bn<32>(a, st);
    return CORR_EINVAL;
}

}  // namespace corr
