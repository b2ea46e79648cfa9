// General tensor-core GEMM for the learned flagger's convolutions (as im2col
// products): D[m][n] = sum_k A[m][k] B[n][k], BF16 operands, FP32
// accumulation in TMEM.
//
// One CTA per (128-row M tile, K split), 128 threads: warp 0 lane 0 streams
// A (128 x 64 BF16) and B (BN x 64 BF16) K-tiles into a ring of shared-memory
// stages with TMA (128-byte swizzle); warp 1 lane 0 issues
// tcgen05.mma.kind::f16 (M = 128, N = BN, K = 16); the four warps read their
// TMEM lanes and store the FP32 tile.  K splits write separate partial tiles
// that launch_split_sum adds in a fixed order.  Waits are bounded as in the
// Gram kernel.
#include "corr.h"
#include "corr_internal.h"

#include <cuda.h>
#include <cudaTypedefs.h>

#include "tc_common.cuh"

namespace corr {

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder();

namespace {

using namespace tc;

constexpr int kGStages = 4;
constexpr int kATile = 128 * 128;      // bytes: 128 rows x 64 BF16

struct __align__(8) GemmShared {
    uint64_t full[kGStages];
    uint64_t empty[kGStages];
    uint64_t accum;
    uint32_t tmem_addr;
    int abort;
};

template <int BN>
__host__ __device__ constexpr uint32_t gemm_idesc() {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

template <int BN>
__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(gemm_idesc<BN>()), "r"(acc)
        : "memory");
}

template <int BN>
__global__ void __launch_bounds__(128, 1) gemm_kernel(const __grid_constant__ CUtensorMap ta,
                                                      const __grid_constant__ CUtensorMap tb, GemmArgs G) {
    constexpr int kBTile = BN * 128;
    constexpr int kStage = kATile + kBTile;
    constexpr uint32_t kCols = BN < 32 ? 32 : BN;
    extern __shared__ __align__(1024) uint8_t gsm_raw[];
    uint8_t* stages = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(gsm_raw) + 1023) & ~uintptr_t(1023));
    GemmShared* sh = reinterpret_cast<GemmShared*>(stages + kGStages * kStage);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.x * 128;
    const int split = blockIdx.y;
    const int k_begin = split * G.k_per_split;
    int k_end = k_begin + G.k_per_split;
    if (k_end > G.K) k_end = G.K;
    const int num_k = k_end > k_begin ? (k_end - k_begin + 63) / 64 : 0;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kGStages; ++s) {
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
                     "r"(kCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = sh->tmem_addr;
    int issued = 0;   // TMA stage loads issued (producer thread)

    if (num_k > 0) {
        if (warp == 0 && lane == 0) {
            for (int it = 0; it < num_k; ++it) {
                const int s = it % kGStages;
                const uint32_t ph = (uint32_t)(it / kGStages) & 1u;
                if (!mbar_wait(&sh->empty[s], ph ^ 1u)) {
                    sh->abort = 1;
                    break;
                }
                mbar_expect_tx(&sh->full[s], kStage);
                tma_load_2d(stages + s * kStage, &ta, &sh->full[s], k_begin + it * 64, m0);
                tma_load_2d(stages + s * kStage + kATile, &tb, &sh->full[s], k_begin + it * 64, 0);
                issued = it + 1;
            }
        } else if (warp == 1 && lane == 0) {
            bool ok = true;
            for (int it = 0; it < num_k && ok; ++it) {
                const int s = it % kGStages;
                const uint32_t ph = (uint32_t)(it / kGStages) & 1u;
                if (!mbar_wait(&sh->full[s], ph)) {
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint64_t da = sdesc(smem_u32(stages + s * kStage));
                const uint64_t db = sdesc(smem_u32(stages + s * kStage + kATile));
#pragma unroll
                for (int kk = 0; kk < 4; ++kk)
                    mma_bf16<BN>(tmem, da + (uint64_t)((kk * 32) >> 4), db + (uint64_t)((kk * 32) >> 4),
                                 (it | kk) != 0 ? 1u : 0u);
                mma_commit(&sh->empty[s]);
            }
            if (!ok) sh->abort = 1;
            mma_commit(&sh->accum);
        }
        __syncwarp();
        if (!mbar_wait(&sh->accum, 0)) sh->abort = 1;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    }
    __syncthreads();
    const int row = m0 + warp * 32 + lane;
    float* D = G.D + ((size_t)split * G.M + row) * BN;
    if (sh->abort) {
        if (threadIdx.x == 0 && G.status) atomicExch(G.status, CORR_ETIMEDOUT);
        if (warp == 0 && lane == 0) drain_loads(sh->full, kGStages, issued, kWaitNs);
    } else if (num_k == 0) {
        if (row < G.M)
            for (int c = 0; c < BN; ++c) D[c] = 0.f;
    } else {
#pragma unroll
        for (int c0 = 0; c0 < BN; c0 += 16) {
            uint32_t r[16];
            tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, r);
            if (row < G.M) {
                float4* o = reinterpret_cast<float4*>(D + c0);
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    o[i] = make_float4(__uint_as_float(r[4 * i]), __uint_as_float(r[4 * i + 1]),
                                       __uint_as_float(r[4 * i + 2]), __uint_as_float(r[4 * i + 3]));
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kCols) : "memory");
    }
}

__global__ void split_sum_kernel(const float* D, int splits, long long mn, float* out) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= mn) return;
    float acc = 0.f;
    for (int s = 0; s < splits; ++s) acc += D[(size_t)s * mn + i];
    out[i] = acc;
}

bool make_map(CUtensorMap* map, const void* base, int K, int rows, int pitch, int box_rows) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return false;
    cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)pitch};
    cuuint32_t box[2] = {64, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int BN>
int launch_bn(const GemmArgs& a, const CUtensorMap& ta, const CUtensorMap& tb, cudaStream_t st) {
    const size_t smem = (size_t)kGStages * (kATile + BN * 128) + sizeof(GemmShared) + 1024;
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(gemm_kernel<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        attr = true;
    }
    dim3 grid((unsigned)((a.M + 127) / 128), (unsigned)a.splits);
    gemm_kernel<BN><<<grid, 128, smem, st>>>(ta, tb, a);
    return CORR_OK;
}

}  // namespace

int launch_gemm(const GemmArgs& a, cudaStream_t st) {
    if (a.M <= 0 || a.K <= 0) return CORR_OK;
    if (a.N != 16 && a.N != 32 && a.N != 64) return CORR_EINVAL;
    if (a.lda % 16 || a.ldb % 16 || a.k_per_split % 64 || a.splits < 1) return CORR_EINVAL;
    if ((long long)a.splits * a.k_per_split < a.K) return CORR_EINVAL;
    if ((reinterpret_cast<uintptr_t>(a.A) & 15) || (reinterpret_cast<uintptr_t>(a.B) & 15)) return CORR_EINVAL;
    CUtensorMap ta, tb;
    if (!make_map(&ta, a.A, a.K, a.M, a.lda, 128) || !make_map(&tb, a.B, a.K, a.N, a.ldb, a.N)) return CORR_EINVAL;
    if (a.N == 16) return launch_bn<16>(a, ta, tb, st);
    if (a.N == 32) return launch_bn<32>(a, ta, tb, st);
    return launch_bn<64>(a, ta, tb, st);
}

void launch_split_sum(const float* D, int splits, long long mn, float* out, cudaStream_t st) {
    if (mn <= 0) return;
    split_sum_kernel<<<(unsigned)((mn + 255) / 256), 256, 0, st>>>(D, splits, mn, out);
}

}  // namespace corr
