// Allocation-free X-engine entry point.
//
// Some callers cannot allocate device memory: real-time loops that forbid
// allocator calls (cudaMalloc and cudaFree can synchronise the device and
// stall the stream that must keep up with the samples), and hosts that own
// the GPU's memory budget themselves (a fixed plan made at start-up, where a
// library allocating behind their back breaks the plan).  For them,
// corr_xengine_noalloc computes the same visibilities as corr_xengine_dev
// without any allocation: its partial-sum scratch is the file-scope device
// array below, which every GPU that loads the library holds until exit.
#include "corr.h"
#include "corr_internal.h"

#include <cstdint>
#include <mutex>
#include <string>

namespace {

// 8 MiB of FP32 partial sums: one group of spectra needs
// (number of 4x4 input blocks A <= B) * 32 * n_chan floats.
constexpr size_t kScratchFloats = (size_t)1 << 21;
static __device__ __align__(256) float g_scratch[kScratchFloats];

constexpr int kMaxDevices = 64;
float* g_scratch_ptr[kMaxDevices] = {};
std::mutex g_mu;

// The device address of g_scratch on the current device, looked up once per
// device (host code may not use the array's name as a device pointer).  The
// address is kept for the life of the process: after cudaDeviceReset the
// cached value would be stale, so calls after a reset are not supported.
int scratch_address(float** out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        corr::set_global_error(std::string("cudaGetDevice: ") + cudaGetErrorString(e));
        return CORR_ECUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) {
        corr::set_global_error("device index out of range for the scratch table");
        return CORR_EINVAL;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p) {
            corr::set_global_error(std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            return CORR_ECUDA;
        }
        g_scratch_ptr[dev] = static_cast<float*>(p);
    }
    *out = g_scratch_ptr[dev];
    return CORR_OK;
}

}  // namespace

extern "C" int corr_xengine_noalloc(const float* d_V, int n_spec, int n_in, int n_chan, float* d_vis,
                                    void* stream) {
    if (!d_V || !d_vis || n_spec < 1 || n_in < 1 || n_in > 256 || n_chan < 1) {
        corr::set_global_error("corr_xengine_noalloc: bad argument");
        return CORR_EINVAL;
    }
    // The X-engine reads V as 16-byte vectors and the finaliser writes
    // complex64 values: misaligned buffers are refused before any launch.
    if ((reinterpret_cast<uintptr_t>(d_V) & 15) != 0 || (reinterpret_cast<uintptr_t>(d_vis) & 7) != 0) {
        corr::set_global_error("corr_xengine_noalloc: d_V must be 16-byte and d_vis 8-byte aligned");
        return CORR_EINVAL;
    }
    const int n_in_pad = (n_in + 3) & ~3;
    const int nb = n_in_pad / 4;
    const int nt = nb * (nb + 1) / 2;
    const size_t per_group = (size_t)nt * 32 * (size_t)n_chan;
    if (per_group > kScratchFloats) {
        corr::set_global_error("corr_xengine_noalloc: n_in/n_chan too large for the 8 MiB scratch "
                               "(one group needs blocks*32*n_chan floats <= 2^21)");
        return CORR_EINVAL;
    }
    // Groups are a grid dimension of the X-engine launch (at most 65535).
    long long max_groups = (long long)(kScratchFloats / per_group);
    if (max_groups > 65535) max_groups = 65535;
    long long G = 64;
    long long groups = (n_spec + G - 1) / G;
    if (groups > max_groups) {
        G = (n_spec + max_groups - 1) / max_groups;
        groups = (n_spec + G - 1) / G;
    }
    float* scratch = nullptr;
    int rc = scratch_address(&scratch);
    if (rc != CORR_OK) return rc;
    // An error left by earlier, unrelated work is reported as such and left
    // in place for its owner, not taken for a failure of these launches.
    cudaError_t e = cudaPeekAtLastError();
    if (e != cudaSuccess) {
        corr::set_global_error(std::string("corr_xengine_noalloc: CUDA error pending before the call: ") +
                               cudaGetErrorString(e));
        return CORR_ECUDA;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    corr::XArgs x{};
    x.V = reinterpret_cast<const float2*>(d_V);
    x.v_origin = 0;
    x.v_mask = -1LL;
    x.n_chan = n_chan;
    x.n_in_pad = n_in_pad;
    x.nt = nt;
    x.int_start = 0;
    x.int_end = n_spec;
    x.s_limit = n_spec;
    x.G = (int)G;
    x.j0 = 0;
    x.n_groups = (int)groups;
    x.part = scratch;
    corr::launch_xengine(x, st);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        corr::set_global_error(std::string("corr_xengine_noalloc: X-engine launch: ") + cudaGetErrorString(e));
        return CORR_ECUDA;
    }
    corr::FinArgs f{};
    f.part = scratch;
    f.n_slots = (int)groups;
    f.nt = nt;
    f.n_chan = n_chan;
    f.n_in = n_in;
    f.scale = 1.0f / (float)n_spec;
    f.R = reinterpret_cast<float2*>(d_vis);
    corr::launch_finalize(f, st);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        corr::set_global_error(std::string("corr_xengine_noalloc: finaliser launch: ") + cudaGetErrorString(e));
        return CORR_ECUDA;
    }
    return CORR_OK;
}
