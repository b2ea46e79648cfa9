// Allocation-free X-engine entry point.
//
// Some callers cannot allocate device memory: code running while a CUDA
// stream is being captured into a graph that must stay replayable, real-time
// loops that forbid allocator calls (which can synchronise the device), and
// hosts that own the GPU's memory budget themselves.  For them,
// corr_xengine_noalloc computes the same visibilities as corr_xengine_dev
// without any allocation: its partial-sum scratch is the file-scope device
// array below, which every GPU that loads the library holds until exit.
#include "corr.h"
#include "corr_internal.h"

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
// device (host code may not use the array's name as a device pointer).
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
    const int n_in_pad = (n_in + 3) & ~3;
    const int nb = n_in_pad / 4;
    const int nt = nb * (nb + 1) / 2;
    const size_t per_group = (size_t)nt * 32 * (size_t)n_chan;
    if (per_group > kScratchFloats) {
        corr::set_global_error("corr_xengine_noalloc: n_in/n_chan too large for the 8 MiB scratch "
                               "(one group needs blocks*32*n_chan floats <= 2^21)");
        return CORR_EINVAL;
    }
    const long long max_groups = (long long)(kScratchFloats / per_group);
    long long G = 64;
    long long groups = (n_spec + G - 1) / G;
    if (groups > max_groups) {
        G = (n_spec + max_groups - 1) / max_groups;
        groups = (n_spec + G - 1) / G;
    }
    float* scratch = nullptr;
    int rc = scratch_address(&scratch);
    if (rc != CORR_OK) return rc;
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
    corr::FinArgs f{};
    f.part = scratch;
    f.n_slots = (int)groups;
    f.nt = nt;
    f.n_chan = n_chan;
    f.n_in = n_in;
    f.scale = 1.0f / (float)n_spec;
    f.R = reinterpret_cast<float2*>(d_vis);
    corr::launch_finalize(f, st);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        corr::set_global_error(std::string("corr_xengine_noalloc launch: ") + cudaGetErrorString(e));
        return CORR_ECUDA;
    }
    return CORR_OK;
}
