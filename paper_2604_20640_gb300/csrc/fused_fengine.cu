// Launcher of the fused F-engine kernel (PFB FIR in shared memory feeding
// the FFT; the kernel is pfb_fft_kernel in fft_core.cuh).
#include "fft_core.cuh"

namespace corr {

namespace {

template <int M, int MODE, int P>
int launch_fused_m(const FusedArgs& a, cudaStream_t st) {
    using FC = FusedCfg<M>;
    static int resident = 0;     // CTAs per SM at this kernel's registers and shared memory
    static int sms = 0;
    const size_t smem = FC::smem_bytes(P);
    if (!resident) {
        if (cudaFuncSetAttribute(pfb_fft_kernel<M, MODE, P>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem) != cudaSuccess)
            return CORR_ECUDA;
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        int r = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&r, pfb_fft_kernel<M, MODE, P>, M / 16, smem) !=
                cudaSuccess || r < 1)
            return CORR_ECUDA;
        if (sms < 1) sms = 152;
        resident = r;
    }
    // One wave of resident CTAs, each over a run of consecutive spectra of
    // one pair (a run's first P-1 frames are read twice: by it and by the
    // run before).
    const long long n = a.f.s_end - a.f.s_begin;
    const int n_groups = a.f.n_in_pad / 2;
    long long runs = (long long)sms * resident / n_groups;
    if (runs > n) runs = n;
    if (runs < 1) runs = 1;
    FusedArgs b = a;
    b.f.spt = a.run > 0 ? a.run : (int)((n + runs - 1) / runs);
    dim3 grid((unsigned)((n + b.f.spt - 1) / b.f.spt), (unsigned)n_groups);
    pfb_fft_kernel<M, MODE, P><<<grid, M / 16, smem, st>>>(b);
    return CORR_OK;
}

template <int MODE>
int launch_fused_mode(const FusedArgs& a, cudaStream_t st) {
    switch (a.f.M) {
        case 1024: if constexpr (MODE >= 2) return launch_fused_m<1024, MODE, 4>(a, st); else return CORR_EINVAL;
        case 2048: if constexpr (MODE >= 2) return launch_fused_m<2048, MODE, 4>(a, st); else return CORR_EINVAL;
        case 4096: if constexpr (MODE >= 2) return launch_fused_m<4096, MODE, 4>(a, st); else return CORR_EINVAL;
        case 8192: return launch_fused_m<8192, MODE, 4>(a, st);
        default: return CORR_EINVAL;
    }
}

}  // namespace

bool fused_f_supported(int M, int taps, int es, int mode) {
    if (es != 1 || taps != 4) return false;
    if (mode == 2 || mode == 3 || mode == 6 || mode == 7) return M >= 1024 && M <= 8192;
    return M == 8192;
}

int launch_fused_f(const FusedArgs& a, cudaStream_t st) {
    const int mode = a.inv ? (a.fp8 ? 7 : 6) : a.f.tiles ? 2 : a.f.phasor ? 1 : a.f.pair_major ? 3 : 0;
    if (!fused_f_supported(a.f.M, a.taps, a.src.es, mode)) return CORR_EINVAL;
    if ((reinterpret_cast<uintptr_t>(a.hs) & 15) != 0) return CORR_EINVAL;
    if (a.f.s_end <= a.f.s_begin) return CORR_OK;
    switch (mode) {
        case 0: return launch_fused_mode<0>(a, st);
        case 1: return launch_fused_mode<1>(a, st);
        case 2: return launch_fused_mode<2>(a, st);
        case 6: return launch_fused_mode<6>(a, st);
        case 7: return launch_fused_mode<7>(a, st);
        default: return launch_fused_mode<3>(a, st);
    }
}

}  // namespace corr
