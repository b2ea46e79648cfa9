// F-engine launchers of the two-kernel path (Sec. 4.2 "F-engine (PFB and
// FFT)"): the polyphase FIR kernel and the FFT kernel, and the FFT's
// twiddle table.  The kernels are in fft_core.cuh.
#include "fft_core.cuh"

namespace corr {

std::vector<float2> fft_twiddle_table(int M) {
    const double pi = 3.14159265358979323846;
    std::vector<float2> t;
    int ns = first_radix(M) == 16 ? 1 : first_radix(M);
    if (first_radix(M) == 16) {
        t.resize(16, make_float2(1.f, 0.f));   // first pass at Ns = 1 (unused)
        ns = 16;
    }
    while (ns < M) {
        for (int r = 0; r < 16; ++r)
            for (int k = 0; k < ns; ++k) {
                const double ang = -2.0 * pi * (double)r * k / (16.0 * ns);
                t.push_back(make_float2((float)std::cos(ang), (float)std::sin(ang)));
            }
        ns *= 16;
    }
    return t;
}

template <int MODE>
static int launch_fft_mode(const FftArgs& a, cudaStream_t st) {
    switch (a.M) {
        case 16: return launch_fft_m<16, MODE>(a, st);
        case 32: return launch_fft_m<32, MODE>(a, st);
        case 64: return launch_fft_m<64, MODE>(a, st);
        case 128: return launch_fft_m<128, MODE>(a, st);
        case 256: return launch_fft_m<256, MODE>(a, st);
        case 512: return launch_fft_m<512, MODE>(a, st);
        case 1024: return launch_fft_m<1024, MODE>(a, st);
        case 2048: return launch_fft_m<2048, MODE>(a, st);
        case 4096: return launch_fft_m<4096, MODE>(a, st);
        case 8192: return launch_fft_m<8192, MODE>(a, st);
        case 16384: return launch_fft_m<16384, MODE>(a, st);
        default: return CORR_EINVAL;
    }
}

int launch_fft(const FftArgs& a, cudaStream_t st) {
    if (a.s_end <= a.s_begin) return CORR_OK;
    if (a.inv) {
        // code words out: the size the fused F-engine leaves to this path
        if (a.M != 16384 || a.iq || a.tiles || a.phasor) return CORR_EINVAL;
        return a.fp8 ? launch_fft_m<16384, 7>(a, st) : launch_fft_m<16384, 6>(a, st);
    }
    if (a.iq) return launch_fft_iq(a, st);
    if (a.tiles) return launch_fft_mode<2>(a, st);
    if (a.phasor) return launch_fft_mode<1>(a, st);
    if (a.pair_major) return launch_fft_mode<3>(a, st);
    return launch_fft_mode<0>(a, st);
}

void launch_fir(const FirArgs& a, cudaStream_t st) {
    const long long n = a.s_end - a.s_begin;
    if (n <= 0) return;
    if (a.iq) {
        launch_fir_iq(a, st);
        return;
    }
    dim3 grid((unsigned)((a.M / 2 + kFirThreads - 1) / kFirThreads), (unsigned)a.n_pairs,
              (unsigned)((n + a.spt - 1) / a.spt));
    switch (a.taps) {
#define CORR_FIR(P)                                                                    \
    case P:                                                                            \
        if (a.src.es == 2) fir_kernel<P, 2><<<grid, kFirThreads, 0, st>>>(a);          \
        else fir_kernel<P, 1><<<grid, kFirThreads, 0, st>>>(a);                        \
        break;
        CORR_FIR(1) CORR_FIR(2) CORR_FIR(3) CORR_FIR(4) CORR_FIR(5) CORR_FIR(6) CORR_FIR(7) CORR_FIR(8)
        CORR_FIR(9) CORR_FIR(10) CORR_FIR(11) CORR_FIR(12) CORR_FIR(13) CORR_FIR(14) CORR_FIR(15) CORR_FIR(16)
#undef CORR_FIR
        default: break;
    }
}

}  // namespace corr

