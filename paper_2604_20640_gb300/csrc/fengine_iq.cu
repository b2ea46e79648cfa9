// Complex (I/Q) input forms of the two F-engine stages (Sec. 4.2: the raw
// samples "converted into complex voltage streams", read as interleaved
// int8 I/Q baseband samples): the FIR filters the I and Q parts of one input
// into z = y_I + j y_Q, and the FFT keeps all M = n_chan channels of Z.  The
// kernels are in fft_core.cuh.
#include "fft_core.cuh"

namespace corr {

void launch_fir_iq(const FirArgs& a, cudaStream_t st) {
    const long long n = a.s_end - a.s_begin;
    if (n <= 0 || a.src.es != 2) return;
    dim3 grid((unsigned)((a.M / 2 + kFirThreads - 1) / kFirThreads), (unsigned)a.n_pairs,
              (unsigned)((n + a.spt - 1) / a.spt));
    switch (a.taps) {
#define CORR_FIR_IQ(P)                                                              \
    case P:                                                                         \
        fir_kernel<P, 2, true><<<grid, kFirThreads, 0, st>>>(a);                    \
        break;
        CORR_FIR_IQ(1) CORR_FIR_IQ(2) CORR_FIR_IQ(3) CORR_FIR_IQ(4) CORR_FIR_IQ(5) CORR_FIR_IQ(6) CORR_FIR_IQ(7)
        CORR_FIR_IQ(8) CORR_FIR_IQ(9) CORR_FIR_IQ(10) CORR_FIR_IQ(11) CORR_FIR_IQ(12) CORR_FIR_IQ(13)
        CORR_FIR_IQ(14) CORR_FIR_IQ(15) CORR_FIR_IQ(16)
#undef CORR_FIR_IQ
        default: break;
    }
}

namespace {

template <int MODE>
int launch_fft_iq_mode(const FftArgs& a, cudaStream_t st) {
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
        default: return CORR_EINVAL;
    }
}

}  // namespace

int launch_fft_iq(const FftArgs& a, cudaStream_t st) {
    if (a.tiles || a.pair_major) return CORR_EINVAL;     // power tiles and the pair-major ring are for real input
    if (a.s_end <= a.s_begin) return CORR_OK;
    return a.phasor ? launch_fft_iq_mode<5>(a, st) : launch_fft_iq_mode<4>(a, st);
}

}  // namespace corr
