"""GB300-native FX correlator hot path (arXiv 2604.20640): polyphase filter
bank + real FFT with fused coarse/fine delay and phase correction, Hermitian
cross-multiply-accumulate and MAD flagging, as hand-written sm_103a CUDA
behind the C ABI of ``libcorr.so`` (``include/corr.h``).

``Correlator`` is a thin ctypes binding; PyTorch only supplies device memory
and streams.  Build the library with :func:`build` (nvcc, in-tree).
"""

from .corr import (  # noqa: F401
    Correlator, Group, FlagNet, CorrError, load_library, LIB_PATH, EXPORTED, tile_mad, calibrate,
    CORR_OK, CORR_EINVAL, CORR_ENOMEM, CORR_ECUDA, CORR_EAGAIN, CORR_ETIMEDOUT, CORR_ESTATE,
    CORR_FP32, CORR_INT8, CORR_FP8, CORR_INT8_BYTES, CORR_INT8_WORDS, CORR_FP8_WORDS,
)


def build(verbose: bool = False) -> str:
    from .build import build_library
    return build_library(verbose=verbose)
