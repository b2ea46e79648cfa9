"""The allocation-free X-engine (corr_xengine_noalloc) against the
allocating one (corr_xengine_dev) and against the FP64 oracle.

corr_xengine_noalloc serves callers that may not allocate device memory: a
real-time loop in which an allocator call could synchronise the device and
stall the stream that keeps up with the samples, or a host that plans the
GPU's memory itself.  Its scratch is a fixed file-scope device array shared
by all calls.  Two calls in a row, with different shapes, must both agree
with corr_xengine_dev and with the oracle's X-engine within the visibility
tolerance of the parity tests (1e-5 relative Frobenius error per channel),
so nothing left in the shared array by one call leaks into the next.  This
file is collected last on purpose.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import fx_oracle as fx  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_20640_gb300.build import build_library
    build_library()


def _random_V(rng, n_spec, n_chan, n_in):
    n_pad = (n_in + 3) // 4 * 4
    V = np.zeros((n_spec, n_chan, n_pad), dtype=np.complex64)
    V[:, :, :n_in] = (rng.standard_normal((n_spec, n_chan, n_in)) +
                      1j * rng.standard_normal((n_spec, n_chan, n_in))).astype(np.complex64)
    return torch.from_numpy(V).to(DEV)


def test_noalloc_matches_allocating_xengine_on_two_calls():
    from paper_2604_20640_gb300 import Correlator
    from paper_2604_20640_gb300.corr import xengine_noalloc
    rng = np.random.default_rng(2024)
    # second call: smaller shape, and a long stream that needs longer groups
    for (n_in, n_chan, n_spec) in [(8, 512, 300), (5, 4096, 700)]:
        V = _random_V(rng, n_spec, n_chan, n_in)
        ref = torch.empty((n_chan, n_in, n_in), dtype=torch.complex64, device=DEV)
        c = Correlator(n_in, 1, n_chan, 4, 16)
        c.xengine_dev(V, n_spec, ref)
        out = torch.full((n_chan, n_in, n_in), complex(np.nan, np.nan), dtype=torch.complex64, device=DEV)
        xengine_noalloc(V, n_spec, n_in, n_chan, out)
        torch.cuda.synchronize()
        R_ref = ref.cpu().numpy().astype(np.complex128)
        R_out = out.cpu().numpy().astype(np.complex128)
        err = fx.rel_frobenius_per_channel(R_out[None], R_ref[None]).max()
        assert err < 1e-5, err
        # and directly against the oracle (V as [n_in][n_spec][n_chan], FP64)
        Vh = V.cpu().numpy()[:, :, :n_in].astype(np.complex128).transpose(2, 0, 1)
        R_or = fx.x_engine(Vh, n_spec)
        err_or = fx.rel_frobenius_per_channel(R_out[None], R_or).max()
        assert err_or < 1e-5, err_or
        c.close()


def test_noalloc_rejects_shapes_beyond_its_scratch():
    from paper_2604_20640_gb300 import CorrError, CORR_EINVAL
    from paper_2604_20640_gb300.corr import xengine_noalloc
    # rejected before any device work, so small placeholder buffers suffice
    V = torch.zeros((4,), dtype=torch.complex64, device=DEV)
    out = torch.zeros((4,), dtype=torch.complex64, device=DEV)
    with pytest.raises(CorrError) as e:
        xengine_noalloc(V, 1, 256, 8192, out)
    assert e.value.code == CORR_EINVAL


def test_noalloc_rejects_a_misaligned_view():
    """A complex64 view one element into a buffer is 8-byte aligned only; the
    X-engine reads V as 16-byte vectors, so the call is refused on the host."""
    from paper_2604_20640_gb300 import CorrError, CORR_EINVAL
    from paper_2604_20640_gb300.corr import xengine_noalloc
    buf = torch.zeros((1 + 16 * 64 * 4,), dtype=torch.complex64, device=DEV)
    out = torch.zeros((64, 4, 4), dtype=torch.complex64, device=DEV)
    with pytest.raises(CorrError) as e:
        xengine_noalloc(buf[1:], 16, 4, 64, out)
    assert e.value.code == CORR_EINVAL
