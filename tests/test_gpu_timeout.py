"""Failure detection of the tensor-core X-engine without a GPU fault.

Every wait of the tcgen05 pipeline (TMA producer, MMA issuer, epilogue) is
bounded by %globaltimer.  With the fault-injection option "inject_stall" the
load producer issues nothing, so the MMA issuer's first wait on a full
barrier runs out after "tc_wait_ms"; the kernel must record CORR_ETIMEDOUT in
the handle's status word, free its tensor memory and return -- the host sees
the status, the call finishes within a bounded time, and the same handle and
context then produce correct results again."""

import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from fxsynth import StreamSpec, delays_for, make_stream  # noqa: E402
from oracle import fx_oracle as fx  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_20640_gb300.build import build_library
    build_library()


def test_tensor_core_wait_expires_and_the_handle_recovers():
    from paper_2604_20640_gb300 import Correlator, CORR_ETIMEDOUT
    n_ant, n_chan, n_int = 8, 64, 512
    n_in = 2 * n_ant
    S = 2 * n_chan * n_int * 2 + 99
    tau, phi = delays_for(n_in, 41)
    x = make_stream(StreamSpec(n_ant=n_ant, n_pol=2, n_samples=S, seed=41, tau=tau, phi=phi))
    xd = torch.from_numpy(x).to(DEV)
    c = Correlator(n_ant, 2, n_chan, 4, n_int, precision=1)
    c.set_delays(tau, phi)
    n = c.n_integrations(S)
    vis = torch.empty((n, n_chan, n_in, n_in), dtype=torch.complex64, device=DEV)
    flags = torch.empty_like(vis, dtype=torch.uint8)
    assert c.device_status() == 0
    c.set_option("tc_wait_ms", 5)
    c.set_option("inject_stall", 1)
    t0 = time.perf_counter()
    c.run_dev(xd, vis, flags)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    assert c.device_status() == CORR_ETIMEDOUT
    assert dt < 10.0                                   # two integrations, 5 ms waits
    assert c.device_status() == 0                      # read clears the word
    # the same handle, same context, no injection: correct again
    c.set_option("inject_stall", 0)
    c.set_option("tc_wait_ms", 2000)
    c.run_dev(xd, vis, flags)
    torch.cuda.synchronize()
    assert c.device_status() == 0
    Ro = fx.correlate(x, n_chan, 4, n_int, tau, phi)[0]
    drho = np.abs(fx.normalised_coefficients(vis.cpu().numpy().astype(np.complex128)) -
                  fx.normalised_coefficients(Ro)).max()
    assert drho < 5e-3
    c.close()


def test_gram_stage_call_reports_the_expired_wait():
    from paper_2604_20640_gb300 import Correlator, CORR_ETIMEDOUT, CORR_INT8
    c = Correlator(2, 1, 16, 4, 8)
    n_chan, K, pitch = 4, 256, 512
    Q = torch.zeros((n_chan, 128, pitch // 2), dtype=torch.bfloat16, device=DEV)
    Q[:, :3, :K] = 2.0
    G = torch.full((n_chan, 128, 128), 7.0, device=DEV)
    c.set_option("tc_wait_ms", 3)
    c.set_option("inject_stall", 1)
    c.gram_dev(Q, n_chan, pitch, K, CORR_INT8, G)
    assert c.device_status() == CORR_ETIMEDOUT
    assert torch.all(G == 7.0)                         # nothing written on expiry
    c.set_option("inject_stall", 0)
    c.gram_dev(Q, n_chan, pitch, K, CORR_INT8, G)
    assert c.device_status() == 0
    assert torch.all(G[:, :3, :3] == 4.0 * K) and torch.all(G[:, 3:, :] == 0) and torch.all(G[:, :, 3:] == 0)
    c.close()
