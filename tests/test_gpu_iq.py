"""Complex (I/Q) input on the GPU against the FP64 oracle (option
"sample_format" = 1; the reading is stated in oracle/fx_oracle.py).

Bars as for real input: visibilities within 1e-5 relative Frobenius error
per channel, channelised voltages within 1e-5 relative L2 per (input,
spectrum), flags identical outside the 1e-4 T band, any chunking of a pushed
stream bit-identical to one device-resident run.  Transform lengths from 16
to 8192 points, odd input counts, negative and beyond-frame coarse delays,
complex tones at positive and negative frequencies.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from fxsynth import StreamSpec, delays_for, make_stream_iq  # noqa: E402
from oracle import fx_oracle as fx  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_20640_gb300.build import build_library
    build_library()


def _corr(n_ant, n_pol, n_chan, taps, n_int, **kw):
    from paper_2604_20640_gb300 import Correlator
    return Correlator(n_ant, n_pol, n_chan, taps, n_int, sample_format=1, **kw)


@pytest.mark.parametrize("n_ant,n_pol,n_chan,n_int,taps", [
    (3, 1, 16, 40, 4), (2, 2, 256, 30, 4), (5, 1, 1024, 12, 8), (3, 2, 4096, 6, 4), (2, 1, 8192, 4, 3),
    (6, 2, 512, 10, 4)])
def test_iq_run_matches_oracle(n_ant, n_pol, n_chan, n_int, taps):
    n_in = n_ant * n_pol
    M = n_chan
    S = M * (2 * n_int + 3) + 77                      # complex samples; ragged tail
    tau, phi = delays_for(n_in, 3 * n_chan + n_in)
    tau = np.asarray(tau).copy()
    tau[-1] = -9.6                                     # negative coarse advance
    if n_in > 2:
        tau[1] = M + 31.2                              # beyond one frame
    tones = [(5.0 / M, 6.0, 0.3), (-(M // 4 + 0.0) / M, 9.0, 1.0)]
    x = make_stream_iq(StreamSpec(n_ant=n_ant, n_pol=n_pol, n_samples=S, seed=n_chan + n_in,
                                  tau=delays_for(n_in, 9)[0], phi=delays_for(n_in, 9)[1], tones=tones))
    c = _corr(n_ant, n_pol, n_chan, taps, n_int, max_delay=20000)
    c.set_delays(tau, phi)
    xd = torch.from_numpy(x).to(DEV)
    n = c.n_integrations(S, include_partial=True)
    vis = torch.empty((n, n_chan, n_in, n_in), dtype=torch.complex64, device=DEV)
    flags = torch.empty((n, n_chan, n_in, n_in), dtype=torch.uint8, device=DEV)
    assert c.run_dev(xd, vis, flags, include_partial=True) == n
    torch.cuda.synchronize()
    w = min(64, n_chan)
    Ro, Fo, To = fx.correlate_iq(x, n_chan, taps, n_int, tau, phi, window=w, partial=True)
    Rg = vis.cpu().numpy().astype(np.complex128)
    assert fx.rel_frobenius_per_channel(Rg, Ro).max() < 1e-5
    A = np.abs(Ro)
    ok = (flags.cpu().numpy() == Fo) | (np.abs(A - To) < 1e-4 * To)
    assert ok.all()
    c.close()


def test_iq_stage_call_matches_oracle_voltages():
    n_ant, n_chan, taps = 3, 2048, 4
    S = n_chan * 30 + 5
    tau, phi = np.array([0.0, 2.7, -13.2]), np.array([0.0, 0.9, -2.0])
    x = make_stream_iq(StreamSpec(n_ant=n_ant, n_pol=1, n_samples=S, seed=4, tones=[(-0.2, 5.0, 0.0)]))
    c = _corr(n_ant, 1, n_chan, taps, 8)
    c.set_delays(tau, phi)
    V = torch.empty((25, n_chan, 4), dtype=torch.complex64, device=DEV)
    c.fengine_dev(torch.from_numpy(x).to(DEV), 3, 25, V)
    torch.cuda.synchronize()
    Vo = fx.f_engine_iq(x, n_chan, taps, tau, phi)[:, 3:28]
    Vg = V.cpu().numpy()[:, :, :n_ant].transpose(2, 0, 1).astype(np.complex128)
    rel = np.linalg.norm(Vg - Vo, axis=2) / np.linalg.norm(Vo, axis=2)
    assert rel.max() < 1e-5
    assert np.all(V.cpu().numpy()[:, :, n_ant:] == 0)
    c.close()


def test_iq_streaming_chunking_is_bit_identical():
    n_ant, n_pol, n_chan, n_int = 2, 2, 1024, 20
    S = n_chan * (3 * n_int + 2) + 501
    tau, phi = delays_for(4, 21)
    x = make_stream_iq(StreamSpec(n_ant=n_ant, n_pol=n_pol, n_samples=S, seed=21, tau=tau, phi=phi))
    c = _corr(n_ant, n_pol, n_chan, 4, n_int)
    c.set_delays(tau, phi)
    n = c.n_integrations(S, include_partial=True)
    vis = torch.empty((n, n_chan, 4, 4), dtype=torch.complex64, device=DEV)
    flags = torch.empty((n, n_chan, 4, 4), dtype=torch.uint8, device=DEV)
    c.run_dev(torch.from_numpy(x).to(DEV), vis, flags, include_partial=True)
    torch.cuda.synchronize()
    c.close()
    cs = _corr(n_ant, n_pol, n_chan, 4, n_int, chunk=7001)
    cs.set_delays(tau, phi)
    pos = 0
    for m in [1001, 3, 20000, S]:
        m = min(m, S - pos)
        if m <= 0:
            break
        cs.push(x[:, 2 * pos:2 * (pos + m)])            # interleaved pairs: 2 elements per sample
        pos += m
    cs.flush()
    v, f = cs.get_vis(), cs.get_flags()
    cs.close()
    assert np.array_equal(v, vis.cpu().numpy()) and np.array_equal(f, flags.cpu().numpy())


def test_iq_option_rejects_unsupported_combinations():
    from paper_2604_20640_gb300 import Correlator, CorrError, CORR_EINVAL
    c = Correlator(2, 1, 256, 4, 8, precision=1)
    with pytest.raises(CorrError) as e:
        c.set_option("sample_format", 1)
    assert e.value.code == CORR_EINVAL
    c.close()
    c = _corr(2, 1, 256, 4, 8)
    with pytest.raises(CorrError) as e:
        c.set_option("precision", 2)
    assert e.value.code == CORR_EINVAL
    with pytest.raises(CorrError) as e:
        c.set_option("sample_bits", 16)
    assert e.value.code == CORR_EINVAL
    x = torch.zeros((2, 2 * 256 * 64 * 2), dtype=torch.int8, device=DEV)
    with pytest.raises(CorrError) as e:
        c.spectrogram_dev(x, 1, torch.empty((2, 1, 1, 64, 256), device=DEV))
    assert e.value.code == CORR_EINVAL
    c.close()
    from paper_2604_20640_gb300 import Correlator as C2
    with pytest.raises(CorrError) as e:
        C2(2, 1, 8, 4, 8, sample_format=1)            # n_chan < 16
    assert e.value.code == CORR_EINVAL
