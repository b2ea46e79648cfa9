"""Parity at the configurations the benchmark times, in the launch
configuration it times them (autotuned ring sizes, full stream lengths).

The streams are the benchmark's own synthetic streams, drawn on the device;
the FP64 oracle recomputes the sampled outputs from the same samples copied
back to the host:

* streaming workload: 4 antennas x 2 pols, 2^28 int8 samples per input,
  4096 channels, n_int 1024 (32 integrations through the pair-major spectra
  ring, several ring wraps): every visibility of two integrations (the first
  and the last) on a 64-channel window holding an injected tone plus a
  spread of single channels, within 1e-5 relative Frobenius error per
  channel, and the window's MAD flags identical outside the 1e-4 T band;
* 64-input precision workload: 2^26 samples per input, 1024 channels,
  n_int 4096 (K = 4096, beyond the K where FP32 Gram sums stay exact),
  int8 and e4m3 codes on the tensor cores: normalised coefficients within
  5e-3 of the full-precision oracle on sampled channels of the first
  integration (pre-pass scales) and the last (scales from the previous
  autocorrelations);
* eight uneven sub-array streams in one captured graph, tensor-core members
  (>= 24 inputs, int8) beside CUDA-core FP32 members, autotuned: every
  member bit-identical to its own run and within the bars above of the
  oracle on its last integration.

The oracle's voltages for an integration come from ``fx.f_engine`` applied
to the slice of the stream that integration reads (one input at a time):
spectrum s reads samples [(s - P + 1) M + d, (s + 1) M + d) with the coarse
advance 0 <= d < M, so a slice from frame s0 - P to frame s1 + 2 (clipped
to the stream) holds every sample the integration's spectra use, and
samples outside the slice are never read by them.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from fxsynth import config_c2, config_c3  # noqa: E402
from fxsynth.streams import C4_SHAPES, config_c4_streams  # noqa: E402
from fxsynth.streams_torch import make_stream_torch  # noqa: E402
from oracle import fx_oracle as fx  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
TAPS = 4


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_20640_gb300.build import build_library
    build_library()


def _oracle_vis(x_dev, n_chan, tau, phi, s0, s1, chans):
    """R[k][a][b] (FP64) of spectra [s0, s1) on channels `chans`, from the
    oracle's F-engine over the slice of the stream those spectra read."""
    M = 2 * n_chan
    d, _ = fx.split_delay(np.asarray(tau, np.float64))
    assert np.all(d >= 0) and np.all(d < M)
    S = x_dev.shape[1]
    f_lo = max(0, s0 - TAPS)
    hi = min(S, (s1 + 2) * M)
    xs = x_dev[:, f_lo * M:hi].cpu().numpy()
    n_in = xs.shape[0]
    V = np.empty((n_in, s1 - s0, len(chans)), np.complex128)
    for a in range(n_in):
        Va = fx.f_engine(xs[a:a + 1], n_chan, TAPS, np.asarray(tau)[a:a + 1], np.asarray(phi)[a:a + 1])[0]
        V[a] = Va[s0 - f_lo:s1 - f_lo][:, chans]
    return np.einsum('ask,bsk->kab', V, V.conj()) / (s1 - s0)


def _rho(R):
    return fx.normalised_coefficients(R)


def test_streaming_workload_full_size_at_its_tuning():
    from paper_2604_20640_gb300 import Correlator
    n_chan, n_int, S = 4096, 1024, 1 << 28
    spec = config_c2(seed=2000, n_samples=S, M=2 * n_chan)
    x = make_stream_torch(spec, device=DEV)
    c = Correlator(4, 2, n_chan, TAPS, n_int)
    c.autotune(x)
    ring, spt, _ = c.tuning()
    c.set_delays(spec.tau, spec.phi)
    n = c.n_integrations(S)
    assert n == 32
    vis = torch.empty((n, n_chan, 8, 8), dtype=torch.complex64, device=DEV)
    flags = torch.empty((n, n_chan, 8, 8), dtype=torch.uint8, device=DEV)
    assert c.run_dev(x, vis, flags) == n
    torch.cuda.synchronize()
    # one 64-channel window around the first tone, plus single channels
    tone_ch = int(round(spec.tones[0][0] * 2 * n_chan))
    w0 = tone_ch // 64 * 64
    singles = [0, 1, 777, 2049, 4095]
    chans = list(range(w0, w0 + 64)) + singles
    for i in (0, n - 1):
        Ro = _oracle_vis(x, n_chan, spec.tau, spec.phi, i * n_int, (i + 1) * n_int, chans)
        Rg = vis[i, chans].cpu().numpy().astype(np.complex128)
        err = fx.rel_frobenius_per_channel(Rg[None], Ro[None]).max()
        assert err < 1e-5, (i, err, ring, spt)
        Fo, _, To = fx.mad_flags(Ro[None, :64], 5.0, 64)
        Fg = flags[i, chans[:64]].cpu().numpy()[None]
        A = np.abs(Ro[None, :64])
        ok = (Fg == Fo) | (np.abs(A - To) < 1e-4 * To)
        assert ok.all(), (i, ring, spt)
        assert Fo[0, tone_ch - w0].any()            # the tone channel is flagged
    c.close()


@pytest.mark.parametrize("prec,name,ints", [(1, "int8", (0, 7)), (2, "e4m3", (7,))])
def test_precision_workload_full_size_at_its_tuning(prec, name, ints):
    from paper_2604_20640_gb300 import Correlator
    n_chan, n_int, S = 1024, 4096, 1 << 26
    spec = config_c3(seed=3000, n_samples=S)
    x = make_stream_torch(spec, device=DEV)
    c = Correlator(32, 2, n_chan, TAPS, n_int, precision=prec)
    c.autotune(x)
    c.set_delays(spec.tau, spec.phi)
    n = c.n_integrations(S)
    assert n == 8
    vis = torch.empty((n, n_chan, 64, 64), dtype=torch.complex64, device=DEV)
    flags = torch.empty((n, n_chan, 64, 64), dtype=torch.uint8, device=DEV)
    assert c.run_dev(x, vis, flags) == n
    torch.cuda.synchronize()
    assert c.device_status() == 0
    chans = [0, 3, 100, 511, 512, 900, 1023]
    for i in ints:
        Ro = _oracle_vis(x, n_chan, spec.tau, spec.phi, i * n_int, (i + 1) * n_int, chans)
        Rg = vis[i, chans].cpu().numpy().astype(np.complex128)
        drho = np.abs(_rho(Rg) - _rho(Ro)).max()
        assert drho < 5e-3, (name, i, drho, c.tuning())
    c.close()


def test_batched_group_with_tensor_core_members_at_its_tuning(tmp_path):
    from paper_2604_20640_gb300 import Correlator, Group
    S = 1 << 24
    specs = config_c4_streams(seed=4000, n_samples=S)
    members, solo, xs, vis, flags = [], [], [], [], []
    cache = str(tmp_path / "tune.txt")
    for spec, (na, nc, ni) in zip(specs, C4_SHAPES):
        prec = 1 if 2 * na >= 24 else 0
        c = Correlator(na, 2, nc, TAPS, ni, precision=prec)
        c.set_delays(spec.tau, spec.phi)
        x = make_stream_torch(spec, device=DEV)
        c.autotune(x, cache)
        n = c.n_integrations(S)
        v = torch.zeros((n, nc, 2 * na, 2 * na), dtype=torch.complex64, device=DEV)
        f = torch.zeros((n, nc, 2 * na, 2 * na), dtype=torch.uint8, device=DEV)
        v2, f2 = torch.zeros_like(v), torch.zeros_like(f)
        c.run_dev(x, v2, f2)
        members.append((c, prec, spec))
        solo.append((v2, f2))
        xs.append(x)
        vis.append(v)
        flags.append(f)
    assert any(p == 1 for _, p, _ in members) and any(p == 0 for _, p, _ in members)
    g = Group([m[0] for m in members])
    g.run_dev(xs, vis, flags)
    torch.cuda.synchronize()
    for (c, prec, spec), x, v, f, (v2, f2) in zip(members, xs, vis, flags, solo):
        assert torch.equal(v, v2) and torch.equal(f, f2)
        assert c.device_status() == 0
        i = v.shape[0] - 1
        chans = [0, 5, c.n_chan // 2 + 1, c.n_chan - 1]
        Ro = _oracle_vis(x, c.n_chan, spec.tau, spec.phi, i * c.n_int, (i + 1) * c.n_int, chans)
        Rg = v[i, chans].cpu().numpy().astype(np.complex128)
        if prec == 0:
            assert fx.rel_frobenius_per_channel(Rg[None], Ro[None]).max() < 1e-5
        else:
            assert np.abs(_rho(Rg) - _rho(Ro)).max() < 5e-3
    g.close()
