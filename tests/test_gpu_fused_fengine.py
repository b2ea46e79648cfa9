"""The fused F-engine (PFB + FFT in one kernel, FIR output kept in shared
memory) against the two-kernel path (FIR kernel, z ring, FFT kernel) and the
FP64 oracle.

The fused kernel keeps the FMA order of the FIR kernel and the FFT kernel's
passes, so every output that does not go through atomic additions must be
bit-identical between the two paths (option "fused_f" 1 and 0):
visibilities and flags of whole streams (pair-major spectra rings at every
fused length, the channel-major ring at M = 8192), the stage call's rotated
spectra, and streams pushed in ragged chunks through the staging buffers.
Dynamic spectra accumulate rows with atomic additions whose order is not
fixed, so they are compared within FP32 rounding.  Delays include negative
advances and advances beyond a frame, which put the edge frames of a
CTA's run on the checked load path.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from fxsynth import StreamSpec, make_stream, delays_for  # noqa: E402
from oracle import fx_oracle as fx  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_20640_gb300.build import build_library
    build_library()


def _run(n_ant, n_pol, n_chan, n_int, x, tau, phi, fused, **opt):
    from paper_2604_20640_gb300 import Correlator
    c = Correlator(n_ant, n_pol, n_chan, 4, n_int, fused_f=fused, max_delay=20000, **opt)
    c.set_delays(tau, phi)
    n_in = n_ant * n_pol
    n = c.n_integrations(x.shape[1], include_partial=True)
    vis = torch.full((n, n_chan, n_in, n_in), complex(np.nan, np.nan), dtype=torch.complex64, device=DEV)
    flags = torch.full((n, n_chan, n_in, n_in), 7, dtype=torch.uint8, device=DEV)
    got = c.run_dev(x, vis, flags, include_partial=True)
    torch.cuda.synchronize()
    c.close()
    return got, vis, flags


# (n_ant, n_pol, n_chan, n_int): pair-major rings at M = 1024 .. 8192 (up to
# 8 inputs), odd input counts (a padding input), and the channel-major ring
# with 12 inputs at M = 8192
SHAPES = [(4, 2, 4096, 40), (4, 1, 1024, 64), (3, 1, 512, 100), (2, 1, 2048, 33), (5, 1, 4096, 20),
          (6, 2, 4096, 24)]


@pytest.mark.parametrize("n_ant,n_pol,n_chan,n_int", SHAPES)
def test_fused_run_is_bit_identical_to_two_kernel_path(n_ant, n_pol, n_chan, n_int):
    n_in = n_ant * n_pol
    M = 2 * n_chan
    S = M * (2 * n_int + 7) + 333                    # ragged tail, partial integration
    tau, phi = delays_for(n_in, n_in * 31 + n_chan)
    tau = np.asarray(tau).copy()
    tau[1 % n_in] = -17.4                            # a negative coarse advance
    if n_in > 2:
        tau[2] = M + 123.6                           # an advance beyond one frame
    spec = StreamSpec(n_ant=n_ant, n_pol=n_pol, n_samples=S, seed=77 + n_chan, tau=None, phi=None)
    x = torch.from_numpy(make_stream(spec)).to(DEV)
    g1, v1, f1 = _run(n_ant, n_pol, n_chan, n_int, x, tau, phi, 1)
    g0, v0, f0 = _run(n_ant, n_pol, n_chan, n_int, x, tau, phi, 0)
    assert g1 == g0 == v1.shape[0]
    assert torch.equal(v1, v0) and torch.equal(f1, f0)
    # and the oracle on the last (partial) integration
    Ro = fx.correlate(x.cpu().numpy(), n_chan, 4, n_int, tau, phi, partial=True)[0]
    err = fx.rel_frobenius_per_channel(v1.cpu().numpy().astype(np.complex128), Ro).max()
    assert err < 1e-5, err


def test_fused_stage_call_matches_two_kernel_path_and_oracle():
    from paper_2604_20640_gb300 import Correlator
    n_chan, n_ant = 4096, 3
    M = 2 * n_chan
    S = M * 40 + 1000
    tau, phi = delays_for(n_ant, 5)
    x = make_stream(StreamSpec(n_ant=n_ant, n_pol=1, n_samples=S, seed=5, tau=tau, phi=phi))
    xd = torch.from_numpy(x).to(DEV)
    outs = []
    for fused in (1, 0):
        c = Correlator(n_ant, 1, n_chan, 4, 16, fused_f=fused)
        c.set_delays(tau, phi)
        V = torch.empty((37, n_chan, 4), dtype=torch.complex64, device=DEV)
        c.fengine_dev(xd, 2, 37, V)                   # spectra 2 .. 38 (the first ones see the zero history)
        torch.cuda.synchronize()
        outs.append(V)
        c.close()
    assert torch.equal(outs[0], outs[1])
    Vo = fx.f_engine(x, n_chan, 4, tau, phi)[:, 2:39]                       # [a][s][k]
    Vg = outs[0].cpu().numpy()[:, :, :n_ant].transpose(2, 0, 1).astype(np.complex128)
    rel = np.linalg.norm(Vg - Vo, axis=2) / np.linalg.norm(Vo, axis=2)
    assert rel.max() < 1e-5, rel.max()
    assert np.all(outs[0].cpu().numpy()[:, :, n_ant:] == 0)                 # the padding input


@pytest.mark.parametrize("n_chan", [4096, 1024])
def test_fused_dynamic_spectra_match_two_kernel_path(n_chan):
    from paper_2604_20640_gb300 import Correlator
    n_row = 3
    M = 2 * n_chan
    S = M * n_row * 64 + 500
    x = make_stream(StreamSpec(n_ant=3, n_pol=1, n_samples=S, seed=9, tones=[(40.3 / M, 8.0, 0.0)]))
    xd = torch.from_numpy(x).to(DEV)
    outs = []
    for fused in (1, 0):
        c = Correlator(3, 1, n_chan, 4, 64, fused_f=fused)
        t = torch.empty((3, 1, n_chan // 256, 64, 256), device=DEV)
        c.spectrogram_dev(xd, n_row, t)
        torch.cuda.synchronize()
        outs.append(t.double().cpu().numpy())
        c.close()
    d = np.abs(outs[0] - outs[1]) / (np.abs(outs[1]) + outs[1].mean())
    assert d.max() < 1e-6, d.max()


def test_fused_streaming_pushes_match_run_dev():
    """Ragged host pushes go through the two staging buffers (a nonzero
    stream base, frames that straddle the end of the pushed samples): the
    results equal one device-resident run bit for bit."""
    from paper_2604_20640_gb300 import Correlator
    n_ant, n_pol, n_chan, n_int = 4, 2, 4096, 24
    M = 2 * n_chan
    S = M * (3 * n_int + 5) + 77
    tau, phi = delays_for(8, 12)
    x = make_stream(StreamSpec(n_ant=n_ant, n_pol=n_pol, n_samples=S, seed=12, tau=tau, phi=phi))
    g, v_run, f_run = _run(n_ant, n_pol, n_chan, n_int, torch.from_numpy(x).to(DEV), tau, phi, 1)
    c = Correlator(n_ant, n_pol, n_chan, 4, n_int, chunk=150001)
    c.set_delays(tau, phi)
    pos = 0
    for n in [70001, 3, 250000, 123457] + [S]:
        n = min(n, S - pos)
        if n <= 0:
            break
        c.push(x[:, pos:pos + n])
        pos += n
    c.flush()
    v, f = c.get_vis(), c.get_flags()
    c.close()
    assert v.shape[0] == g
    assert np.array_equal(v, v_run.cpu().numpy()) and np.array_equal(f, f_run.cpu().numpy())


# (n_ant, n_pol, n_chan, n_int) of the reduced-precision pipelines whose
# F-engine writes the codes itself: M = 1024 .. 8192, a padding input, 64
# inputs, integration lengths that are not multiples of the Gram kernel's
# 64- or 128-spectrum tiles, a partial last integration
CODE_SHAPES = [(2, 1, 512, 37), (3, 2, 1024, 45), (5, 1, 2048, 22), (32, 2, 1024, 70), (12, 2, 4096, 9)]


@pytest.mark.parametrize("prec", [1, 2])
@pytest.mark.parametrize("n_ant,n_pol,n_chan,n_int", CODE_SHAPES)
@pytest.mark.parametrize("run", [0, 5])
def test_fused_codes_are_bit_identical_to_requantiser(prec, n_ant, n_pol, n_chan, n_int, run):
    """With fixed scales (from the first ring fill after the pre-pass on)
    the fused F-engine requantises in its epilogue and writes 4-byte code
    words straight into the integration's word buffer instead of spectra;
    with fused_f = 0 the requantiser makes the same words from the U = 2Y
    spectra of the two-kernel F-engine.  Same codes, so the visibilities
    and flags agree bit for bit (runs of 5 spectra per CTA and 1 MiB rings
    put launch and run boundaries at odd columns)."""
    n_in = n_ant * n_pol
    M = 2 * n_chan
    S = M * (3 * n_int + 9) + 101
    tau, phi = delays_for(n_in, 5 * n_in + n_chan)
    tau = np.asarray(tau).copy()
    tau[0] = -6.3
    spec = StreamSpec(n_ant=n_ant, n_pol=n_pol, n_samples=S, seed=900 + n_chan + n_in, tau=tau, phi=phi,
                      tones=[(0.1, 8.0, 0.2)])
    x = torch.from_numpy(make_stream(spec)).to(DEV)
    g1, v1, f1 = _run(n_ant, n_pol, n_chan, n_int, x, tau, phi, 1, precision=prec, fir_spt=run, ring_mb=1)
    g0, v0, f0 = _run(n_ant, n_pol, n_chan, n_int, x, tau, phi, 0, precision=prec, ring_mb=1)
    assert g1 == g0 == v1.shape[0] >= 4
    assert torch.equal(v1, v0) and torch.equal(f1, f0)
    assert torch.isfinite(torch.view_as_real(v1)).all()
