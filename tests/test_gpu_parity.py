"""GPU parity of the CUDA hot path against the FP64 oracle (through the C ABI).

Tolerances (FP32 path):
  * channelised voltages: relative L2 error per (input, spectrum) < 1e-5;
  * visibilities: relative Frobenius error per channel < 1e-5;
  * flags: identical except where |A - T| < 1e-4 T (A, T in FP64);
  * any two chunkings of one stream: bit-identical.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from fxsynth import StreamSpec, make_stream, config_c1  # noqa: E402
from oracle import fx_oracle as fx  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_20640_gb300.build import build_library
    build_library()


def _corr(*a, **k):
    from paper_2604_20640_gb300 import Correlator
    return Correlator(*a, **k)


def _stream(n_in, S, seed, tau=None, phi=None, **kw):
    return make_stream(StreamSpec(n_ant=n_in, n_pol=1, n_samples=S, seed=seed, tau=tau, phi=phi, **kw))


def _vis_err(Rg, Ro):
    return fx.rel_frobenius_per_channel(np.asarray(Rg).astype(np.complex128), Ro)


def _flags_ok(Fg, Ro, Fo, To):
    A = np.abs(Ro)
    return (Fg == Fo) | (np.abs(A - To) < 1e-4 * To)


def _fengine(c, x, s0, n_spec):
    xd = torch.from_numpy(x).to(DEV)
    V = torch.full((n_spec, c.n_chan, c.n_in_pad), complex(np.nan, np.nan), dtype=torch.complex64, device=DEV)
    c.fengine_dev(xd, s0, n_spec, V)
    torch.cuda.synchronize()
    return V.cpu().numpy()


# ---------------------------------------------------------------------------
# F-engine alone
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("n_chan", [8, 16, 32, 64, 128, 256, 512, 1024, 2048, 4096, 8192])
def test_fengine_matches_oracle_all_lengths(n_chan):
    M, P, n_in = 2 * n_chan, 4, 3
    n_spec = 11
    S = M * n_spec + min(37, M - 1)        # ragged tail
    tau = np.array([0.0, 13.4, -6.6])
    phi = np.array([0.3, -2.0, 1.1])
    x = _stream(n_in, S, seed=n_chan, tau=tau, phi=phi)
    c = _corr(n_in, 1, n_chan, P, 4)
    c.set_delays(tau, phi)
    Vg = _fengine(c, x, 0, n_spec)
    Vo = fx.f_engine(x, n_chan, P, tau, phi)
    assert Vo.shape[1] == n_spec
    for a in range(n_in):
        num = np.linalg.norm(Vg[:, :, a] - Vo[a], axis=1)
        den = np.linalg.norm(Vo[a], axis=1)
        assert np.all(num <= 1e-5 * den + 1e-6), (a, (num / np.maximum(den, 1e-30)).max())
    assert np.all(Vg[:, :, n_in:] == 0)     # padding inputs are zero


@pytest.mark.parametrize("taps", [1, 2, 3, 8, 16])
def test_fengine_taps_and_subrange(taps):
    n_chan, n_in = 64, 4
    M = 2 * n_chan
    S = M * 40
    tau = np.array([0.0, 3.0, 40.0, 17.5])
    x = _stream(n_in, S, seed=taps, tau=tau)
    c = _corr(n_in, 1, n_chan, taps, 8)
    c.set_delays(tau)
    Vo = fx.f_engine(x, n_chan, taps, tau)
    for s0, n in [(0, 40), (7, 9), (39, 1)]:
        Vg = _fengine(c, x, s0, n)
        for a in range(n_in):
            num = np.linalg.norm(Vg[:, :, a] - Vo[a, s0:s0 + n], axis=1)
            den = np.linalg.norm(Vo[a, s0:s0 + n], axis=1)
            assert np.all(num <= 1e-5 * den + 1e-6)


def test_fengine_delays_beyond_stream_read_zero():
    n_chan, n_in = 32, 2
    M = 2 * n_chan
    S = M * 6
    x = _stream(n_in, S, seed=5)
    tau = np.array([float(S + 10), -float(S + 10)])
    c = _corr(n_in, 1, n_chan, 4, 2, max_delay=S + 100)
    c.set_delays(tau)
    Vg = _fengine(c, x, 0, 6)
    assert np.all(Vg[:, :, :2] == 0)


def test_fengine_tone_lands_in_its_channel():
    n_chan, P = 512, 4
    M = 2 * n_chan
    k0 = 77
    n = np.arange(M * 12)
    x = np.clip(np.rint(60 * np.cos(2 * np.pi * k0 * n / M + 0.4)), -128, 127).astype(np.int8)[None, :]
    x = np.repeat(x, 2, axis=0)
    c = _corr(2, 1, n_chan, P, 4)
    Vg = _fengine(c, x, 0, 12)
    for s in range(P - 1, 12):
        assert np.argmax(np.abs(Vg[s, :, 0])) == k0


# ---------------------------------------------------------------------------
# X-engine and flagging alone
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("n_in,n_chan,n_spec", [(1, 64, 7), (2, 32, 100), (4, 256, 130), (5, 64, 64),
                                                (8, 512, 257), (12, 64, 33), (16, 128, 65), (64, 32, 70)])
def test_xengine_matches_oracle(n_in, n_chan, n_spec):
    rng = np.random.default_rng(n_in * 1000 + n_chan)
    n_pad = (n_in + 3) // 4 * 4
    V = np.zeros((n_spec, n_chan, n_pad), dtype=np.complex64)
    V[:, :, :n_in] = (rng.standard_normal((n_spec, n_chan, n_in)) +
                      1j * rng.standard_normal((n_spec, n_chan, n_in))).astype(np.complex64)
    c = _corr(n_in, 1, n_chan, 4, 16)
    Vd = torch.from_numpy(V).to(DEV)
    R = torch.empty((n_chan, n_in, n_in), dtype=torch.complex64, device=DEV)
    c.xengine_dev(Vd, n_spec, R)
    torch.cuda.synchronize()
    Ro = fx.x_engine(np.transpose(V[:, :, :n_in].astype(np.complex128), (2, 0, 1)), n_spec)[0]
    Rg = R.cpu().numpy()
    assert _vis_err(Rg[None], Ro[None]).max() < 1e-5
    assert np.all(Rg == np.conj(np.swapaxes(Rg, -1, -2)))          # exactly Hermitian
    assert np.all(np.einsum('kaa->ka', Rg).imag == 0)


def test_xengine_dev_rejects_misaligned_buffers():
    """V is read as 16-byte vectors: a complex64 view one element into a
    buffer is refused on the host (CORR_EINVAL), before any launch."""
    from paper_2604_20640_gb300 import CorrError, CORR_EINVAL
    c = _corr(4, 1, 64, 4, 16)
    buf = torch.zeros((1 + 16 * 64 * 4,), dtype=torch.complex64, device=DEV)
    R = torch.empty((64, 4, 4), dtype=torch.complex64, device=DEV)
    with pytest.raises(CorrError) as e:
        c.xengine_dev(buf[1:], 16, R)
    assert e.value.code == CORR_EINVAL


def test_xengine_dev_long_stream_beyond_the_grid_limit():
    """More than 64 x 65535 spectra: the partial-sum groups are lengthened so
    that their count stays a legal grid dimension; the result still matches
    the oracle (one channel, one input, so the buffer stays small)."""
    n_spec = 64 * 65535 + 1000
    rng = np.random.default_rng(5)
    V = np.zeros((n_spec, 8, 4), dtype=np.complex64)
    V[:, :, 0] = (rng.standard_normal((n_spec, 8)) + 1j * rng.standard_normal((n_spec, 8))).astype(np.complex64)
    c = _corr(1, 1, 8, 4, 16)
    R = torch.empty((8, 1, 1), dtype=torch.complex64, device=DEV)
    c.xengine_dev(torch.from_numpy(V).to(DEV), n_spec, R)
    torch.cuda.synchronize()
    Ro = np.mean(np.abs(V[:, :, 0].astype(np.complex128)) ** 2, axis=0)
    # 65535 partial slots summed in order in FP32: rounding grows like
    # u sqrt(n) ~ 1.5e-5 here, so this check of the grid split allows 1e-4
    assert np.max(np.abs(R.cpu().numpy()[:, 0, 0].real - Ro) / Ro) < 1e-4


# the last four have >= 16384 (window, baseline) items per call: a group of
# 4 lanes per item instead of a warp (the last: 16650 items, so the last warp
# holds groups past the end that must store nothing)
@pytest.mark.parametrize("window,n_chan,n_in", [(64, 256, 3), (64, 64, 1), (32, 128, 4), (8, 8, 2), (256, 512, 2),
                                                (64, 1024, 40), (32, 512, 28), (16, 256, 64), (64, 128, 74)])
def test_mad_flags_match_oracle(window, n_chan, n_in):
    rng = np.random.default_rng(window + n_chan)
    n_vis = 3
    R = (rng.rayleigh(1.0, (n_vis, n_chan, n_in, n_in)) *
         np.exp(1j * rng.uniform(0, 6.3, (n_vis, n_chan, n_in, n_in))))
    hit = rng.random(R.shape) < 0.05
    R[hit] *= 20.0                                           # outliers
    R[1, :window, 0, 0] = 2.0                                # MAD = 0 window
    R[1, 3, 0, 0] = 3.0
    R = (R + np.conj(np.swapaxes(R, -1, -2))) / 2            # Hermitian
    R = np.ascontiguousarray(R.astype(np.complex64))
    c = _corr(n_in, 1, n_chan, 4, 16, flag_window=window)
    Rd = torch.from_numpy(R).to(DEV)
    F = torch.full(R.shape, 7, dtype=torch.uint8, device=DEV)
    c.flag_dev(Rd, n_vis, F)
    torch.cuda.synchronize()
    Fo, Ao, To = fx.mad_flags(R.astype(np.complex128), 5.0, window)
    ok = _flags_ok(F.cpu().numpy(), R.astype(np.complex128), Fo, To)
    assert ok.all(), np.argwhere(~ok)[:5]
    assert F.cpu().numpy()[1, 3, 0, 0] == 1


# ---------------------------------------------------------------------------
# Whole path
# ---------------------------------------------------------------------------

def _run_dev(c, x, partial=False):
    xd = torch.from_numpy(x).to(DEV)
    n = c.n_integrations(x.shape[1], partial)
    vis = torch.empty((max(n, 1), c.n_chan, c.n_in, c.n_in), dtype=torch.complex64, device=DEV)
    flags = torch.empty((max(n, 1), c.n_chan, c.n_in, c.n_in), dtype=torch.uint8, device=DEV)
    got = c.run_dev(xd, vis, flags, include_partial=partial)
    torch.cuda.synchronize()
    assert got == n
    return vis.cpu().numpy()[:n], flags.cpu().numpy()[:n]


@pytest.mark.parametrize("n_chan,n_int,n_in,partial", [(1024, 512, 4, False), (256, 100, 5, True),
                                                       (64, 3, 8, True), (4096, 64, 8, False),
                                                       (8192, 16, 2, True)])
def test_run_dev_matches_oracle(n_chan, n_int, n_in, partial):
    M = 2 * n_chan
    S = M * (n_int * 3 + (n_int // 2 if partial else 0)) + 333
    rng = np.random.default_rng(n_chan)
    tau = np.concatenate([[0.0], rng.uniform(0, 40, n_in - 1)])
    phi = rng.uniform(0, 2 * np.pi, n_in)
    x = _stream(n_in, S, seed=n_chan + n_in, tau=tau, phi=phi)
    c = _corr(n_in, 1, n_chan, 4, n_int)
    c.set_delays(tau, phi)
    Rg, Fg = _run_dev(c, x, partial)
    Ro, Fo, To = fx.correlate(x, n_chan, 4, n_int, tau, phi, partial=partial)
    assert Rg.shape == Ro.shape
    assert _vis_err(Rg, Ro).max() < 1e-5
    assert _flags_ok(Fg, Ro, Fo, To).all()


def test_c1_full_size_matches_oracle():
    spec = config_c1()                                  # 4 x 2^22 samples
    x = make_stream(spec)
    tau, phi = np.asarray(spec.tau), np.asarray(spec.phi)
    c = _corr(4, 1, 1024, 4, 512)
    c.set_delays(tau, phi)
    Rg, Fg = _run_dev(c, x)
    Ro, Fo, To = fx.correlate(x, 1024, 4, 512, tau, phi)
    assert Rg.shape == (4, 1024, 4, 4)
    assert _vis_err(Rg, Ro).max() < 1e-5
    assert _flags_ok(Fg, Ro, Fo, To).all()
    # the same stream through the host streaming API
    c2 = _corr(4, 1, 1024, 4, 512)
    c2.set_delays(tau, phi)
    c2.push(x)
    c2.flush()
    assert np.array_equal(c2.get_vis(), Rg)
    assert np.array_equal(c2.get_flags(), Fg)


# ---------------------------------------------------------------------------
# Streaming: chunking invariance, flush, delay changes
# ---------------------------------------------------------------------------

def _push_all(c, x, sizes):
    pos = 0
    for n in sizes:
        c.push(x[:, pos:pos + n])
        pos += n
    assert pos == x.shape[1]


def test_streaming_chunking_is_bit_identical_and_matches_oracle():
    n_chan, n_int, n_in = 128, 24, 4
    M = 2 * n_chan
    S = M * (n_int * 4 + 7) + 51
    tau = np.array([0.0, 9.7, 33.2, 2.0])
    phi = np.array([0.0, 1.0, 2.0, 3.0])
    x = _stream(n_in, S, seed=77, tau=tau, phi=phi)
    outs = []
    rng = np.random.default_rng(3)
    plans = [[S], [1] * 300 + [S - 300], [257, 13, 4099, 1, 3] + [S - 4373]]
    sizes = []
    left = S
    while left > 0:
        n = int(min(left, rng.integers(1, 3 * M)))
        sizes.append(n)
        left -= n
    plans.append(sizes)
    for plan in plans:
        c = _corr(n_in, 1, n_chan, 4, n_int, chunk=1000)
        c.set_delays(tau, phi)
        _push_all(c, x, plan)
        c.flush()
        outs.append((c.get_vis(), c.get_flags()))
    for v, f in outs[1:]:
        assert np.array_equal(v, outs[0][0])
        assert np.array_equal(f, outs[0][1])
    Ro, Fo, To = fx.correlate(x, n_chan, 4, n_int, tau, phi, partial=True)
    assert outs[0][0].shape == Ro.shape
    assert _vis_err(outs[0][0], Ro).max() < 1e-5
    assert _flags_ok(outs[0][1], Ro, Fo, To).all()


def test_delay_change_applies_at_integration_boundary():
    n_chan, n_int, n_in = 64, 10, 3
    M = 2 * n_chan
    S = M * n_int * 3
    t0, p0 = np.array([0.0, 5.0, 20.0]), np.array([0.0, 0.5, 1.0])
    t1, p1 = np.array([0.0, -3.2, 11.6]), np.array([0.2, -0.5, 2.0])
    x = _stream(n_in, S, seed=11)
    c = _corr(n_in, 1, n_chan, 4, n_int)
    c.set_delays(t0, p0)
    first = M * n_int + 20                       # integration 0 done, 1 not started
    c.push(x[:, :first])
    assert c.pending() == 1
    c.set_delays(t1, p1)
    c.push(x[:, first:])
    c.flush()
    Rg, Fg = c.get_vis(), c.get_flags()
    Ro, Fo, To = fx.correlate(x, n_chan, 4, n_int, schedule=[(t0, p0), (t1, p1), (t1, p1)])
    assert _vis_err(Rg, Ro).max() < 1e-5
    assert _flags_ok(Fg, Ro, Fo, To).all()


def test_empty_and_tiny_streams():
    c = _corr(2, 1, 32, 4, 4)
    c.push(np.zeros((2, 0), np.int8))
    c.flush()
    assert c.get_vis().shape[0] == 0
    c.reset()
    x = _stream(2, 63, seed=1)                   # shorter than one frame
    c.push(x)
    c.flush()
    assert c.get_vis().shape[0] == 0
    from paper_2604_20640_gb300 import CorrError, CORR_ESTATE
    with pytest.raises(CorrError) as e:
        c.push(x)
    assert e.value.code == CORR_ESTATE


def test_push_dev_matches_push():
    n_chan, n_int, n_in = 256, 16, 4
    M = 2 * n_chan
    S = M * n_int * 3 + 100
    x = _stream(n_in, S, seed=21)
    c1 = _corr(n_in, 1, n_chan, 4, n_int)
    c1.push(x)
    c1.flush()
    c2 = _corr(n_in, 1, n_chan, 4, n_int)
    xd = torch.from_numpy(x).to(DEV)
    c2.push_dev(xd[:, :5000])
    c2.push_dev(xd[:, 5000:])
    c2.flush()
    assert np.array_equal(c1.get_vis(), c2.get_vis())


def test_results_popped_into_pinned_and_pageable_buffers_agree():
    n_chan, n_int, n_in = 256, 8, 4
    M = 2 * n_chan
    S = M * n_int * 5 + 300
    x = _stream(n_in, S, seed=23)
    ref = _corr(n_in, 1, n_chan, 4, n_int)
    ref.push(x)
    ref.flush()
    Rv, Rf = ref.get_vis(), ref.get_flags()
    assert Rv.shape[0] == 5
    c = _corr(n_in, 1, n_chan, 4, n_int)
    c.push(x)
    c.flush()
    shape = (6, n_chan, n_in, n_in)
    pv = torch.full(shape, 7 + 7j, dtype=torch.complex64).pin_memory()
    pf = torch.full(shape, 9, dtype=torch.uint8).pin_memory()
    v1 = c.get_vis(max_int=2, out=pv)                 # pinned: DMA from the device slots
    f1 = c.get_flags(max_int=3, out=np.zeros(shape, np.uint8))   # pageable
    assert v1.shape[0] == 2 and f1.shape[0] == 3
    assert np.array_equal(v1.numpy(), Rv[:2]) and np.array_equal(f1, Rf[:3])
    assert (pv[2:].numpy() == 7 + 7j).all()           # nothing written past the count
    v2 = c.get_vis(out=np.zeros(shape, np.complex64))
    f2 = c.get_flags(out=pf)
    assert np.array_equal(v2, Rv[2:]) and np.array_equal(f2.numpy(), Rf[3:])
    assert (pf[2:].numpy() == 9).all()
    assert c.get_vis(out=pv).shape[0] == 0 and c.get_flags(out=pf).shape[0] == 0
    from paper_2604_20640_gb300 import CorrError
    for bad in (torch.zeros(shape, dtype=torch.complex64, device=DEV),       # device tensor
                np.zeros((6, n_chan, n_in, n_in + 1), np.complex64),         # wrong shape
                np.zeros(shape, np.complex128)):                              # wrong type
        with pytest.raises(CorrError):
            c.get_vis(max_int=1, out=bad)


def test_results_without_host_images_after_pinned_pops():
    """After a pop into pinned memory, new results get no host image (the next
    pinned pop takes them by DMA from the device slots); a pop into pageable
    memory, or a checkpoint, makes the image on demand.  Every route gives
    the results of a stream popped the usual way."""
    n_chan, n_int, n_in = 256, 8, 4
    M = 2 * n_chan
    third = M * n_int * 2
    S = 3 * third + 300
    x = _stream(n_in, S, seed=29)
    ref = _corr(n_in, 1, n_chan, 4, n_int)
    ref.push(x)
    ref.flush()
    Rv, Rf = ref.get_vis(), ref.get_flags()
    assert Rv.shape[0] == 6
    c = _corr(n_in, 1, n_chan, 4, n_int)
    shape = (8, n_chan, n_in, n_in)
    pv = torch.zeros(shape, dtype=torch.complex64).pin_memory()
    pf = torch.zeros(shape, dtype=torch.uint8).pin_memory()
    c.push(x[:, :third])
    vs = [c.get_vis(out=pv).numpy().copy()]
    fs = [c.get_flags(out=pf).numpy().copy()]            # pinned: later results skip the image
    c.push(x[:, third:2 * third])
    vs.append(c.get_vis())                               # pageable: image made on demand
    fs.append(c.get_flags(out=pf).numpy().copy())        # pinned again
    c.push(x[:, 2 * third:])
    c.flush()
    state = c.save_state()                               # queued results without images
    c2 = _corr(n_in, 1, n_chan, 4, n_int)
    c2.load_state(state)
    vs.append(c2.get_vis())
    fs.append(c2.get_flags())
    assert np.array_equal(np.concatenate(vs), Rv) and np.array_equal(np.concatenate(fs), Rf)


def test_stage_times_and_stage_mask():
    n_chan, n_int, n_in = 256, 8, 4
    M = 2 * n_chan
    S = M * n_int * 4
    xd = torch.from_numpy(_stream(n_in, S, seed=5)).to(DEV)
    c = _corr(n_in, 1, n_chan, 4, n_int)
    vis = torch.empty((4, n_chan, n_in, n_in), dtype=torch.complex64, device=DEV)
    flags = torch.empty((4, n_chan, n_in, n_in), dtype=torch.uint8, device=DEV)
    c.set_option("stage_timing", 1)
    c.stage_times()
    c.run_dev(xd, vis, flags)
    ms, n = c.stage_times()
    # with at most 8 inputs the flags are made in the finalisation launch
    assert all(n[i] > 0 and ms[i] > 0 for i in range(4)) and n[4] == n[5] == n[6] == 0
    c.set_option("stage_mask", 1 << 1)                # the FFT alone
    c.run_dev(xd, vis, flags)
    ms2, n2 = c.stage_times()
    assert n2[1] == n[1] and ms2[1] > 0
    assert all(n2[i] == 0 and ms2[i] == 0 for i in (0, 2, 3, 4, 5, 6))
    c.set_option("stage_timing", 0)
    c.run_dev(xd, vis, flags)
    assert sum(c.stage_times()[1]) == 0
    from paper_2604_20640_gb300 import CorrError
    for bad in (-1, 128, 2.5):
        with pytest.raises(CorrError):
            c.set_option("stage_mask", bad)


@pytest.mark.parametrize("window,wname,taps", [(1, "kaiser", 8), (1, "kaiser", 4), (2, "none", 1), (0, "hann", 8)])
def test_fengine_window_options_match_oracle(window, wname, taps):
    n_chan, n_in = 512, 3
    M = 2 * n_chan
    S = M * 30 + 5
    tau = np.array([0.0, 7.0, 21.3])
    phi = np.array([0.0, 1.0, -0.5])
    x = _stream(n_in, S, seed=40 + taps, tau=tau, phi=phi)
    c = _corr(n_in, 1, n_chan, taps, 8)
    c.set_option("window", window)
    c.set_option("kaiser_beta", 8.0)
    c.set_delays(tau, phi)
    Vg = _fengine(c, x, 0, 30)
    Vo = fx.f_engine(x, n_chan, taps, tau, phi, pfb_window=wname, beta=8.0)
    for a in range(n_in):
        num = np.linalg.norm(Vg[:, :, a] - Vo[a], axis=1)
        den = np.linalg.norm(Vo[a], axis=1)
        assert np.all(num <= 1e-5 * den + 1e-6)
    R, F = _run_dev(c, x, True)
    Ro, Fo, To = fx.correlate(x, n_chan, taps, 8, tau, phi, partial=True, pfb_window=wname, beta=8.0)
    assert _vis_err(R, Ro).max() < 1e-5
    assert _flags_ok(F, Ro, Fo, To).all()


def test_leakage_of_the_gpu_filter_banks():
    """Channel response measured through the GPU F-engine with a dithered
    tone swept across one channel (Fig. 4's comparison) for the plain FFT
    (window 2, one tap), the 4-tap Hann PFB and the 8-tap Kaiser PFB:
    response of the next channel to a tone at a channel centre, worst
    response two or more channels away, and the channel-edge response.
    The FP64 filter responses are -44.4 dB (Hann 4) and -83 dB (Kaiser 8)
    one channel away; the dither floor here is about -68 dB."""
    n_chan = 256
    M = 2 * n_chan
    k0 = 64
    offsets = np.linspace(-0.5, 0.5, 21)
    S = M * 80
    n = np.arange(S)
    # triangular dither turns the int8 rounding error into a white floor
    # instead of harmonic spurs
    rng = np.random.default_rng(3)
    x = np.stack([np.round(120 * np.cos(2 * np.pi * (k0 + d) * n / M) + rng.uniform(-0.5, 0.5, S)
                           + rng.uniform(-0.5, 0.5, S)) for d in offsets]).clip(-128, 127).astype(np.int8)
    out = {}
    for name, window, taps in (("fft", 2, 1), ("hann4", 0, 4), ("kaiser8", 1, 8)):
        c = _corr(len(offsets), 1, n_chan, taps, 8)
        c.set_option("window", window)
        V = _fengine(c, x, 16, 64)[:, :, :len(offsets)]
        P = np.mean(np.abs(V) ** 2, axis=0)          # [n_chan][tone]
        mid = offsets.size // 2
        peak = P[k0, mid]
        adjacent = max(P[k0 + 1, mid], P[k0 - 1, mid]) / peak
        far = np.max(np.delete(P, np.arange(k0 - 1, k0 + 2), axis=0)[:, :]) / peak
        far2 = np.max(np.delete(P, np.arange(k0 - 2, k0 + 3), axis=0)) / peak
        edge = P[k0, 0] / peak
        out[name] = {"adjacent": 10 * np.log10(adjacent), "beyond_1ch": 10 * np.log10(far),
                     "beyond_2ch": 10 * np.log10(far2), "edge": 10 * np.log10(edge)}
    print({k: {m: round(float(v), 1) for m, v in d.items()} for k, d in out.items()})
    assert out["fft"]["beyond_2ch"] > -20.0                        # rectangular sidelobes (-17.9 dB)
    assert abs(out["hann4"]["adjacent"] + 44.4) < 3.0              # the Hann-4 response one channel away
    assert out["kaiser8"]["adjacent"] < out["hann4"]["adjacent"] - 15.0
    assert out["hann4"]["beyond_2ch"] < -60.0 and out["kaiser8"]["beyond_2ch"] < -60.0
    assert abs(out["hann4"]["edge"] + 6.1) < 0.5 and abs(out["kaiser8"]["edge"] + 6.0) < 0.5


# ---------------------------------------------------------------------------
# 16-bit padded input (14-bit ADC values in int16, Sec. 3)
# ---------------------------------------------------------------------------

def _stream16(n_in, S, seed, tau=None, phi=None):
    return make_stream(StreamSpec(n_ant=n_in, n_pol=1, n_samples=S, seed=seed, tau=tau, phi=phi, sigma=1000.0,
                                  bits=14))


@pytest.mark.parametrize("n_chan", [16, 256, 4096])
def test_fengine_16bit_matches_oracle(n_chan):
    M = 2 * n_chan
    n_in, n_spec = 3, 9
    S = M * n_spec + min(29, M - 1)
    tau = np.array([0.0, 11.3, -5.6])
    phi = np.array([0.2, -1.0, 2.0])
    x = _stream16(n_in, S, seed=n_chan + 5, tau=tau, phi=phi)
    assert x.dtype == np.int16 and np.abs(x).max() > 127
    c = _corr(n_in, 1, n_chan, 4, 4, sample_bits=16)
    c.set_delays(tau, phi)
    Vg = _fengine(c, x, 0, n_spec)
    Vo = fx.f_engine(x, n_chan, 4, tau, phi)
    for a in range(n_in):
        num = np.linalg.norm(Vg[:, :, a] - Vo[a], axis=1)
        den = np.linalg.norm(Vo[a], axis=1)
        assert np.all(num <= 1e-5 * den + 1e-6)


def test_16bit_stream_run_push_and_widening():
    n_chan, n_int, n_in = 256, 24, 4
    M = 2 * n_chan
    S = M * (n_int * 3 + 5) + 77
    tau = np.array([0.0, 9.7, 33.2, -2.0])
    phi = np.array([0.0, 0.5, -1.5, 2.5])
    x = _stream16(n_in, S, seed=31, tau=tau, phi=phi)
    c = _corr(n_in, 1, n_chan, 4, n_int, sample_bits=16)
    c.set_delays(tau, phi)
    R, F = _run_dev(c, x, True)
    Ro, Fo, To = fx.correlate(x, n_chan, 4, n_int, tau, phi, partial=True)
    assert _vis_err(R, Ro).max() < 1e-5
    assert _flags_ok(F, Ro, Fo, To).all()
    # host pushes in uneven pieces: bit-identical to the device run
    c2 = _corr(n_in, 1, n_chan, 4, n_int, sample_bits=16, chunk=3000)
    c2.set_delays(tau, phi)
    _push_all(c2, x, [1000, 7, 33333, S - 34340])
    c2.flush()
    assert np.array_equal(c2.get_vis(), R)
    # an int8 stream widened to int16 correlates bit-identically to the int8 path
    x8 = _stream(n_in, S, seed=32, tau=tau, phi=phi)
    c8 = _corr(n_in, 1, n_chan, 4, n_int)
    c8.set_delays(tau, phi)
    c16 = _corr(n_in, 1, n_chan, 4, n_int, sample_bits=16)
    c16.set_delays(tau, phi)
    R8, F8 = _run_dev(c8, x8, True)
    R16, F16 = _run_dev(c16, x8.astype(np.int16), True)
    assert np.array_equal(R8, R16) and np.array_equal(F8, F16)
