"""Pins of the FP64 oracle against facts fixed outside the oracle itself.

Each test checks the oracle against a closed form, a special case that reduces
to an independent library routine, hand-worked values from ``tests/golden``,
an invariant of the mathematics, or brute force on tiny inputs.  Together they
are chosen so that a dropped term, a wrong sign, a wrong index or a swapped
operand anywhere in the oracle fails at least one of them.
"""

import itertools
import json
import math
import os

import numpy as np
import pytest

from oracle import fx_oracle as fx
from fxsynth import StreamSpec, make_stream

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _load(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


# --------------------------------------------------------------------------
# Filter-bank prototype
# --------------------------------------------------------------------------

def test_pfb_coefficients_match_library_window_and_sinc():
    scipy_win = pytest.importorskip("scipy.signal.windows")
    for M, P in [(8, 4), (64, 4), (2048, 4), (16, 8), (32, 1)]:
        L = M * P
        h = fx.pfb_coefficients(M, P)
        ref = scipy_win.hann(L, sym=True) * np.sinc((np.arange(L) - (L - 1) / 2.0) / M)
        np.testing.assert_allclose(h, ref, rtol=0, atol=1e-15)
        np.testing.assert_allclose(h, h[::-1], rtol=0, atol=1e-15)   # symmetric prototype
        assert h[0] == 0.0 and abs(h[-1]) < 1e-15           # Hann end points


def test_pfb_leakage_below_rectangular():
    # Fig. 4: the PFB suppresses sidelobes relative to a rectangular FFT.  For
    # a tone Delta bins away from a channel centre the steady-state channel
    # response is |sum_n h[n] e^{-j 2 pi Delta n / M}|^2 (the filter's DTFT).
    M, P = 64, 4
    h = fx.pfb_coefficients(M, P)
    n = np.arange(M * P)
    delta = np.linspace(1.0, M / 2, 4000)
    pfb = np.abs(np.exp(-2j * np.pi * np.outer(delta, n) / M) @ h) ** 2 / h.sum() ** 2
    rect = np.abs(np.exp(-2j * np.pi * np.outer(delta, np.arange(M)) / M).sum(axis=1)) ** 2 / M ** 2
    assert 10 * np.log10(pfb.max()) < -40.0        # Hann-sinc, 4 taps
    assert 10 * np.log10(rect.max()) > -14.0       # rectangular: -13 dB first sidelobe
    # -6 dB at the channel edge (adjacent channels cross at half power).
    edge = np.abs(np.exp(-1j * np.pi * n / M) @ h) ** 2 / h.sum() ** 2
    assert abs(10 * np.log10(edge) + 6.0) < 0.5


def test_bessel_i0_and_kaiser_window_match_library():
    x = np.linspace(0.0, 30.0, 301)
    np.testing.assert_allclose(fx.bessel_i0(x), np.i0(x), rtol=1e-14, atol=0)
    for L, beta in [(16, 8.0), (65536, 8.0), (1000, 3.5), (7, 0.0)]:
        np.testing.assert_allclose(fx.pfb_window(L, "kaiser", beta), np.kaiser(L, beta), rtol=0, atol=1e-13)


def _channel_response(h, M, delta):
    n = np.arange(h.size)
    return np.abs(np.exp(-2j * np.pi * np.outer(delta, n) / M) @ h) ** 2 / h.sum() ** 2


def test_kaiser_8_tap_pfb_leakage_below_hann_4_tap():
    # Fig. 4's 8-tap Kaiser (beta = 8) prototype: far sidelobes well below the
    # 4-tap Hann-sinc and far below the rectangular FFT; its passband is
    # flatter (smaller scalloping at the channel edge).
    M = 64
    hk = fx.pfb_coefficients(M, 8, "kaiser", 8.0)
    hh = fx.pfb_coefficients(M, 4)
    assert np.allclose(hk, hk[::-1], atol=1e-15)
    far = np.linspace(2.0, M / 2, 3000)
    lk = 10 * np.log10(_channel_response(hk, M, far).max())
    lh = 10 * np.log10(_channel_response(hh, M, far).max())
    assert lk < -60.0 and lk < lh - 10.0
    edge_k = 10 * np.log10(_channel_response(hk, M, np.array([0.5]))[0])
    edge_h = 10 * np.log10(_channel_response(hh, M, np.array([0.5]))[0])
    assert abs(edge_k + 6.0) < 1.0 and abs(edge_h + 6.0) < 0.5
    # "none" with one tap is the plain DFT's unit coefficients
    assert np.array_equal(fx.pfb_coefficients(M, 1, "none"), np.ones(M))


# --------------------------------------------------------------------------
# Channeliser
# --------------------------------------------------------------------------

def test_dft_hand_worked_values():
    for c in _load("dft_small.json")["cases"]:
        Y = fx.dft_brute(np.array(c["y"], dtype=np.float64))
        np.testing.assert_allclose(Y.real, c["re"], atol=1e-12)
        np.testing.assert_allclose(Y.imag, c["im"], atol=1e-12)


@pytest.mark.parametrize("M", [4, 16, 64, 256, 2048])
def test_dft_brute_equals_numpy_rfft(M):
    rng = np.random.default_rng(M)
    y = rng.standard_normal((3, M))
    ref = np.fft.rfft(y, axis=-1)[:, : M // 2]
    Yb = fx.dft_brute(y)
    Yf = fx.channelise(y)
    scale = np.abs(ref).max()
    assert np.abs(Yb - ref).max() < 1e-11 * scale * math.log2(M)
    assert np.abs(Yf - Yb).max() < 1e-11 * scale * math.log2(M)


def test_one_tap_unit_filter_is_plain_dft():
    # P = 1 with h = 1 is a plain per-frame DFT (library routine).
    M, S = 32, 32 * 9
    rng = np.random.default_rng(5)
    x = rng.integers(-128, 128, size=(2, S)).astype(np.int8)
    V = fx.f_engine(x, M // 2, 1, h=np.ones(M))
    ref = np.fft.rfft(x.astype(np.float64).reshape(2, S // M, M), axis=-1)[..., : M // 2]
    np.testing.assert_allclose(V, ref, atol=1e-9)
    Vb = fx.f_engine(x, M // 2, 1, h=np.ones(M), brute=True)
    np.testing.assert_allclose(Vb, ref, atol=1e-9)


def test_fir_tap_order_against_sliding_dot_product():
    # Non-symmetric h so that a reversed tap order cannot hide.
    M, P, S = 8, 3, 8 * 7
    rng = np.random.default_rng(11)
    h = rng.standard_normal(P * M)
    x = rng.standard_normal(S)
    y = fx.pfb_fir(x, h, M, P)
    for s in range(S // M):
        for m in range(M):
            acc = 0.0
            for n in range(P * M):          # pM + m = n, frame index s-P+1+p
                if n % M != m:
                    continue
                idx = (s - P + 1) * M + n
                if idx >= 0:
                    acc += h[n] * x[idx]
            assert abs(acc - y[s, m]) < 1e-12


def test_tone_lands_in_its_channel_closed_form():
    M, P, k0, A, theta = 64, 4, 5, 37.0, 0.7
    S = M * 12
    n = np.arange(S)
    x = A * np.cos(2 * np.pi * k0 * n / M + theta)
    h = fx.pfb_coefficients(M, P)
    Y = fx.channelise(fx.pfb_fir(x, h, M, P))
    g = h.reshape(P, M).sum(axis=0)
    m = np.arange(M)
    expect = (A / 2) * np.exp(1j * theta) * g.sum() + \
             (A / 2) * np.exp(-1j * theta) * np.sum(g * np.exp(-4j * np.pi * k0 * m / M))
    for s in range(P - 1, S // M):
        assert abs(Y[s, k0] - expect) < 1e-9 * abs(expect)
        assert np.argmax(np.abs(Y[s])) == k0


def test_white_noise_power():
    # E|Y_k|^2 = sigma^2 sum_n h[n]^2 for white noise (k != 0).
    M, P, sig = 64, 4, 3.0
    rng = np.random.default_rng(21)
    n_spec = 4000
    x = rng.standard_normal(M * n_spec) * sig
    h = fx.pfb_coefficients(M, P)
    Y = fx.channelise(fx.pfb_fir(x, h, M, P))[P - 1:, 1:]
    p = np.abs(Y) ** 2
    expect = sig ** 2 * np.sum(h ** 2)
    se = p.std() / math.sqrt(p.size)
    assert abs(p.mean() - expect) < 5 * se


# --------------------------------------------------------------------------
# Delay compensation
# --------------------------------------------------------------------------

def test_split_delay_hand_values():
    for tau, d, r in _load("split_delay.json")["cases"]:
        dd, rr = fx.split_delay(tau)
        assert int(dd) == d and abs(float(rr) - r) < 1e-12


def test_coarse_shift_hand_values():
    x = np.array([1, 2, 3, 4, 5], dtype=np.float64)
    np.testing.assert_array_equal(fx.coarse_shift(x, 2), [3, 4, 5, 0, 0])
    np.testing.assert_array_equal(fx.coarse_shift(x, -1), [0, 1, 2, 3, 4])
    np.testing.assert_array_equal(fx.coarse_shift(x, 0), x)
    np.testing.assert_array_equal(fx.coarse_shift(x, 7), [0, 0, 0, 0, 0])


def _source_only(n_in, S, tau, phi, seed=3):
    spec = StreamSpec(n_ant=n_in, n_pol=1, n_samples=S, seed=seed, noise_frac=0.0,
                      src_frac=1.0, tau=tau, phi=phi, block=1 << 14)
    return make_stream(spec)


def test_integer_delay_correction_aligns_inputs_exactly():
    n_chan, P = 32, 4
    M = 2 * n_chan
    tau = np.array([0.0, 3.0, 17.0, 40.0])
    x = _source_only(4, M * 40, tau, None)
    V = fx.f_engine(x, n_chan, P, tau=tau)
    last = V.shape[1] - 1                       # tail frame sees zero fill
    for a in range(1, 4):
        np.testing.assert_array_equal(V[a, :last], V[0, :last])
    R = fx.x_engine(V[:, :last], n_int=last)
    for a in range(4):
        np.testing.assert_allclose(R[0, :, 0, a], R[0, :, 0, 0], rtol=1e-13, atol=0)


def test_uncorrected_delay_gives_phase_slope_2pi_f_tau():
    n_chan, P = 64, 4
    M = 2 * n_chan
    tau = np.array([0.0, 5.0, -3.0])
    x = _source_only(3, M * 400, tau, None)
    R = fx.correlate(x, n_chan, P, n_int=400)[0][0]
    k = np.arange(n_chan)
    for a in (1, 2):
        ph = np.unwrap(np.angle(R[1:-1, 0, a]))
        slope = np.polyfit(k[1:-1], ph, 1)[0]
        assert abs(slope - 2 * np.pi * tau[a] / M) < 0.01 * 2 * np.pi / M


def test_fractional_delay_and_phase_correction_flatten_phase():
    n_chan, P = 64, 4
    M = 2 * n_chan
    tau = np.array([0.0, 7.3, 22.6, 39.9])
    phi = np.array([0.0, 1.0, -2.0, 2.9])
    x = _source_only(4, M * 512, tau, phi)
    R_on = fx.correlate(x, n_chan, P, n_int=512, tau=tau, phi=phi)[0][0]
    R_off = fx.correlate(x, n_chan, P, n_int=512)[0][0]
    band = slice(4, n_chan - 4)
    for a in (1, 2, 3):
        assert np.abs(np.angle(R_on[band, 0, a])).max() < 0.05
        # Without correction the phase is far from flat.
        assert np.abs(np.angle(R_off[band, 0, a])).max() > 1.0


# --------------------------------------------------------------------------
# X-engine
# --------------------------------------------------------------------------

def test_x_engine_brute_force_loops():
    rng = np.random.default_rng(2)
    n_in, n_spec, n_chan = 3, 7, 4
    V = rng.standard_normal((n_in, n_spec, n_chan)) + 1j * rng.standard_normal((n_in, n_spec, n_chan))
    R = fx.x_engine(V, n_int=3, partial=True)
    assert R.shape == (3, n_chan, n_in, n_in)
    for i, (s0, s1) in enumerate([(0, 3), (3, 6), (6, 7)]):
        for k in range(n_chan):
            for a in range(n_in):
                for b in range(n_in):
                    acc = 0j
                    for s in range(s0, s1):
                        acc += V[a, s, k] * complex(V[b, s, k].real, -V[b, s, k].imag)
                    assert abs(acc / (s1 - s0) - R[i, k, a, b]) < 1e-12
    assert fx.x_engine(V, n_int=3).shape[0] == 2


def test_identical_inputs_cross_equals_auto_and_hermitian_psd():
    rng = np.random.default_rng(9)
    x = rng.integers(-60, 60, size=(3, 64 * 50)).astype(np.int8)
    x[2] = x[0]
    R, _, _ = fx.correlate(x, 32, 4, n_int=25)
    np.testing.assert_allclose(R[..., 0, 2], R[..., 0, 0], rtol=1e-13)
    np.testing.assert_array_equal(R[..., 0, 0].imag, 0.0)
    assert np.all(R[..., 0, 0].real >= 0)
    np.testing.assert_allclose(R, np.conj(np.swapaxes(R, -1, -2)), rtol=0, atol=1e-9)
    ev = np.linalg.eigvalsh(R)
    assert ev.min() > -1e-9 * ev.max()


# --------------------------------------------------------------------------
# MAD flagging (Eq. 2)
# --------------------------------------------------------------------------

def test_mad_hand_worked_cases():
    for c in _load("mad_cases.json")["cases"]:
        A = np.array(c["A"], dtype=np.float64)
        assert fx.median_exact(A) == pytest.approx(c["median"], abs=1e-12)
        med = fx.median_exact(A)
        assert fx.median_exact(np.abs(A - med)) == pytest.approx(c["mad"], abs=1e-12)
        T = fx.mad_threshold(A, c["sigma"])
        assert T == pytest.approx(c["T"], abs=1e-9)
        assert list((A > T).astype(int)) == c["flags"]


def test_median_against_numpy_and_permutations():
    rng = np.random.default_rng(4)
    for n in [1, 2, 3, 7, 8, 64, 65]:
        v = rng.standard_normal(n)
        assert fx.median_exact(v) == pytest.approx(float(np.median(v)), abs=1e-15)
    base = [3.0, -1.0, 7.5, 7.5, 0.25, 2.0]
    vals = {fx.median_exact(np.array(p)) for p in itertools.permutations(base)}
    assert vals == {0.5 * (2.0 + 3.0)}


def test_mad_flags_windows_are_aligned_and_independent():
    n_chan, w = 128, 64
    rng = np.random.default_rng(8)
    R = (1.0 + 0.01 * rng.standard_normal((1, n_chan, 2, 2))).astype(np.complex128)
    R[0, 10, 0, 1] = 50.0        # outlier in window 0, baseline (0,1)
    R[0, 100, 1, 1] = 50.0       # outlier in window 1, auto (1,1)
    flags, A, T = fx.mad_flags(R, 5.0, w)
    assert flags[0, 10, 0, 1] == 1 and flags[0, 100, 1, 1] == 1
    assert flags.sum() == 2
    # Thresholds are constant inside a window and follow Eq. 2 there.
    for k0 in (0, 64):
        blk = A[0, k0:k0 + w, 0, 1]
        assert np.all(T[0, k0:k0 + w, 0, 1] == fx.mad_threshold(blk, 5.0))


def test_partial_integration_divides_by_actual_count():
    rng = np.random.default_rng(1)
    V = np.ones((1, 10, 2), dtype=np.complex128) * 2.0
    R = fx.x_engine(V, n_int=4, partial=True)
    assert R.shape[0] == 3
    np.testing.assert_allclose(R[:, :, 0, 0], 4.0)


def test_sampled_oracle_matches_full_oracle():
    rng = np.random.default_rng(17)
    n_chan, P = 32, 4
    M = 2 * n_chan
    x = rng.integers(-128, 128, size=(3, M * 20)).astype(np.int8)
    tau = np.array([0.0, 5.4, -2.7])
    phi = np.array([0.1, -1.0, 2.0])
    V = fx.f_engine(x, n_chan, P, tau, phi)
    spectra, chans = [0, 3, 19], [0, 7, 31]
    Vs = fx.f_engine_sampled(x, n_chan, P, tau, phi, spectra, chans)
    np.testing.assert_allclose(Vs, V[:, spectra][:, :, chans], rtol=1e-10, atol=1e-9)
