"""Pins of the complex (I/Q) input oracle (Sec. 4.2, complex voltage streams;
the reading is stated in oracle/fx_oracle.py): hand-worked DFTs, numpy's FFT
as the library routine, closed-form complex tones at positive and negative
frequencies, the real path as the special case Q = 0, and the signed channel
frequencies in the delay correction (a fractionally delayed complex source
has a flat cross-phase after correction in both halves of the band, and the
phase slope 2 pi f_k tau before it)."""

import json
import os

import numpy as np
import pytest

from oracle import fx_oracle as fx

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "dft_complex_small.json")


def _interleave(z):
    """complex [n_in][S] -> interleaved [n_in][2S] (I, Q, I, Q, ...)."""
    out = np.empty(z.shape[:-1] + (2 * z.shape[-1],))
    out[..., 0::2] = z.real
    out[..., 1::2] = z.imag
    return out


def test_complex_dft_hand_cases_and_frequencies():
    g = json.load(open(GOLDEN))
    for c in g["dft"]:
        y = np.array(c["y_re"]) + 1j * np.array(c["y_im"])
        Y = np.array(c["Y_re"]) + 1j * np.array(c["Y_im"])
        np.testing.assert_allclose(fx.dft_brute_complex(y), Y, atol=1e-12)
    np.testing.assert_array_equal(fx.channel_frequency_iq(8), g["frequencies_M8"])


def test_complex_dft_matches_library():
    rng = np.random.default_rng(3)
    y = rng.standard_normal((5, 64)) + 1j * rng.standard_normal((5, 64))
    np.testing.assert_allclose(fx.dft_brute_complex(y), np.fft.fft(y, axis=-1), atol=1e-10)


def test_iq_deinterleave():
    x = np.array([[1, -2, 3, 4, -5, 6]], dtype=np.int8)
    np.testing.assert_array_equal(fx.iq_to_complex(x), [[1 - 2j, 3 + 4j, -5 + 6j]])


@pytest.mark.parametrize("sign", [1, -1])
def test_complex_tone_lands_in_its_signed_channel(sign):
    """x[n] = A e^{+-j pi n / 2}, exact in int8 (A, 0, -A, 0 / 0, +-A, 0, -+A):
    after the P-1 start-up spectra, Y[M/4] (positive tone) or Y[3M/4]
    (negative tone) = A sum_n h[n], and the other tone's bin holds
    A sum_n h[n] (-1)^n."""
    M, P, A = 64, 4, 20
    n = np.arange(M * 12)
    z = A * np.exp(sign * 1j * np.pi * n / 2)
    x = np.round(_interleave(z[None])).astype(np.int8)
    V = fx.f_engine_iq(x, M, P)[0, P - 1:]
    h = fx.pfb_coefficients(M, P)
    k_on, k_off = (M // 4, 3 * M // 4) if sign > 0 else (3 * M // 4, M // 4)
    np.testing.assert_allclose(V[:, k_on], A * h.sum(), rtol=1e-12)
    np.testing.assert_allclose(V[:, k_off], A * np.sum(h * (-1.0) ** np.arange(h.size)), atol=1e-9)


def test_real_input_is_the_q_zero_case():
    """With Q = 0 and M = 2 n_chan, channels 0 .. n_chan-1 of the complex path
    are the real path's channels (same prototype, same delay phases)."""
    rng = np.random.default_rng(11)
    n_chan, P, S = 32, 4, 64 * 20
    I = rng.integers(-60, 60, size=(3, S)).astype(np.int8)
    tau, phi = np.array([0.0, 3.3, -7.8]), np.array([0.0, 1.1, -0.4])
    x = _interleave(I.astype(np.float64) + 0j)
    V_iq = fx.f_engine_iq(x, 2 * n_chan, P, tau, phi)
    V_re = fx.f_engine(I, n_chan, P, tau, phi)
    np.testing.assert_allclose(V_iq[:, :, :n_chan], V_re, rtol=1e-12, atol=1e-9)


def test_fractional_delay_phase_in_both_halves_of_the_band():
    """Input 1 is input 0's complex white source delayed by tau = 3.3 samples
    (exact, by a circular phase ramp over the stream).  Before correction the
    cross-phase follows +2 pi f_k tau with f_k signed; with the delay applied
    it is flat in every channel.  The channel centred on +-fs/2 (k = M/2)
    straddles the band edge, where a delay's phase jumps between the two
    sides, so it is left out of both checks."""
    rng = np.random.default_rng(5)
    M, P, S, tau = 32, 4, 32 * 600, 3.3
    s = rng.standard_normal(S) + 1j * rng.standard_normal(S)
    f = np.fft.fftfreq(S)
    s1 = np.fft.ifft(np.fft.fft(s) * np.exp(-2j * np.pi * f * tau))
    x = _interleave(50.0 * np.stack([s, s1]))
    fk = fx.channel_frequency_iq(M)
    keep = np.arange(M) != M // 2
    R0 = fx.x_engine(fx.f_engine_iq(x, M, P), 600)[0]
    ph0 = np.angle(R0[:, 0, 1] * np.exp(-2j * np.pi * fk * tau))
    assert np.abs(ph0[keep]).max() < 0.05
    R1 = fx.x_engine(fx.f_engine_iq(x, M, P, [0.0, tau]), 600)[0]
    assert np.abs(np.angle(R1[keep, 0, 1])).max() < 0.05
    # unsigned frequencies (k / M throughout) would leave 2 pi tau in the upper half
    wrong = np.angle(R0[:, 0, 1] * np.exp(-2j * np.pi * (np.arange(M) / M) * tau))
    assert np.abs(wrong[M // 2 + 1:]).min() > 1.0


def test_iq_visibilities_hermitian_and_identical_inputs():
    rng = np.random.default_rng(2)
    n_chan, P, n_int = 16, 4, 8
    z = rng.integers(-50, 50, size=(1, 2 * n_chan * n_int * 3)).astype(np.int8)
    x = np.concatenate([z, z, rng.integers(-50, 50, size=z.shape).astype(np.int8)])
    R, F, T = fx.correlate_iq(x, n_chan, P, n_int, window=16)
    np.testing.assert_allclose(R, np.conj(np.swapaxes(R, -1, -2)), atol=1e-9)
    np.testing.assert_allclose(R[..., 0, 1], R[..., 0, 0], rtol=1e-12)
    assert F.shape == R.shape
