"""Pins of the oracle parts that no other pin reaches: the parity measures
every visibility test relies on, and the requantisation scale rule with its
schedule (pre-pass for the first integration, previous autocorrelations
after that).

The measures are checked against hand-worked two-channel cases
(tests/golden/checker_cases.json).  The scale schedule is checked on a
stream whose channelised voltage has a closed form: a quarter-band tone
x[n] = A cos(pi n / 2) = A, 0, -A, 0, ... (exact in int8), one tap, so that
spectrum s depends on frame s alone and Y_s[M/4] = A * sum_{m even} h[m]
(the DFT row e^{-j pi m / 2} = (-j)^m times the tone is A at even m and 0
at odd m).  The amplitude steps inside the first integration, so the
pre-pass over its first 64 spectra, the whole-integration mean and the
previous integration's autos all give different scales.
"""

import json
import os

import numpy as np
import pytest

from oracle import fx_oracle as fx
from oracle import requant_oracle as rq

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "checker_cases.json")


def _case():
    return json.load(open(GOLDEN))


def test_rel_frobenius_per_channel_hand_case():
    c = _case()["rel_frobenius"]
    ref = np.array(c["ref_re"]) + 1j * np.array(c["ref_im"])
    test = np.array(c["test_re"]) + 1j * np.array(c["test_im"])
    got = fx.rel_frobenius_per_channel(test, ref)
    assert got.shape == (1, 2)                      # one value per (integration, channel)
    np.testing.assert_allclose(got, c["expect"], rtol=1e-14)


def test_normalised_coefficients_hand_case():
    c = _case()["normalised"]
    R = np.array(c["R_re"]) + 1j * np.array(c["R_im"])
    rho = np.array(c["rho_re"]) + 1j * np.array(c["rho_im"])
    np.testing.assert_allclose(fx.normalised_coefficients(R), rho, rtol=1e-14, atol=1e-15)
    # with a leading integration axis the result is the same per integration
    np.testing.assert_allclose(fx.normalised_coefficients(R[None]), rho[None], rtol=1e-14, atol=1e-15)


@pytest.mark.parametrize("dtype,P,sigma", [
    ("int8", 2.0 * 24 ** 2, 1.0),           # sigma = sqrt(P/2)/24 off DC
    ("int8", 9 * 2.0 * 24 ** 2, 3.0),
    ("e4m3", 2.0 * 64 ** 2, 1.0),           # sigma = sqrt(P/2)/64
    ("e4m3", 0.25 * 2.0 * 64 ** 2, 0.5),
    ("int8", 0.0, 1.0),                     # no power: unit scale
])
def test_scales_from_power_hand_values(dtype, P, sigma):
    # channel 1 of a two-channel row (channel 0 is the DC bin, below)
    assert rq.scales_from_power(np.array([[1.0, P]]), dtype)[0, 1] == pytest.approx(sigma, rel=1e-15)


@pytest.mark.parametrize("dtype,g", [("int8", 24.0), ("e4m3", 64.0)])
def test_scale_of_the_real_dc_channel(dtype, g):
    """The DC bin of a real transform is real, so its one component carries
    the whole power: sigma = sqrt(P)/g there, sqrt(P/2)/g elsewhere."""
    P = np.array([[g ** 2, 2.0 * g ** 2, 4.0 * g ** 2], [9 * g ** 2, 0.0, 2.0 * g ** 2]])
    np.testing.assert_allclose(rq.scales_from_power(P, dtype), [[1.0, 1.0, np.sqrt(2.0)], [3.0, 1.0, 1.0]],
                               rtol=1e-15)


def _tone_step_stream(M, n_int, a1, a2):
    """One input: frames 0..63 carry the quarter-band tone at amplitude a1,
    every later frame at a2 (two integrations of n_int frames)."""
    n_frames = 2 * n_int
    amp = np.where(np.arange(n_frames) < 64, a1, a2)
    pattern = np.tile([1, 0, -1, 0], M // 4)
    return (amp[:, None] * pattern[None, :]).reshape(1, -1).astype(np.int8)


@pytest.mark.parametrize("dtype", ["int8", "e4m3"])
def test_scale_schedule_on_a_tone_step(dtype):
    n_chan, n_int, a1, a2 = 8, 128, 20, 40
    M = 2 * n_chan
    k0 = M // 4
    x = _tone_step_stream(M, n_int, a1, a2)
    h = fx.pfb_coefficients(M, 1)
    H = h[0::2].sum()                                  # Y_s[k0] = A H
    R, S = rq.correlate_quantized(x, n_chan, 1, n_int, dtype=dtype)
    assert R.shape[0] == 2
    g = {"int8": 24.0, "e4m3": 64.0}[dtype]
    # integration 0: pre-pass over its first 64 spectra, all at a1 (k0 > 0:
    # the component power is half of |V|^2)
    s0 = np.sqrt((a1 * H) ** 2 / 2.0) / g
    assert S[0, 0, k0] == pytest.approx(s0, rel=1e-12)
    # its codes: a1 H / s0 = g sqrt(2) for 64 spectra, 2 g sqrt(2) for the rest
    c1, c2 = rq.quantize(np.array([g * np.sqrt(2.0), 2 * g * np.sqrt(2.0)]), dtype)
    if dtype == "int8":
        assert (c1, c2) == (34.0, 68.0)                # 33.94 -> 34, 67.88 -> 68
    else:
        assert (c1, c2) == (88.0, 176.0)               # e4m3 steps of 8 and 16 there
    raa0 = s0 ** 2 * (64 * c1 ** 2 + (n_int - 64) * c2 ** 2) / n_int
    assert R[0, k0, 0, 0].real == pytest.approx(raa0, rel=1e-12)
    # integration 1: scales from integration 0's autocorrelation
    s1 = np.sqrt(raa0 / 2.0) / g
    assert S[1, 0, k0] == pytest.approx(s1, rel=1e-12)
    c3 = rq.quantize(np.array([a2 * H / s1]), dtype)[0]
    assert R[1, k0, 0, 0].real == pytest.approx(s1 ** 2 * c3 ** 2, rel=1e-12)
