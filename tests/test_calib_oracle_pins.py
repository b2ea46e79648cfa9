"""Pins of the calibration oracle (Sec. 7, Eq. 3): exact recovery on
analytic visibilities, the delay spectrum's closed-form peak, and recovery of
the delays and phases injected into a synthetic stream, with the phases flat
after the correction is applied."""

import numpy as np

from fxsynth import StreamSpec, make_stream
from oracle import calib_oracle as co
from oracle import fx_oracle as fx


def test_exact_recovery_on_analytic_visibilities():
    n_chan = 512
    M = 2 * n_chan
    k = np.arange(n_chan)
    for dtau, dphi in [(13.37, 0.8), (-20.6, -2.9), (0.0, 0.0), (41.124, 3.0)]:
        R = 3.0 * np.exp(1j * (2 * np.pi * k * dtau / M - dphi))
        tau, phi = co.calibrate_baseline(R, M, np.ones(n_chan, bool), 64.0)
        assert abs(tau - dtau) < 1e-9
        assert abs(np.angle(np.exp(1j * (phi - dphi)))) < 1e-9


def test_delay_spectrum_peak_closed_form():
    # on the grid the aligned sum is the number of weighted channels; one
    # sample off it is |sin(pi n / M) / sin(pi / M)| (n channels)
    n_chan, M = 256, 512
    k = np.arange(n_chan)
    R = np.exp(2j * np.pi * k * 7.25 / M)
    w = np.ones(n_chan)
    w[:10] = 0
    t, D = co.delay_spectrum(R, w, M, 16.0)
    assert abs(t[np.argmax(D)] - 7.25) < 1e-12
    assert abs(D.max() - 246.0) < 1e-9
    i1 = int(np.argmax(D)) + co.GRID
    n = 246
    assert abs(D[i1] - abs(np.sin(np.pi * n / M) / np.sin(np.pi / M))) < 1e-9


def test_recovers_injected_delays_and_flattens_phase():
    n_chan, n_int = 512, 256
    M = 2 * n_chan
    tau = np.array([0.0, 7.3, -11.8, 29.45])
    phi = np.array([0.0, 1.2, -0.7, 2.5])
    x = make_stream(StreamSpec(n_ant=4, n_pol=1, n_samples=M * n_int, seed=77, tau=tau, phi=phi,
                               src_frac=0.2))
    R, _, _ = fx.correlate(x, n_chan, 4, n_int)          # correlator without delay correction
    t_hat, p_hat = co.calibrate(R[0], ref=0, k_lo=8, k_hi=n_chan - 8, max_delay=48.0)
    assert np.max(np.abs(t_hat - tau)) < 0.05
    assert np.max(np.abs(np.angle(np.exp(1j * (p_hat - phi))))) < 0.05
    # closing the loop: with the solution applied the phases are flat
    R2, _, _ = fx.correlate(x, n_chan, 4, n_int, t_hat, p_hat)
    for a in range(1, 4):
        ph = np.angle(R2[0, 8:n_chan - 8, 0, a])
        assert abs(np.angle(np.mean(np.exp(1j * ph)))) < 0.05
        t2, _ = co.calibrate_baseline(R2[0, :, 0, a], M, np.arange(n_chan) >= 8, 48.0)
        assert abs(t2) < 0.05


def test_unwrap_about_the_mean_matches_sequential_unwrap_when_clean_and_resists_outliers():
    n_chan = 1024
    M = 2 * n_chan
    k = np.arange(n_chan)
    R = 5.0 * np.exp(1j * (2 * np.pi * k * 3.1 / M - 0.4))
    mask = np.ones(n_chan, bool)
    t1, p1 = co.calibrate_baseline(R, M, mask, 16.0)
    assert abs(t1 - 3.1) < 1e-9 and abs(p1 - 0.4) < 1e-9
    # one weak channel with its phase flipped: a sequential unwrap of the
    # residual phase would carry a 2 pi step into the whole upper band
    R2 = R.copy()
    R2[300] = -0.05 * R[300] * np.exp(0.2j)
    t2, p2 = co.calibrate_baseline(R2, M, mask, 16.0)
    assert abs(t2 - 3.1) < 1e-3 and abs(p2 - 0.4) < 1e-3
