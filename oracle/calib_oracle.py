"""FP64 oracle of the delay / phase calibration -- TEST INFRASTRUCTURE ONLY.

Sec. 7 calibrates in three serial steps on the visibilities of each baseline
(ref, a), over a clean band of channels:

1. coarse group delay: the peak of the delay spectrum, the Fourier transform
   of the visibilities along frequency;
2. fine delay: a weighted linear fit to the unwrapped phase against
   frequency, tau_residual = (1 / 2 pi) d phi / d nu (Eq. 3);
3. residual phase: the argument of the mean complex vector once the delay is
   removed.

Readings (also listed in the design notes):
* Units: channel k sits at nu_k = k / M cycles per sample (M = 2 n_chan);
  delays are in samples.  With x_a delayed by tau_a and rotated by +phi_a
  (the synthetic streams' convention), R_ref,a[k] = <V_ref conj(V_a)> has
  argument 2 pi k (tau_a - tau_ref) / M - (phi_a - phi_ref), so the solution
  (tau_a - tau_ref, phi_a - phi_ref) is what ``corr_set_delays`` takes to
  flatten the phases.
* The delay spectrum is evaluated directly on a grid of trial delays
  t = -T, -T + 1/4, ..., T (T = ``max_delay``), weighting each channel by 1
  (unflagged) or 0 (flagged or outside [k_lo, k_hi)); the first maximum of
  its magnitude wins.
* The fine fit weights channels by |R|, on the phase of R[k] with the coarse
  slope removed.  The phase is unwrapped about the band's mean vector c0
  (psi_k = arg c0 + wrap(arg R_k - arg c0)): the coarse step leaves at most
  1/8 sample of delay, i.e. at most pi/8 of drift across the band, so there
  is no 2 pi ambiguity to resolve, and an isolated channel whose noisy phase
  sits near +-pi stays one outlier instead of adding 2 pi to every later
  channel as a sequential unwrap would.  On noise-free data the two agree.
"""

from __future__ import annotations

import numpy as np

GRID = 4   # trial delays per sample


def delay_spectrum(R: np.ndarray, w: np.ndarray, M: int, max_delay: float) -> tuple:
    """(trial delays t, |sum_k w_k R_k exp(-j 2 pi k t / M)|) for one baseline."""
    k = np.arange(R.size, dtype=np.float64)
    t = np.arange(-int(round(max_delay * GRID)), int(round(max_delay * GRID)) + 1, dtype=np.float64) / GRID
    ph = np.exp(-2j * np.pi * np.outer(t, k) / M)
    return t, np.abs(ph @ (w * R))


def calibrate_baseline(R: np.ndarray, M: int, mask: np.ndarray, max_delay: float) -> tuple:
    """(tau, phi) of one baseline's visibilities R[k] (complex, FP64)."""
    R = np.asarray(R, np.complex128)
    w0 = mask.astype(np.float64)
    t, D = delay_spectrum(R, w0, M, max_delay)
    t_c = t[int(np.argmax(D))]
    k = np.arange(R.size, dtype=np.float64)
    sel = mask.astype(bool)
    Rc = R * np.exp(-2j * np.pi * k * t_c / M)
    c0 = np.sum(Rc[sel])
    psi = np.angle(c0) + np.angle(Rc[sel] * np.conj(c0))
    wk = np.abs(R[sel])
    # weighted least squares psi = c + b k
    kk = k[sel]
    W = wk.sum()
    kb = (wk * kk).sum() / W
    pb = (wk * psi).sum() / W
    b = (wk * (kk - kb) * (psi - pb)).sum() / (wk * (kk - kb) ** 2).sum()
    tau = t_c + b * M / (2.0 * np.pi)
    c = np.sum(R[sel] * np.exp(-2j * np.pi * kk * tau / M))
    phi = -np.angle(c)
    return float(tau), float(phi)


def calibrate(R: np.ndarray, ref: int = 0, k_lo: int = 0, k_hi=None, max_delay: float = 64.0,
              flags=None) -> tuple:
    """Per-input (tau, phi) relative to input ``ref`` from visibilities
    R[k][a][b] of one integration (flags[k][a][b] nonzero = excluded)."""
    R = np.asarray(R)
    n_chan, n_in = R.shape[0], R.shape[1]
    M = 2 * n_chan
    k_hi = n_chan if k_hi is None else k_hi
    tau = np.zeros(n_in)
    phi = np.zeros(n_in)
    band = np.zeros(n_chan, bool)
    band[k_lo:k_hi] = True
    for a in range(n_in):
        if a == ref:
            continue
        mask = band.copy()
        if flags is not None:
            mask &= np.asarray(flags)[:, ref, a] == 0
        tau[a], phi[a] = calibrate_baseline(R[:, ref, a], M, mask, max_delay)
    return tau, phi
