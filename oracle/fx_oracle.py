"""FP64 oracle of the FX correlator hot path -- TEST INFRASTRUCTURE ONLY.

Every function is the plain definition of one step, written in numpy float64 /
complex128, with no blocking, fusion or reordering beyond what the definition
states.  Library primitives used as single steps: ``numpy.fft.rfft`` (the
channeliser at full size; pinned against :func:`dft_brute`), ``numpy.einsum``
(the correlation sum) and ``numpy.sort`` (order statistics).

Paper passages followed (arXiv 2604.20640):

* Eq. 1 (Sec. 4.1): cross-power spectrum S_ij(nu) = < V_i V_j^* e^{j 2 pi nu tau_g,ij} >,
  the geometric delay compensated by a linear phase, <.> a time integration.
* Sec. 4.2, "F-engine (PFB and FFT)": raw samples unpacked to voltages, a
  polyphase-filter-bank weighting, then an FFT (Fig. 4 shows the PFB's lower
  sidelobes against a rectangular-window FFT).
* Sec. 4.2, "X-engine and integration" and Algorithm 1: V_i V_j^* for all
  baselines accumulated over the integration interval.
* Eq. 2 (Sec. 7): MAD sigma clipping, T = median(A) + sigma * MAD(A) * 1.4826,
  sigma = 5, on visibility amplitude A.

Readings where the paper is silent (each also recorded in the design notes):

1. Prototype filter: symmetric Hann window (denominator L-1) times a sinc with
   cutoff 1/M centred at (L-1)/2, L = P*M, unnormalised.
2. Zero history before the first sample: spectrum s (s = 0 .. S//M - 1) uses
   frames s-P+1 .. s, frames before the stream are zero.
3. Real samples, M = 2*n_chan point real transform, DC kept, Nyquist dropped.
4. Forward transform sign e^{-j...}, unscaled.
5. Delay correction per input: coarse advance by d = floor(tau + 1/2) samples
   (x'[n] = x[n+d], zero outside the stream), then the fine phase
   exp(+j 2 pi k r / M) with r = tau - d, then the instrument phase exp(-j phi).
   Eq. 1's per-baseline factor exp(j 2 pi nu (tau_i - tau_j)) factorises into
   these per-input terms.
6. <.> is the mean over n_int consecutive spectra; a partial last integration
   is emitted only at end of stream, divided by its actual count.
7. Visibility R[k][a][b] = <V_a[k] conj(V_b[k])>, full Hermitian matrix.
8. MAD flagging per integration, per baseline (a, b) (autos included), on
   windows of ``window`` channels aligned at channel 0; A = |R_ab|; even-count
   median = mean of the two middle order statistics; MAD = 0 not special-cased;
   flag = A > T (strict, upper one-sided).
"""

from __future__ import annotations

import math
from typing import Optional, Sequence

import numpy as np

MAD_TO_SIGMA = 1.4826   # Eq. 2


# --------------------------------------------------------------------------
# F-engine
# --------------------------------------------------------------------------

def bessel_i0(x) -> np.ndarray:
    """Modified Bessel function of the first kind, order 0, from its power
    series I0(x) = sum_k ((x/2)^k / k!)^2 (all terms positive), summed until
    a term no longer changes the FP64 sum."""
    x = np.asarray(x, np.float64)
    q = (x / 2.0) ** 2
    term = np.ones_like(x)
    total = np.ones_like(x)
    k = 0
    while True:
        k += 1
        term = term * q / (k * k)
        if np.all(term <= 1e-17 * total):
            return total
        total = total + term


def pfb_window(L: int, kind: str = "hann", beta: float = 8.0) -> np.ndarray:
    """Taper of the prototype filter, n = 0 .. L-1: symmetric Hann
    0.5 - 0.5 cos(2 pi n / (L-1)) (reading 1), or Kaiser
    I0(beta sqrt(1 - (2n/(L-1) - 1)^2)) / I0(beta) (the 8-tap, beta = 8
    window of Fig. 4)."""
    n = np.arange(L, dtype=np.float64)
    if kind == "hann":
        return 0.5 - 0.5 * np.cos(2.0 * np.pi * n / (L - 1))
    if kind == "kaiser":
        r = 2.0 * n / (L - 1) - 1.0
        return bessel_i0(beta * np.sqrt(np.maximum(0.0, 1.0 - r * r))) / bessel_i0(np.array(beta))
    raise ValueError(kind)


def pfb_coefficients(M: int, P: int, window: str = "hann", beta: float = 8.0) -> np.ndarray:
    """Prototype FIR h[n], n = 0 .. P*M-1 (Sec. 4.2 PFB weighting; reading 1):
    the taper times a sinc of cutoff 1/M centred at (L-1)/2.  ``window =
    "none"`` gives h = 1 (with P = 1 the plain per-frame DFT, the
    rectangular-FFT reference of Fig. 4)."""
    L = P * M
    if L < 2:
        raise ValueError("P*M must be at least 2")
    if window == "none":
        return np.ones(L)
    n = np.arange(L, dtype=np.float64)
    w = pfb_window(L, window, beta)
    x = (n - (L - 1) / 2.0) / M
    sinc = np.ones(L)
    nz = x != 0.0
    sinc[nz] = np.sin(np.pi * x[nz]) / (np.pi * x[nz])
    return w * sinc


def split_delay(tau) -> tuple:
    """Coarse integer advance d = floor(tau + 1/2) and fine remainder r = tau - d."""
    tau = np.asarray(tau, dtype=np.float64)
    d = np.floor(tau + 0.5)
    return d.astype(np.int64), tau - d


def coarse_shift(x: np.ndarray, d: int) -> np.ndarray:
    """x'[n] = x[n + d] for 0 <= n + d < S, else 0 (reading 5)."""
    x = np.asarray(x, dtype=np.float64)
    S = x.shape[-1]
    out = np.zeros(S)
    lo, hi = max(0, -d), min(S, S - d)
    if hi > lo:
        out[lo:hi] = x[lo + d: hi + d]
    return out


def pfb_fir(xp: np.ndarray, h: np.ndarray, M: int, P: int) -> np.ndarray:
    """y[s][m] = sum_p h[pM + m] x'[(s - P + 1 + p) M + m], zero frames before 0."""
    n_spec = xp.shape[-1] // M
    frames = xp[: n_spec * M].reshape(n_spec, M)
    y = np.zeros((n_spec, M))
    for p in range(P):
        shift = P - 1 - p               # frame index s - shift
        if shift >= n_spec:
            continue
        y[shift:] += h[p * M:(p + 1) * M][None, :] * frames[: n_spec - shift]
    return y


def dft_brute(y: np.ndarray) -> np.ndarray:
    """Y[k] = sum_m y[m] e^{-j 2 pi k m / M}, k = 0 .. M/2-1, by direct summation."""
    M = y.shape[-1]
    k = np.arange(M // 2)[:, None]
    m = np.arange(M)[None, :]
    W = np.exp(-2j * np.pi * ((k * m) % M) / M)
    return y @ W.T


def channelise(y: np.ndarray) -> np.ndarray:
    """Same sum as :func:`dft_brute`, through numpy's FFT (library step)."""
    M = y.shape[-1]
    return np.fft.rfft(y, axis=-1)[..., : M // 2]


def fine_correct(Y: np.ndarray, r: float, phi: float, M: int) -> np.ndarray:
    """V[k] = Y[k] exp(j (2 pi k r / M - phi))  (Eq. 1 phase term; reading 5)."""
    k = np.arange(Y.shape[-1])
    return Y * np.exp(1j * (2.0 * np.pi * k * r / M - phi))


def f_engine(x: np.ndarray, n_chan: int, taps: int, tau=None, phi=None,
             h: Optional[np.ndarray] = None, brute: bool = False, pfb_window: str = "hann",
             beta: float = 8.0) -> np.ndarray:
    """Channelised, delay-corrected voltages V[a][s][k] (complex128).

    ``x`` is ``[n_in][S]``; ``tau`` total delays in samples, ``phi`` instrument
    phases in radians (both per input, default 0).
    """
    x = np.asarray(x)
    n_in = x.shape[0]
    M = 2 * n_chan
    if h is None:
        h = pfb_coefficients(M, taps, pfb_window, beta)
    tau = np.zeros(n_in) if tau is None else np.asarray(tau, np.float64)
    phi = np.zeros(n_in) if phi is None else np.asarray(phi, np.float64)
    d, r = split_delay(tau)
    n_spec = x.shape[1] // M
    V = np.empty((n_in, n_spec, n_chan), dtype=np.complex128)
    for a in range(n_in):
        xp = coarse_shift(x[a], int(d[a]))
        y = pfb_fir(xp, h, M, taps)
        Y = dft_brute(y) if brute else channelise(y)
        V[a] = fine_correct(Y, float(r[a]), float(phi[a]), M)
    return V


def f_engine_sampled(x: np.ndarray, n_chan: int, taps: int, tau, phi, spectra: Sequence[int],
                     chans: Sequence[int]) -> np.ndarray:
    """V[a][i][j] for spectrum ``spectra[i]`` and channel ``chans[j]`` only.

    Each value is the direct sum of the definition (filter then one DFT row),
    so it scales to streams of any length.
    """
    x = np.asarray(x)
    n_in = x.shape[0]
    M = 2 * n_chan
    h = pfb_coefficients(M, taps)
    d, r = split_delay(np.asarray(tau, np.float64))
    phi = np.asarray(phi, np.float64)
    chans = np.asarray(chans)
    m = np.arange(M)
    rows = np.exp(-2j * np.pi * ((chans[:, None] * m[None, :]) % M) / M)
    S = x.shape[1]
    out = np.empty((n_in, len(spectra), len(chans)), dtype=np.complex128)
    for a in range(n_in):
        rot = np.exp(1j * (2.0 * np.pi * chans * r[a] / M - phi[a]))
        for i, s in enumerate(spectra):
            y = np.zeros(M)
            for p in range(taps):
                f = s - taps + 1 + p
                if f < 0:
                    continue
                idx = f * M + m + d[a]
                ok = (idx >= 0) & (idx < S)
                xs = np.zeros(M)
                xs[ok] = x[a, idx[ok]]
                y += h[p * M:(p + 1) * M] * xs
            out[a, i] = (rows @ y) * rot
    return out


# --------------------------------------------------------------------------
# X-engine and integration
# --------------------------------------------------------------------------

def x_engine(V: np.ndarray, n_int: int, partial: bool = False) -> np.ndarray:
    """R[i][k][a][b] = (1/count) sum_{s in integration i} V_a,s[k] conj(V_b,s[k])."""
    n_in, n_spec, n_chan = V.shape
    n_full = n_spec // n_int
    starts = [i * n_int for i in range(n_full)]
    if partial and n_spec % n_int:
        starts.append(n_full * n_int)
    R = np.empty((len(starts), n_chan, n_in, n_in), dtype=np.complex128)
    for i, s0 in enumerate(starts):
        s1 = min(s0 + n_int, n_spec)
        blk = V[:, s0:s1, :]
        R[i] = np.einsum('ask,bsk->kab', blk, blk.conj()) / (s1 - s0)
    return R


# --------------------------------------------------------------------------
# MAD flagging (Eq. 2)
# --------------------------------------------------------------------------

def median_exact(v: np.ndarray) -> float:
    """Median by sorting; even count -> mean of the two middle order statistics."""
    s = np.sort(np.asarray(v, dtype=np.float64).ravel())
    n = s.size
    if n == 0:
        raise ValueError("median of empty set")
    if n % 2:
        return float(s[n // 2])
    return 0.5 * (float(s[n // 2 - 1]) + float(s[n // 2]))


def mad_threshold(A: np.ndarray, sigma: float = 5.0) -> float:
    """T = median(A) + sigma * MAD(A) * 1.4826 with MAD = median(|A - median(A)|)."""
    med = median_exact(A)
    mad = median_exact(np.abs(np.asarray(A, np.float64) - med))
    return med + sigma * mad * MAD_TO_SIGMA


def mad_flags(R: np.ndarray, sigma: float = 5.0, window: int = 64):
    """Flags[i][k][a][b] (uint8) and the thresholds T[i][k][a][b] for R[i][k][a][b]."""
    n_i, n_chan, n_in, _ = R.shape
    w = min(window, n_chan)
    if n_chan % w:
        raise ValueError("n_chan must be a multiple of the flag window")
    A = np.abs(R)
    T = np.empty(A.shape)
    for i in range(n_i):
        for a in range(n_in):
            for b in range(n_in):
                for k0 in range(0, n_chan, w):
                    T[i, k0:k0 + w, a, b] = mad_threshold(A[i, k0:k0 + w, a, b], sigma)
    flags = (A > T).astype(np.uint8)
    return flags, A, T


# --------------------------------------------------------------------------
# Whole hot path
# --------------------------------------------------------------------------

def correlate(x: np.ndarray, n_chan: int, taps: int, n_int: int, tau=None, phi=None,
              sigma: float = 5.0, window: int = 64, partial: bool = False,
              schedule: Optional[Sequence[tuple]] = None, pfb_window: str = "hann", beta: float = 8.0):
    """Visibilities R[i][k][a][b] and MAD flags for a whole stream (Algorithm 1).

    ``schedule`` optionally gives one ``(tau, phi)`` per integration (a delay
    change takes effect at an integration boundary); otherwise ``tau``/``phi``
    hold throughout.
    """
    if schedule is None:
        V = f_engine(x, n_chan, taps, tau, phi, pfb_window=pfb_window, beta=beta)
    else:
        M = 2 * n_chan
        n_spec = np.asarray(x).shape[1] // M
        V = None
        cache = {}
        for i, (t, p) in enumerate(schedule):
            s0, s1 = i * n_int, min((i + 1) * n_int, n_spec)
            if s0 >= n_spec:
                break
            key = (tuple(np.asarray(t, np.float64)), tuple(np.asarray(p, np.float64)))
            if key not in cache:
                cache[key] = f_engine(x, n_chan, taps, t, p, pfb_window=pfb_window, beta=beta)
            if V is None:
                V = np.empty_like(cache[key])
            V[:, s0:s1] = cache[key][:, s0:s1]
    R = x_engine(V, n_int, partial=partial)
    flags, A, T = mad_flags(R, sigma, window)
    return R, flags, T


# --------------------------------------------------------------------------
# Complex (I/Q) input
# --------------------------------------------------------------------------
# Sec. 4.2 says the raw samples are "converted into complex voltage streams";
# reading 3 takes real samples (the default).  The other reading, selectable
# per correlator:
#
# * each input is a stream of complex baseband samples x[n] = I[n] + j Q[n],
#   stored interleaved (I0, Q0, I1, Q1, ...) as int8 (or int16);
# * the PFB is the same real prototype over M = n_chan branches applied to the
#   complex samples (I and Q filtered alike; zero history, zero outside the
#   stream, coarse advance d in complex samples);
# * an M-point complex DFT (e^{-j...}, unscaled) keeps all M channels, in FFT
#   order: channel k sits at f_k = k / M cycles per sample for k < M/2 and
#   at (k - M) / M above (the negative frequencies);
# * the fine delay and instrument phase are exp(j (2 pi f_k r - phi)).

def iq_to_complex(x_iq: np.ndarray) -> np.ndarray:
    """[n_in][2S] interleaved (I, Q) samples -> complex128 [n_in][S]."""
    x_iq = np.asarray(x_iq, dtype=np.float64)
    return x_iq[..., 0::2] + 1j * x_iq[..., 1::2]


def channel_frequency_iq(M: int) -> np.ndarray:
    """f_k (cycles per sample) of the M channels of an M-point complex DFT."""
    k = np.arange(M)
    return np.where(k < M // 2, k, k - M) / M


def dft_brute_complex(y: np.ndarray) -> np.ndarray:
    """Y[k] = sum_m y[m] e^{-j 2 pi k m / M}, all k = 0 .. M-1, by direct summation."""
    M = y.shape[-1]
    k = np.arange(M)[:, None]
    m = np.arange(M)[None, :]
    W = np.exp(-2j * np.pi * ((k * m) % M) / M)
    return y @ W.T


def f_engine_iq(x_iq: np.ndarray, n_chan: int, taps: int, tau=None, phi=None,
                brute: bool = False) -> np.ndarray:
    """Channelised, delay-corrected voltages V[a][s][k] of complex input
    (k = 0 .. n_chan-1, M = n_chan)."""
    xc = iq_to_complex(x_iq)
    n_in = xc.shape[0]
    M = n_chan
    h = pfb_coefficients(M, taps)
    tau = np.zeros(n_in) if tau is None else np.asarray(tau, np.float64)
    phi = np.zeros(n_in) if phi is None else np.asarray(phi, np.float64)
    d, r = split_delay(tau)
    f = channel_frequency_iq(M)
    n_spec = xc.shape[1] // M
    V = np.empty((n_in, n_spec, M), dtype=np.complex128)
    for a in range(n_in):
        # the shift and the FIR are real and linear: apply them to I and Q
        y = (pfb_fir(coarse_shift(xc[a].real, int(d[a])), h, M, taps) +
             1j * pfb_fir(coarse_shift(xc[a].imag, int(d[a])), h, M, taps))
        Y = dft_brute_complex(y) if brute else np.fft.fft(y, axis=-1)
        V[a] = Y * np.exp(1j * (2.0 * np.pi * f * r[a] - phi[a]))
    return V


def correlate_iq(x_iq: np.ndarray, n_chan: int, taps: int, n_int: int, tau=None, phi=None,
                 sigma: float = 5.0, window: int = 64, partial: bool = False):
    """Visibilities and MAD flags of a complex-input stream (as :func:`correlate`)."""
    V = f_engine_iq(x_iq, n_chan, taps, tau, phi)
    R = x_engine(V, n_int, partial=partial)
    flags, A, T = mad_flags(R, sigma, window)
    return R, flags, T


def rel_frobenius_per_channel(R_test: np.ndarray, R_ref: np.ndarray) -> np.ndarray:
    """||R_test[.., k] - R_ref[.., k]||_F / ||R_ref[.., k]||_F per (integration, channel)."""
    num = np.sqrt(np.sum(np.abs(R_test - R_ref) ** 2, axis=(-2, -1)))
    den = np.sqrt(np.sum(np.abs(R_ref) ** 2, axis=(-2, -1)))
    return num / np.maximum(den, 1e-300)


def normalised_coefficients(R: np.ndarray) -> np.ndarray:
    """rho_ab = R_ab / sqrt(R_aa R_bb) per channel."""
    d = np.sqrt(np.abs(np.einsum('...aa->...a', R)))
    return R / np.maximum(d[..., :, None] * d[..., None, :], 1e-300)
