"""Seeded int8 baseband streams shaped like a small L-band interferometer.

Recipe (all randomness from a Philox bit generator keyed by ``seed``):

* receiver noise: independent N(0, noise_frac * sigma^2) per input and sample;
* a common sky source of variance ``src_frac * sigma^2`` seen by every input,
  delayed by ``tau[a]`` samples and rotated by the instrument phase ``phi[a]``
  (positive frequencies multiplied by exp(+j phi), i.e. the instrument adds
  +phi that the correlator later removes).  Integer delays with zero phase are
  applied as exact sample shifts of one long source sequence; otherwise the
  source is synthesised per block of ``block`` samples in the frequency domain
  (a circular delay inside each block);
* narrowband tones ``(freq cycles/sample, amplitude, phase)`` common to all
  inputs;
* linear chirps ``(t0, t1, f0, f1, amplitude)`` common to all inputs;
* broadband bursts: each ``burst_frame``-sample frame carries, with
  probability ``burst_frac``, extra white noise of power ``burst_gain`` times
  the receiver noise, common to all inputs;
* everything summed, rounded half-to-even and clipped to [-128, 127]
  (``bits`` = 8, int8 output; the 8-bit truncated recorder mode), or to
  [-2^(bits-1), 2^(bits-1) - 1] stored as int16 for larger ``bits`` (14: the
  ADC width of the 16-bit padded recorder mode).

The module holds no part of the correlator (no filter bank, channeliser,
correlator or flagger).
"""

from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence, Tuple

import numpy as np


@dataclasses.dataclass
class StreamSpec:
    n_ant: int
    n_pol: int
    n_samples: int
    seed: int
    sigma: float = 16.0
    noise_frac: float = 1.0                    # receiver noise power / sigma^2
    src_frac: float = 0.05
    tau: Optional[Sequence[float]] = None      # per input, samples (truth)
    phi: Optional[Sequence[float]] = None      # per input, radians (truth)
    tones: Sequence[Tuple[float, float, float]] = ()
    chirps: Sequence[Tuple[int, int, float, float, float]] = ()
    burst_frac: float = 0.0
    burst_frame: int = 2048
    burst_gain: float = 10.0
    block: int = 1 << 16
    bits: int = 8

    @property
    def n_in(self) -> int:
        return self.n_ant * self.n_pol


def _rng(seed: int, stream: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(key=[int(seed) & ((1 << 64) - 1), int(stream)]))


def _source_exact(spec: StreamSpec, tau_int: np.ndarray, out: np.ndarray) -> None:
    """Add the common source as exact integer sample shifts of one sequence."""
    dmin, dmax = int(tau_int.min()), int(tau_int.max())
    rng = _rng(spec.seed, 1)
    amp = math.sqrt(spec.src_frac) * spec.sigma
    span = spec.n_samples + (dmax - dmin)
    s = rng.standard_normal(span) * amp
    for a in range(spec.n_in):
        # x_a[n] = s[n - tau_a]; s is indexed from n = dmin - dmax.
        off = dmax - int(tau_int[a])
        out[a] += s[off: off + spec.n_samples]


def _source_freq(spec: StreamSpec, tau: np.ndarray, phi: np.ndarray, out: np.ndarray) -> None:
    """Add the common source with fractional delays / phases, per block."""
    rng = _rng(spec.seed, 1)
    amp = math.sqrt(spec.src_frac) * spec.sigma
    B = min(spec.block, spec.n_samples)
    f = np.arange(B // 2 + 1) / B
    rot = np.exp(-2j * np.pi * f[None, :] * tau[:, None])
    ph = np.exp(1j * phi)[:, None] * np.ones((1, B // 2 + 1))
    ph[:, 0] = 1.0
    if B % 2 == 0:
        ph[:, -1] = 1.0
    filt = rot * ph
    for b0 in range(0, spec.n_samples, B):
        n = min(B, spec.n_samples - b0)
        s = rng.standard_normal(B) * amp
        Sf = np.fft.rfft(s)
        blk = np.fft.irfft(Sf[None, :] * filt, n=B, axis=1)
        out[:, b0:b0 + n] += blk[:, :n]


def make_stream(spec: StreamSpec, return_float: bool = False):
    """Return int8 samples ``[n_in][n_samples]`` (and the float sum if asked)."""
    n_in, S = spec.n_in, spec.n_samples
    x = _rng(spec.seed, 0).standard_normal((n_in, S))
    x *= spec.sigma * math.sqrt(spec.noise_frac)
    if spec.src_frac > 0:
        tau = np.zeros(n_in) if spec.tau is None else np.asarray(spec.tau, np.float64)
        phi = np.zeros(n_in) if spec.phi is None else np.asarray(spec.phi, np.float64)
        if np.all(tau == np.round(tau)) and np.all(phi == 0):
            _source_exact(spec, np.round(tau).astype(np.int64), x)
        else:
            _source_freq(spec, tau, phi, x)
    n = np.arange(S, dtype=np.float64)
    for (freq, amp, theta) in spec.tones:
        x += amp * np.cos(2 * np.pi * freq * n + theta)[None, :]
    for (t0, t1, f0, f1, amp) in spec.chirps:
        t0, t1 = max(0, int(t0)), min(S, int(t1))
        if t1 <= t0:
            continue
        t = np.arange(t1 - t0, dtype=np.float64)
        rate = (f1 - f0) / max(1, (t1 - t0))
        x[:, t0:t1] += amp * np.cos(2 * np.pi * (f0 * t + 0.5 * rate * t * t))[None, :]
    if spec.burst_frac > 0:
        rng = _rng(spec.seed, 2)
        n_fr = S // spec.burst_frame
        hit = np.nonzero(rng.random(n_fr) < spec.burst_frac)[0]
        g = math.sqrt(spec.burst_gain) * spec.sigma
        for fr in hit:
            a0 = fr * spec.burst_frame
            x[:, a0:a0 + spec.burst_frame] += rng.standard_normal(spec.burst_frame)[None, :] * g
    lim = 1 << (spec.bits - 1)
    q = np.clip(np.rint(x), -lim, lim - 1).astype(np.int8 if spec.bits <= 8 else np.int16)
    if return_float:
        return q, x
    return q


def make_stream_iq(spec: StreamSpec) -> np.ndarray:
    """Complex baseband counterpart of :func:`make_stream`: int8 ``[n_in][2 S]``
    with each input's (I, Q) pairs interleaved.  Circular complex receiver
    noise of power sigma^2 (sigma^2 / 2 per part), a common complex source at
    src_frac of it, delayed by tau_a (per block, by a phase ramp over signed
    frequencies) and rotated by phi_a, complex tones (freq in cycles per
    sample, may be negative; amplitude per part), rounded half to even and
    clipped to int8 per part."""
    n_in, S = spec.n_in, spec.n_samples
    rng = _rng(spec.seed, 11)
    sc = spec.sigma * math.sqrt(spec.noise_frac / 2.0)
    x = (rng.standard_normal((n_in, S)) + 1j * rng.standard_normal((n_in, S))) * sc
    if spec.src_frac > 0:
        tau = np.zeros(n_in) if spec.tau is None else np.asarray(spec.tau, np.float64)
        phi = np.zeros(n_in) if spec.phi is None else np.asarray(spec.phi, np.float64)
        amp = spec.sigma * math.sqrt(spec.src_frac / 2.0)
        B = min(spec.block, S)
        f = np.fft.fftfreq(B)
        filt = np.exp(-2j * np.pi * f[None, :] * tau[:, None]) * np.exp(1j * phi)[:, None]
        src = _rng(spec.seed, 12)
        for b0 in range(0, S, B):
            n = min(B, S - b0)
            s_blk = (src.standard_normal(B) + 1j * src.standard_normal(B)) * amp
            x[:, b0:b0 + n] += np.fft.ifft(np.fft.fft(s_blk)[None, :] * filt, axis=1)[:, :n]
    t = np.arange(S, dtype=np.float64)
    for (freq, amp, theta) in spec.tones:
        x += amp * np.exp(1j * (2 * np.pi * freq * t + theta))[None, :]
    lim = 1 << (spec.bits - 1)
    out = np.empty((n_in, 2 * S), dtype=np.int8)
    out[:, 0::2] = np.clip(np.rint(x.real), -lim, lim - 1)
    out[:, 1::2] = np.clip(np.rint(x.imag), -lim, lim - 1)
    return out


def delays_for(n_in: int, seed: int, max_delay: float = 40.0, integer: bool = False):
    """Per-input geometric delays in [0, max_delay] (input 0 at 0) and phases."""
    rng = _rng(seed, 7)
    tau = rng.uniform(0.0, max_delay, n_in)
    tau[0] = 0.0
    if integer:
        tau = np.round(tau)
    phi = rng.uniform(0.0, 2 * np.pi, n_in)
    return tau, phi


def tone_amplitude(sigma: float, M: int, db: float) -> float:
    """Tone amplitude whose power in one bin of a rectangular M-point DFT is
    ``db`` decibels above that of N(0, sigma^2) noise."""
    return 2.0 * sigma * math.sqrt(10 ** (db / 10.0) / M)


def config_c1(seed: int = 1000, n_samples: int = 1 << 22) -> StreamSpec:
    """4 antennas x 1 pol, noise sigma=16 + 5 % common source, 0-40 sample delays."""
    tau, phi = delays_for(4, seed)
    return StreamSpec(n_ant=4, n_pol=1, n_samples=n_samples, seed=seed, tau=tau, phi=phi)


def config_c2(seed: int = 2000, n_samples: int = 1 << 28, M: int = 8192) -> StreamSpec:
    """4 antennas x 2 pols, 3 tones at +20 dB and 1 % bursts at +10 dB."""
    tau, phi = delays_for(8, seed)
    # Tones in the lower quarter of the band (where satellite navigation sits
    # in a 1050-1550 MHz baseband), at bin centres of an M-point transform.
    chans = [int(M // 2 * 0.12) + 1, int(M // 2 * 0.18) + 3, int(M // 2 * 0.24) + 5]
    amp = tone_amplitude(16.0, M, 20.0)
    tones = [(c / M, amp, 0.3 * i) for i, c in enumerate(chans)]
    return StreamSpec(n_ant=4, n_pol=2, n_samples=n_samples, seed=seed, tau=tau, phi=phi,
                      tones=tones, burst_frac=0.01, burst_frame=M, burst_gain=10.0)


def config_c3(seed: int = 3000, n_samples: int = 1 << 26) -> StreamSpec:
    """32 antennas x 2 pols, C1 content."""
    tau, phi = delays_for(64, seed)
    return StreamSpec(n_ant=32, n_pol=2, n_samples=n_samples, seed=seed, tau=tau, phi=phi)


# Eight sub-array streams: (n_ant, n_chan, n_int); n_pol = 2 throughout.
C4_SHAPES: List[Tuple[int, int, int]] = [
    (4, 512, 4096), (6, 1024, 2048), (8, 2048, 1024), (12, 4096, 512),
    (16, 8192, 256), (24, 512, 1024), (32, 1024, 512), (32, 2048, 256),
]


def config_c4_streams(seed: int = 4000, n_samples: int = 1 << 24) -> List[StreamSpec]:
    out = []
    for i, (na, nc, ni) in enumerate(C4_SHAPES):
        tau, phi = delays_for(2 * na, seed + i)
        out.append(StreamSpec(n_ant=na, n_pol=2, n_samples=n_samples, seed=seed + i,
                              tau=tau, phi=phi))
    return out
