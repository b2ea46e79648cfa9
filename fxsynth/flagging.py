"""Seeded (time x channel) power tiles with injected RFI and their truth masks,
for training and scoring the learned flagger.

Recipe (layout decisions from a numpy Philox generator keyed by ``seed``;
noise from a torch generator seeded from it):

* a tile is ``rows`` x ``chans`` pixels (64 x 256); each pixel is the mean
  of ``n_row`` powers |n + s|^2 of one channel, n complex Gaussian receiver
  noise of power b[k] g[r] and s the RFI voltage -- the statistics of the
  autocorrelation power of a channelised voltage stream averaged over
  ``n_row`` spectra;
* bandpass b[k] = c (1 + sum of three random cosines of at most 3 cycles per
  tile, amplitudes <= 0.15), overall level c = 10^U(-1, 1); slow row gain
  g[r] = 1 + 0.05 sin(2 pi r / 64 + theta);
* RFI events, each with interference-to-noise ratio INR (per spectrum,
  relative to the local noise power), drawn per tile:
  - narrowband tones: 1-3 channels wide, on for all rows or a segment of
    4-64 rows, INR 10^(U(-8, 15) / 10), constant amplitude, random phase per
    spectrum;
  - chirps: a line k(r) = k0 + slope (r - r0), |slope| 0.25-4 channels per
    row, 1-2 channels wide, 16-64 rows long, INR 10^(U(-8, 12) / 10);
  - broadband bursts: 1-4 rows over the whole tile or a sub-band of >= 64
    channels, noise-like, INR 10^(U(-8, 6) / 10);
* truth = 1 on every pixel that received RFI power.

The module holds no part of the flagger (no normalisation, network or
threshold rule).
"""

from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass
class TileSpec:
    rows: int = 64
    chans: int = 256
    n_row: int = 16
    max_tones: int = 3
    max_chirps: int = 2
    max_bursts: int = 2
    p_clean: float = 0.15          # probability that a tile has no RFI at all


def _events(rng: np.random.Generator, spec: TileSpec):
    """List of (kind, pixel mask [rows][chans] bool, INR) for one tile."""
    R, C = spec.rows, spec.chans
    out = []
    if rng.random() < spec.p_clean:
        return out
    rr = np.arange(R)[:, None]
    cc = np.arange(C)[None, :]
    for _ in range(rng.integers(0, spec.max_tones + 1)):
        w = int(rng.integers(1, 4))
        k0 = int(rng.integers(0, C - w + 1))
        if rng.random() < 0.5:
            r0, r1 = 0, R
        else:
            ln = int(rng.integers(4, 65))
            r0 = int(rng.integers(0, R - min(ln, R) + 1))
            r1 = min(R, r0 + ln)
        m = (rr >= r0) & (rr < r1) & (cc >= k0) & (cc < k0 + w)
        out.append(("tone", m, 10 ** (rng.uniform(-8, 15) / 10)))
    for _ in range(rng.integers(0, spec.max_chirps + 1)):
        ln = int(rng.integers(16, 65))
        r0 = int(rng.integers(0, R - min(ln, R) + 1))
        r1 = min(R, r0 + ln)
        slope = rng.uniform(0.25, 4.0) * (1 if rng.random() < 0.5 else -1)
        k0 = rng.uniform(0, C)
        w = int(rng.integers(1, 3))
        kc = np.floor(k0 + slope * (np.arange(R) - r0))[:, None]
        m = (rr >= r0) & (rr < r1) & (cc >= kc) & (cc < kc + w)
        # a steep chirp crosses several channels within one row
        if abs(slope) > 1:
            k_lo = np.floor(k0 + slope * (np.arange(R) - r0 - 0.5))[:, None]
            k_hi = np.floor(k0 + slope * (np.arange(R) - r0 + 0.5))[:, None]
            lo, hi = np.minimum(k_lo, k_hi), np.maximum(k_lo, k_hi)
            m = (rr >= r0) & (rr < r1) & (cc >= lo) & (cc <= hi + w - 1)
        out.append(("chirp", m, 10 ** (rng.uniform(-8, 12) / 10)))
    for _ in range(rng.integers(0, spec.max_bursts + 1)):
        ln = int(rng.integers(1, 5))
        r0 = int(rng.integers(0, R - ln + 1))
        if rng.random() < 0.5:
            k0, k1 = 0, C
        else:
            bw = int(rng.integers(64, C + 1))
            k0 = int(rng.integers(0, C - bw + 1))
            k1 = k0 + bw
        m = (rr >= r0) & (rr < r0 + ln) & (cc >= k0) & (cc < k1)
        out.append(("burst", m, 10 ** (rng.uniform(-8, 6) / 10)))
    return out


def make_tiles(n_tiles: int, seed: int, device="cpu", spec: TileSpec = TileSpec(), return_kinds: bool = False):
    """(power [n][rows][chans] float32, truth [n][rows][chans] uint8) as torch
    tensors on ``device``; with ``return_kinds`` also a uint8 map of the RFI
    kind per pixel (0 none, 1 tone, 2 chirp, 3 burst; later events win)."""
    import torch

    rng = np.random.Generator(np.random.Philox(key=[int(seed) & ((1 << 64) - 1), 0x7F1A6]))
    R, C, L = spec.rows, spec.chans, spec.n_row
    noise_pow = np.empty((n_tiles, R, C))
    tone_pow = np.zeros((n_tiles, R, C))          # coherent (constant-amplitude) RFI power
    burst_pow = np.zeros((n_tiles, R, C))         # noise-like RFI power
    truth = np.zeros((n_tiles, R, C), np.uint8)
    kinds = np.zeros((n_tiles, R, C), np.uint8)
    kcode = {"tone": 1, "chirp": 2, "burst": 3}
    k = np.arange(C)
    for t in range(n_tiles):
        c = 10 ** rng.uniform(-1, 1)
        b = np.ones(C)
        for _ in range(3):
            b += rng.uniform(0, 0.15) * np.cos(2 * np.pi * rng.uniform(0, 3) * k / C + rng.uniform(0, 2 * np.pi))
        g = 1 + 0.05 * np.sin(2 * np.pi * np.arange(R) / 64 + rng.uniform(0, 2 * np.pi))
        noise_pow[t] = c * g[:, None] * b[None, :]
        for kind, m, inr in _events(rng, spec):
            tgt = burst_pow if kind == "burst" else tone_pow
            tgt[t][m] += inr * noise_pow[t][m]
            truth[t][m] = 1
            kinds[t][m] = kcode[kind]
    gen = torch.Generator(device=device)
    gen.manual_seed(int(rng.integers(0, 2 ** 62)))
    shape = (n_tiles, R, C, L)
    var = torch.as_tensor(noise_pow + burst_pow, dtype=torch.float32, device=device)[..., None]
    amp = torch.as_tensor(np.sqrt(tone_pow), dtype=torch.float32, device=device)[..., None]
    re = torch.randn(shape, generator=gen, device=device) * torch.sqrt(var / 2)
    im = torch.randn(shape, generator=gen, device=device) * torch.sqrt(var / 2)
    ph = torch.rand(shape, generator=gen, device=device) * (2 * math.pi)
    re = re + amp * torch.cos(ph)
    im = im + amp * torch.sin(ph)
    power = (re * re + im * im).mean(dim=-1).contiguous()
    tr = torch.as_tensor(truth, device=device)
    if return_kinds:
        return power, tr, torch.as_tensor(kinds, device=device)
    return power, tr
