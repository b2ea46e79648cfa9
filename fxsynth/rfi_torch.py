"""Seeded int8 voltage streams with injected RFI, drawn on a device, for the
learned-flagger workload (32 inputs, 4096 channels, dynamic-spectrum rows of
``n_row`` spectra, 64-row tiles).

Recipe, per input and per batch of ``row_blocks`` x 64 rows (random layout
from a numpy Philox generator keyed by ``(seed, batch)``; noise from a torch
generator seeded from it):

* receiver noise N(0, sigma^2), sigma = 16;
* narrowband RFI, interference-to-noise ratio INR given in dB of power in one
  bin of a rectangular M-point DFT relative to the noise (the convention of
  ``tone_amplitude``), drawn from ``nb_db``:
  - tones at a random frequency inside a random channel, on for the whole
    batch or for a segment of 4-64 rows, random phase;
  - linear chirps of 16-64 rows drifting 0.25-4 channels per row;
* broadband bursts of 1-4 rows, over the whole band or a sub-band of >= 1/16
  of it: Gaussian noise band-limited in the frequency domain, per-channel
  INR drawn from ``bb_db`` (0-30 dB; above about 18 dB the sum saturates the
  int8 samples, as an 8-bit recorder does);
* the sum rounded half-to-even and clipped to int8 (``total``);
* the narrowband and the broadband RFI alone, each scaled by a per-input gain
  (``g_nb``, ``g_bb``) that brings its peak to about 120 and quantised the
  same way, so that the same F-engine can measure the RFI power each pixel
  received (``nb``, ``bb``);
* ``noise_only(...)``: a stream of the receiver noise alone, for the
  per-channel noise level.

The module holds no part of the correlator or the flagger.
"""

from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass
class RfiSpec:
    n_in: int = 32
    n_chan: int = 4096
    n_row: int = 256
    row_blocks: int = 1
    seed: int = 5000
    sigma: float = 16.0
    nb_db: tuple = (0.0, 30.0)
    bb_db: tuple = (0.0, 30.0)
    tones_per_tile: float = 1.5        # mean number per 64 x 256 tile
    chirps_per_tile: float = 0.6
    bursts_per_block: float = 1.2      # mean number per input and 64-row block

    @property
    def M(self) -> int:
        return 2 * self.n_chan

    @property
    def rows(self) -> int:
        return 64 * self.row_blocks

    @property
    def n_samples(self) -> int:
        return self.rows * self.n_row * self.M


def _amp(sigma: float, M: int, db: float) -> float:
    return 2.0 * sigma * math.sqrt(10 ** (db / 10.0) / M)


def _quantise(x, gain):
    import torch
    return torch.clamp(torch.round(x * gain), -128, 127).to(torch.int8)


def make_rfi_batch(spec: RfiSpec, batch: int, device="cuda"):
    """dict(total, nb, bb: int8 [n_in][n_samples]; g_nb, g_bb: float [n_in])."""
    import torch

    rng = np.random.Generator(np.random.Philox(key=[int(spec.seed) & ((1 << 63) - 1), 0x5C5 + int(batch)]))
    gen = torch.Generator(device=device)
    gen.manual_seed(int(rng.integers(0, 2 ** 62)))
    M, S, R, L = spec.M, spec.n_samples, spec.rows, spec.n_row
    n_tiles_per_input = spec.row_blocks * (spec.n_chan // 256)
    spr = L * M                                            # samples per row
    out = {k: torch.empty((spec.n_in, S), dtype=torch.int8, device=device) for k in ("total", "nb", "bb")}
    g_nb = np.ones(spec.n_in)
    g_bb = np.ones(spec.n_in)
    for a in range(spec.n_in):
        nb = torch.zeros(S, dtype=torch.float32, device=device)
        bb = torch.zeros(S, dtype=torch.float32, device=device)
        for _ in range(rng.poisson(spec.tones_per_tile * n_tiles_per_input)):
            f = (rng.integers(0, spec.n_chan) + rng.uniform(0.05, 0.95)) / M
            if rng.random() < 0.5:
                r0, r1 = 0, R
            else:
                ln = int(rng.integers(4, 65))
                r0 = int(rng.integers(0, max(1, R - ln + 1)))
                r1 = min(R, r0 + ln)
            # phase in cycles per block of 2^16 samples t = t_b + tau: the
            # block's start frac(f t_b) in FP64, plus frac(f tau) from one
            # shared table, summed in FP32 (below 2 cycles: 2^-23 resolution)
            amp = _amp(spec.sigma, M, rng.uniform(*spec.nb_db))
            ph0 = rng.uniform(0, 2 * math.pi)
            n = (r1 - r0) * spr
            blk = 1 << 16
            tb = torch.arange(r0 * spr, r1 * spr, blk, device=device, dtype=torch.float64)
            base = torch.remainder(f * tb, 1.0).to(torch.float32)
            loc = torch.remainder(f * torch.arange(blk, device=device, dtype=torch.float64), 1.0).to(torch.float32)
            cyc = base[:, None] + loc[None, :]
            cyc.mul_(2 * math.pi).add_(ph0).cos_().mul_(amp)
            nb[r0 * spr:r1 * spr] += cyc.reshape(-1)[:n]
            del cyc
        for _ in range(rng.poisson(spec.chirps_per_tile * n_tiles_per_input)):
            ln = int(rng.integers(16, 65))
            r0 = int(rng.integers(0, max(1, R - ln + 1)))
            r1 = min(R, r0 + ln)
            slope = rng.uniform(0.25, 4.0) * (1 if rng.random() < 0.5 else -1)    # channels per row
            f0 = (rng.uniform(0, spec.n_chan)) / M
            rate = slope / M / spr                                                # cycles / sample^2
            # per block of 2^16 samples: start phase and local frequency in
            # FP64, then the linear term in 32-bit fixed point and the small
            # quadratic term (under one cycle per block) in FP32
            n = (r1 - r0) * spr
            blk = 1 << 16
            t0 = torch.arange(0, n, blk, device=device, dtype=torch.float64)
            ph0 = torch.remainder(f0 * t0 + 0.5 * rate * t0 * t0, 1.0)
            fq = (torch.round(torch.remainder(f0 + rate * t0, 1.0) * 2.0 ** 32).to(torch.int64)) & 0xFFFFFFFF
            tau = torch.arange(blk, device=device, dtype=torch.int64)
            lin = ((fq[:, None] * tau[None, :]) & 0xFFFFFFFF).to(torch.float32) * (1.0 / 2.0 ** 32)
            quad = (0.5 * rate) * tau.to(torch.float32) ** 2
            cyc = ph0.to(torch.float32)[:, None] + lin + quad[None, :]
            nb[r0 * spr:r1 * spr] += _amp(spec.sigma, M, rng.uniform(*spec.nb_db)) * torch.cos(
                (2 * math.pi) * torch.remainder(cyc, 1.0)).reshape(-1)[:n]
        for _ in range(rng.poisson(spec.bursts_per_block * spec.row_blocks)):
            ln = int(rng.integers(1, 5))
            r0 = int(rng.integers(0, R - ln + 1))
            n = ln * spr
            w = torch.randn(n, generator=gen, device=device, dtype=torch.float32)
            w *= spec.sigma * math.sqrt(10 ** (rng.uniform(*spec.bb_db) / 10.0))
            if rng.random() >= 0.5:
                bw = int(rng.integers(spec.n_chan // 16, spec.n_chan + 1))
                k0 = int(rng.integers(0, spec.n_chan - bw + 1))
                W = torch.fft.rfft(w)
                i0, i1 = k0 * n // M, (k0 + bw) * n // M
                W[:i0] = 0
                W[i1:] = 0
                w = torch.fft.irfft(W, n=n)
            bb[r0 * spr:r0 * spr + n] += w
        noise = torch.randn(S, generator=gen, device=device, dtype=torch.float32) * spec.sigma
        out["total"][a] = _quantise(noise + nb + bb, 1.0)
        del noise
        m_nb = float(nb.abs().max())
        m_bb = float(bb.abs().max())
        g_nb[a] = 120.0 / m_nb if m_nb > 0 else 1.0
        g_bb[a] = 120.0 / m_bb if m_bb > 0 else 1.0
        out["nb"][a] = _quantise(nb, g_nb[a])
        out["bb"][a] = _quantise(bb, g_bb[a])
    out["g_nb"] = g_nb
    out["g_bb"] = g_bb
    return out


def noise_only(spec: RfiSpec, n_samples: int, device="cuda", seed: int = 99):
    """int8 [1][n_samples] of the receiver noise alone."""
    import torch
    gen = torch.Generator(device=device)
    gen.manual_seed(int(spec.seed) * 7919 + seed)
    x = torch.randn((1, n_samples), generator=gen, device=device, dtype=torch.float32) * spec.sigma
    return _quantise(x, 1.0)
