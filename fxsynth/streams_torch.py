"""Bulk version of :mod:`fxsynth.streams` drawn with torch's RNG on a device.

Same recipe as :func:`fxsynth.streams.make_stream` (receiver noise, a common
source delayed by ``tau`` and rotated by ``phi`` per input in the frequency
domain per block, tones, chirps, broadband bursts, round-half-even and clip
to int8), but generated block by block on ``device`` so multi-GiB streams
take well under a second.  The random numbers differ from the numpy
generator's; parity checks copy the slice they need back to the host.
"""

from __future__ import annotations

import math

import torch

from .streams import StreamSpec


def make_stream_torch(spec: StreamSpec, device="cuda", block: int = 1 << 22) -> torch.Tensor:
    n_in, S = spec.n_in, spec.n_samples
    g = torch.Generator(device=device)
    g.manual_seed(int(spec.seed) & ((1 << 63) - 1))
    lim = 1 << (spec.bits - 1)
    out = torch.empty((n_in, S), dtype=torch.int8 if spec.bits <= 8 else torch.int16, device=device)
    B = min(block, S)
    if spec.burst_frac > 0:
        B = max(spec.burst_frame, (B // spec.burst_frame) * spec.burst_frame)
    tau = torch.zeros(n_in, dtype=torch.float64) if spec.tau is None else torch.tensor(spec.tau, dtype=torch.float64)
    phi = torch.zeros(n_in, dtype=torch.float64) if spec.phi is None else torch.tensor(spec.phi, dtype=torch.float64)
    f = torch.arange(B // 2 + 1, dtype=torch.float64) / B
    filt = torch.exp(-2j * math.pi * f[None, :] * tau[:, None])
    ph = torch.exp(1j * phi)[:, None].expand(n_in, B // 2 + 1).clone()
    ph[:, 0] = 1.0
    if B % 2 == 0:
        ph[:, -1] = 1.0
    filt = (filt * ph).to(torch.complex64).to(device)
    amp_src = math.sqrt(spec.src_frac) * spec.sigma
    amp_noise = spec.sigma * math.sqrt(spec.noise_frac)
    for b0 in range(0, S, B):
        n = min(B, S - b0)
        x = torch.randn((n_in, B), generator=g, device=device, dtype=torch.float32) * amp_noise
        if spec.src_frac > 0:
            s = torch.randn(B, generator=g, device=device, dtype=torch.float32) * amp_src
            x += torch.fft.irfft(torch.fft.rfft(s)[None, :] * filt, n=B, dim=1)
        if spec.tones or spec.chirps:
            t = torch.arange(b0, b0 + B, device=device, dtype=torch.float64)
            for (freq, amp, theta) in spec.tones:
                cyc = torch.remainder(freq * t, 1.0)
                x += (amp * torch.cos(2 * math.pi * cyc + theta)).to(torch.float32)[None, :]
            for (t0, t1, f0, f1, amp) in spec.chirps:
                lo, hi = max(t0, b0), min(t1, b0 + B)
                if hi <= lo:
                    continue
                tt = torch.arange(lo - t0, hi - t0, device=device, dtype=torch.float64)
                rate = (f1 - f0) / max(1, (t1 - t0))
                cyc = torch.remainder(f0 * tt + 0.5 * rate * tt * tt, 1.0)
                x[:, lo - b0:hi - b0] += (amp * torch.cos(2 * math.pi * cyc)).to(torch.float32)[None, :]
        if spec.burst_frac > 0:
            nf = B // spec.burst_frame
            hit = torch.rand(nf, generator=g, device=device) < spec.burst_frac
            burst = torch.randn((nf, spec.burst_frame), generator=g, device=device) * (
                math.sqrt(spec.burst_gain) * spec.sigma)
            x += (burst * hit[:, None]).reshape(1, B)
        out[:, b0:b0 + n] = torch.clamp(torch.round(x[:, :n]), -lim, lim - 1).to(out.dtype)
    return out
