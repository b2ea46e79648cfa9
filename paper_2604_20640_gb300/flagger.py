"""Training and inference driver of the learned RFI flagger (all arithmetic in
libcorr.so; this module only sequences calls).

``train`` runs Adam steps on batches produced by a caller-supplied function
``batch(step) -> (power [B][64][256] CUDA float32, truth [B][64][256] CUDA
uint8)``; the power tiles are normalised on the GPU (ln(P / tile median))
before each step.
"""

from __future__ import annotations

from typing import Callable, List, Optional

from .corr import FlagNet


def train(net: FlagNet, batch: Callable[[int], tuple], steps: int, lr: float = 1e-3,
          lr_final: Optional[float] = None, stream=None) -> List[float]:
    """Adam training; the learning rate decays geometrically to ``lr_final``
    (default lr / 10) over ``steps``.  Returns the loss of every step."""
    import torch

    lr_final = lr / 10 if lr_final is None else lr_final
    losses = []
    x = None
    for i in range(steps):
        power, truth = batch(i)
        if x is None or x.shape != power.shape:
            x = torch.empty_like(power)
        net.prepare(power, x, stream=stream)
        r = lr * (lr_final / lr) ** (i / max(1, steps - 1))
        losses.append(net.train_step(x, truth, r, stream=stream))
    return losses


def flag(net: FlagNet, power, c_min: float = 0.9, sigma: float = 5.0, stream=None):
    """(flags uint8 [B][64][256], confidence [B]) of power tiles."""
    import torch

    flags = torch.empty(power.shape, dtype=torch.uint8, device=power.device)
    conf = torch.empty(power.shape[0], dtype=torch.float32, device=power.device)
    net.flag(power, flags, conf, c_min=c_min, sigma=sigma, stream=stream)
    return flags, conf


def noise_level(corr, noise, n_row: int):
    """Per-channel mean autocorrelation power [n_chan] of a noise-only
    stream ``noise`` (int8 [1][S] on the device, S >= 64 n_row M) through
    ``corr``'s F-engine (a one-input correlator)."""
    import torch

    M = 2 * corr.n_chan
    rows = (noise.shape[1] // M // n_row) // 64 * 64
    t = torch.empty((1, rows // 64, corr.n_chan // 256, 64, 256), device=noise.device)
    corr.spectrogram_dev(noise, n_row, t)
    # [1][rb][cb][64][256] -> mean over rows -> [cb * 256]
    return t.mean(dim=(0, 1, 3)).reshape(-1)


def power_tiles(corr, samples, n_row: int, out=None):
    """Dynamic-spectrum tiles [n_in * rows/64 * n_chan/256][64][256] of an
    int8 stream [n_in][S] on the device."""
    import torch

    M = 2 * corr.n_chan
    rows = (samples.shape[1] // M // n_row) // 64 * 64
    shape = (corr.n_in, rows // 64, corr.n_chan // 256, 64, 256)
    if out is None:
        out = torch.empty(shape, device=samples.device)
    corr.spectrogram_dev(samples, n_row, out.view(shape))
    return out.view(-1, 64, 256)


def truth_tiles(corr, nb, bb, g_nb, g_bb, level, n_row: int, thresh: float = 0.1):
    """Truth masks of RFI streams: a pixel is RFI when the power the RFI alone
    puts there, measured through the same F-engine, exceeds ``thresh`` times
    the channel's noise level.  ``nb``/``bb`` are the narrowband and
    broadband RFI quantised with per-input gains ``g_nb``/``g_bb``.
    Returns (truth, truth_nb, truth_bb) as uint8 tiles."""
    import torch

    dev = nb.device
    p_nb = power_tiles(corr, nb, n_row)
    p_bb = power_tiles(corr, bb, n_row)
    n_in = corr.n_in
    per_in = p_nb.shape[0] // n_in
    inv_nb = torch.as_tensor(1.0 / (g_nb ** 2), dtype=torch.float32, device=dev).repeat_interleave(per_in)
    inv_bb = torch.as_tensor(1.0 / (g_bb ** 2), dtype=torch.float32, device=dev).repeat_interleave(per_in)
    cb = corr.n_chan // 256
    lvl = level.view(cb, 1, 256).repeat(per_in // cb, 1, 1).repeat(n_in, 1, 1)       # [tiles][1][256]
    a = p_nb * inv_nb[:, None, None]
    b = p_bb * inv_bb[:, None, None]
    t_nb = a > thresh * lvl
    t_bb = b > thresh * lvl
    truth = (a + b) > thresh * lvl
    return truth.to(torch.uint8), t_nb.to(torch.uint8), t_bb.to(torch.uint8)
