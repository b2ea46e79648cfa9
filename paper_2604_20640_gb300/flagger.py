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
