"""Train and score the learned RFI flagger on dynamic spectra from this
F-engine (the flagging workload: 32 inputs, 4096 channels, rows of 256
spectra, 64 x 256 tiles), with synthetic RFI streams from ``fxsynth``.

    python -m paper_2604_20640_gb300.train_flagnet --steps 2000 --out weights.npy

Batches of streams are drawn on the GPU, channelised by the F-engine into
power tiles, and labelled through the same F-engine: a pixel is RFI when the
RFI alone puts more than 0.1 x the channel's noise level there.
"""

from __future__ import annotations

import argparse
import time

import numpy as np

from . import flagger
from .corr import Correlator, FlagNet

N_ROW = 256
TRUTH_FRACTION = 0.1


class TileSource:
    """Power tiles and truth masks of seeded RFI streams (``fxsynth.rfi_torch``)."""

    def __init__(self, n_in: int = 8, n_chan: int = 4096, n_row: int = N_ROW, seed: int = 5000, device="cuda"):
        from fxsynth.rfi_torch import RfiSpec, noise_only
        self.spec = RfiSpec(n_in=n_in, n_chan=n_chan, n_row=n_row, seed=seed)
        self.device = device
        self.corr = Correlator(n_in, 1, n_chan, 4, 256)
        one = Correlator(1, 1, n_chan, 4, 256)
        self.level = flagger.noise_level(one, noise_only(self.spec, self.spec.n_samples, device), n_row)
        one.close()

    def batch(self, index: int, with_parts: bool = False):
        """(power [B][64][256], truth uint8 [B][64][256][, truth_nb, truth_bb, streams])."""
        from fxsynth.rfi_torch import make_rfi_batch
        b = make_rfi_batch(self.spec, index, self.device)
        power = flagger.power_tiles(self.corr, b["total"], self.spec.n_row)
        truth, t_nb, t_bb = flagger.truth_tiles(self.corr, b["nb"], b["bb"], b["g_nb"], b["g_bb"], self.level,
                                                self.spec.n_row, TRUTH_FRACTION)
        if with_parts:
            return power, truth, t_nb, t_bb, b
        return power, truth


def train(net: FlagNet, src: TileSource, steps: int, tiles_per_step: int = 32, lr: float = 1e-3,
          first_batch: int = 0, log=None):
    """Adam over F-engine tiles; each drawn batch is shuffled and used once."""
    import torch
    pool_p, pool_t = None, None
    pos = 0
    nb = first_batch
    gen = torch.Generator(device="cpu")
    gen.manual_seed(src.spec.seed)

    def next_batch(i):
        nonlocal pool_p, pool_t, pos, nb
        if pool_p is None or pos + tiles_per_step > pool_p.shape[0]:
            p, t = src.batch(nb)
            nb += 1
            perm = torch.randperm(p.shape[0], generator=gen).to(p.device)
            pool_p, pool_t, pos = p[perm], t[perm], 0
        out = pool_p[pos:pos + tiles_per_step], pool_t[pos:pos + tiles_per_step]
        pos += tiles_per_step
        if log and i % 100 == 0:
            log(i)
        return out

    return flagger.train(net, next_batch, steps, lr=lr)


def _pr(pred, truth):
    tp = int((pred & truth).sum())
    fp = int((pred & ~truth).sum())
    fn = int((~pred & truth).sum())
    return tp / max(1, tp + fp), tp / max(1, tp + fn)


def evaluate(net: FlagNet, power, truth, t_nb, t_bb, c_min: float = 0.9):
    """dict of precision / recall (overall, narrowband-only and broadband-only
    truth) for the net alone, MAD alone (along channels as in the paper,
    along time, and their union) and the hybrid at ``c_min``."""
    import torch
    from .corr import tile_mad
    out = {}
    t = truth.bool()
    for name, cm in (("net", -1.0), ("mad", 2.0), ("mad_time", None), ("mad_union", None), ("hybrid", c_min)):
        if cm is None:
            f = torch.empty(power.shape, dtype=torch.uint8, device=power.device)
            tile_mad(power, f, axes=2 if name == "mad_time" else 3)
            conf = None
        else:
            f, conf = flagger.flag(net, power, c_min=cm)
        f = f.bool()
        p, r = _pr(f, t)
        _, r_nb = _pr(f, t_nb.bool())
        _, r_bb = _pr(f, t_bb.bool())
        out[name] = {"precision": round(p, 4), "recall": round(r, 4), "recall_narrowband": round(r_nb, 4),
                     "recall_broadband": round(r_bb, 4)}
        if name == "hybrid":
            out[name]["tiles_on_mad"] = int((conf < cm).sum())
    out["truth_fraction"] = float(t.float().mean())
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--tiles", type=int, default=32)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--seed", type=int, default=5000)
    ap.add_argument("--init", type=int, default=0, help="seed of the He-normal initialisation")
    ap.add_argument("--eval-inputs", type=int, default=8,
                    help="inputs of the held-out evaluation batch (32: the flagging workload's 512 tiles)")
    ap.add_argument("--out", required=True)
    args = ap.parse_args()
    import torch
    torch.cuda.init()
    src = TileSource(seed=args.seed)
    net = FlagNet(init_params(args.init))
    t0 = time.time()
    losses = train(net, src, args.steps, args.tiles, args.lr,
                   log=lambda i: print("step %d  %.1f s" % (i, time.time() - t0), flush=True))
    np.save(args.out, net.get_params())
    t_train = time.time() - t0
    ev = src if args.eval_inputs == 8 else TileSource(n_in=args.eval_inputs, seed=args.seed + 1)
    p, t, tn, tb, _ = ev.batch(10 ** 6, with_parts=True)
    print({"loss_first": float(np.mean(losses[:10])), "loss_last": float(np.mean(losses[-50:])),
           "steps": args.steps, "tiles_drawn": args.steps * args.tiles, "eval_tiles": int(p.shape[0]),
           "train_seconds": round(t_train, 1), "eval": evaluate(net, p, t, tn, tb)})


def init_params(seed: int = 0) -> np.ndarray:
    """He-normal weights, zero biases, flattened layer by layer (w[o][c][u][v], b[o])."""
    rng = np.random.default_rng(seed)
    out = []
    for ci, co in ((1, 32), (32, 32), (32, 32), (32, 1)):
        out.append(rng.standard_normal(co * ci * 25) * np.sqrt(2.0 / (ci * 25)))
        out.append(np.zeros(co))
    return np.concatenate(out).astype(np.float32)


if __name__ == "__main__":
    main()
