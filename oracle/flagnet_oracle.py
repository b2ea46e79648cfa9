"""FP64 oracle of the learned RFI flagger -- TEST INFRASTRUCTURE ONLY.

The paper flags RFI with the MAD rule of Eq. 2 (Sec. 7) and shows the
dynamic spectra the flagger works on (Sec. 5).  The learned flagger is the
build's own addition: a small convolutional network that marks RFI pixels in
(time x channel) tiles of autocorrelation power, with MAD as the fallback on
tiles where the network is not confident.

Network (readings, also listed in the design notes):
  4 layers of 5x5 cross-correlation with zero padding 2 ("same" size),
  channels 1 -> 32 -> 32 -> 32 -> 1, ReLU after layers 1-3, a logistic
  output per pixel; loss = mean binary cross-entropy against the truth mask,
  computed from the logits.  Input pixel = ln(P / median(P over the tile)).
  Tile confidence = mean over pixels of |2p - 1|; below c_min the tile's
  flags come from the MAD rule applied along each row over aligned windows
  of 64 channels (Eq. 2 with sigma = 5).
"""

from __future__ import annotations

import numpy as np

from . import fx_oracle as fx

LAYERS = [(1, 32), (32, 32), (32, 32), (32, 1)]
KS = 5
PAD = 2


def init_params(seed: int = 0):
    """He-normal weights, zero biases: list of (w [Co][Ci][5][5], b [Co])."""
    rng = np.random.default_rng(seed)
    out = []
    for ci, co in LAYERS:
        std = np.sqrt(2.0 / (ci * KS * KS))
        out.append((rng.standard_normal((co, ci, KS, KS)) * std, np.zeros(co)))
    return out


def conv2d(x: np.ndarray, w: np.ndarray, b: np.ndarray) -> np.ndarray:
    """y[n,o,i,j] = b[o] + sum_{c,u,v} w[o,c,u,v] x[n,c,i+u-2,j+v-2] (zero outside)."""
    n, ci, H, W = x.shape
    co = w.shape[0]
    xp = np.zeros((n, ci, H + 2 * PAD, W + 2 * PAD))
    xp[:, :, PAD:PAD + H, PAD:PAD + W] = x
    y = np.broadcast_to(b[None, :, None, None], (n, co, H, W)).copy()
    for u in range(KS):
        for v in range(KS):
            y += np.einsum('oc,nchw->nohw', w[:, :, u, v], xp[:, :, u:u + H, v:v + W])
    return y


def conv2d_backward(x: np.ndarray, w: np.ndarray, dy: np.ndarray):
    """Gradients (dx, dw, db) of sum(dy * conv2d(x, w, b))."""
    n, ci, H, W = x.shape
    xp = np.zeros((n, ci, H + 2 * PAD, W + 2 * PAD))
    xp[:, :, PAD:PAD + H, PAD:PAD + W] = x
    dxp = np.zeros_like(xp)
    dw = np.zeros_like(w)
    for u in range(KS):
        for v in range(KS):
            dw[:, :, u, v] = np.einsum('nohw,nchw->oc', dy, xp[:, :, u:u + H, v:v + W])
            dxp[:, :, u:u + H, v:v + W] += np.einsum('oc,nohw->nchw', w[:, :, u, v], dy)
    return dxp[:, :, PAD:PAD + H, PAD:PAD + W], dw, dy.sum(axis=(0, 2, 3))


def forward(params, x: np.ndarray):
    """Logits z and the cached activations of the net for input x [n,1,H,W]."""
    acts = [x]
    h = x
    for li, (w, b) in enumerate(params):
        z = conv2d(h, w, b)
        h = np.maximum(z, 0.0) if li < len(params) - 1 else z
        acts.append(h)
    return h, acts


def sigmoid(z):
    return 0.5 * (1.0 + np.tanh(0.5 * z))


def bce_from_logits(z: np.ndarray, t: np.ndarray) -> float:
    """mean(softplus(z) - t z) = mean(-t ln p - (1 - t) ln(1 - p)), p = sigmoid(z)."""
    return float(np.mean(np.logaddexp(0.0, z) - t * z))


def loss_and_grads(params, x: np.ndarray, t: np.ndarray):
    z, acts = forward(params, x)
    L = bce_from_logits(z, t)
    dz = (sigmoid(z) - t) / z.size
    grads = [None] * len(params)
    g = dz
    for li in range(len(params) - 1, -1, -1):
        w, b = params[li]
        dx, dw, db = conv2d_backward(acts[li], w, g)
        grads[li] = (dw, db)
        if li > 0:
            g = dx * (acts[li] > 0)          # ReLU of the previous layer
    return L, grads


def flatten_params(params) -> np.ndarray:
    """One vector, layer by layer: w[o][c][u][v] then b[o]."""
    return np.concatenate([np.concatenate([w.ravel(), b.ravel()]) for w, b in params])


def unflatten_params(vec: np.ndarray):
    out, off = [], 0
    for ci, co in LAYERS:
        nw = co * ci * KS * KS
        out.append((np.asarray(vec[off:off + nw], np.float64).reshape(co, ci, KS, KS),
                    np.asarray(vec[off + nw:off + nw + co], np.float64)))
        off += nw + co
    return out


def dynamic_spectrum(x: np.ndarray, n_chan: int, taps: int, n_row: int, tau=None) -> np.ndarray:
    """Autocorrelation power P[a][r][k] = mean over spectra s in
    [r n_row, (r + 1) n_row) of |V_a,s[k]|^2, r < floor(n_spec / n_row): the
    (time x channel) dynamic spectra of Sec. 5, from the F-engine of
    Sec. 4.2 (coarse and fine delay as in Eq. 1; the phase factor has unit
    modulus and drops out)."""
    V = fx.f_engine(x, n_chan, taps, tau, None)
    n_in, n_spec, _ = V.shape
    rows = n_spec // n_row
    p = np.abs(V[:, :rows * n_row, :]) ** 2
    return p.reshape(n_in, rows, n_row, n_chan).mean(axis=2)


def to_tiles(P: np.ndarray, th: int = 64, tw: int = 256) -> np.ndarray:
    """[n_in][rows][n_chan] -> [n_in][rows / th][n_chan / tw][th][tw]."""
    n_in, rows, n_chan = P.shape
    return P.reshape(n_in, rows // th, th, n_chan // tw, tw).transpose(0, 1, 3, 2, 4)


def tile_input(power: np.ndarray) -> np.ndarray:
    """ln(P / median(P)) per tile; power [..., H, W] > 0."""
    med = np.median(power.reshape(*power.shape[:-2], -1), axis=-1)[..., None, None]
    return np.log(power / med)


def confidence(p: np.ndarray) -> np.ndarray:
    """Mean over a tile's pixels of |2p - 1|."""
    return np.mean(np.abs(2.0 * p - 1.0), axis=(-2, -1))


def mad_tile_flags(power: np.ndarray, sigma: float = 5.0, window: int = 64, axes: int = 1) -> np.ndarray:
    """Eq. 2 on (time x channel) tiles.  axes & 1: along each row over
    aligned windows of ``window`` channels; axes & 2: along each channel over
    the tile's rows (the time direction); both: the union of the two."""
    H, W = power.shape[-2:]
    out = np.zeros(power.shape, np.uint8)
    flat = power.reshape(-1, H, W)
    of = out.reshape(-1, H, W)
    for t in range(flat.shape[0]):
        if axes & 1:
            for r in range(H):
                for k0 in range(0, W, window):
                    seg = flat[t, r, k0:k0 + window]
                    of[t, r, k0:k0 + window] |= (seg > fx.mad_threshold(seg, sigma)).astype(np.uint8)
        if axes & 2:
            for k in range(W):
                seg = flat[t, :, k]
                of[t, :, k] |= (seg > fx.mad_threshold(seg, sigma)).astype(np.uint8)
    return out


def precision_recall(pred: np.ndarray, truth: np.ndarray):
    pred = pred.astype(bool)
    truth = truth.astype(bool)
    tp = np.sum(pred & truth)
    fp = np.sum(pred & ~truth)
    fn = np.sum(~pred & truth)
    prec = tp / max(1, tp + fp)
    rec = tp / max(1, tp + fn)
    return float(prec), float(rec)
