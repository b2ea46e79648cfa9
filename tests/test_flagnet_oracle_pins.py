"""Pins of the learned-flagger oracle: convolution against a library routine,
gradients against finite differences in FP64, the loss against its direct
formula, and the MAD fallback against the Eq. 2 oracle."""

import numpy as np
import pytest

from oracle import flagnet_oracle as fn
from oracle import fx_oracle as fx


def test_conv_matches_library_correlate2d():
    sig = pytest.importorskip("scipy.signal")
    rng = np.random.default_rng(0)
    x = rng.standard_normal((2, 3, 7, 9))
    w = rng.standard_normal((4, 3, 5, 5))
    b = rng.standard_normal(4)
    y = fn.conv2d(x, w, b)
    for n in range(2):
        for o in range(4):
            ref = b[o] + sum(sig.correlate2d(x[n, c], w[o, c], mode="same", boundary="fill")
                             for c in range(3))
            np.testing.assert_allclose(y[n, o], ref, rtol=1e-12, atol=1e-12)


def test_bce_from_logits_equals_direct_formula():
    rng = np.random.default_rng(1)
    z = rng.standard_normal(100) * 3
    t = (rng.random(100) < 0.3).astype(float)
    p = 1 / (1 + np.exp(-z))
    direct = -np.mean(t * np.log(p) + (1 - t) * np.log(1 - p))
    assert abs(fn.bce_from_logits(z, t) - direct) < 1e-12


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(2)
    params = [(w * 0.5, rng.standard_normal(b.shape) * 0.1) for w, b in fn.init_params(3)]
    # narrow the net so the check is quick: keep the architecture, small tile
    x = rng.standard_normal((2, 1, 6, 7))
    t = (rng.random((2, 1, 6, 7)) < 0.4).astype(float)
    L, grads = fn.loss_and_grads(params, x, t)
    eps = 1e-6
    for li in range(4):
        w, b = params[li]
        for idx in [(0, 0, 2, 2), (w.shape[0] - 1, w.shape[1] - 1, 0, 4), (w.shape[0] // 2, 0, 3, 1)]:
            wp = w.copy(); wp[idx] += eps
            wm = w.copy(); wm[idx] -= eps
            pp = list(params); pp[li] = (wp, b)
            pm = list(params); pm[li] = (wm, b)
            fd = (fn.loss_and_grads(pp, x, t)[0] - fn.loss_and_grads(pm, x, t)[0]) / (2 * eps)
            assert abs(fd - grads[li][0][idx]) <= 1e-6 * max(1e-3, abs(fd)) + 1e-9, (li, idx)
        for o in [0, b.shape[0] - 1]:
            bp = b.copy(); bp[o] += eps
            bm = b.copy(); bm[o] -= eps
            pp = list(params); pp[li] = (w, bp)
            pm = list(params); pm[li] = (w, bm)
            fd = (fn.loss_and_grads(pp, x, t)[0] - fn.loss_and_grads(pm, x, t)[0]) / (2 * eps)
            assert abs(fd - grads[li][1][o]) <= 1e-6 * max(1e-3, abs(fd)) + 1e-9, (li, o)


def test_param_count():
    n = sum(w.size + b.size for w, b in fn.init_params())
    assert n == 52897


def test_mad_fallback_is_eq2_per_row_window():
    rng = np.random.default_rng(4)
    P = rng.rayleigh(1.0, (3, 4, 128)) + 0.1
    P[1, 2, 70] = 40.0
    F = fn.mad_tile_flags(P)
    assert F[1, 2, 70] == 1
    for t in range(3):
        for r in range(4):
            for k0 in (0, 64):
                seg = P[t, r, k0:k0 + 64]
                assert np.array_equal(F[t, r, k0:k0 + 64], (seg > fx.mad_threshold(seg, 5.0)).astype(np.uint8))


def test_tile_input_and_confidence():
    P = np.full((2, 3), 4.0)
    P[0, 0] = 4.0 * np.e
    np.testing.assert_allclose(fn.tile_input(P), np.log(P / 4.0))
    assert fn.confidence(np.array([[0.0, 1.0], [0.5, 0.5]])) == 0.5
    pr, rc = fn.precision_recall(np.array([1, 1, 0, 0]), np.array([1, 0, 1, 0]))
    assert pr == 0.5 and rc == 0.5
