"""Pins of the learned-flagger oracle: convolution against a library routine,
gradients against finite differences in FP64, the loss against its direct
formula, and the MAD fallback against the Eq. 2 oracle."""

import math

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


def test_params_flatten_order_and_roundtrip():
    params = fn.init_params(7)
    v = fn.flatten_params(params)
    assert v.size == 52897
    # layer 0: 32 x 1 x 5 x 5 weights, then 32 biases; layer 1 starts at 832
    assert v[0] == params[0][0][0, 0, 0, 0] and v[7] == params[0][0][0, 0, 1, 2]
    assert v[25] == params[0][0][1, 0, 0, 0] and v[800] == params[0][1][0]
    assert v[832 + 25 * 3 + 5 * 4 + 1] == params[1][0][0, 3, 4, 1]
    back = fn.unflatten_params(v)
    for (w, b), (w2, b2) in zip(params, back):
        assert np.array_equal(w, w2) and np.array_equal(b, b2)


def test_dynamic_spectrum_tone_closed_form():
    # A tone A cos(2 pi k0 n / M + theta) at a channel centre gives
    # |Y[k0]|^2 = |A/2 e^{j theta} G(0) + A/2 e^{-j theta} G(2 k0)|^2 in every
    # spectrum after the P - 1 filter-fill spectra (G the folded-filter DFT).
    M, P, k0, A, theta, n_row = 64, 4, 5, 37.0, 0.7, 4
    n = np.arange(M * 24)
    x = (A * np.cos(2 * np.pi * k0 * n / M + theta))[None, :]
    D = fn.dynamic_spectrum(x, M // 2, P, n_row)
    h = fx.pfb_coefficients(M, P)
    g = h.reshape(P, M).sum(axis=0)
    m = np.arange(M)
    y = (A / 2) * np.exp(1j * theta) * g.sum() + \
        (A / 2) * np.exp(-1j * theta) * np.sum(g * np.exp(-4j * np.pi * k0 * m / M))
    assert D.shape == (1, 6, 32)
    for r in range(1, 6):
        assert abs(D[0, r, k0] - abs(y) ** 2) < 1e-9 * abs(y) ** 2
        assert np.argmax(D[0, r]) == k0


def test_dynamic_spectrum_white_noise_level_and_delay_invariance():
    # E P = sigma^2 sum h^2 away from DC; an integer delay only shifts time.
    M, P, sig, n_row = 64, 4, 3.0, 50
    rng = np.random.default_rng(5)
    x = rng.standard_normal((1, M * 4000)) * sig
    D = fn.dynamic_spectrum(x, M // 2, P, n_row)[0, 1:, 1:]
    expect = sig ** 2 * np.sum(fx.pfb_coefficients(M, P) ** 2)
    se = D.std() / math.sqrt(D.size)
    assert abs(D.mean() - expect) < 5 * se
    x2 = np.concatenate([np.zeros((1, 3 * M)), x[:, :M * 200]], axis=1)
    D2 = fn.dynamic_spectrum(x2, M // 2, P, 1, tau=np.array([3.0 * M]))
    D1 = fn.dynamic_spectrum(x[:, :M * 200], M // 2, P, 1)
    np.testing.assert_allclose(D2[0, :190], D1[0, :190], rtol=1e-9, atol=1e-9)


def test_to_tiles_index_map():
    P = np.arange(2 * 128 * 512, dtype=float).reshape(2, 128, 512)
    T = fn.to_tiles(P)
    assert T.shape == (2, 2, 2, 64, 256)
    # input 1, row 64 + 3, channel 256 + 7 -> tile (1, 1, 1), pixel (3, 7)
    assert T[1, 1, 1, 3, 7] == P[1, 67, 263] == 1 * 128 * 512 + 67 * 512 + 263


def test_time_direction_mad_is_eq2_per_channel_and_union():
    rng = np.random.default_rng(8)
    P = rng.rayleigh(1.0, (2, 64, 128)) + 0.1
    P[1, 10:12, :] += 30.0          # a broadband burst: rows 10-11 raised in every channel
    F_row = fn.mad_tile_flags(P, axes=1)
    F_time = fn.mad_tile_flags(P, axes=2)
    F_both = fn.mad_tile_flags(P, axes=3)
    assert F_time[1, 10:12, :].all()                  # seen along time
    assert F_row[1, 10:12, :].sum() < 0.1 * 2 * 128   # not along the raised row itself
    assert np.array_equal(F_both, F_row | F_time)
    for k in (0, 77):
        seg = P[0, :, k]
        assert np.array_equal(F_time[0, :, k], (seg > fx.mad_threshold(seg, 5.0)).astype(np.uint8))
