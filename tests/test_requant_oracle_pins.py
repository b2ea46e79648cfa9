"""Pins of the reduced-precision oracle (int8 / e4m3 requantisation, exact
Gram matrix, rescaling) against hand-worked values, an independent library
conversion, brute force and the full-precision oracle."""

import numpy as np
import pytest

from oracle import fx_oracle as fx
from oracle import requant_oracle as rq
from fxsynth import config_c1, make_stream


def test_int8_rounding_hand_values():
    x = np.array([1.5, 2.5, -0.5, -1.5, 126.6, 200.0, -200.0, 0.49, -127.5])
    np.testing.assert_array_equal(rq.quantize_int8(x), [2, 2, -0.0, -2, 127, 127, -127, 0, -127])


def test_e4m3_hand_values():
    x = np.array([448.0, 500.0, -1e9, 1.0625, 1.1875, 2.0 ** -10, 3 * 2.0 ** -10, 0.0, -3.3])
    expect = [448.0, 448.0, -448.0, 1.0, 1.25, 0.0, 2.0 ** -8, 0.0, -3.25]
    np.testing.assert_array_equal(rq.e4m3_round(x), expect)


def test_e4m3_matches_library_conversion():
    torch = pytest.importorskip("torch")
    if not hasattr(torch, "float8_e4m3fn"):
        pytest.skip("torch without float8")
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.uniform(-448, 448, 20000), rng.uniform(-0.05, 0.05, 20000),
                        rng.standard_normal(20000) * 64])
    x = np.clip(x, -448, 448)
    ref = torch.tensor(x, dtype=torch.float64).to(torch.float8_e4m3fn).to(torch.float64).numpy()
    np.testing.assert_array_equal(rq.e4m3_round(x), ref)


def test_e4m3_decode_matches_library_and_hand_values():
    b = np.arange(256, dtype=np.uint8)
    v = rq.e4m3_decode(b)
    assert v[0x00] == 0.0 and v[0x38] == 1.0 and v[0x7E] == 448.0 and v[0x01] == 2.0 ** -9
    assert v[0xB8] == -1.0 and np.isnan(v[0x7F]) and np.isnan(v[0xFF])
    torch = pytest.importorskip("torch")
    if not hasattr(torch, "float8_e4m3fn"):
        pytest.skip("torch without float8")
    ref = torch.from_numpy(b.copy()).view(torch.float8_e4m3fn).to(torch.float64).numpy()
    ok = ~np.isnan(ref)
    np.testing.assert_array_equal(v[ok], ref[ok])
    assert np.all(np.isnan(v[~ok]))
    # decode(round(x)) is idempotent on the grid
    np.testing.assert_array_equal(rq.e4m3_round(v[ok]), v[ok])


def test_gram_brute_force():
    rng = np.random.default_rng(1)
    Q = rng.integers(-127, 128, size=(2, 6, 9)).astype(np.int8)
    G = rq.gram(Q)
    for c in range(2):
        for r in range(6):
            for s in range(6):
                assert G[c, r, s] == sum(int(Q[c, r, k]) * int(Q[c, s, k]) for k in range(9))


def test_visibilities_from_gram_equal_direct_sum():
    rng = np.random.default_rng(2)
    N, K, C = 3, 11, 4
    qr = rng.integers(-127, 128, size=(N, K, C)).astype(np.int64)
    qi = rng.integers(-127, 128, size=(N, K, C)).astype(np.int64)
    G = rq.gram(rq.stacked_rows(qr, qi))
    Cv = rq.visibilities_from_gram(G, N)
    q = qr + 1j * qi
    for c in range(C):
        for a in range(N):
            for b in range(N):
                direct = sum(q[a, k, c] * np.conj(q[b, k, c]) for k in range(K))
                assert Cv[c, a, b] == direct


def test_quantized_correlation_close_to_full_precision():
    # The quantisation error of rho is statistical (~1/sqrt(K)); the 5e-3
    # bound is for integrations of thousands of spectra (K = 2048 here).
    spec = config_c1(seed=1234, n_samples=2048 * 2048 * 2)
    x = make_stream(spec)
    tau, phi = np.asarray(spec.tau), np.asarray(spec.phi)
    R = fx.correlate(x, 1024, 4, 2048, tau, phi)[0]
    rho = fx.normalised_coefficients(R)
    for dt in ("int8", "e4m3"):
        Rq, S = rq.correlate_quantized(x, 1024, 4, 2048, tau, phi, dtype=dt)
        rho_q = fx.normalised_coefficients(Rq)
        assert np.abs(rho_q - rho).max() < 5e-3, dt
        assert S.shape == (2, 4, 1024)
