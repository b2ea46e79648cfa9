"""Learned flagger on the GPU against the FP64 oracle: input normalisation,
forward logits and gradients (BF16 operands, FP32 accumulation), the MAD
fallback (Eq. 2 per row window), the confidence switch, the dynamic spectra
from the F-engine, and a trained net against MAD on held-out synthetic RFI.

Tolerances.  The convolutions round inputs, weights and activations to BF16
(unit roundoff u = 2^-9).  A dot product of terms with random signs then has
a relative error of about sqrt(2) u from the operand roundings plus u from
storing the activation, ~0.35 % per layer; four layers compound to ~0.7 %
rms.  The bar is 1.5 % relative Frobenius error on the logits and 3 % on each
layer's gradient (whose operands carry the forward error as well).
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle import flagnet_oracle as fn  # noqa: E402
from oracle import fx_oracle as fx  # noqa: E402
from fxsynth.flagging import TileSpec, make_tiles  # noqa: E402
from fxsynth.streams import StreamSpec, make_stream  # noqa: E402


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2604_20640_gb300 as pkg
    pkg.load_library()
    return pkg


def _params(seed):
    rng = np.random.default_rng(seed + 100)
    return [(w, rng.standard_normal(b.shape) * 0.05) for w, b in fn.init_params(seed)]


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_prepare_matches_oracle(lib):
    power, _ = make_tiles(3, seed=11, device="cuda")
    net = lib.FlagNet()
    x = torch.empty_like(power)
    net.prepare(power, x)
    ref = fn.tile_input(power.double().cpu().numpy())
    np.testing.assert_allclose(x.cpu().numpy(), ref, rtol=0, atol=2e-6 * np.abs(ref).max() + 2e-6)


def test_forward_matches_oracle(lib):
    params = _params(5)
    power, _ = make_tiles(2, seed=12, device="cuda")
    xr = fn.tile_input(power.double().cpu().numpy())
    net = lib.FlagNet(fn.flatten_params(params))
    x = torch.as_tensor(xr, dtype=torch.float32, device="cuda")
    z = torch.empty_like(x)
    net.forward(x, z)
    torch.cuda.synchronize()
    zr, _ = fn.forward(params, xr[:, None])
    zr = zr[:, 0]
    assert _rel(z.double().cpu().numpy(), zr) < 0.015
    assert net.status() == 0


def test_params_roundtrip(lib):
    v = fn.flatten_params(_params(9)).astype(np.float32)
    net = lib.FlagNet(v)
    assert np.array_equal(net.get_params(), v)


def test_loss_and_gradients_match_oracle(lib):
    params = _params(6)
    power, truth = make_tiles(1, seed=13, device="cuda")
    xr = fn.tile_input(power.double().cpu().numpy())
    net = lib.FlagNet(fn.flatten_params(params))
    x = torch.as_tensor(xr, dtype=torch.float32, device="cuda")
    loss, g = net.loss_grad(x, truth)
    tr = truth.cpu().numpy().astype(np.float64)
    L, grads = fn.loss_and_grads(params, xr[:, None], tr[:, None])
    assert abs(loss - L) < 2e-3 * abs(L)
    gr = fn.unflatten_params(g)
    for li in range(4):
        assert _rel(gr[li][0], grads[li][0]) < 0.03, li
        assert _rel(gr[li][1], grads[li][1]) < 0.03, li


def test_mad_fallback_equals_eq2(lib):
    power, _ = make_tiles(4, seed=14, device="cuda")
    net = lib.FlagNet(fn.flatten_params(_params(1)))
    flags = torch.empty(power.shape, dtype=torch.uint8, device="cuda")
    conf = torch.empty(4, device="cuda")
    net.flag(power, flags, conf, c_min=2.0)        # confidence <= 1: always MAD
    P = power.double().cpu().numpy()
    ref = fn.mad_tile_flags(P)
    got = flags.cpu().numpy()
    diff = np.argwhere(got != ref)
    # a disagreement may only sit on the FP32 rounding of the threshold
    for t, r, k in diff:
        k0 = (k // 64) * 64
        T = fx.mad_threshold(P[t, r, k0:k0 + 64], 5.0)
        assert abs(P[t, r, k] - T) <= 1e-5 * T
    assert len(diff) <= 2
    assert got.sum() > 0


def test_confidence_switch(lib):
    power, _ = make_tiles(6, seed=15, device="cuda")
    net = lib.FlagNet(fn.flatten_params(_params(2)))
    x = torch.empty_like(power)
    z = torch.empty_like(power)
    net.prepare(power, x)
    net.forward(x, z)
    f_net = torch.empty(power.shape, dtype=torch.uint8, device="cuda")
    f_mad = torch.empty_like(f_net)
    f_mix = torch.empty_like(f_net)
    conf = torch.empty(6, device="cuda")
    net.flag(power, f_net, conf, c_min=0.0)
    net.flag(power, f_mad, None, c_min=2.0)
    c = conf.cpu().numpy()
    # confidence against its definition on the GPU's own logits
    ref_c = fn.confidence(fn.sigmoid(z.double().cpu().numpy()))
    np.testing.assert_allclose(c, ref_c, rtol=0, atol=1e-5)
    assert torch.equal(f_net, (z > 0).to(torch.uint8))
    c_min = float(np.median(c))
    net.flag(power, f_mix, None, c_min=c_min)
    for t in range(6):
        want = f_net[t] if c[t] >= c_min else f_mad[t]
        assert torch.equal(f_mix[t], want), t


def test_bad_arguments(lib):
    net = lib.FlagNet()
    with pytest.raises(lib.CorrError):
        net.set_params(np.zeros(10, np.float32))
    x = torch.zeros((1, 64, 256), device="cuda")
    with pytest.raises(lib.CorrError):
        net.train_step(x, torch.zeros((1, 64, 256), dtype=torch.uint8, device="cuda"), -1.0)


@pytest.mark.parametrize("n_chan,rows,n_row,tau", [(256, 64, 4, None), (512, 128, 3, [0.0, 5.0, -2.6])])
def test_spectrogram_matches_oracle(lib, n_chan, rows, n_row, tau):
    M = 2 * n_chan
    n_in = 2 if tau is None else 3
    n_samples = (rows * n_row + 5) * M + 77          # a ragged tail the spectra never reach
    spec = StreamSpec(n_ant=n_in, n_pol=1, n_samples=n_samples, seed=31,
                      tones=[(20.3 / M, 6.0, 0.0)], chirps=[(0, n_samples, 40 / M, 200 / M, 5.0)],
                      burst_frac=0.05, burst_frame=M * n_row)
    x = make_stream(spec)
    c = lib.Correlator(n_in, 1, n_chan, 4, 64)
    if tau is not None:
        c.set_delays(np.asarray(tau))
    d = torch.as_tensor(x, device="cuda")
    tiles = torch.full((n_in, rows // 64, n_chan // 256, 64, 256), 7.0, device="cuda")
    c.spectrogram_dev(d, n_row, tiles)
    torch.cuda.synchronize()
    ref = fn.to_tiles(fn.dynamic_spectrum(x, n_chan, 4, n_row, None if tau is None else np.asarray(tau))[:, :rows])
    assert ref.shape == tiles.shape
    got = tiles.double().cpu().numpy()
    scale = ref.mean(axis=(-2, -1), keepdims=True)
    assert np.max(np.abs(got - ref) / (ref + scale)) < 2e-5


def test_spectrogram_rejects_bad_shapes(lib):
    c = lib.Correlator(2, 1, 128, 4, 64)
    d = torch.zeros((2, 256 * 64 * 4), dtype=torch.int8, device="cuda")
    with pytest.raises(lib.CorrError):
        c.spectrogram_dev(d, 1, torch.zeros(1, device="cuda"))      # n_chan % 256
    c2 = lib.Correlator(2, 1, 256, 4, 64)
    with pytest.raises(lib.CorrError):
        c2.spectrogram_dev(d[:, :512 * 10], 1, torch.zeros(1, device="cuda"))   # fewer than 64 rows


def test_training_learns_and_beats_mad(lib):
    from paper_2604_20640_gb300 import flagger
    net = lib.FlagNet(fn.flatten_params(fn.init_params(0)))
    spec = TileSpec()
    losses = flagger.train(net, lambda i: make_tiles(16, seed=1000 + i, device="cuda", spec=spec),
                           steps=600, lr=2e-3)
    assert np.isfinite(losses).all()
    assert np.mean(losses[-50:]) < 0.6 * np.mean(losses[:5])
    assert net.status() == 0
    power, truth = make_tiles(64, seed=7, device="cuda", spec=spec)
    f_net, _ = flagger.flag(net, power, c_min=0.0)
    f_mad, _ = flagger.flag(net, power, c_min=2.0)
    t = truth.cpu().numpy()
    p_net, r_net = fn.precision_recall(f_net.cpu().numpy(), t)
    p_mad, r_mad = fn.precision_recall(f_mad.cpu().numpy(), t)
    print("net precision %.3f recall %.3f | MAD precision %.3f recall %.3f" % (p_net, r_net, p_mad, r_mad))
    assert r_net > r_mad + 0.15
    assert p_net > 0.8


def test_noise_level_matches_filter_energy(lib):
    # E|Y_k|^2 = sigma_q^2 sum_n h[n]^2 for white noise away from DC, with
    # sigma_q^2 = 16^2 + 1/12 for int8-rounded N(0, 16^2) (no clipping at 8 sigma)
    from fxsynth.rfi_torch import RfiSpec, noise_only
    from paper_2604_20640_gb300 import flagger
    spec = RfiSpec(n_in=1, n_chan=1024, n_row=64)
    one = lib.Correlator(1, 1, 1024, 4, 64)
    lvl = flagger.noise_level(one, noise_only(spec, spec.n_samples, "cuda"), 64).cpu().numpy()
    expect = (16.0 ** 2 + 1.0 / 12) * np.sum(fx.pfb_coefficients(2048, 4) ** 2)
    # 64 rows x 64 spectra per channel: relative standard error 1/64 per channel
    assert abs(np.mean(lvl[4:-4]) / expect - 1) < 3e-3
    assert np.max(np.abs(lvl[4:-4] / expect - 1)) < 6 / 64


def test_c5_pipeline_trained_net_beats_mad(lib):
    from paper_2604_20640_gb300 import train_flagnet
    src = train_flagnet.TileSource(n_in=4, n_chan=1024, n_row=64, seed=321)
    net = lib.FlagNet(train_flagnet.init_params(0))
    losses = train_flagnet.train(net, src, 400, 32, 1e-3)
    assert np.mean(losses[-40:]) < 0.5 * np.mean(losses[:5])
    p, t, tn, tb, _ = src.batch(10 ** 6, with_parts=True)
    q = train_flagnet.evaluate(net, p, t, tn, tb)
    print(q)
    assert 0.005 < q["truth_fraction"] < 0.5
    assert q["net"]["recall"] > q["mad"]["recall"] + 0.1
    assert q["net"]["precision"] > 0.8
    assert q["net"]["recall_broadband"] > q["mad"]["recall_broadband"]


@pytest.mark.parametrize("axes", [1, 2, 3])
def test_tile_mad_matches_oracle(lib, axes):
    power, _ = make_tiles(3, seed=20 + axes, device="cuda")
    flags = torch.empty(power.shape, dtype=torch.uint8, device="cuda")
    lib.tile_mad(power, flags, axes=axes)
    P = power.double().cpu().numpy()
    ref = fn.mad_tile_flags(P, axes=axes)
    got = flags.cpu().numpy()
    diff = np.argwhere(got != ref)
    for t, r, k in diff:        # only FP32 rounding of a threshold may differ
        near = False
        if axes & 1:
            k0 = (k // 64) * 64
            T = fx.mad_threshold(P[t, r, k0:k0 + 64], 5.0)
            near |= abs(P[t, r, k] - T) <= 1e-5 * T
        if axes & 2:
            T = fx.mad_threshold(P[t, :, k], 5.0)
            near |= abs(P[t, r, k] - T) <= 1e-5 * T
        assert near
    assert len(diff) <= 3 and got.sum() > 0
