"""Delay / phase calibration on the GPU (Sec. 7, Eq. 3) against the FP64
oracle on the same visibilities, and the closed loop: visibilities of a
stream with injected delays and phases -> solution -> corr_set_delays ->
flat phases."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from fxsynth import StreamSpec, make_stream  # noqa: E402
from oracle import calib_oracle as co  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2604_20640_gb300 as pkg
    pkg.load_library()
    return pkg


def _vis(lib, x, n_chan, n_int, n_in, tau=None, phi=None):
    c = lib.Correlator(n_in, 1, n_chan, 4, n_int)
    if tau is not None:
        c.set_delays(tau, phi)
    n = c.n_integrations(x.shape[1])
    v = torch.empty((n, n_chan, n_in, n_in), dtype=torch.complex64, device="cuda")
    f = torch.empty(v.shape, dtype=torch.uint8, device="cuda")
    c.run_dev(torch.from_numpy(x).cuda(), v, f)
    torch.cuda.synchronize()
    return v, f


@pytest.mark.parametrize("n_chan,n_in", [(512, 4), (2048, 6)])
def test_calibration_matches_oracle_and_closes_the_loop(lib, n_chan, n_in):
    M = 2 * n_chan
    n_int = 128
    rng = np.random.default_rng(n_chan)
    tau = np.concatenate([[0.0], rng.uniform(-30, 30, n_in - 1)])
    phi = np.concatenate([[0.0], rng.uniform(-3, 3, n_in - 1)])
    x = make_stream(StreamSpec(n_ant=n_in, n_pol=1, n_samples=M * n_int, seed=n_chan + 1, tau=tau, phi=phi,
                               src_frac=0.2))
    v, f = _vis(lib, x, n_chan, n_int, n_in)
    k_lo, k_hi = 8, n_chan - 8
    t_g, p_g = lib.calibrate(v[0], None, 0, k_lo, k_hi, 40.0)
    R = v[0].cpu().numpy().astype(np.complex128)
    t_o, p_o = co.calibrate(R, 0, k_lo, k_hi, 40.0)
    assert np.max(np.abs(t_g - t_o)) < 1e-4
    assert np.max(np.abs(np.angle(np.exp(1j * (p_g - p_o))))) < 1e-4
    # the injected truth, and flat phases once the solution is applied
    assert np.max(np.abs(t_g - tau)) < 0.05
    assert np.max(np.abs(np.angle(np.exp(1j * (p_g - phi))))) < 0.05
    v2, _ = _vis(lib, x, n_chan, n_int, n_in, t_g, p_g)
    t2, p2 = lib.calibrate(v2[0], None, 0, k_lo, k_hi, 40.0)
    assert np.max(np.abs(t2)) < 0.05 and np.max(np.abs(np.angle(np.exp(1j * p2)))) < 0.05


def test_calibration_honours_flags_and_band(lib):
    n_chan, n_in, n_int = 256, 3, 128
    M = 2 * n_chan
    tau = np.array([0.0, 5.5, -9.25])
    phi = np.array([0.0, 0.4, -1.1])
    x = make_stream(StreamSpec(n_ant=n_in, n_pol=1, n_samples=M * n_int, seed=9, tau=tau, phi=phi, src_frac=0.2,
                               tones=[(40.5 / M, 60.0, 0.0)]))
    v, _ = _vis(lib, x, n_chan, n_int, n_in)
    flags = torch.zeros(v.shape[1:], dtype=torch.uint8, device="cuda")
    flags[38:44] = 1                        # the tone's channels
    t_g, p_g = lib.calibrate(v[0], flags, 0, 4, n_chan - 4, 20.0)
    fl = flags.cpu().numpy()
    t_o, p_o = co.calibrate(v[0].cpu().numpy().astype(np.complex128), 0, 4, n_chan - 4, 20.0, flags=fl)
    assert np.max(np.abs(t_g - t_o)) < 1e-4
    assert np.max(np.abs(np.angle(np.exp(1j * (p_g - p_o))))) < 1e-4
    with pytest.raises(lib.CorrError):
        lib.calibrate(v[0], None, 0, 10, 11, 20.0)     # fewer than two channels
