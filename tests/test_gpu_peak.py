"""The FP32 peak probe (corr_peak_fp32) that sets the F-engine's arithmetic
ceiling: its rate must scale with the work (twice the FMAs in twice the
time, within clock noise) and sit in the plausible range for one device
(above 10 TFLOP/s; below 152 SMs x 128 lanes x 4 FLOP x 2.1 GHz for the
packed form, the most any FP32 pipe arrangement of this device could give)."""

import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_20640_gb300.build import build_library
    build_library()


@pytest.mark.parametrize("packed", [False, True])
def test_peak_probe_is_consistent(packed):
    from paper_2604_20640_gb300.corr import peak_fp32
    t1, ms1 = peak_fp32(packed, 2048)
    t2, ms2 = peak_fp32(packed, 4096)
    assert 10.0 < t2 < 152 * 128 * 4 * 2.1e9 / 1e12
    assert 1.5 < ms2 / ms1 < 2.5
    assert abs(t2 / t1 - 1.0) < 0.25


def test_peak_probe_rejects_bad_arguments():
    from paper_2604_20640_gb300 import CorrError, CORR_EINVAL
    from paper_2604_20640_gb300.corr import peak_fp32
    with pytest.raises(CorrError) as e:
        peak_fp32(False, 0)
    assert e.value.code == CORR_EINVAL
