"""CPU checks of the C ABI: the library builds, loads and exports every
function ``include/corr.h`` declares, and fails loudly without a GPU."""

import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "corr.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:[A-Za-z_][\w\s\*]*?)\b(corr_\w+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def lib_path():
    from paper_2604_20640_gb300.build import build_library
    return build_library()


def test_header_declares_the_boundary_calls():
    names = declared_functions()
    for n in ["corr_create", "corr_set_delays", "corr_push", "corr_get_vis", "corr_get_flags",
              "corr_flush", "corr_destroy", "corr_last_error", "corr_set_option"]:
        assert n in names


def test_library_exports_every_declared_symbol(lib_path):
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT\s+(corr_\w+)", out))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    import paper_2604_20640_gb300 as pkg
    assert sorted(pkg.EXPORTED) == declared_functions()


def test_library_loads_and_rejects_bad_shapes_without_gpu(lib_path):
    import paper_2604_20640_gb300 as pkg
    L = pkg.load_library()
    for fn in pkg.EXPORTED:
        assert hasattr(L, fn)
    with pytest.raises(pkg.CorrError) as e:
        pkg.Correlator(4, 1, 1000, 4, 16)          # n_chan not a power of two
    assert e.value.code == pkg.CORR_EINVAL
    with pytest.raises(pkg.CorrError) as e:
        pkg.Correlator(4, 1, 1024, 0, 16)          # taps < 1
    assert e.value.code == pkg.CORR_EINVAL


def test_missing_library_fails_loudly(tmp_path):
    import paper_2604_20640_gb300.corr as corr
    saved = corr._lib
    try:
        corr._lib = None
        with pytest.raises(corr.CorrError):
            corr.load_library(str(tmp_path / "nope.so"))
    finally:
        corr._lib = saved


def test_result_buffer_validation_on_the_host():
    """get_vis / get_flags take caller buffers [>= n][n_chan][n_in][n_in]:
    C-contiguous numpy arrays or CPU tensors of the right type; anything
    else is rejected before the library is called."""
    import types
    import numpy as np
    from paper_2604_20640_gb300 import Correlator, CorrError
    me = types.SimpleNamespace(n_chan=8, n_in=3)
    check = Correlator._result_out
    good = np.zeros((4, 8, 3, 3), np.complex64)
    ptr, view = check(me, good, 4, np.complex64)
    assert ptr == good.ctypes.data and view is good
    check(me, good, 2, np.complex64)                                   # larger than needed
    for bad, n in [(np.zeros((4, 8, 3, 3), np.complex128), 4),          # wrong type
                   (np.zeros((4, 8, 3, 4), np.complex64), 4),           # wrong shape
                   (np.zeros((3, 8, 3, 3), np.complex64), 4),           # too short
                   (np.zeros((4, 8, 3, 3, 2), np.complex64)[..., 0], 4),  # not contiguous
                   ([[0]], 1)]:                                         # not an array
        with pytest.raises(CorrError):
            check(me, bad, n, np.complex64)
    torch = pytest.importorskip("torch")
    t = torch.zeros((4, 8, 3, 3), dtype=torch.uint8)
    ptr, view = check(me, t, 4, np.uint8)
    assert ptr == t.data_ptr() and view is t
    for bad in (torch.zeros((4, 8, 3, 3), dtype=torch.int8), torch.zeros((4, 3, 8, 3), dtype=torch.uint8),
                torch.zeros((4, 8, 3, 6), dtype=torch.uint8)[..., ::2]):
        with pytest.raises(CorrError):
            check(me, bad, 4, np.uint8)


def test_noalloc_refuses_misaligned_buffers_before_any_cuda_call(lib_path):
    """corr_xengine_noalloc reads V as 16-byte vectors and writes complex64
    results: a V pointer off a 16-byte boundary, or a result pointer off an
    8-byte one, is refused with CORR_EINVAL on the host.  The check runs
    before the first CUDA call, so it needs no GPU (the addresses are never
    dereferenced)."""
    import paper_2604_20640_gb300 as pkg
    L = pkg.load_library()
    good_v, good_r = 0x10000, 0x20000
    for v, r in [(good_v + 8, good_r), (good_v + 4, good_r), (good_v, good_r + 4)]:
        rc = L.corr_xengine_noalloc(v, 16, 4, 64, r, None)
        assert rc == pkg.CORR_EINVAL
        assert b"aligned" in L.corr_last_error(None)
