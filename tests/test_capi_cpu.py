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
