"""CPU checks of the C ABI: libtem.so builds for sm_103a, loads, and exports
every function include/tem.h declares; the Python binding declares the same
set.  No compute call is made (there may be no GPU)."""
import os
import re
import ctypes

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "tem.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int|int64_t|const char \*)\s*(tem_\w+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_2605_19951_gb300 import build, tem
    if not os.path.exists(tem.LIB_PATH):
        build.build()
    return ctypes.CDLL(tem.LIB_PATH)


def test_header_declares_core_calls():
    names = _declared()
    for core in ("tem_create", "tem_mesh", "tem_poles", "tem_sources", "tem_factor", "tem_forward",
                 "tem_jvp", "tem_jtvp", "tem_lsqr", "tem_destroy"):
        assert core in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_header():
    from paper_2605_19951_gb300 import tem
    assert sorted(tem.SIGNATURES) == _declared()


def test_binding_refuses_cpu_tensors():
    torch = pytest.importorskip("torch")
    from paper_2605_19951_gb300 import tem
    with pytest.raises(TypeError):
        tem._dev(torch.zeros(3, dtype=torch.float64))
