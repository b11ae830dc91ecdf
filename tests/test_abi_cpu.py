"""Host-side checks of the C ABI that need no GPU: the library builds, loads, and exports every
function include/ichee.h declares; the binding's structures match the header's sizes."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib_path():
    from paper_2409_03568_gb300 import build
    return build.build()


def test_library_exports_every_declared_function(lib_path):
    from paper_2409_03568_gb300 import ichee
    names = ichee.header_functions()
    assert len(names) >= 16
    lib = ctypes.CDLL(lib_path)
    for name in names:
        assert hasattr(lib, name), name
    assert set(ichee._SIGS) == set(names)


def test_binding_structs_match_header_layout():
    from paper_2409_03568_gb300 import ichee
    with open(os.path.join(ROOT, "include", "ichee.h")) as f:
        text = f.read()
    assert "ICHEE_MAX_PRIMES 8" in text
    assert ctypes.sizeof(ichee.Params) == 48 + 8 + 4 + 4   # 12 words, the double, gauss_bound, tail padding
    assert ctypes.sizeof(ichee.CtImgMeta) == 4 * 4 + 8
    assert ctypes.sizeof(ichee.CacheDesc) == 6 * 4
    enum_ops = re.findall(r"ICHEE_OP_(\w+)\s*=\s*(\d+)", text)
    for name, val in enum_ops:
        assert getattr(ichee, "OP_" + name) == int(val)


def test_last_error_is_empty_string_initially():
    from paper_2409_03568_gb300 import ichee
    assert isinstance(ichee.ichee_last_error(), str)
