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


def test_null_arguments_are_refused_without_a_launch(lib_path):
    """Argument checks come first and report a status and a message; no call aborts. Every call
    below gets a null handle or a null pointer, so none of them reaches the GPU."""
    from paper_2409_03568_gb300 import ichee
    L = ichee._lib
    calls = {
        "ichee_ctx_create": lambda: L.ichee_ctx_create(None, 0, None),
        "ichee_keygen": lambda: L.ichee_keygen(None, 1, 0, None),
        "ichee_ct_bytes": lambda: L.ichee_ct_bytes(None, 0, None),
        "ichee_encrypt_image": lambda: L.ichee_encrypt_image(None, None, None, 1, 1, 1, 0, None, None, None),
        "ichee_eval": lambda: L.ichee_eval(None, 0, None, None, None, None, None, 0, None, None, None),
        "ichee_decrypt_image": lambda: L.ichee_decrypt_image(None, None, None, None, None),
        "ichee_encrypt_batch": lambda: L.ichee_encrypt_batch(None, None, None, None, 0, None, None, None),
        "ichee_decrypt_batch": lambda: L.ichee_decrypt_batch(None, None, None, None, 0, None),
        "ichee_set_tuned_shape": lambda: L.ichee_set_tuned_shape(None, 1, 256, 0),
        "ichee_buffer_bytes_left": lambda: L.ichee_buffer_bytes_left(None, None),
        "ichee_server_submit": lambda: L.ichee_server_submit(None, None, None),
        "ichee_stream_status": lambda: L.ichee_stream_status(None, None),
    }
    for name, call in calls.items():
        status = call()
        assert status == ichee.EINVAL, (name, status)
        assert ichee.ichee_last_error(), name


def test_context_creation_without_a_device_fails_cleanly(lib_path):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    from paper_2409_03568_gb300 import ichee
    with pytest.raises(ichee.IcheeError) as e:
        ichee.Context(log_n=10, prime_bits=[30, 30], log2_scale=25)
    assert e.value.status == ichee.ECUDA and "cudaSetDevice" in str(e.value)
