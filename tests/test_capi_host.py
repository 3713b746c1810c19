"""Host-only checks of the C-ABI library: it builds, loads, exports every symbol
include/*.h declares, and reports errors as status codes (no GPU needed)."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def rc():
    from paper_1211_5595_gb300 import build
    build.build()
    import paper_1211_5595_gb300 as rc
    rc.lib()
    return rc


def declared_symbols(header):
    text = open(os.path.join(ROOT, "include", header)).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return set(re.findall(r"\b(rc_[a-z0-9_]+)\s*\(", text))


def test_headers_are_known():
    # every header of include/ is checked against its library below
    assert sorted(f for f in os.listdir(os.path.join(ROOT, "include")) if f.endswith(".h")) == ["rc.h", "rc_probe.h"]


def test_every_declared_symbol_is_exported(rc):
    names = declared_symbols("rc.h")
    assert len(names) >= 16
    lib = C.CDLL(rc.LIB_PATH)
    missing = [n for n in sorted(names) if not hasattr(lib, n)]
    assert not missing, missing
    # the binding wraps every declared call under the same name
    assert names <= set(rc.SIGNATURES), sorted(names - set(rc.SIGNATURES))
    for n in names:
        assert callable(getattr(rc, n)), n


def test_debug_library_exports_the_same_calls(rc):
    """The debug build (device index checks) is the same interface."""
    from paper_1211_5595_gb300 import build
    lib = C.CDLL(build.DEBUG_LIB)
    missing = [n for n in sorted(declared_symbols("rc.h")) if not hasattr(lib, n)]
    assert not missing, missing


def test_probe_library_exports_its_header(rc):
    """The measurement probes live in their own library, outside the
    raycasting interface."""
    from paper_1211_5595_gb300 import build
    names = declared_symbols("rc_probe.h")
    assert names == {"rc_probe_read_l1", "rc_probe_read_l2", "rc_probe_l1_bytes"}
    lib = C.CDLL(build.PROBE_LIB)
    assert all(hasattr(lib, n) for n in names)
    assert not (names & declared_symbols("rc.h"))
    lib.rc_probe_read_l1.argtypes = [C.c_void_p, C.c_size_t, C.c_int, C.c_void_p]
    # invalid arguments are refused before any launch (cudaErrorInvalidValue = 1)
    assert lib.rc_probe_read_l1(None, 16, 1, None) == 1
    assert lib.rc_probe_read_l1(C.c_void_p(16), 1 << 20, 1, None) == 1


def test_status_strings(rc):
    assert rc.rc_status_string(rc.RC_OK) == "ok"
    assert rc.rc_status_string(rc.RC_ERR_INVALID_ARG) == "invalid argument"
    assert rc.rc_status_string(99) == "unknown status"


def test_null_arguments_are_status_codes(rc):
    L = rc.lib()
    assert L.rc_context_create(0, None, None) == rc.RC_ERR_INVALID_ARG
    assert L.rc_volume_upload(None, None, 0, 0) == rc.RC_ERR_INVALID_ARG
    assert "vol is NULL" in rc.rc_last_error(None)
    p = rc.RenderParams().c()
    assert L.rc_render(None, None, C.byref(p), None, None) == rc.RC_ERR_INVALID_ARG
    assert L.rc_render_backward(None, None, C.byref(p), None, None) == rc.RC_ERR_INVALID_ARG
    assert L.rc_tf_set(None, None, 0, 0) == rc.RC_ERR_INVALID_ARG
    assert L.rc_tf2d_set(None, None, 0, 0, C.c_float(1.0), 0) == rc.RC_ERR_INVALID_ARG
    assert L.rc_tf2d_set_device(None, None, 0, 0, C.c_float(1.0), 0) == rc.RC_ERR_INVALID_ARG
    assert L.rc_camera_set(None, None) == rc.RC_ERR_INVALID_ARG
    assert L.rc_volume_brick_dims(None, None) == rc.RC_ERR_INVALID_ARG
    assert L.rc_context_destroy(None) == rc.RC_OK
    assert L.rc_volume_destroy(None) == rc.RC_OK


def test_binding_raises_rcerror(rc):
    with pytest.raises(rc.RCError):
        rc.rc_render(None, None, rc.RenderParams(), None)


@pytest.mark.skipif(os.path.exists("/dev/nvidia0"), reason="a GPU is present")
def test_context_without_gpu_is_an_error_not_a_crash(rc):
    out = C.c_void_p()
    st = rc.lib().rc_context_create(0, None, C.byref(out))
    assert st in (rc.RC_ERR_CUDA, rc.RC_ERR_INVALID_ARG)
    assert out.value is None
