"""Host-side checks of the CUDA library: it builds for sm_103a, it loads, and it
exports every entry point that include/nnca.h declares (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "nnca.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(nnca_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libnnca():
    from paper_2203_14832_gb300 import _build
    path = _build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for s in ["nnca_build", "nnca_matvec", "nnca_matvec_host", "nnca_destroy", "nnca_get_stats", "nnca_export",
              "nnca_last_error", "nnca_status_string"]:
        assert s in syms


def test_library_exports_every_declared_symbol(libnnca):
    for s in declared_symbols():
        assert hasattr(libnnca, s), s


def test_binding_names_match(libnnca):
    from paper_2203_14832_gb300 import nnca
    for s in declared_symbols():
        if s != "nnca_status_string":
            assert hasattr(nnca, s), s


def test_calls_without_a_device_fail_cleanly(libnnca):
    """Argument checks run on the host before any device work."""
    libnnca.nnca_build.restype = ctypes.c_int
    out = ctypes.c_void_p()
    st = libnnca.nnca_build(None, None, ctypes.c_int64(10), None, ctypes.c_int64(0), 0, None, ctypes.byref(out))
    assert st == 1 and not out.value
    libnnca.nnca_status_string.restype = ctypes.c_char_p
    assert libnnca.nnca_status_string(1) == b"invalid argument"
    libnnca.nnca_last_error.restype = ctypes.c_char_p
    assert b"NULL" in libnnca.nnca_last_error(None)


def test_unknown_m2l_form_is_rejected_on_the_host(libnnca):
    """nnca_config.m2l_form takes NNCA_M2L_AUTO or NNCA_M2L_FULL; anything else fails
    before any device call."""
    from paper_2203_14832_gb300 import nnca
    libnnca.nnca_build.restype = ctypes.c_int
    libnnca.nnca_last_error.restype = ctypes.c_char_p
    for form, ok in ((nnca.M2L_AUTO, True), (nnca.M2L_FULL, True), (2, False), (-1, False)):
        cfg = nnca.Config(m2l_form=form).c()
        out = ctypes.c_void_p()
        pts = (ctypes.c_double * 30)()   # host memory: a valid form fails later, at the device check
        st = libnnca.nnca_build(ctypes.byref(cfg), pts, ctypes.c_int64(10), None, ctypes.c_int64(0), 0, None,
                                ctypes.byref(out))
        assert st == 1 and not out.value
        msg = libnnca.nnca_last_error(None)
        assert (b"m2l_form" in msg) != ok, msg
