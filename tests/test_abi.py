"""The C ABI library builds for sm_103a and exports every function include/caspt2.h
declares; host-only entry points answer without a GPU."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def so():
    from paper_1606_01273_gb300 import build as b
    if not os.path.exists(b.LIB):
        b.build()
    return C.CDLL(b.LIB)


def _declared():
    hdr = open(os.path.join(ROOT, "include", "caspt2.h")).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    return sorted(set(re.findall(r"\b(caspt2_\w+)\s*\(", hdr)))


def test_every_declared_symbol_is_exported(so):
    names = _declared()
    assert len(names) >= 12
    missing = [n for n in names if not hasattr(so, n)]
    assert not missing, missing


def test_host_only_entry_points(so):
    so.caspt2_strerror.restype = C.c_char_p
    assert so.caspt2_strerror(0) == b"ok"
    assert b"invalid" in so.caspt2_strerror(-1)
    so.caspt2_supported_classes.restype = C.c_uint
    assert so.caspt2_supported_classes() == 0xFF
    so.caspt2_create.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
    assert so.caspt2_create(None, None, None) == -1      # EINVAL before touching the GPU
    so.caspt2_get_kernel_launches.restype = C.c_long
    so.caspt2_get_kernel_launches.argtypes = [C.c_void_p]
    assert so.caspt2_get_kernel_launches(None) == -1
    so.caspt2_densities.argtypes = [C.c_void_p, C.c_uint, C.c_void_p]
    assert so.caspt2_densities(None, 0xFF, None) == -1
    so.caspt2_get_densities.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p,
                                        C.c_void_p]
    assert so.caspt2_get_densities(None, 0, None, None, None, None) == -1
    so.caspt2_get_status.argtypes = [C.c_void_p, C.c_void_p]
    assert so.caspt2_get_status(None, None) == -1
    so.caspt2_solve.argtypes = [C.c_void_p, C.c_void_p]
    assert so.caspt2_solve(None, None) == -1
    so.caspt2_amplitude_size.argtypes = [C.c_void_p, C.c_int]
    so.caspt2_amplitude_size.restype = C.c_long
    assert so.caspt2_amplitude_size(None, 0) == -1
    for fn in (so.caspt2_get_amplitudes, so.caspt2_get_lambda):
        fn.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p]
        assert fn(None, 0, 0, 0, 0, None, None) == -1


def test_server_entry_points_reject_null(so):
    """Serving entry points validate their arguments before touching the device."""
    so.caspt2_server_create.argtypes = [C.c_void_p, C.c_size_t, C.c_int]
    assert so.caspt2_server_create(None, 0, 2) == -1
    so.caspt2_server_submit.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
    assert so.caspt2_server_submit(None, None, None) == -1
    so.caspt2_server_wait.argtypes = [C.c_void_p, C.c_long, C.c_int, C.c_void_p]
    assert so.caspt2_server_wait(None, 1, 0, None) == -1


def test_options_precision_defaults_and_validation(so):
    """The precision form is opt-in (plain FP64 by default, 7 slices) and bad values are
    rejected before any device work."""
    import paper_1606_01273_gb300 as cp
    o = cp.default_options()
    assert o.precision == cp.FP64 and o.slices == 7
    dims = cp.Dims(2, 2, 2, 4, 1)
    h = C.c_void_p()
    assert o.degen_thresh == 1e-8
    for bad in (dict(precision=7), dict(precision=cp.BF16X, slices=0),
                dict(precision=cp.BF16X, slices=8), dict(degen_thresh=-1.0)):
        ob = cp.default_options(**bad)
        assert cp.lib().caspt2_create(C.byref(h), C.byref(dims), C.byref(ob)) == cp.EINVAL


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    import paper_1606_01273_gb300 as cp
    monkeypatch.setattr(cp, "LIBPATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(cp, "_lib", None)
    with pytest.raises(RuntimeError):
        cp.lib()
