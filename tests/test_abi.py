"""The C-ABI library loads and exports every entry point declared in include/rcb.h (no GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "rcb.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(rcb_[a-z_]+)\s*\(", src)) - {"rcb_alloc_fn", "rcb_free_fn"})


@pytest.fixture(scope="module")
def libpath():
    import paper_1108_0028_gb300 as rcb
    return rcb.build()


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    names = _declared()
    assert "rcb_build" in names and "rcb_gravity_backward" in names
    for n in names:
        assert hasattr(lib, n), n
    import paper_1108_0028_gb300 as rcb
    assert sorted(rcb.SYMBOLS) == sorted(names)


def test_strerror_and_argument_checks_need_no_gpu(libpath):
    import paper_1108_0028_gb300 as rcb
    lib = rcb.lib()
    assert lib.rcb_strerror(0) == b"ok"
    assert lib.rcb_strerror(-3) == b"output capacity too small"
    p = rcb.rcb_params(12, 1, 0.5, 0, 0)
    h = ctypes.c_void_p(None)
    # null pointers and invalid sizes are rejected on the host before any CUDA call
    assert lib.rcb_build(None, None, None, 10, ctypes.byref(p), None, None, None, None, ctypes.byref(h)) == -1
    bad = rcb.rcb_params(0, 1, 0.5, 0, 0)
    one = ctypes.c_void_p(1)
    assert lib.rcb_build(one, one, one, 10, ctypes.byref(bad), None, None, None, None, ctypes.byref(h)) == -1
    bad = rcb.rcb_params(12, 7, 0.5, 0, 0)
    assert lib.rcb_build(one, one, one, 10, ctypes.byref(bad), None, None, None, None, ctypes.byref(h)) == -1
    bad = rcb.rcb_params(12, 1, -0.1, 0, 0)
    assert lib.rcb_build(one, one, one, 10, ctypes.byref(bad), None, None, None, None, ctypes.byref(h)) == -1
    assert lib.rcb_build(one, one, one, 0, ctypes.byref(p), None, None, None, None, ctypes.byref(h)) == -1
    assert lib.rcb_build(one, one, one, 1 << 31, ctypes.byref(p), None, None, None, None, ctypes.byref(h)) == -1
    # unknown flag bits, and the two alternative splits together, are rejected
    bad = rcb.rcb_params(12, 1, 0.5, 16, 0)
    assert lib.rcb_build(one, one, one, 10, ctypes.byref(bad), None, None, None, None, ctypes.byref(h)) == -1
    bad = rcb.rcb_params(12, 1, 0.5, rcb.RCB_FLAG_CENTRE_OF_NUMBER | rcb.RCB_FLAG_MEDIAN_SPLIT, 0)
    assert lib.rcb_build(one, one, one, 10, ctypes.byref(bad), None, None, None, None, ctypes.byref(h)) == -1
    assert lib.rcb_gravity(None, None, None, None) == -1
    assert lib.rcb_set_precision(None, 0) == -1
    lib.rcb_free(None)


def test_binding_refuses_without_library(tmp_path, monkeypatch):
    import paper_1108_0028_gb300 as rcb
    monkeypatch.setattr(rcb, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(rcb, "_lib", None)
    with pytest.raises(RuntimeError):
        rcb.lib()


def test_flag_values_match_the_header():
    import paper_1108_0028_gb300 as rcb
    src = open(os.path.join(ROOT, "include", "rcb.h")).read()
    found = {k: int(v) for k, v in re.findall(r"#define (RCB_FLAG_[A-Z_]+) (\d+)u", src)}
    assert found == {k: getattr(rcb, k) for k in found}
    assert set(found) == {"RCB_FLAG_TIMING", "RCB_FLAG_CENTRE_OF_NUMBER", "RCB_FLAG_MAC_ONLY", "RCB_FLAG_MEDIAN_SPLIT"}
