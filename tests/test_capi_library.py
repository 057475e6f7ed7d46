"""CPU checks of the C ABI: libpwl.so builds for sm_103a, loads, exports
every entry point include/pwl.h declares, and the binding declares exactly
those.  Host-only calls (version, workspace sizes, argument validation that
fails before any CUDA call) run without a GPU; nothing launches a kernel."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pwl.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pwl_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1510_02975_gb300 import _build, _capi
    _build.build()
    return _capi.load()


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("pwl_design", "pwl_project", "pwl_table_build", "pwl_eval", "pwl_eval_backward"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_binding_covers_the_header():
    from paper_1510_02975_gb300 import _capi
    assert sorted(_capi.SIGNATURES) == _declared()


def test_exported_symbols_match_nm():
    from paper_1510_02975_gb300 import _build
    import subprocess
    out = subprocess.run(["nm", "-D", "--defined-only", _build.LIB], capture_output=True, text=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if " T " in ln}
    for name in _declared():
        assert name in exported, name


def test_host_only_calls(lib):
    assert lib.pwl_version() == 10000
    assert lib.pwl_design_workspace_size(0, 0) == 0
    w1 = lib.pwl_design_workspace_size(4096, 0)
    w2 = lib.pwl_design_workspace_size(4096, 64 * 4096)
    assert w1 == w2 and w1 >= 8 * (2 * 64 * 4096)
    assert lib.pwl_project_workspace_size(100) >= 16 * 100 + 32 * 101


def test_validation_fails_before_any_cuda_call(lib):
    from paper_1510_02975_gb300 import _capi
    F = _capi.make_func({"kind": "gaussian", "a": 1.0, "b": -1.0, "p": [1, 0, 1]})
    st = lib.pwl_design(ctypes.byref(F), 10, 0, 0, None, None, 0, None)
    assert st == _capi.PWL_EINVAL
    assert b"interval" in lib.pwl_last_error()
    F = _capi.make_func({"kind": "gaussian", "a": -1.0, "b": 1.0, "p": [1, 0, 0]})
    assert lib.pwl_design(ctypes.byref(F), 10, 0, 0, None, None, 0, None) == _capi.PWL_EINVAL
    F = _capi.make_func({"kind": "gaussian", "a": -1.0, "b": 1.0, "p": [1, 0, 1]})
    assert lib.pwl_design(ctypes.byref(F), 0, 0, 0, None, None, 0, None) == _capi.PWL_EINVAL
    assert lib.pwl_design(ctypes.byref(F), 10, 0, 7, None, None, 0, None) == _capi.PWL_EINVAL
    assert lib.pwl_project(ctypes.byref(F), None, 10, 5, 8, 0, None, None, 0, None) == _capi.PWL_EINVAL
    out = ctypes.c_void_p()
    assert lib.pwl_table_build(None, None, 10, 0, 0, ctypes.byref(out), None) == _capi.PWL_EINVAL
    assert lib.pwl_eval(None, None, None, 10, 0, None) == _capi.PWL_EINVAL
    assert lib.pwl_table_destroy(None) == _capi.PWL_OK


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    from paper_1510_02975_gb300 import _capi
    monkeypatch.setattr(_capi, "_lib", None)
    monkeypatch.setattr(_capi, "library_path", lambda: str(tmp_path / "missing.so"))
    with pytest.raises(ImportError):
        _capi.load()


def test_product_path_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_1510_02975_gb300")
    for dirpath, _, files in os.walk(pkg):
        for fn in files:
            if fn.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, fn)).read()
                assert "import oracle" not in text and "from oracle" not in text, fn
                assert "pwl_oracle" not in text, fn
