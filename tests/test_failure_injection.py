"""Failure detection without a GPU fault (CPU part): the device-allocation
hook of the library makes the calls that allocate fail with PWL_ENOMEM.
No device is needed: the hook refuses the allocation before any CUDA call
that could succeed, and the calls must return cleanly with a NULL handle."""
import ctypes

import pytest

PWL_OK, PWL_EINVAL, PWL_ENOMEM = 0, 1, 2


@pytest.fixture(scope="module")
def lib():
    from paper_1510_02975_gb300 import _build, _capi
    _build.build()
    return _capi.load()


def _func(kind=0):
    from paper_1510_02975_gb300 import _capi
    return _capi.make_func({"kind": ["gaussian", "lorentzian", "bessel_j0"][kind], "a": -4.0, "b": 4.0,
                            "p": [1.0, 0.0, 1.0] if kind < 2 else [1.0, 1.0]})


def test_table_build_reports_enomem_and_returns_no_handle(lib):
    fake = ctypes.c_void_p(0x10000)  # never dereferenced: the first allocation fails
    out = ctypes.c_void_p(0x1234)
    try:
        assert lib.pwl_test_fail_allocations(0) == PWL_OK
        st = lib.pwl_table_build(fake, fake, 64, 0, 0, ctypes.byref(out), None)
        assert st == PWL_ENOMEM
        assert out.value is None
        assert b"cudaMalloc(table)" in lib.pwl_last_error()
    finally:
        lib.pwl_test_fail_allocations(-1)


def test_batch_create_reports_enomem_and_returns_no_handle(lib):
    from paper_1510_02975_gb300 import _capi
    funcs = (_capi.PwlFunc * 3)(_func(0), _func(1), _func(2))
    ns = (ctypes.c_int64 * 3)(16, 100, 1000)
    out = ctypes.c_void_p(0x1234)
    try:
        lib.pwl_test_fail_allocations(0)
        st = lib.pwl_batch_create(funcs, ns, 3, 0, 0, ctypes.byref(out))
        assert st == PWL_ENOMEM
        assert not out.value
    finally:
        lib.pwl_test_fail_allocations(-1)


def test_argument_errors_come_before_allocation(lib):
    # validation fails first: the hook is never consulted
    out = ctypes.c_void_p()
    try:
        lib.pwl_test_fail_allocations(0)
        assert lib.pwl_table_build(None, None, 64, 0, 0, ctypes.byref(out), None) == PWL_EINVAL
        assert lib.pwl_batch_inject_wait_timeout(None, 1, 1000) == PWL_EINVAL
    finally:
        lib.pwl_test_fail_allocations(-1)
