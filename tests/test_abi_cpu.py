"""C-ABI checks that need no GPU: the library builds, loads, exports every
function include/*.h declares, and rejects bad arguments on the host before
touching the device."""
import ctypes
import os

import pytest

from util import header_functions

import paper_1612_09001_gb300 as dpd
from paper_1612_09001_gb300 import _lib, build


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(build.LIB_PATH):
        build.build()
    return _lib.load()


def test_every_declared_function_is_exported(lib):
    names = header_functions()
    assert len(names) >= 8
    for n in names:
        assert hasattr(lib, n), f"{n} declared in include/ but not exported"


def test_binding_covers_header():
    assert set(header_functions()) == set(_lib.SIGNATURES)


def test_cpu_library_exports_its_header():
    from paper_1612_09001_gb300 import cpu
    build.build_cpu()
    names = header_functions("dpd_cpu.h")
    assert set(names) == {"dpd_cpu_apply", "dpd_cpu_max_threads"}
    lib = cpu.load()
    for n in names:
        assert hasattr(lib, n), f"{n} declared in include/dpd_cpu.h but not exported"


def test_status_strings(lib):
    for code, name in _lib.STATUS.items():
        assert lib.dpd_status_string(code).decode() == name


def test_create_rejects_bad_models(lib):
    h = ctypes.c_void_p()
    # even orders (the paper's order sets are odd, Sec. 2.1) and models past the
    # built range are unsupported (2); negative values and no branch at all are
    # invalid (1)
    for P, Q, M in [(2, 1, 1), (1, 4, 0), (13, 1, 1), (1, 1, 8), (12, 0, 0)]:
        assert lib.dpd_create(P, Q, M, ctypes.byref(h)) == 2, (P, Q, M)
    for P, Q, M in [(0, 0, 1), (1, 1, -1), (-1, 1, 0), (1, -3, 0)]:
        assert lib.dpd_create(P, Q, M, ctypes.byref(h)) == 1, (P, Q, M)
    assert lib.dpd_create(5, 5, 2, None) == 1


def test_null_handle_calls(lib):
    assert lib.dpd_destroy(None) == 0
    k = ctypes.c_int()
    assert lib.dpd_num_coeffs(None, ctypes.byref(k)) == 1
    assert lib.dpd_apply(None, None, None, 10, None) == 1
    assert lib.dpd_set_coeffs(None, None, 3, 0, None) == 1
    assert lib.dpd_sync_status(None, None) == 1
    assert lib.dpd_set_fwd_launch(None, 0, 4, 8, 4, 0, 1, 0) == 1


def test_num_coeffs_formula():
    assert dpd.num_coeffs(9, 9, 4) == 51
    assert dpd.num_coeffs(11, 11, 7) == 97
    assert dpd.num_coeffs(5, 3, 4) == 26
    assert dpd.num_coeffs(7, 0, 3) == 17


def test_launch_counter_starts_at_zero_without_gpu(lib):
    assert lib.dpd_kernel_launches() >= 0
