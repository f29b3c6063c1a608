"""The C-ABI library loads and exports every function include/ib.h declares.

CPU only: no compute call is made.  On a machine without a usable sm_103a
device, ib_create must fail loudly (IB_ERR_CUDA) rather than fall back.
"""
import ctypes as C

import pytest

from paper_math_0301321_gb300 import binding, build


@pytest.fixture(scope="module")
def lib():
    build.build()
    return binding.load()


def test_header_declares_the_boundary():
    names = binding.header_functions()
    for want in ("ib_create", "ib_set_structure", "ib_set_state", "ib_get_state", "ib_step", "ib_spread",
                 "ib_interp", "ib_fluid_solve", "ib_adjoint_step", "ib_bin_sort", "ib_get_bin_order", "ib_get_mean_velocity", "ib_sync", "ib_destroy",
                 "ib_last_error", "ib_info"):
        assert want in names


def test_library_exports_every_declared_symbol(lib):
    for name in binding.header_functions():
        assert hasattr(lib, name), name


def test_create_rejects_bad_arguments_without_touching_the_gpu(lib):
    d = binding.ib_grid_desc((C.c_int32 * 3)(33, 32, 32), 1 / 32, 1.0, 0.02, 1e-5, binding.IB_FP32, None, 0)
    h = C.c_void_p()
    assert lib.ib_create(C.byref(d), C.byref(h)) == binding.IB_ERR_UNSUPPORTED
    assert b"33" in lib.ib_last_error()
    d = binding.ib_grid_desc((C.c_int32 * 3)(32, 32, 32), -1.0, 1.0, 0.02, 1e-5, binding.IB_FP32, None, 0)
    assert lib.ib_create(C.byref(d), C.byref(h)) == binding.IB_ERR_ARG
    assert lib.ib_create(None, C.byref(h)) == binding.IB_ERR_ARG
    assert lib.ib_destroy(None) == binding.IB_OK


def test_create_fails_loudly_without_a_device(lib):
    from conftest import cuda_available
    if cuda_available():
        pytest.skip("a CUDA device is present")
    d = binding.ib_grid_desc((C.c_int32 * 3)(32, 32, 32), 1 / 32, 1.0, 0.02, 1e-5, binding.IB_FP32, None, 0)
    h = C.c_void_p()
    assert lib.ib_create(C.byref(d), C.byref(h)) == binding.IB_ERR_CUDA
    assert not h.value
