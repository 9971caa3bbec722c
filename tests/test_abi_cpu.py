"""CPU-side checks of the C ABI: the library builds, loads, exports every
function include/reg.h declares, and rejects invalid arguments before any
CUDA call (no GPU needed)."""
import ctypes
import math
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1503_00757_gb300 import build as b
    if not os.path.exists(b.LIB_PATH):
        b.build()
    from paper_1503_00757_gb300.binding import lib as load
    return load()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "reg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(reg_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ["reg_create", "reg_gradient", "reg_hessian_matvec", "reg_solve", "reg_detgrad",
                 "reg_destroy", "reg_set_images", "reg_set_stream"]:
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_invalid_arguments_rejected_without_gpu(lib):
    from paper_1503_00757_gb300.binding import reg_grid
    h = ctypes.c_void_p()
    bad = [
        (reg_grid(48, 64), 4, 1, 1e-2, math.inf, 0.0),    # not a power of two
        (reg_grid(8, 64), 4, 1, 1e-2, math.inf, 0.0),     # below 16
        (reg_grid(2048, 64), 4, 1, 1e-2, math.inf, 0.0),  # above 1024
        (reg_grid(64, 64), 0, 1, 1e-2, math.inf, 0.0),    # nt < 1
        (reg_grid(64, 64), 4, 4, 1e-2, math.inf, 0.0),    # bad norm (H1, H2, H3 only)
        (reg_grid(64, 64), 4, 1, 0.0, math.inf, 0.0),     # beta <= 0
        (reg_grid(64, 64), 4, 1, 1e-2, -1.0, 0.0),        # gamma < 0
        (reg_grid(64, 64), 4, 1, 1e-2, math.inf, 1.0),    # shear out of range
        (reg_grid(64, 64), 4, 2, 1e-2, math.inf, 0.5),    # shear needs H1
        (reg_grid(64, 64), 4, 1, -1e-3, 1e-3, 0.5),       # beta_v must be positive
    ]
    for args in bad:
        assert lib.reg_create(*args, ctypes.byref(h)) == 1
        assert not h.value
    assert lib.reg_last_error()


def test_new_entry_points_reject_invalid_arguments_without_gpu(lib):
    from paper_1503_00757_gb300.binding import reg_grid
    h = ctypes.c_void_p()
    # warm-start network: sizes must be powers of two in [32, 1024], batch in [1, 256]
    assert lib.reg_net_create(48, 64, 4, ctypes.byref(h)) == 1
    assert lib.reg_net_create(64, 64, 0, ctypes.byref(h)) == 1
    assert lib.reg_net_create(2048, 64, 4, ctypes.byref(h)) == 1
    # batch executor: at most 256 workers
    assert lib.reg_executor_create(1000, ctypes.byref(h)) == 1
    assert lib.reg_solve_batch(None, -1, None, 1) == 1
    # allocation-free gradient: scratch limit of 512 x 512 nodes
    assert lib.reg_spectral_grad_static(reg_grid(1024, 512), None, None, None) == 1
    assert b"scratch" in lib.reg_last_error()
    assert lib.reg_spectral_grad_static(reg_grid(12, 16), None, None, None) == 1
    # autotuner: grid and nt checked before any CUDA call
    R, C, P, ms = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
    assert lib.reg_autotune(reg_grid(96, 64), 4, 1, 0, ctypes.byref(R), ctypes.byref(C), ctypes.byref(P), None,
                            ctypes.byref(ms)) == 1
    assert lib.reg_autotune(reg_grid(64, 64), 0, 1, 0, None, None, None, None, None) == 1
    # FP32 peak: the output pointer is checked before any CUDA call
    assert lib.reg_fp32_peak(None, None) == 1
    assert lib.reg_autotune(reg_grid(64, 64), 4, 17, 0, None, None, None, None, None) == 1
    assert lib.reg_tile_config(None, ctypes.byref(R), ctypes.byref(C), ctypes.byref(P), None) == 1
    assert lib.reg_set_tiles(None, 4, 2, 0) == 1
    assert lib.reg_net_set_output_scale(None, ctypes.c_float(1.0)) == 1
    assert lib.reg_set_pdl(None, 1) == 1


def test_network_entry_points_reject_invalid_arguments_without_gpu(lib):
    """The tensor-core network's entry points check their arguments before any CUDA call."""
    f = ctypes.c_float()
    assert lib.reg_net_set_conv_kernel(None, 1) == 1
    assert lib.reg_net_set_record(None, 1) == 1
    assert lib.reg_net_layer_tensor(None, 0, 0, 1, ctypes.byref(f)) == 1
    assert lib.reg_net_forward_fine(None, ctypes.byref(f), 1, ctypes.byref(f)) == 1
    assert b"NULL" in lib.reg_last_error()


def test_3d_entry_points_reject_invalid_arguments_without_gpu(lib):
    """reg3_* validate sizes and pointers before any CUDA call."""
    h = ctypes.c_void_p()
    inf = float("inf")
    assert lib.reg3_create(12, 16, 16, 4, 1e-2, inf, ctypes.byref(h)) == 1   # not a power of two
    assert lib.reg3_create(16, 16, 512, 4, 1e-2, inf, ctypes.byref(h)) == 1  # axis above 256
    assert lib.reg3_create(16, 16, 16, 0, 1e-2, inf, ctypes.byref(h)) == 1   # nt
    assert lib.reg3_create(16, 16, 16, 4, 0.0, inf, ctypes.byref(h)) == 1    # beta
    assert lib.reg3_create(16, 16, 16, 4, 1e-2, -1.0, ctypes.byref(h)) == 1  # gamma
    assert lib.reg3_gradient(None, None, None, None) == 1
    assert lib.reg3_hessian_matvec(None, None, None) == 1
    assert lib.reg3_set_images(None, None, None) == 1
    assert lib.reg3_solve(None, None, 1e-2, 10, 10, None) == 1
