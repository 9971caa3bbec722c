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
        (reg_grid(64, 64), 4, 3, 1e-2, math.inf, 0.0),    # bad norm
        (reg_grid(64, 64), 4, 1, 0.0, math.inf, 0.0),     # beta <= 0
        (reg_grid(64, 64), 4, 1, 1e-2, -1.0, 0.0),        # gamma < 0
        (reg_grid(64, 64), 4, 1, 1e-2, math.inf, 1.0),    # shear out of range
        (reg_grid(64, 64), 4, 2, 1e-2, math.inf, 0.5),    # shear needs H1
        (reg_grid(64, 64), 4, 1, 1e-2, 1e-3, 0.5),        # shear needs w = 0
    ]
    for args in bad:
        assert lib.reg_create(*args, ctypes.byref(h)) == 1
        assert not h.value
    assert lib.reg_last_error()
