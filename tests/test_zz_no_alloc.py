"""The allocation-free spectral gradient (reg_spectral_grad_static), called
through the C ABI, must agree with the context-based reg_spectral_grad on two
calls in a row (the second call reuses the scratch the first one left behind).
Kept in a file of its own that pytest collects last."""
import ctypes

import numpy as np
import pytest

from paper_1503_00757_gb300 import synth

pytestmark = pytest.mark.gpu

OP_TOL = 1e-5


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_static_gradient_matches_context_gradient_twice(torch_cuda):
    torch = torch_cuda
    from paper_1503_00757_gb300.binding import Context, lib, reg_grid

    L = lib()
    for call, (n1, n2, seed) in enumerate([(256, 256, 11), (64, 128, 12)]):
        f_np = synth.smooth_field(n1, n2, min(n1, n2) // 4, np.random.default_rng(seed), decay=0.5)
        f = torch.tensor(f_np, dtype=torch.float32, device="cuda")
        ref = torch.empty(2, n1, n2, device="cuda")
        ctx = Context(n1, n2, 1)
        ctx.spectral_grad(f, ref)
        out = torch.full((2, n1, n2), float("nan"), device="cuda")
        rc = L.reg_spectral_grad_static(reg_grid(n1, n2), ctypes.c_void_p(f.data_ptr()),
                                        ctypes.c_void_p(out.data_ptr()), None)
        assert rc == 0, L.reg_last_error()
        torch.cuda.synchronize()
        a, b = out.cpu().numpy().astype(np.float64), ref.cpu().numpy().astype(np.float64)
        assert np.isfinite(a).all()
        assert _rel(a, b) < OP_TOL, (call, _rel(a, b))
        ctx.close()


def test_static_gradient_rejects_grids_beyond_the_scratch(torch_cuda):
    torch = torch_cuda
    from paper_1503_00757_gb300.binding import lib, reg_grid

    L = lib()
    f = torch.zeros(1024, 1024, device="cuda")
    out = torch.zeros(2, 1024, 1024, device="cuda")
    rc = L.reg_spectral_grad_static(reg_grid(1024, 1024), ctypes.c_void_p(f.data_ptr()),
                                    ctypes.c_void_p(out.data_ptr()), None)
    assert rc == 1
    assert b"scratch" in L.reg_last_error()


_FIRST_CALL_ON_NONBLOCKING_STREAM = r"""
import ctypes, sys
import numpy as np
import torch
sys.path.insert(0, sys.argv[1])
from paper_1503_00757_gb300 import synth
from paper_1503_00757_gb300.binding import Context, lib, reg_grid
L = lib()
n1 = n2 = 128
f_np = synth.smooth_field(n1, n2, 32, np.random.default_rng(5), decay=0.5)
s = torch.cuda.Stream()  # torch creates its pool streams with cudaStreamNonBlocking
with torch.cuda.stream(s):
    f = torch.tensor(f_np, dtype=torch.float32, device="cuda")
    out = torch.full((2, n1, n2), float("nan"), device="cuda")
s.synchronize()
# the first call of the process on this device: its set-up, then kernels on the non-blocking stream
rc = L.reg_spectral_grad_static(reg_grid(n1, n2), ctypes.c_void_p(f.data_ptr()),
                                ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(s.cuda_stream))
assert rc == 0, L.reg_last_error()
s.synchronize()
ref = torch.empty(2, n1, n2, device="cuda")
ctx = Context(n1, n2, 1)
ctx.spectral_grad(f, ref)
torch.cuda.synchronize()
a, b = out.cpu().numpy().astype(np.float64), ref.cpu().numpy().astype(np.float64)
err = float(np.linalg.norm(a - b) / np.linalg.norm(b))
assert np.isfinite(a).all() and err < 1e-5, err
print("ok", err)
"""


def test_first_call_of_a_process_on_a_nonblocking_stream(torch_cuda):
    """In a fresh process (so that this is the device's first call and runs its set-up),
    the first call is issued on a cudaStreamNonBlocking stream: its kernels must see the
    twiddle table that the set-up uploaded."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", _FIRST_CALL_ON_NONBLOCKING_STREAM, root],
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.strip().startswith("ok")
