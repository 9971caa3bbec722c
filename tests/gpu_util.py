"""Helpers shared by the GPU parity tests (marshalling and error records only)."""
import json
import math
import os

import numpy as np

# Every parity check made through ``check`` is recorded here (quantity, measured error,
# tolerance, and the conditioning factor where the tolerance carries one); conftest writes
# the list to the file named by REG_PARITY_LOG at the end of the session.
RECORDS = []


def dev():
    import torch
    return torch.device("cuda:0")


def to_gpu(a):
    import torch
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float32, device=dev())


def to_np(t):
    return t.detach().cpu().numpy().astype(np.float64)


def rel_l2(a, b):
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(np.asarray(a, dtype=np.float64) - b) / max(np.linalg.norm(b), 1e-300))


def check(quantity, err, tol, **extra):
    """Assert err < tol and keep the pair for the error-vs-FP64 table."""
    test = os.environ.get("PYTEST_CURRENT_TEST", "").split(" ")[0]
    rec = {"test": test, "quantity": quantity, "err": float(err), "tol": float(tol)}
    rec.update({k: (float(v) if isinstance(v, (int, float, np.floating)) else v) for k, v in extra.items()})
    RECORDS.append(rec)
    assert err < tol, f"{quantity}: error {err:.3e} is not below the tolerance {tol:.3e}"


def check_rel(quantity, got, ref, tol, **extra):
    """Relative L2 error of got against the FP64 reference, checked and recorded."""
    e = rel_l2(got, ref)
    check(quantity, e, tol, **extra)
    return e


def write_records(path):
    with open(path, "w") as f:
        json.dump(RECORDS, f, indent=1)


def make_ctx(n1, n2, nt, regnorm=1, beta=1e-2, gamma=math.inf, shear=0.0):
    from paper_1503_00757_gb300.binding import Context
    return Context(n1, n2, nt, regnorm=regnorm, beta=beta, gamma=gamma, shear=shear)
