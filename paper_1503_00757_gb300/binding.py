"""Thin Python binding of libreg.so (include/reg.h).

Argument marshalling only: every step of the computation runs in the CUDA
kernels behind the C ABI.  Field arguments are torch CUDA float32 tensors
(contiguous, 16-byte aligned); the binding passes their device pointers.
If the library has not been built this module raises on first use; there is
no CPU fallback.
"""
import ctypes
import math
import os

from .build import LIB_PATH

REG_H1, REG_H2, REG_H3 = 1, 2, 3
REG_NT_FIXED, REG_NT_CFL = 0, 1
REG_CONV_MMA_SYNC, REG_CONV_TCGEN05 = 0, 1
REG_NET_INPUT, REG_NET_OUTPUT, REG_NET_OUTPUT_GRAD = 0, 1, 2
STATUS = {0: "REG_OK", 1: "REG_ERR_ARG", 2: "REG_ERR_CUDA", 3: "REG_ERR_NOMEM", 4: "REG_ERR_NAN",
          5: "REG_ERR_LINESEARCH", 6: "REG_ERR_PCG_MAXIT", 7: "REG_ERR_TIMEOUT", 8: "REG_WARN_CFL",
          9: "REG_ERR_STATE", 10: "REG_ERR_MAXIT"}


class reg_grid(ctypes.Structure):
    _fields_ = [("n1", ctypes.c_int), ("n2", ctypes.c_int)]


class reg_solve_opts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("maxit_newton", ctypes.c_int), ("maxit_pcg", ctypes.c_int),
                ("armijo_c1", ctypes.c_double), ("armijo_rho", ctypes.c_double), ("max_ls", ctypes.c_int),
                ("nt_policy", ctypes.c_int), ("cfl_max", ctypes.c_double), ("warm_start", ctypes.c_int)]


class reg_solve_stats(ctypes.Structure):
    _fields_ = [("n_newton", ctypes.c_int), ("n_mv", ctypes.c_int), ("n_pde", ctypes.c_int),
                ("n_ls", ctypes.c_int), ("n_pcg_maxit", ctypes.c_int), ("status", ctypes.c_int),
                ("nt_used", ctypes.c_int), ("cfl_warn", ctypes.c_int), ("J0", ctypes.c_double),
                ("J", ctypes.c_double), ("gnorm_rel", ctypes.c_double), ("rnorm_rel_sq", ctypes.c_double),
                ("cfl", ctypes.c_double)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


class reg_batch_item(ctypes.Structure):
    _fields_ = [("grid", reg_grid), ("nt", ctypes.c_int), ("regnorm", ctypes.c_int), ("beta", ctypes.c_double),
                ("gamma", ctypes.c_double), ("shear", ctypes.c_double), ("mT", ctypes.c_void_p),
                ("mR", ctypes.c_void_p), ("v", ctypes.c_void_p), ("want_detgrad", ctypes.c_int),
                ("stats", reg_solve_stats), ("detgrad", ctypes.c_double * 5), ("status", ctypes.c_int)]


_P = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double
_SIGS = {
    "reg_last_error": ([], ctypes.c_char_p),
    "reg_default_opts": ([ctypes.POINTER(reg_solve_opts)], None),
    "reg_create": ([reg_grid, _I, _I, _D, _D, _D, ctypes.POINTER(_P)], _I),
    "reg_destroy": ([_P], None),
    "reg_set_stream": ([_P, _P], _I),
    "reg_set_images": ([_P, _P, _P], _I),
    "reg_spectral_grad": ([_P, _P, _P], _I),
    "reg_spectral_div": ([_P, _P, _P], _I),
    "reg_apply_reg": ([_P, _P, _P], _I),
    "reg_apply_proj": ([_P, _P, _P], _I),
    "reg_apply_precond": ([_P, _P, _P], _I),
    "reg_apply_precond_sqrt": ([_P, _P, _P, _I], _I),
    "reg_objective": ([_P, _P, _P, ctypes.POINTER(_D)], _I),
    "reg_gradient": ([_P, _P, _P, ctypes.POINTER(_D)], _I),
    "reg_hessian_matvec": ([_P, _P, _P], _I),
    "reg_body_force": ([_P, _P], _I),
    "reg_solve": ([_P, _P, ctypes.POINTER(reg_solve_opts), ctypes.POINTER(reg_solve_stats)], _I),
    "reg_register_host": ([_P, _P, _P, _P, ctypes.POINTER(reg_solve_opts), ctypes.POINTER(reg_solve_stats)], _I),
    "reg_detgrad": ([_P, _P, _P, ctypes.POINTER(_D)], _I),
    "reg_kernel_timing": ([_P, _I], _I),
    "reg_kernel_time": ([_P, _I, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(_D), ctypes.POINTER(_D)], _I),
    "reg_launch_count": ([_P], ctypes.c_longlong),
    "reg_spectral_grad_static": ([reg_grid, _P, _P, _P], _I),
    "reg_set_params": ([_P, _I, _I, _D, _D, _D], _I),
    "reg_solve_batch": ([ctypes.POINTER(reg_batch_item), _I, ctypes.POINTER(reg_solve_opts), _I], _I),
    "reg_executor_create": ([_I, ctypes.POINTER(_P)], _I),
    "reg_executor_solve": ([_P, ctypes.POINTER(reg_batch_item), _I, ctypes.POINTER(reg_solve_opts)], _I),
    "reg_executor_destroy": ([_P], None),
    "reg_autotune": ([reg_grid, _I, _I, _I, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I),
                      ctypes.POINTER(_I), ctypes.POINTER(_D)], _I),
    "reg_tile_config": ([_P, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I)], _I),
    "reg_set_tiles": ([_P, _I, _I, _I], _I),
    "reg_set_pdl": ([_P, _I], _I),
    "reg_set_transport": ([_P, _I], _I),
    "reg_set_hessian": ([_P, _I], _I),
    "reg_displacement": ([_P, _P, _P], _I),
    "reg_label_overlap": ([_P, _P, _P, _P, _P, ctypes.POINTER(_D)], _I),
    "reg_transport_config": ([_P, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I)], _I),
    "reg_fp32_peak": ([ctypes.POINTER(_D), ctypes.POINTER(_D)], _I),
    "reg_net_create": ([_I, _I, _I, ctypes.POINTER(_P)], _I),
    "reg_net_destroy": ([_P], None),
    "reg_net_num_params": ([_P], ctypes.c_longlong),
    "reg_net_set_stream": ([_P, _P], _I),
    "reg_net_set_params": ([_P, _P], _I),
    "reg_net_get_params": ([_P, _P], _I),
    "reg_net_forward": ([_P, _P, _I, _P], _I),
    "reg_net_set_output_scale": ([_P, ctypes.c_float], _I),
    "reg_net_loss_grad": ([_P, _P, _P, _I, ctypes.POINTER(_D), _P], _I),
    "reg_net_train_step": ([_P, _P, _P, _I, ctypes.c_float, ctypes.POINTER(_D)], _I),
    "reg3_create": ([_I, _I, _I, _I, _D, _D, ctypes.POINTER(_P)], _I),
    "reg3_destroy": ([_P], None),
    "reg3_set_stream": ([_P, _P], _I),
    "reg3_set_images": ([_P, _P, _P], _I),
    "reg3_gradient": ([_P, _P, _P, ctypes.POINTER(_D)], _I),
    "reg3_hessian_matvec": ([_P, _P, _P], _I),
    "reg3_solve": ([_P, _P, _D, _I, _I, _P], _I),
    "reg_net_forward_fine": ([_P, _P, _I, _P], _I),
    "reg_net_set_conv_kernel": ([_P, _I], _I),
    "reg_net_set_record": ([_P, _I], _I),
    "reg_net_layer_tensor": ([_P, _I, _I, _I, _P], _I),
}

_lib = None


def lib():
    """Load libreg.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, (args, res) in _SIGS.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _lib = L
    return _lib


class RegError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def _check(st):
    if st != 0:
        raise RegError(st, lib().reg_last_error().decode())
    return st


def _ptr(t, numel=None, name="tensor"):
    if t is None:
        return None
    import torch
    if not isinstance(t, torch.Tensor) or t.device.type != "cuda" or t.dtype != torch.float32:
        raise TypeError(f"{name} must be a CUDA float32 tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{name} has {t.numel()} elements, expected {numel}")
    return ctypes.c_void_p(t.data_ptr())


def default_opts(**kw):
    o = reg_solve_opts()
    lib().reg_default_opts(ctypes.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def spectral_grad_static(f, grad_f, stream=None):
    """Allocation-free spectral gradient (reg_spectral_grad_static): f (n1, n2),
    grad_f (2, n1, n2) CUDA float32 tensors; no context, no device allocation."""
    n1, n2 = f.shape[-2], f.shape[-1]
    handle = None if stream is None else ctypes.c_void_p(stream.cuda_stream)
    _check(lib().reg_spectral_grad_static(reg_grid(n1, n2), _ptr(f, n1 * n2, "f"), _ptr(grad_f, 2 * n1 * n2, "grad_f"),
                                          handle))


def autotune(n1, n2, nt=4, concurrency=1, force=False):
    """FFT tiles and launch mode for an n1 x n2 grid (reg_autotune) timed with `concurrency`
    solves at once: (rows per row CTA, columns per column CTA, prefetch flag, PDL flag,
    ms per matvec of the winner, or -1 if the grid was already tuned)."""
    R, C, P, D, ms = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
    _check(lib().reg_autotune(reg_grid(n1, n2), nt, concurrency, 1 if force else 0, ctypes.byref(R), ctypes.byref(C),
                              ctypes.byref(P), ctypes.byref(D), ctypes.byref(ms)))
    return R.value, C.value, P.value, D.value, ms.value


def fp32_peak():
    """Measured FP32 FMA throughput of the current device (reg_fp32_peak):
    (TFLOP/s, ms per launch of the FMA kernel)."""
    tf, ms = ctypes.c_double(), ctypes.c_double()
    _check(lib().reg_fp32_peak(ctypes.byref(tf), ctypes.byref(ms)))
    return tf.value, ms.value


def _batch_items(pairs):
    n = len(pairs)
    arr = (reg_batch_item * n)()
    for i, p in enumerate(pairs):
        n1, n2 = p["mT"].shape[-2], p["mT"].shape[-1]
        it = arr[i]
        it.grid = reg_grid(n1, n2)
        it.nt, it.regnorm = int(p["nt"]), int(p.get("regnorm", REG_H1))
        it.beta, it.gamma, it.shear = float(p["beta"]), float(p.get("gamma", math.inf)), float(p.get("shear", 0.0))
        it.mT = _ptr(p["mT"], n1 * n2, "mT")
        it.mR = _ptr(p["mR"], n1 * n2, "mR")
        it.v = _ptr(p["v"], 2 * n1 * n2, "v")
        it.want_detgrad = int(p.get("detgrad", 0))
    return arr


def _batch_stats(arr):
    out = []
    for i in range(len(arr)):
        d = arr[i].stats.as_dict()
        d["rc"] = arr[i].status
        if arr[i].want_detgrad:
            d["detgrad"] = tuple(arr[i].detgrad)
        out.append(d)
    return out


class Executor:
    """Persistent batch executor (reg_executor_*): worker streams and per-size
    contexts survive across solve() calls."""

    def __init__(self, nworkers=8):
        h = ctypes.c_void_p()
        _check(lib().reg_executor_create(int(nworkers), ctypes.byref(h)))
        self.h = h

    def solve(self, pairs, opts=None, check=True):
        """Same arguments and results as solve_batch."""
        arr = _batch_items(pairs)
        o = opts if opts is not None else default_opts()
        rc = lib().reg_executor_solve(self.h, arr, len(pairs), ctypes.byref(o))
        if check:
            _check(rc)
        return rc, _batch_stats(arr)

    def close(self):
        if self.h:
            lib().reg_executor_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def solve_batch(pairs, opts=None, nworkers=8, check=True):
    """Batched registration (reg_solve_batch).  pairs: list of dicts with CUDA
    float32 tensors mT (n1, n2), mR (n1, n2), v (2, n1, n2), the problem
    parameters nt, regnorm, beta, gamma, shear and optionally detgrad=1.  v is
    overwritten with each solution.  Returns (status, list of per-pair stats
    dicts, with "detgrad" when requested)."""
    arr = _batch_items(pairs)
    o = opts if opts is not None else default_opts()
    rc = lib().reg_solve_batch(arr, len(pairs), ctypes.byref(o), int(nworkers))
    if check:
        _check(rc)
    return rc, _batch_stats(arr)


class Net:
    """Warm-start network (reg_net_*): H x W images, batches of up to max_batch."""

    def __init__(self, H, W, max_batch, stream=None):
        h = ctypes.c_void_p()
        _check(lib().reg_net_create(H, W, max_batch, ctypes.byref(h)))
        self.h, self.H, self.W = h, H, W
        self.nparams = lib().reg_net_num_params(h)
        if stream is not None:
            _check(lib().reg_net_set_stream(h, ctypes.c_void_p(stream.cuda_stream)))

    def close(self):
        if self.h:
            lib().reg_net_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, p):
        _check(lib().reg_net_set_params(self.h, _ptr(p, self.nparams, "params")))

    def get_params(self, p):
        _check(lib().reg_net_get_params(self.h, _ptr(p, self.nparams, "params")))

    def forward(self, images, v_out):
        B = images.shape[0]
        n = B * 2 * self.H * self.W
        _check(lib().reg_net_forward(self.h, _ptr(images, n, "images"), B, _ptr(v_out, n, "v_out")))

    def forward_fine(self, images, v_out):
        """Warm start for pairs on the doubled grid: images and v_out are B x 2 x 2H x 2W."""
        B = images.shape[0]
        n = B * 2 * 4 * self.H * self.W
        _check(lib().reg_net_forward_fine(self.h, _ptr(images, n, "images"), B, _ptr(v_out, n, "v_out")))

    def set_output_scale(self, scale):
        """reg_net_forward returns scale times the projected prediction (warm-start damping)."""
        _check(lib().reg_net_set_output_scale(self.h, float(scale)))

    def loss_grad(self, images, targets, grads=None):
        B = images.shape[0]
        n = B * 2 * self.H * self.W
        loss = ctypes.c_double()
        _check(lib().reg_net_loss_grad(self.h, _ptr(images, n, "images"), _ptr(targets, n, "targets"), B,
                                       ctypes.byref(loss), _ptr(grads, self.nparams, "grads")))
        return loss.value

    def train_step(self, images, targets, lr):
        B = images.shape[0]
        n = B * 2 * self.H * self.W
        loss = ctypes.c_double()
        _check(lib().reg_net_train_step(self.h, _ptr(images, n, "images"), _ptr(targets, n, "targets"), B,
                                        ctypes.c_float(lr), ctypes.byref(loss)))
        return loss.value


    def set_conv_kernel(self, kind):
        """REG_CONV_TCGEN05 (default) or REG_CONV_MMA_SYNC."""
        _check(lib().reg_net_set_conv_kernel(self.h, int(kind)))

    def set_record(self, on=True):
        _check(lib().reg_net_set_record(self.h, 1 if on else 0))

    def layer_tensor(self, kind, layer, out):
        """Layer tensor of the last pass into out (device, B x C x H x W floats)."""
        _check(lib().reg_net_layer_tensor(self.h, int(kind), int(layer), out.shape[0], _ptr(out, out.numel(), "out")))


class Context3D:
    """One 3-D registration problem (reg3_*): H1 seminorm on an n1 x n2 x n3 periodic box."""

    def __init__(self, n1, n2, n3, nt, beta=1e-2, gamma=math.inf, stream=None):
        h = ctypes.c_void_p()
        _check(lib().reg3_create(n1, n2, n3, nt, float(beta), float(gamma), ctypes.byref(h)))
        self.h, self.N = h, n1 * n2 * n3
        if stream is not None:
            _check(lib().reg3_set_stream(h, ctypes.c_void_p(stream.cuda_stream)))

    def close(self):
        if self.h:
            lib().reg3_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_images(self, mT, mR):
        _check(lib().reg3_set_images(self.h, _ptr(mT, self.N, "mT"), _ptr(mR, self.N, "mR")))

    def gradient(self, v, g_out):
        J = ctypes.c_double()
        _check(lib().reg3_gradient(self.h, _ptr(v, 3 * self.N, "v"), _ptr(g_out, 3 * self.N, "g"), ctypes.byref(J)))
        return J.value

    def hessian_matvec(self, vt, Hvt_out):
        _check(lib().reg3_hessian_matvec(self.h, _ptr(vt, 3 * self.N, "vt"), _ptr(Hvt_out, 3 * self.N, "Hvt")))

    def solve(self, v_out, tol=1e-2, maxit_newton=50, maxit_pcg=100, check=True):
        """Algorithm 1 from v = 0 into v_out; returns the stats as a dict."""
        st = (ctypes.c_double * 7)()
        rc = lib().reg3_solve(self.h, _ptr(v_out, 3 * self.N, "v"), float(tol), int(maxit_newton), int(maxit_pcg),
                              ctypes.cast(st, ctypes.c_void_p))
        if check:
            _check(rc)
        keys = ("n_newton", "n_mv", "n_ls", "gnorm_rel", "J", "status", "J0")
        d = {k: st[i] for i, k in enumerate(keys)}
        for k in ("n_newton", "n_mv", "n_ls", "status"):
            d[k] = int(d[k])
        d["rc"] = rc
        return d


def flatten_params(params):
    """Oracle parameter list [(W, b), ...] -> flat array in the reg_net order."""
    import numpy as np
    return np.concatenate([np.concatenate([W.ravel(), b.ravel()]) for W, b in params])


def unflatten_params(flat, channels):
    import numpy as np
    out, o = [], 0
    for cin, cout in zip(channels[:-1], channels[1:]):
        W = np.asarray(flat[o:o + cout * cin * 9]).reshape(cout, cin, 3, 3)
        o += cout * cin * 9
        b = np.asarray(flat[o:o + cout])
        o += cout
        out.append((W, b))
    return out


class Context:
    """Owns one reg_ctx (one registration problem on one grid)."""

    def __init__(self, n1, n2, nt, regnorm=REG_H1, beta=1e-2, gamma=math.inf, shear=0.0, stream=None):
        self.n1, self.n2, self.N = n1, n2, n1 * n2
        h = ctypes.c_void_p()
        _check(lib().reg_create(reg_grid(n1, n2), nt, regnorm, beta, gamma, shear, ctypes.byref(h)))
        self.h = h
        if stream is not None:
            self.set_stream(stream)

    def close(self):
        if self.h:
            lib().reg_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, nt, regnorm=REG_H1, beta=1e-2, gamma=math.inf, shear=0.0):
        _check(lib().reg_set_params(self.h, nt, regnorm, beta, gamma, shear))

    def set_stream(self, stream):
        """stream: a torch.cuda.Stream (or None for the legacy default stream)."""
        handle = None if stream is None else ctypes.c_void_p(stream.cuda_stream)
        _check(lib().reg_set_stream(self.h, handle))

    def set_images(self, mT, mR):
        _check(lib().reg_set_images(self.h, _ptr(mT, self.N, "mT"), _ptr(mR, self.N, "mR")))

    def spectral_grad(self, f, out):
        _check(lib().reg_spectral_grad(self.h, _ptr(f, self.N), _ptr(out, 2 * self.N)))

    def spectral_div(self, u, out):
        _check(lib().reg_spectral_div(self.h, _ptr(u, 2 * self.N), _ptr(out, self.N)))

    def apply_reg(self, v, out):
        _check(lib().reg_apply_reg(self.h, _ptr(v, 2 * self.N), _ptr(out, 2 * self.N)))

    def apply_proj(self, b, out):
        _check(lib().reg_apply_proj(self.h, _ptr(b, 2 * self.N), _ptr(out, 2 * self.N)))

    def apply_precond(self, r, out):
        _check(lib().reg_apply_precond(self.h, _ptr(r, 2 * self.N), _ptr(out, 2 * self.N)))

    def apply_precond_sqrt(self, x, out, inverse=False):
        _check(lib().reg_apply_precond_sqrt(self.h, _ptr(x, 2 * self.N), _ptr(out, 2 * self.N), 1 if inverse else 0))

    def objective(self, v, m1=None):
        J = ctypes.c_double()
        _check(lib().reg_objective(self.h, _ptr(v, 2 * self.N), _ptr(m1, self.N), ctypes.byref(J)))
        return J.value

    def gradient(self, v, g):
        J = ctypes.c_double()
        _check(lib().reg_gradient(self.h, _ptr(v, 2 * self.N), _ptr(g, 2 * self.N), ctypes.byref(J)))
        return J.value

    def hessian_matvec(self, vt, Hvt):
        _check(lib().reg_hessian_matvec(self.h, _ptr(vt, 2 * self.N), _ptr(Hvt, 2 * self.N)))

    def body_force(self, b):
        """Body force of the last gradient or incremental body force of the last matvec (before K)."""
        _check(lib().reg_body_force(self.h, _ptr(b, 2 * self.N)))

    def solve(self, v, opts=None, check=True):
        """Newton-Krylov solve; v (2, n1, n2) is overwritten.  Returns the stats dict."""
        st = reg_solve_stats()
        o = opts if opts is not None else default_opts()
        rc = lib().reg_solve(self.h, _ptr(v, 2 * self.N, "v"), ctypes.byref(o), ctypes.byref(st))
        if check:
            _check(rc)
        d = st.as_dict()
        d["rc"] = rc
        return d

    def register_host(self, mT_host, mR_host, v_host, opts=None, check=True):
        """Solve from host float32 buffers (numpy arrays or pinned CPU tensors)."""
        import numpy as np

        def hptr(a, n, writable=False):
            if hasattr(a, "data_ptr"):
                if a.device.type != "cpu" or a.dtype.__str__() != "torch.float32" or not a.is_contiguous():
                    raise TypeError("host buffers must be contiguous CPU float32")
                if a.numel() != n:
                    raise ValueError("bad host buffer size")
                return ctypes.c_void_p(a.data_ptr())
            if not (isinstance(a, np.ndarray) and a.dtype == np.float32 and a.flags["C_CONTIGUOUS"]):
                raise TypeError("host buffers must be contiguous float32")
            if a.size != n:
                raise ValueError("bad host buffer size")
            return ctypes.c_void_p(a.ctypes.data)

        st = reg_solve_stats()
        o = opts if opts is not None else default_opts()
        rc = lib().reg_register_host(self.h, hptr(mT_host, self.N), hptr(mR_host, self.N),
                                     hptr(v_host, 2 * self.N, True), ctypes.byref(o), ctypes.byref(st))
        if check:
            _check(rc)
        d = st.as_dict()
        d["rc"] = rc
        return d

    def detgrad(self, v, detF=None):
        """Returns (min det F1, mean det F1, max det F1, max D, mean D)."""
        stats = (ctypes.c_double * 5)()
        _check(lib().reg_detgrad(self.h, _ptr(v, 2 * self.N), _ptr(detF, self.N), stats))
        return tuple(stats)

    def kernel_timing(self, enable):
        _check(lib().reg_kernel_timing(self.h, int(enable)))

    def kernel_time(self, kclass):
        """(launches, milliseconds, algorithmic bytes) of kernel class kclass since timing was enabled."""
        n = ctypes.c_longlong()
        ms = ctypes.c_double()
        by = ctypes.c_double()
        _check(lib().reg_kernel_time(self.h, kclass, ctypes.byref(n), ctypes.byref(ms), ctypes.byref(by)))
        return n.value, ms.value, by.value

    def launch_count(self):
        return lib().reg_launch_count(self.h)

    def tile_config(self):
        """(rows per row-kernel CTA, spectrum columns per column-kernel CTA, prefetch flag, PDL flag)
        of this context."""
        R, C, P, D = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(lib().reg_tile_config(self.h, ctypes.byref(R), ctypes.byref(C), ctypes.byref(P), ctypes.byref(D)))
        return R.value, C.value, P.value, D.value

    def set_pdl(self, enable):
        """Programmatic dependent launch on (default) or off for this context's kernels."""
        _check(lib().reg_set_pdl(self.h, 1 if enable else 0))

    def set_tiles(self, R, C, P=0):
        """Launch with R rows per row-kernel CTA, C spectrum columns per column-kernel CTA and
        operand prefetch P in the RK2 row kernels (R = C = 0: default rule)."""
        _check(lib().reg_set_tiles(self.h, R, C, P))

    def set_transport(self, cluster):
        """Transport solves in the cluster-resident kernel (True) or the row/column kernel pairs (False)."""
        _check(lib().reg_set_transport(self.h, 1 if cluster else 0))

    def transport_config(self):
        """(cluster path in use, CTAs per cluster, clusters that fit on the device at once)."""
        a, b, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(lib().reg_transport_config(self.h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
        return a.value, b.value, c.value

    def set_hessian(self, full):
        """Full Newton Hessian (True) or Gauss-Newton (False, default) for matvecs and solves."""
        _check(lib().reg_set_hessian(self.h, 1 if full else 0))

    def displacement(self, v, u_out):
        """Displacement u_1 of the flow of v (the deformation map is y = x - u_1)."""
        _check(lib().reg_displacement(self.h, _ptr(v, 2 * self.N, "v"), _ptr(u_out, 2 * self.N, "u_out")))

    def label_overlap(self, v, labels_T, labels_R, transported=None):
        """(Jaccard, Dice, false positive error, false negative error) of the template labels
        transported with v against the reference labels; transported (optional) receives the
        smoothed, transported template labels before the threshold."""
        out = (ctypes.c_double * 4)()
        _check(lib().reg_label_overlap(self.h, _ptr(v, 2 * self.N, "v"), _ptr(labels_T, self.N, "labels_T"),
                                       _ptr(labels_R, self.N, "labels_R"), _ptr(transported, self.N, "transported"),
                                       out))
        return tuple(out)
