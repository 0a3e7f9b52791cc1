"""Thin Python binding of libgpsparse (C ABI in include/gpsparse.h).

Argument marshalling only: every step of assembly, solve, log-determinant and
gradient runs in the CUDA kernels of the library.  Arrays may be torch tensors
on the GPU (passed as device pointers, ordered on the current torch stream) or
host arrays (torch CPU tensors / numpy), which the library copies itself.

The library must have been built (``paper_2205_09070_gb300.build.build()``);
there is no fallback of any kind when it is missing.
"""

from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

from . import build as _build

GP_OK = 0
GP_ERR_INVALID_ARG = 1
GP_ERR_CUDA = 2
GP_ERR_OOM = 3
GP_ERR_NOT_CONVERGED = 4
GP_ERR_NOT_SPD = 5
GP_ERR_TIMEOUT = 6
GP_ERR_NOT_ASSEMBLED = 7
GP_ERR_UNSUPPORTED = 8

GP_FP64 = 0
GP_FP32_MIXED = 1

GP_FLAG_TIME_KERNELS = 1
GP_FLAG_SPMM_CPASYNC = 2
GP_FLAG_SPMM_TMA = 4
GP_FLAG_SPMM_TMA_WIDE = 8
GP_FLAG_LOGDET_TAYLOR = 16
GP_FLAG_SPMM_CPASYNC_WIDE = 32
GP_FLAG_SPMM_WINDOW = 64
GP_FLAG_FAULT_OOM = 128
GP_FLAG_FAULT_NOT_SPD = 256
GP_FLAG_FAULT_NAN = 512
GP_FLAG_BATCH_STREAMS = 1024

GP_SPMM_CPASYNC = 0
GP_SPMM_TMA = 1
GP_SPMM_TMA_WIDE = 2
GP_SPMM_CPASYNC_WIDE = 3
GP_SPMM_WINDOW = 4
SPMM_FLAGS = {"cpasync": GP_FLAG_SPMM_CPASYNC, "tma": GP_FLAG_SPMM_TMA, "tma_wide": GP_FLAG_SPMM_TMA_WIDE,
              "cpasync_wide": GP_FLAG_SPMM_CPASYNC_WIDE, "window": GP_FLAG_SPMM_WINDOW}

EXPORTED = ["gp_n_params", "gp_default_opts", "gp_create", "gp_destroy", "gp_set_stream", "gp_assemble",
            "gp_get_csr", "gp_get_csr_noalloc", "gp_solve", "gp_predict", "gp_lml", "gp_lml_grad",
            "gp_lml_grad_batched", "gp_status_string", "gp_sparsity_estimate", "gp_augmented", "gp_predict_var",
            "gp_train"]

GP_OBJ_LML = 0
GP_OBJ_AUGMENTED = 1
GP_OBJ_CONSTRAINED = 2
OBJECTIVES = {"lml": GP_OBJ_LML, "augmented": GP_OBJ_AUGMENTED, "constrained": GP_OBJ_CONSTRAINED}


GP_CORE_NONE = 0
GP_CORE_SQEXP = 1


class KernelDesc(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int32), ("n_funcs", ctypes.c_int32), ("n_bumps", ctypes.c_int32),
                ("beta", ctypes.c_double), ("core", ctypes.c_int32)]


class TrainOpts(ctypes.Structure):
    _fields_ = [("objective", ctypes.c_int32), ("n_steps", ctypes.c_int32), ("lr", ctypes.c_double),
                ("beta1", ctypes.c_double), ("beta2", ctypes.c_double), ("eps", ctypes.c_double),
                ("domain_volume", ctypes.c_double), ("s_max", ctypes.c_double), ("max_halvings", ctypes.c_int32)]


class Opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("n_probes", ctypes.c_int32), ("lanczos_steps", ctypes.c_int32),
                ("max_iter", ctypes.c_int32), ("cg_rtol", ctypes.c_double), ("seed", ctypes.c_uint64),
                ("check_every", ctypes.c_int32), ("flags", ctypes.c_int32), ("precond_block", ctypes.c_int32),
                ("batch_workers", ctypes.c_int32)]


class Info(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("n_active", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("iters", ctypes.c_int32), ("status_detail", ctypes.c_int32), ("max_rel_resid", ctypes.c_double),
                ("quad_form", ctypes.c_double), ("logdet", ctypes.c_double), ("logdet_stderr", ctypes.c_double),
                ("t_assemble_ms", ctypes.c_double), ("t_solve_ms", ctypes.c_double),
                ("t_grad_ms", ctypes.c_double), ("cell_size", ctypes.c_double), ("n_cells", ctypes.c_int64),
                ("launches", ctypes.c_int64), ("n_spmm", ctypes.c_int32), ("kp", ctypes.c_int32),
                ("t_spmm_kernel_ms", ctypes.c_double), ("t_fill_kernel_ms", ctypes.c_double),
                ("t_adjoint_kernel_ms", ctypes.c_double), ("lanczos_iters", ctypes.c_int32),
                ("precond_block", ctypes.c_int32), ("spmm_variant", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class GPError(RuntimeError):
    def __init__(self, status: int, where: str):
        super().__init__(f"{where}: {status_string(status)} (status {status})")
        self.status = status


_LIB = None


def library_path() -> str:
    return _build.LIB


def load(path: str | None = None) -> ctypes.CDLL:
    """Load libgpsparse.so (raises if it has not been built)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = path or library_path()
    if not os.path.exists(path):
        raise RuntimeError(f"libgpsparse.so not found at {path}: build it with "
                           "paper_2205_09070_gb300.build.build() (nvcc, sm_103a)")
    lib = ctypes.CDLL(path)
    vp, i64, i32, dp = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p
    lib.gp_n_params.argtypes = [ctypes.POINTER(KernelDesc)]
    lib.gp_n_params.restype = i64
    lib.gp_default_opts.argtypes = [ctypes.POINTER(Opts)]
    lib.gp_default_opts.restype = None
    lib.gp_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(KernelDesc), ctypes.c_int, vp]
    lib.gp_destroy.argtypes = [vp]
    lib.gp_set_stream.argtypes = [vp, vp]
    lib.gp_assemble.argtypes = [vp, dp, i64, dp, ctypes.POINTER(Opts), ctypes.POINTER(Info)]
    lib.gp_get_csr.argtypes = [vp, dp, dp, dp, dp, ctypes.POINTER(i64)]
    lib.gp_get_csr_noalloc.argtypes = [vp, dp, dp, dp, dp, ctypes.POINTER(i64)]
    lib.gp_solve.argtypes = [vp, dp, dp, ctypes.POINTER(Opts), ctypes.POINTER(Info)]
    lib.gp_predict.argtypes = [vp, dp, dp, i64, dp, ctypes.POINTER(Opts), ctypes.POINTER(Info)]
    lib.gp_predict_var.argtypes = [vp, dp, i64, dp, ctypes.POINTER(Opts), ctypes.POINTER(Info)]
    lib.gp_lml.argtypes = [vp, dp, dp, i64, dp, ctypes.POINTER(Opts), ctypes.POINTER(ctypes.c_double),
                           ctypes.POINTER(Info)]
    lib.gp_lml_grad.argtypes = [vp, dp, dp, i64, dp, ctypes.POINTER(Opts), ctypes.POINTER(ctypes.c_double), dp,
                                ctypes.POINTER(Info)]
    lib.gp_lml_grad_batched.argtypes = [vp, i32, dp, dp, dp, dp, ctypes.POINTER(Opts), dp, dp,
                                        ctypes.POINTER(Info)]
    lib.gp_sparsity_estimate.argtypes = [ctypes.POINTER(KernelDesc), dp, ctypes.c_double, dp, dp]
    lib.gp_augmented.argtypes = [ctypes.POINTER(KernelDesc), dp, ctypes.c_double, ctypes.c_double, dp, dp, dp, dp]
    lib.gp_train.argtypes = [vp, dp, dp, i64, dp, ctypes.POINTER(Opts), ctypes.POINTER(TrainOpts), dp,
                             ctypes.POINTER(Info)]
    lib.gp_status_string.argtypes = [ctypes.c_int]
    lib.gp_status_string.restype = ctypes.c_char_p
    for name in ("gp_create", "gp_destroy", "gp_set_stream", "gp_assemble", "gp_get_csr", "gp_get_csr_noalloc",
                 "gp_solve", "gp_predict", "gp_predict_var", "gp_lml", "gp_sparsity_estimate", "gp_augmented",
                 "gp_lml_grad", "gp_lml_grad_batched"):
        getattr(lib, name).restype = ctypes.c_int
    _LIB = lib
    return lib


def status_string(status: int) -> str:
    return load().gp_status_string(status).decode()


def sparsity_estimate(dim: int, n_funcs: int, n_bumps: int, h, domain_volume: float, beta: float = 1.0,
                      core: int = GP_CORE_NONE):
    """(s, d s / d h): the sparsity bound of the paper's kernel (host-side)."""
    d = KernelDesc(dim, n_funcs, n_bumps, beta, core)
    hh = np.ascontiguousarray(h, dtype=np.float64)
    s = ctypes.c_double()
    g = np.zeros(hh.shape[0], np.float64)
    st = load().gp_sparsity_estimate(ctypes.byref(d), hh.ctypes.data, float(domain_volume), ctypes.byref(s),
                                     g.ctypes.data)
    if st != GP_OK:
        raise GPError(st, "gp_sparsity_estimate")
    return s.value, g


def augmented_objective(dim: int, n_funcs: int, n_bumps: int, h, domain_volume: float, lml: float, lml_grad,
                        beta: float = 1.0, core: int = GP_CORE_NONE):
    """(value, gradient, s) of (2 - s(h)) ln L(h) given ln L and its gradient;
    with lml_grad None only the value and s are formed (gradient None)."""
    d = KernelDesc(dim, n_funcs, n_bumps, beta, core)
    hh = np.ascontiguousarray(h, dtype=np.float64)
    v = ctypes.c_double()
    s = ctypes.c_double()
    if lml_grad is None:
        st = load().gp_augmented(ctypes.byref(d), hh.ctypes.data, float(domain_volume), float(lml), None,
                                 ctypes.byref(v), None, ctypes.byref(s))
        if st != GP_OK:
            raise GPError(st, "gp_augmented")
        return v.value, None, s.value
    lg = np.ascontiguousarray(lml_grad, dtype=np.float64)
    if lg.shape != hh.shape:
        raise ValueError("lml_grad must have one entry per hyperparameter")
    g = np.zeros(hh.shape[0], np.float64)
    st = load().gp_augmented(ctypes.byref(d), hh.ctypes.data, float(domain_volume), float(lml), lg.ctypes.data,
                             ctypes.byref(v), g.ctypes.data, ctypes.byref(s))
    if st != GP_OK:
        raise GPError(st, "gp_augmented")
    return v.value, g, s.value


def default_opts(**kw) -> Opts:
    o = Opts()
    load().gp_default_opts(ctypes.byref(o))
    for k, v in kw.items():
        if k == "precision" and isinstance(v, str):
            v = {"fp64": GP_FP64, "fp32": GP_FP32_MIXED, "fp32_mixed": GP_FP32_MIXED}[v]
        setattr(o, k, v)
    return o


def _ptr(a):
    """(pointer, keepalive) for a torch tensor (any device) or numpy array."""
    if a is None:
        return None, None
    try:
        import torch
        if isinstance(a, torch.Tensor):
            if not a.is_contiguous():
                a = a.contiguous()
            return a.data_ptr(), a
    except ImportError:  # pragma: no cover
        pass
    arr = np.ascontiguousarray(a)
    return arr.ctypes.data, arr


def _stream_handle(device: int):
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream(device).cuda_stream
    except ImportError:  # pragma: no cover
        pass
    return None


@dataclass
class CSR:
    row_ptr: np.ndarray   # n_active + 1
    col: np.ndarray       # nnz, internal (Morton) indices
    val: np.ndarray       # nnz, unscaled K entries
    perm: np.ndarray      # n_active, original index of each internal row


class GP:
    """One library context: a kernel family (dim, n_funcs, n_bumps, beta, core) on one device."""

    def __init__(self, dim: int, n_funcs: int, n_bumps: int, beta: float = 1.0, device: int = 0,
                 core: int = GP_CORE_NONE):
        self._lib = load()
        self.desc = KernelDesc(dim, n_funcs, n_bumps, beta, core)
        self.device = device
        self._stream = _stream_handle(device)
        h = ctypes.c_void_p()
        self._check(self._lib.gp_create(ctypes.byref(h), ctypes.byref(self.desc), device, self._stream), "gp_create")
        self._h = h
        self.n_params = int(self._lib.gp_n_params(ctypes.byref(self.desc)))

    def _hyper(self, h, n_inst=None):
        """Hyperparameters as a contiguous float64 host array of the right length."""
        hh = np.ascontiguousarray(np.asarray(h, dtype=np.float64)).reshape(-1)
        want = self.n_params * (1 if n_inst is None else n_inst)
        if hh.shape[0] != want:
            raise ValueError(f"expected {want} hyperparameters, got {hh.shape[0]}")
        return hh

    def _check(self, st: int, where: str, allow=(GP_OK,)):
        if st not in allow:
            raise GPError(st, where)
        return st

    def _sync_stream(self):
        s = _stream_handle(self.device)
        if s != self._stream:
            self._check(self._lib.gp_set_stream(self._h, s), "gp_set_stream")
            self._stream = s

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.gp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # pragma: no cover
            pass

    # -------------------------------------------------------------- calls
    def assemble(self, x, h, precision=GP_FP32_MIXED) -> dict:
        self._sync_stream()
        n = int(x.shape[0])
        xp, xk = _ptr(x)
        hh = self._hyper(h)
        o = default_opts(precision=precision)
        info = Info()
        self._check(self._lib.gp_assemble(self._h, xp, n, hh.ctypes.data, ctypes.byref(o), ctypes.byref(info)),
                    "gp_assemble")
        return info.as_dict()

    def get_csr(self) -> CSR:
        sizes = (ctypes.c_int64 * 2)()
        self._check(self._lib.gp_get_csr(self._h, None, None, None, None, sizes), "gp_get_csr")
        na, nnz = int(sizes[0]), int(sizes[1])
        rp = np.zeros(na + 1, np.int64)
        col = np.zeros(max(nnz, 1), np.int32)
        val = np.zeros(max(nnz, 1), np.float64)
        perm = np.zeros(max(na, 1), np.int32)
        self._check(self._lib.gp_get_csr(self._h, rp.ctypes.data, col.ctypes.data, val.ctypes.data,
                                         perm.ctypes.data, sizes), "gp_get_csr")
        return CSR(rp, col[:nnz], val[:nnz], perm[:na])

    def solve(self, y, alpha=None, opts: Opts | None = None, allow_not_converged=False):
        self._sync_stream()
        o = opts or default_opts()
        yp, yk = _ptr(y)
        if alpha is None:
            alpha = np.zeros(int(y.shape[0]), np.float64)
        ap, ak = _ptr(alpha)
        info = Info()
        allow = (GP_OK, GP_ERR_NOT_CONVERGED) if allow_not_converged else (GP_OK,)
        self._check(self._lib.gp_solve(self._h, yp, ap, ctypes.byref(o), ctypes.byref(info)), "gp_solve", allow)
        return alpha, info.as_dict()

    def predict(self, y, xstar, mean=None, opts: Opts | None = None, allow_not_converged=False):
        """Posterior mean at the test points xstar (n_star x dim) given the
        targets y of the assembled points; mean is allocated like xstar's rows
        if not given (numpy for host input, torch on the device for device input)."""
        self._sync_stream()
        o = opts or default_opts()
        yp, yk = _ptr(y)
        xp, xk = _ptr(xstar)
        ns = int(xstar.shape[0])
        if mean is None:
            if isinstance(xstar, np.ndarray):
                mean = np.zeros(ns, np.float64)
            else:
                import torch
                mean = torch.zeros(ns, dtype=torch.float64, device=xstar.device)
        mp, mk = _ptr(mean)
        info = Info()
        allow = (GP_OK, GP_ERR_NOT_CONVERGED) if allow_not_converged else (GP_OK,)
        self._check(self._lib.gp_predict(self._h, yp, xp, ns, mp, ctypes.byref(o), ctypes.byref(info)),
                    "gp_predict", allow)
        return mean, info.as_dict()

    def predict_var(self, xstar, var=None, opts: Opts | None = None, allow_not_converged=False):
        """Posterior variance k(x*, x*) - kappa^T K^-1 kappa of the latent
        function at the test points xstar (n_star x dim) with the last
        assembled K; var is allocated like the mean in predict if not given."""
        self._sync_stream()
        o = opts or default_opts()
        xp, xk = _ptr(xstar)
        ns = int(xstar.shape[0])
        if var is None:
            if isinstance(xstar, np.ndarray):
                var = np.zeros(ns, np.float64)
            else:
                import torch
                var = torch.zeros(ns, dtype=torch.float64, device=xstar.device)
        vp_, vk = _ptr(var)
        info = Info()
        allow = (GP_OK, GP_ERR_NOT_CONVERGED) if allow_not_converged else (GP_OK,)
        self._check(self._lib.gp_predict_var(self._h, xp, ns, vp_, ctypes.byref(o), ctypes.byref(info)),
                    "gp_predict_var", allow)
        return var, info.as_dict()

    def lml(self, x, y, h, opts: Opts | None = None, allow_not_converged=False):
        self._sync_stream()
        o = opts or default_opts()
        xp, xk = _ptr(x)
        yp, yk = _ptr(y)
        hh = self._hyper(h)
        out = ctypes.c_double()
        info = Info()
        allow = (GP_OK, GP_ERR_NOT_CONVERGED) if allow_not_converged else (GP_OK,)
        self._check(self._lib.gp_lml(self._h, xp, yp, int(x.shape[0]), hh.ctypes.data, ctypes.byref(o),
                                     ctypes.byref(out), ctypes.byref(info)), "gp_lml", allow)
        return out.value, info.as_dict()

    def lml_grad(self, x, y, h, opts: Opts | None = None, grad=None, allow_not_converged=False):
        self._sync_stream()
        o = opts or default_opts()
        xp, xk = _ptr(x)
        yp, yk = _ptr(y)
        hh = self._hyper(h)
        if grad is None:
            grad = np.zeros(self.n_params, np.float64)
        gp_, gk = _ptr(grad)
        out = ctypes.c_double()
        info = Info()
        allow = (GP_OK, GP_ERR_NOT_CONVERGED) if allow_not_converged else (GP_OK,)
        self._check(self._lib.gp_lml_grad(self._h, xp, yp, int(x.shape[0]), hh.ctypes.data, ctypes.byref(o),
                                          ctypes.byref(out), gp_, ctypes.byref(info)), "gp_lml_grad", allow)
        return out.value, grad, info.as_dict()

    def train(self, x, y, h, opts: Opts | None = None, objective="lml", n_steps=10, lr=0.01, beta1=0.0,
              beta2=0.0, eps=0.0, domain_volume=1.0, s_max=0.0, max_halvings=0, allow_not_converged=False):
        """gp_train: Adam ascent on ln L, (2 - s) ln L or ln L with s < s_max.
        Returns (h after the steps, trace rows (objective, ln L, s) at each
        iterate, info of the last evaluation)."""
        self._sync_stream()
        o = opts or default_opts()
        t = TrainOpts(OBJECTIVES[objective] if isinstance(objective, str) else int(objective), int(n_steps),
                      float(lr), float(beta1), float(beta2), float(eps), float(domain_volume), float(s_max),
                      int(max_halvings))
        xp, xk = _ptr(x)
        yp, yk = _ptr(y)
        hh = self._hyper(h).copy()
        trace = np.zeros((max(int(n_steps), 0) + 1, 3), np.float64)
        info = Info()
        allow = (GP_OK, GP_ERR_NOT_CONVERGED) if allow_not_converged else (GP_OK,)
        self._check(self._lib.gp_train(self._h, xp, yp, int(x.shape[0]), hh.ctypes.data, ctypes.byref(o),
                                       ctypes.byref(t), trace.ctypes.data, ctypes.byref(info)), "gp_train", allow)
        return hh, trace, info.as_dict()

    def lml_grad_batched(self, offsets, x, y, h, opts: Opts | None = None, with_grad=True):
        self._sync_stream()
        o = opts or default_opts()
        off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
        n_inst = off.shape[0] - 1
        xp, xk = _ptr(x)
        yp, yk = _ptr(y)
        hh = self._hyper(h, n_inst)
        lml = np.zeros(n_inst, np.float64)
        grad = np.zeros((n_inst, self.n_params), np.float64) if with_grad else None
        info = Info()
        self._check(self._lib.gp_lml_grad_batched(self._h, n_inst, off.ctypes.data, xp, yp, hh.ctypes.data,
                                                  ctypes.byref(o), lml.ctypes.data,
                                                  grad.ctypes.data if with_grad else None, ctypes.byref(info)),
                    "gp_lml_grad_batched")
        return lml, grad, info.as_dict()
