"""Thin Python binding of libgnp.so (declarations in include/gnp.h).

Argument marshalling only: every step of the method runs in the library's CUDA
kernels.  Device buffers are torch CUDA tensors (contiguous, the dtype each entry
point documents); streams default to torch's current stream.  A missing library
raises at the first call, there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgnp.so")

GNP_OK = 0
STATUS = {0: "GNP_OK", 1: "GNP_ERR_INVALID_ARG", 2: "GNP_ERR_INVALID_CSR", 3: "GNP_ERR_OOM",
          4: "GNP_ERR_CUDA", 5: "GNP_ERR_BREAKDOWN", 6: "GNP_ERR_STAGNATION",
          7: "GNP_ERR_RESIDUAL_MISMATCH", 8: "GNP_ERR_NOT_CONVERGED", 9: "GNP_ERR_TIMEOUT",
          10: "GNP_ERR_NAN", 11: "GNP_ERR_BUSY"}
LAYER_PAPER, LAYER_RESID = 0, 1
H_FP32, H_BF16 = 0, 1


class GnpError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class GnpConfig(C.Structure):
    _fields_ = [("L", C.c_int), ("form", C.c_int), ("hprec", C.c_int), ("batch", C.c_int),
                ("arnoldi_m", C.c_int), ("lr", C.c_float), ("beta1", C.c_float),
                ("beta2", C.c_float), ("eps", C.c_float), ("seed", C.c_ulonglong),
                ("sample_mode", C.c_int), ("no_scale", C.c_int)]


class _SolveInfo(C.Structure):
    _fields_ = [("iters", C.c_int), ("restarts", C.c_int), ("status", C.c_int),
                ("rel_res_est", C.c_double), ("rel_res_true", C.c_double),
                ("seconds", C.c_double), ("res_history", C.POINTER(C.c_double)),
                ("res_history_len", C.c_int), ("hessenberg", C.POINTER(C.c_double)),
                ("hessenberg_cols", C.c_int), ("cycles", C.c_int), ("gconv_launches", C.c_int),
                ("gconv_ms", C.c_double), ("time_history", C.POINTER(C.c_double))]


class _ServerConfig(C.Structure):
    _fields_ = [("max_bytes", C.c_size_t), ("max_active", C.c_int), ("restart", C.c_int), ("grouped", C.c_int)]


class _ServerStats(C.Structure):
    _fields_ = [("queued", C.c_int), ("active", C.c_int), ("used_bytes", C.c_size_t),
                ("rounds", C.c_longlong), ("completed", C.c_longlong), ("max_active_seen", C.c_longlong)]


_lib = None


def lib():
    """Load libgnp.so (built in-tree by paper_2406_00809_gb300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                           "`python -m paper_2406_00809_gb300.build`")
    L = C.CDLL(LIB_PATH)
    vp, i, d, f = C.c_void_p, C.c_int, C.c_double, C.c_float
    pp = C.POINTER(C.c_void_p)
    sig = {
        "gnp_status_string": (C.c_char_p, [i]),
        "gnp_last_error": (C.c_char_p, []),
        "gnp_weight_count": (i, [i]),
        "gnp_mat_create": (i, [i, C.c_longlong, vp, vp, vp, i, vp, pp]),
        "gnp_mat_destroy": (None, [vp]),
        "gnp_mat_info": (i, [vp, C.POINTER(i), C.POINTER(C.c_longlong)]),
        "gnp_gamma": (i, [vp, C.POINTER(d), vp]),
        "gnp_spmv": (i, [vp, vp, vp, vp]),
        "gnp_create": (i, [vp, C.POINTER(GnpConfig), vp, pp]),
        "gnp_destroy": (None, [vp]),
        "gnp_model_gamma": (i, [vp, C.POINTER(d)]),
        "gnp_get_weights": (i, [vp, vp, C.POINTER(i)]),
        "gnp_set_weights": (i, [vp, vp, i]),
        "gnp_set_hprec": (i, [vp, i]),
        "gnp_apply": (i, [vp, vp, vp, vp]),
        "gnp_apply_trace": (i, [vp, vp, vp, vp, vp]),
        "gnp_layer_apply": (i, [vp, i, vp, vp, vp]),
        "gnp_forward_batch": (i, [vp, vp, i, vp, vp]),
        "gnp_backward_batch": (i, [vp, vp, vp, vp]),
        "gnp_sample_batch": (i, [vp, i, vp, vp]),
        "gnp_train_step_pairs": (i, [vp, vp, i, C.POINTER(f), vp]),
        "gnp_train_step": (i, [vp, C.POINTER(f), vp]),
        "gnp_train": (i, [vp, i, C.POINTER(f), vp]),
        "gnp_train_history": (i, [vp, i, vp, C.POINTER(f), vp]),
        "gnp_set_weights_device": (i, [vp, vp, i, vp]),
        "gnp_train_release": (i, [vp]),
        "gnp_philox4x32_10": (i, [vp, C.c_uint, C.c_uint, i, vp, vp]),
        "fgmres_solve": (i, [vp, vp, vp, vp, i, d, i, C.POINTER(_SolveInfo), vp]),
        "fgmres_solve_timeout": (i, [vp, vp, vp, vp, i, d, i, d, C.POINTER(_SolveInfo), vp]),
        "fgmres_solve_precond": (i, [vp, vp, vp, vp, i, d, i, d, C.POINTER(_SolveInfo), vp]),
        "fgmres_solve_multi": (i, [vp, vp, vp, i, vp, i, d, i, C.POINTER(_SolveInfo), vp]),
        "gnp_apply_multi": (i, [vp, vp, i, vp, vp]),
        "gnp_precond_create": (i, [vp, i, vp, i, d, pp]),
        "gnp_precond_destroy": (None, [vp]),
        "gnp_precond_apply": (i, [vp, vp, vp, vp]),
        "gnp_iter_auc": (d, [C.POINTER(C.c_double), i, d]),
        "gnp_time_auc": (d, [C.POINTER(C.c_double), C.POINTER(C.c_double), i, d]),
        "gnp_profile_gconv": (i, [i]),
        "gnp_kernel_faults": (i, [i]),
        "gnp_gamma_noalloc": (i, [i, C.c_longlong, vp, vp, vp, vp, vp]),
        "gnp_server_create": (i, [C.POINTER(_ServerConfig), pp]),
        "gnp_server_submit": (i, [vp, vp, vp, vp, vp, d, i, C.POINTER(C.c_longlong)]),
        "gnp_server_poll": (i, [vp, C.c_longlong, C.POINTER(_SolveInfo)]),
        "gnp_server_wait": (i, [vp, C.c_longlong, d, C.POINTER(_SolveInfo)]),
        "gnp_server_stats": (i, [vp, C.POINTER(_ServerStats)]),
        "gnp_server_destroy": (None, [vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name, None)
        if fn is None:
            continue
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def _check(status: int):
    if status != GNP_OK:
        raise GnpError(status, lib().gnp_last_error().decode())


def _stream(stream):
    if stream is None:
        import torch
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


def _dptr(t, dtype=None, name="tensor"):
    """Device pointer of a contiguous CUDA torch tensor (checked)."""
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA torch tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    return C.c_void_p(t.data_ptr())


def weight_count(L: int) -> int:
    return lib().gnp_weight_count(L)


def status_string(s: int) -> str:
    return lib().gnp_status_string(s).decode()


# --------------------------------------------------------------------- matrices

class Mat:
    """Owner of a gnp_mat handle (freed with the object)."""

    def __init__(self, handle, n, nnz):
        self.h = handle
        self.n = n
        self.nnz = nnz

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.gnp_mat_destroy(self.h)
            self.h = None


def gnp_mat_create(row_ptr, col, val, stream=None) -> Mat:
    """CSR (int32 row_ptr/col, float64 val) from numpy arrays or CUDA tensors."""
    out = C.c_void_p()
    if isinstance(row_ptr, np.ndarray):
        rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
        cl = np.ascontiguousarray(col, dtype=np.int32)
        vl = np.ascontiguousarray(val, dtype=np.float64)
        n = rp.size - 1
        nnz = cl.size
        _check(lib().gnp_mat_create(n, nnz, rp.ctypes.data, cl.ctypes.data, vl.ctypes.data, 0,
                                    _stream(stream), C.byref(out)))
    else:
        import torch
        n = row_ptr.numel() - 1
        nnz = col.numel()
        _check(lib().gnp_mat_create(n, nnz, _dptr(row_ptr, torch.int32, "row_ptr"),
                                    _dptr(col, torch.int32, "col"), _dptr(val, torch.float64, "val"),
                                    1, _stream(stream), C.byref(out)))
    return Mat(out, n, nnz)


def mat_from_csr(A) -> Mat:
    """From an ``inputs.CSR``."""
    return gnp_mat_create(A.row_ptr, A.col, A.val)


def gnp_gamma(A: Mat, stream=None) -> float:
    g = C.c_double()
    _check(lib().gnp_gamma(A.h, C.byref(g), _stream(stream)))
    return g.value


def gnp_gamma_noalloc(row_ptr, col, val, gamma_out, stream=None):
    """gamma (Eq. 6) of a device CSR into the device scalar gamma_out, allocating
    nothing (scratch is a fixed array inside the library; n <= 2^20)."""
    import torch
    n = row_ptr.numel() - 1
    _check(lib().gnp_gamma_noalloc(n, col.numel(), _dptr(row_ptr, torch.int32, "row_ptr"),
                                   _dptr(col, torch.int32, "col"), _dptr(val, torch.float64, "val"),
                                   _dptr(gamma_out, torch.float64, "gamma_out"), _stream(stream)))
    return gamma_out


def gnp_spmv(A: Mat, x, y, stream=None):
    import torch
    _check(lib().gnp_spmv(A.h, _dptr(x, torch.float64, "x"), _dptr(y, torch.float64, "y"), _stream(stream)))
    return y


# --------------------------------------------------------------------- model

SAMPLE_MIX, SAMPLE_X_NORMAL, SAMPLE_B_NORMAL = 0, 1, 2


def make_config(L=8, form=LAYER_PAPER, hprec=H_FP32, batch=16, arnoldi_m=40, lr=1e-3,
                beta1=0.9, beta2=0.999, eps=1e-8, seed=0, sample_mode=SAMPLE_MIX,
                no_scale=False) -> GnpConfig:
    return GnpConfig(L, form, hprec, batch, arnoldi_m, lr, beta1, beta2, eps, seed, sample_mode,
                     1 if no_scale else 0)


class Model:
    def __init__(self, handle, A: Mat, cfg: GnpConfig):
        self.h = handle
        self.A = A  # keep the matrix alive
        self.cfg = cfg
        self.hprec = cfg.hprec

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.gnp_destroy(self.h)
            self.h = None


def gnp_create(A: Mat, cfg: GnpConfig, weights) -> Model:
    w = np.ascontiguousarray(weights, dtype=np.float32)
    if w.size != weight_count(cfg.L):
        raise ValueError(f"weights: {w.size} floats, expected {weight_count(cfg.L)}")
    out = C.c_void_p()
    _check(lib().gnp_create(A.h, C.byref(cfg), w.ctypes.data, C.byref(out)))
    return Model(out, A, cfg)


PRECOND_IDENTITY, PRECOND_GNP, PRECOND_JACOBI, PRECOND_GMRES = 0, 1, 2, 3


class Precond:
    """A right preconditioner handle (gnp_precond): identity, GNP, Jacobi or inner GMRES."""

    def __init__(self, handle, A: Mat, kind: int, M: Model | None):
        self.h = handle
        self.A = A
        self.kind = kind
        self.M = M  # keep the model alive

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.gnp_precond_destroy(self.h)
            self.h = None


def gnp_precond_create(A: Mat, kind: int, M: Model | None = None, inner_iters: int = 10,
                       inner_rtol: float = 1e-6) -> Precond:
    out = C.c_void_p()
    _check(lib().gnp_precond_create(A.h, kind, M.h if M is not None else None, inner_iters, inner_rtol,
                                    C.byref(out)))
    return Precond(out, A, kind, M)


def gnp_precond_apply(P: Precond, v, z, stream=None):
    """z = P(v) for float64 CUDA vectors."""
    import torch
    _check(lib().gnp_precond_apply(P.h, _dptr(v, torch.float64, "v"), _dptr(z, torch.float64, "z"),
                                   _stream(stream)))


def gnp_model_gamma(M: Model) -> float:
    g = C.c_double()
    _check(lib().gnp_model_gamma(M.h, C.byref(g)))
    return g.value


def gnp_get_weights(M: Model) -> np.ndarray:
    cnt = C.c_int(0)
    _check(lib().gnp_get_weights(M.h, None, C.byref(cnt)))
    w = np.zeros(cnt.value, dtype=np.float32)
    _check(lib().gnp_get_weights(M.h, w.ctypes.data, C.byref(cnt)))
    return w


def gnp_set_weights(M: Model, weights):
    w = np.ascontiguousarray(weights, dtype=np.float32)
    _check(lib().gnp_set_weights(M.h, w.ctypes.data, w.size))


def gnp_set_hprec(M: Model, hprec: int):
    _check(lib().gnp_set_hprec(M.h, hprec))
    M.hprec = hprec


def gnp_apply(M: Model, v, z, stream=None):
    """z (float32 [n]) = M(v) (float64 [n])."""
    import torch
    _check(lib().gnp_apply(M.h, _dptr(v, torch.float64, "v"), _dptr(z, torch.float32, "z"),
                           _stream(stream)))
    return z


def gnp_apply_trace(M: Model, v, z, hidden, stream=None):
    import torch
    _check(lib().gnp_apply_trace(M.h, _dptr(v, torch.float64, "v"), _dptr(z, torch.float32, "z"),
                                 _dptr(hidden, torch.float32, "hidden"), _stream(stream)))
    return z


# --------------------------------------------------------------------- training

def gnp_layer_apply(M: Model, layer: int, Hin, Hout, stream=None):
    """One Res-GCONV layer (Eq. 7) on caller hidden blocks [n, 16] of the model's precision
    (torch.float32 for H_FP32, torch.bfloat16 for H_BF16)."""
    import torch
    dt = torch.bfloat16 if M.hprec == H_BF16 else torch.float32
    for t, nm in ((Hin, "Hin"), (Hout, "Hout")):
        if t.numel() != M.A.n * 16:
            raise ValueError(f"{nm} must hold n x 16 = {M.A.n * 16} values, got {t.numel()}")
    _check(lib().gnp_layer_apply(M.h, int(layer), _dptr(Hin, dt, "Hin"), _dptr(Hout, dt, "Hout"),
                                 _stream(stream)))


def gnp_forward_batch(M: Model, b, z, B=None, stream=None):
    """z = M(b) for a node-major batch b (float32 [n, B] or flat [n*B])."""
    import torch
    if B is None:
        B = b.shape[1] if b.dim() == 2 else M.cfg.batch
    _check(lib().gnp_forward_batch(M.h, _dptr(b, torch.float32, "b"), B, _dptr(z, torch.float32, "z"),
                                   _stream(stream)))
    return z


def gnp_backward_batch(M: Model, dz, grad, stream=None):
    import torch
    _check(lib().gnp_backward_batch(M.h, _dptr(dz, torch.float32, "dz"), _dptr(grad, torch.float32, "grad"),
                                    _stream(stream)))
    return grad


def gnp_sample_batch(M: Model, step: int, x, stream=None):
    import torch
    _check(lib().gnp_sample_batch(M.h, step, _dptr(x, torch.float32, "x"), _stream(stream)))
    return x


def gnp_train_step_pairs(M: Model, x, B=None, stream=None) -> float:
    """One training step on solutions x (float32 [n, B] or flat [n*B], node-major)."""
    import torch
    if B is None:
        B = x.shape[1] if x.dim() == 2 else M.cfg.batch
    loss = C.c_float(0.0)
    _check(lib().gnp_train_step_pairs(M.h, _dptr(x, torch.float32, "x"), B, C.byref(loss),
                                      _stream(stream)))
    return loss.value


def gnp_train_step(M: Model, stream=None) -> float:
    loss = C.c_float(0.0)
    _check(lib().gnp_train_step(M.h, C.byref(loss), _stream(stream)))
    return loss.value


def gnp_train_release(M: Model):
    _check(lib().gnp_train_release(M.h))


def gnp_set_weights_device(M: Model, w, stream=None):
    import torch
    _check(lib().gnp_set_weights_device(M.h, _dptr(w, torch.float32, "w"), w.numel(), _stream(stream)))


def gnp_philox4x32_10(ctr, key0: int, key1: int, out, stream=None):
    """ctr, out: int32 CUDA tensors of shape [count, 4] (uint32 bit patterns)."""
    import torch
    _check(lib().gnp_philox4x32_10(_dptr(ctr, torch.int32, "ctr"), key0, key1, ctr.shape[0],
                                   _dptr(out, torch.int32, "out"), _stream(stream)))
    return out


def gnp_train(M: Model, steps: int, stream=None) -> float:
    best = C.c_float(0.0)
    _check(lib().gnp_train(M.h, steps, C.byref(best), _stream(stream)))
    return best.value


def gnp_train_history(M: Model, steps: int, stream=None):
    """(per-step losses, best loss) of `steps` training steps."""
    losses = np.zeros(steps, dtype=np.float32)
    best = C.c_float(0.0)
    _check(lib().gnp_train_history(M.h, steps, losses.ctypes.data if steps else None, C.byref(best),
                                   _stream(stream)))
    return losses, best.value


# --------------------------------------------------------------------- solver

def gnp_profile_gconv(on: bool):
    _check(lib().gnp_profile_gconv(1 if on else 0))


def gnp_kernel_faults(reset: bool = True) -> int:
    """Bounded device waits that gave up since the last reset (-1: unreadable)."""
    return int(lib().gnp_kernel_faults(1 if reset else 0))


@dataclass
class SolveInfo:
    status: int
    iters: int
    restarts: int
    rel_res_est: float
    rel_res_true: float
    seconds: float
    history: np.ndarray = field(default_factory=lambda: np.zeros(0))
    times: np.ndarray | None = None
    hessenberg: np.ndarray | None = None
    cycles: int = 0
    gconv_launches: int = 0
    gconv_ms: float = 0.0

    @property
    def status_name(self) -> str:
        return STATUS.get(self.status, str(self.status))


def fgmres_solve(A: Mat, b, x, M: Model | Precond | None = None, restart=30, rtol=1e-8, maxiters=1000,
                 stream=None, history=True, hessenberg=False, check=False, timeout=0.0,
                 times=False) -> SolveInfo:
    """Solve A x = b (float64 CUDA tensors; x holds x0 on entry).  timeout > 0 (seconds)
    calls fgmres_solve_timeout; times=True also returns the per-iteration device times."""
    import torch
    info = _SolveInfo()
    hist = np.zeros(maxiters + 1) if history else None
    thist = np.zeros(maxiters + 1) if times else None
    hess = np.zeros((restart, restart + 1)) if hessenberg else None
    if hist is not None:
        info.res_history = hist.ctypes.data_as(C.POINTER(C.c_double))
    if thist is not None:
        info.time_history = thist.ctypes.data_as(C.POINTER(C.c_double))
    if hess is not None:
        info.hessenberg = hess.ctypes.data_as(C.POINTER(C.c_double))
    args = (A.h, _dptr(b, torch.float64, "b"), _dptr(x, torch.float64, "x"), M.h if M is not None else None,
            restart, rtol, maxiters)
    if isinstance(M, Precond):
        st = lib().fgmres_solve_precond(*args, timeout, C.byref(info), _stream(stream))
    elif timeout != 0.0:
        st = lib().fgmres_solve_timeout(*args, timeout, C.byref(info), _stream(stream))
    else:
        st = lib().fgmres_solve(*args, C.byref(info), _stream(stream))
    if check:
        _check(st)
    elif st not in STATUS:
        _check(st)
    out = SolveInfo(st, info.iters, info.restarts, info.rel_res_est, info.rel_res_true, info.seconds,
                    cycles=info.cycles, gconv_launches=info.gconv_launches, gconv_ms=info.gconv_ms)
    if hist is not None:
        out.history = hist[:info.res_history_len].copy()
    if thist is not None:
        out.times = thist[:info.iters + 1].copy()
    if hess is not None:
        cols = info.hessenberg_cols
        out.hessenberg = hess.T[:cols + 1, :cols].copy()  # column-major (m+1) x m
    return out


def gnp_apply_multi(M: Model, V, Z, stream=None):
    """Z[:, r] = M(V[:, r]) for [n, k] tensors (V float64, Z float32, row-major)."""
    import torch
    _check(lib().gnp_apply_multi(M.h, _dptr(V, torch.float64, "V"), V.shape[1], _dptr(Z, torch.float32, "Z"),
                                 _stream(stream)))


def fgmres_solve_multi(A: Mat, B, X, M: Model | None = None, restart=30, rtol=1e-8, maxiters=1000,
                       stream=None, history=True, times=False) -> list:
    """Solve the k systems A X[:, r] = B[:, r] together (float64 CUDA tensors of shape [n, k],
    row-major, so element (i, r) is at i*k + r; X holds x0 on entry).  Returns k SolveInfo."""
    import torch
    if B.dim() != 2 or X.shape != B.shape:
        raise ValueError("B and X must be [n, k] tensors of the same shape")
    k = B.shape[1]
    infos = (_SolveInfo * k)()
    hists = [np.zeros(maxiters + 1) if history else None for _ in range(k)]
    thists = [np.zeros(maxiters + 1) if times else None for _ in range(k)]
    for r in range(k):
        if hists[r] is not None:
            infos[r].res_history = hists[r].ctypes.data_as(C.POINTER(C.c_double))
        if thists[r] is not None:
            infos[r].time_history = thists[r].ctypes.data_as(C.POINTER(C.c_double))
    st = lib().fgmres_solve_multi(A.h, _dptr(B, torch.float64, "B"), _dptr(X, torch.float64, "X"), k,
                                  M.h if M is not None else None, restart, rtol, maxiters, infos, _stream(stream))
    if st not in STATUS or st in (1, 3, 4):  # invalid argument, out of memory, CUDA error
        _check(st)
    out = []
    for r in range(k):
        info = infos[r]
        o = SolveInfo(info.status, info.iters, info.restarts, info.rel_res_est, info.rel_res_true, info.seconds,
                      cycles=info.cycles)
        if hists[r] is not None:
            o.history = hists[r][:info.res_history_len].copy()
        if thists[r] is not None:
            o.times = thists[r][:info.iters + 1].copy()
        out.append(o)
    return out


def iter_auc(history, rtol: float) -> float:
    """Iter-AUC of a residual history (Sec. 3 "Evaluation metrics"), computed by the library."""
    h = np.ascontiguousarray(history, dtype=np.float64)
    return float(lib().gnp_iter_auc(h.ctypes.data_as(C.POINTER(C.c_double)), len(h), rtol))


def time_auc(history, times, rtol: float) -> float:
    """Time-AUC of a residual history and its per-iteration times (seconds)."""
    h = np.ascontiguousarray(history, dtype=np.float64)
    t = np.ascontiguousarray(times, dtype=np.float64)
    if len(t) != len(h):
        raise ValueError("history and times differ in length")
    return float(lib().gnp_time_auc(h.ctypes.data_as(C.POINTER(C.c_double)),
                                    t.ctypes.data_as(C.POINTER(C.c_double)), len(h), rtol))


# --------------------------------------------------------------------- autograd

def gnp_function(M: Model):
    """torch.autograd.Function computing z = M(b) for a node-major batch b [n, B]
    with the weight blob w (float32 CUDA [count]) as the differentiable input; the
    backward is the library's hand-written kernel (gnp_backward_batch).  Only the
    weights receive a gradient (tau = ||b|| carries none, Sec. 2.3)."""
    import torch

    class GnpFunction(torch.autograd.Function):
        @staticmethod
        def forward(ctx, w, b):
            gnp_set_weights_device(M, w.detach().contiguous())
            z = torch.empty_like(b)
            gnp_forward_batch(M, b.contiguous(), z, B=b.shape[1] if b.dim() == 2 else None)
            return z

        @staticmethod
        def backward(ctx, dz):
            g = torch.empty(weight_count(M.cfg.L), dtype=torch.float32, device=dz.device)
            gnp_backward_batch(M, dz.contiguous(), g)
            return g, None

    return GnpFunction


# --------------------------------------------------------------------- server

class Server:
    """Continuous-batching solve server (gnp_server_*).  Keeps the buffers of every
    submitted request alive until it is collected.  grouped=True: the requests whose GNP
    runs on the short-row layer kernels advance in grouped steps (one launch per kernel
    for all of them); results equal lone fgmres_solve calls with GNP_ORTHO=cgs2."""

    def __init__(self, max_bytes: int, max_active: int = 64, restart: int = 30, grouped: bool = False):
        cfg = _ServerConfig(max_bytes, max_active, restart, 1 if grouped else 0)
        out = C.c_void_p()
        _check(lib().gnp_server_create(C.byref(cfg), C.byref(out)))
        self.h = out
        self._keep = {}

    def submit(self, A: Mat, M: "Model | None", b, x, rtol=1e-8, maxiters=1000) -> int:
        import torch
        t = C.c_longlong()
        _check(lib().gnp_server_submit(self.h, A.h, M.h if M is not None else None,
                                       _dptr(b, torch.float64, "b"), _dptr(x, torch.float64, "x"),
                                       rtol, maxiters, C.byref(t)))
        self._keep[t.value] = (A, M, b, x)
        return t.value

    def _result(self, st, info):
        return SolveInfo(st, info.iters, info.restarts, info.rel_res_est, info.rel_res_true, info.seconds,
                         cycles=info.cycles)

    def poll(self, ticket: int):
        """None while queued or running, else the SolveInfo (seconds = latency)."""
        info = _SolveInfo()
        st = lib().gnp_server_poll(self.h, ticket, C.byref(info))
        if st == 11:  # GNP_ERR_BUSY
            return None
        if st == 1:
            _check(st)
        self._keep.pop(ticket, None)
        return self._result(st, info)

    def wait(self, ticket: int, timeout: float = 600.0):
        info = _SolveInfo()
        st = lib().gnp_server_wait(self.h, ticket, timeout, C.byref(info))
        if st in (1, 9):
            _check(st)
        self._keep.pop(ticket, None)
        return self._result(st, info)

    def stats(self) -> dict:
        s = _ServerStats()
        _check(lib().gnp_server_stats(self.h, C.byref(s)))
        return {k: getattr(s, k) for k, _ in _ServerStats._fields_}

    def close(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.gnp_server_destroy(self.h)
            self.h = None
            self._keep.clear()

    def __del__(self):
        self.close()
