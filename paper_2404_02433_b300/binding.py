"""Thin ctypes binding of libetc (include/etc.h).

Argument marshalling only: every step of the solve runs in the CUDA library.
Functions keep the C names (``etc_create_rve`` ...).  ``RVE`` wraps a handle
for tensors: device tensors are passed as device pointers, host tensors and
numpy arrays as host pointers (the library copies with cudaMemcpyDefault).
There is no CPU fallback: a missing or unloadable library raises.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, byref, c_double, c_int, c_void_p

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libetc.so")

ETC_OK, ETC_EINVAL, ETC_ENOMEM, ETC_ECUDA, ETC_ENOCONV, ETC_EBREAKDOWN, ETC_ESTATE = range(7)
ETC_PREC_FP64, ETC_PREC_MIXED, ETC_PREC_MIXED_F64 = 0, 1, 2
ETC_REF_LP, ETC_REF_ONES, ETC_REF_USER = 0, 1, 2
ETC_INIT_ZERO, ETC_INIT_LINEAR = 0, 1

EXPORTED = (
    "etc_default_opts", "etc_create_rve", "etc_destroy_rve", "etc_set_reference_params",
    "etc_solve_direction", "etc_get_solution", "etc_effective_tensor", "etc_loading_dims",
    "etc_apply_operator", "etc_apply_operator_df", "etc_apply_preconditioner", "etc_dct_planes",
    "etc_status_string",
    "etc_last_error", "etc_profile_iteration", "etc_transform_tiles", "etc_kernel_launches",
    "etc_apply_reference_inverse_static", "etc_convert_check", "etc_gradient",
    "etc_batch_create", "etc_batch_run", "etc_batch_destroy", "etc_effective_tensor_batch",
    "etc_solve_general", "etc_split_check", "etc_fp64_fma_rate", "etc_batch_queued",
    "etc_residual_history",
)


class EtcOpts(ctypes.Structure):
    _fields_ = [("rtol", c_double), ("maxit", c_int), ("precision", c_int),
                ("true_residual", c_int), ("batch_queue", c_int), ("init", c_int)]


class EtcInfo(ctypes.Structure):
    _fields_ = [("iters", c_int), ("status", c_int), ("relres", c_double),
                ("true_relres", c_double), ("kref", c_double * 5), ("cond_bound", c_double),
                ("kappa_in", c_double), ("column", c_double * 3), ("t_setup_ms", c_double),
                ("t_solve_ms", c_double), ("kappa_energy", c_double)]

    def as_dict(self):
        return {"iters": self.iters, "status": self.status, "relres": self.relres,
                "true_relres": self.true_relres, "kref": list(self.kref),
                "cond_bound": self.cond_bound, "kappa_in": self.kappa_in,
                "column": list(self.column), "t_setup_ms": self.t_setup_ms,
                "t_solve_ms": self.t_solve_ms, "kappa_energy": self.kappa_energy}


class EtcError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"libetc status {status}: {msg}")
        self.status = status


_lib = None


def load_library(path: str | None = None):
    """Load libetc.so (built in-tree by ``build.build()``); raise if absent."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise ImportError(f"libetc.so not found at {p}; run paper_2404_02433_b300/build.py")
    lib = ctypes.CDLL(p)
    vp, dp, ip = c_void_p, POINTER(c_double), POINTER(c_int)
    sig = {
        "etc_default_opts": ([POINTER(EtcOpts)], c_int),
        "etc_create_rve": ([c_int, c_int, c_int, c_double, c_double, c_double, vp, vp, vp, vp,
                            POINTER(c_void_p)], c_int),
        "etc_destroy_rve": ([vp], c_int),
        "etc_set_reference_params": ([vp, c_int, c_int, dp, dp], c_int),
        "etc_solve_direction": ([vp, c_int, c_double, c_double, POINTER(EtcOpts), dp,
                                 POINTER(EtcInfo)], c_int),
        "etc_get_solution": ([vp, c_int, vp], c_int),
        "etc_effective_tensor": ([vp, POINTER(EtcOpts), dp, POINTER(EtcInfo)], c_int),
        "etc_loading_dims": ([vp, c_int, ip], c_int),
        "etc_apply_operator": ([vp, c_int, vp, vp], c_int),
        "etc_apply_operator_df": ([vp, c_int, vp, vp, POINTER(c_double)], c_int),
        "etc_apply_preconditioner": ([vp, c_int, c_int, vp, vp], c_int),
        "etc_dct_planes": ([vp, c_int, c_int, vp, vp], c_int),
        "etc_status_string": ([c_int], ctypes.c_char_p),
        "etc_last_error": ([vp], ctypes.c_char_p),
        "etc_profile_iteration": ([vp, c_int, c_int, c_int, dp], c_int),
        "etc_transform_tiles": ([vp, c_int, c_int, ip], c_int),
        "etc_kernel_launches": ([], ctypes.c_ulonglong),
        "etc_apply_reference_inverse_static": ([c_int, c_int, c_int, dp, vp, vp, vp], c_int),
        "etc_convert_check": ([vp, vp, vp, vp, ctypes.c_longlong, vp], c_int),
        "etc_split_check": ([vp, vp, ctypes.c_longlong, vp], c_int),
        "etc_fp64_fma_rate": ([c_int, dp, vp], c_int),
        "etc_gradient": ([vp, c_int, c_double, c_double, POINTER(EtcOpts), c_int, vp, dp,
                          POINTER(EtcInfo)], c_int),
        "etc_batch_create": ([c_int, POINTER(c_void_p), POINTER(EtcOpts), POINTER(c_void_p)],
                             c_int),
        "etc_batch_run": ([vp, dp, POINTER(EtcInfo), dp], c_int),
        "etc_batch_destroy": ([vp], c_int),
        "etc_batch_queued": ([vp], c_int),
        "etc_residual_history": ([vp, dp, c_int, ip, ip], c_int),
        "etc_solve_general": ([vp, c_int, vp, vp, vp, POINTER(EtcOpts), POINTER(EtcInfo)], c_int),
        "etc_effective_tensor_batch": ([c_int, POINTER(c_void_p), POINTER(EtcOpts), dp,
                                        POINTER(EtcInfo)], c_int),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def _ptr(a):
    """Raw pointer of a contiguous float64 torch tensor or numpy array (or None)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return ctypes.c_void_p(a.data_ptr())
    import numpy as np
    if not (isinstance(a, np.ndarray) and a.flags["C_CONTIGUOUS"]):
        raise ValueError("array must be C-contiguous")
    return ctypes.c_void_p(a.ctypes.data)


def _check(status, handle=None, ok=(ETC_OK,), thread_reason=False):
    """Raise EtcError unless status is in ok.  The message is the handle's last
    error, or with thread_reason the reason etc_last_error(NULL) keeps for the
    handle-less calls (create, batch create, the allocation-free apply)."""
    if status in ok:
        return status
    lib = load_library()
    msg = lib.etc_last_error(handle if handle else None).decode() if (handle or thread_reason) else ""
    if not msg:
        msg = lib.etc_status_string(status).decode()
    raise EtcError(status, msg)


def make_opts(rtol=1e-8, maxit=5000, precision=ETC_PREC_FP64, true_residual=1, batch_queue=0,
              init=ETC_INIT_ZERO):
    o = EtcOpts()
    _check(load_library().etc_default_opts(byref(o)))
    o.rtol, o.maxit, o.precision, o.true_residual = rtol, maxit, precision, true_residual
    o.batch_queue, o.init = batch_queue, init
    return o


# -------------------------------------------------------------- C-named calls
def etc_create_rve(nx, ny, nz, lx, ly, lz, kx, ky=None, kz=None, stream=None):
    lib = load_library()
    h = c_void_p()
    st = lib.etc_create_rve(nx, ny, nz, lx, ly, lz, _ptr(kx), _ptr(ky), _ptr(kz),
                            c_void_p(stream) if stream else None, byref(h))
    _check(st, thread_reason=True)
    return h


def etc_destroy_rve(h):
    return _check(load_library().etc_destroy_rve(h))


def etc_solve_direction(h, direction, p_in=1.0, p_out=0.0, opts=None):
    lib = load_library()
    k = c_double()
    info = EtcInfo()
    st = lib.etc_solve_direction(h, direction, p_in, p_out, byref(opts) if opts else None,
                                 byref(k), byref(info))
    _check(st, h, ok=(ETC_OK, ETC_ENOCONV, ETC_EBREAKDOWN))
    return st, k.value, info


def etc_effective_tensor(h, opts=None):
    lib = load_library()
    K = (c_double * 9)()
    info = (EtcInfo * 3)()
    st = lib.etc_effective_tensor(h, byref(opts) if opts else None, K, info)
    _check(st, h, ok=(ETC_OK, ETC_ENOCONV, ETC_EBREAKDOWN))
    return st, [K[i] for i in range(9)], [info[i] for i in range(3)]


def etc_set_reference_params(h, direction, mode, kref=None):
    lib = load_library()
    kin = (c_double * 5)(*(kref or [1.0] * 5))
    kout = (c_double * 5)()
    _check(lib.etc_set_reference_params(h, direction, mode, kin, kout), h)
    return [kout[i] for i in range(5)]


def etc_get_solution(h, direction, dst):
    return _check(load_library().etc_get_solution(h, direction, _ptr(dst)), h)


def etc_loading_dims(h, direction):
    d = (c_int * 3)()
    _check(load_library().etc_loading_dims(h, direction, d), h)
    return (d[0], d[1], d[2])


def etc_apply_operator(h, direction, w, q):
    return _check(load_library().etc_apply_operator(h, direction, _ptr(w), _ptr(q)), h)


def etc_apply_operator_df(h, direction, w, q):
    """q = A w by the mixed path's double-float operator (w FP32, q FP64); returns w.q."""
    wq = c_double()
    _check(load_library().etc_apply_operator_df(h, direction, _ptr(w), _ptr(q), byref(wq)), h)
    return wq.value


def etc_apply_preconditioner(h, direction, precision, r, z):
    return _check(load_library().etc_apply_preconditioner(h, direction, precision, _ptr(r),
                                                          _ptr(z)), h)


def etc_dct_planes(h, direction, inverse, x, y):
    return _check(load_library().etc_dct_planes(h, direction, int(inverse), _ptr(x), _ptr(y)), h)


def etc_profile_iteration(h, direction, precision, iters):
    ms = (c_double * 6)()
    _check(load_library().etc_profile_iteration(h, direction, precision, iters, ms), h)
    return [ms[i] for i in range(6)]


def etc_transform_tiles(h, direction, precision):
    tiles = (c_int * 3)()
    _check(load_library().etc_transform_tiles(h, direction, precision, tiles), h)
    return [tiles[i] for i in range(3)]


def etc_apply_reference_inverse_static(n0, n1, n2, kref, r, z, stream=None):
    """Allocation-free preconditioner apply (returns the raw status)."""
    k = (c_double * 5)(*kref)
    return load_library().etc_apply_reference_inverse_static(
        n0, n1, n2, k, _ptr(r), _ptr(z), c_void_p(stream) if stream else None)


def etc_fp64_fma_rate(iters=20000, stream=None):
    """Measured FP64 FMA rate of the current device in TFLOP/s."""
    v = c_double()
    _check(load_library().etc_fp64_fma_rate(iters, byref(v), c_void_p(stream) if stream else None))
    return v.value


def etc_convert_check(f_in, d_out, d_in, f_out, stream=None):
    return _check(load_library().etc_convert_check(_ptr(f_in), _ptr(d_out), _ptr(d_in),
                                                   _ptr(f_out), f_in.numel(),
                                                   c_void_p(stream) if stream else None))


def etc_split_check(d, hilo, stream=None):
    """hilo (2n float32): (hi, lo) of each binary64 value of d, as the mixed matvec splits it."""
    return _check(load_library().etc_split_check(_ptr(d), _ptr(hilo), d.numel(),
                                                 c_void_p(stream) if stream else None))


def etc_gradient(h, direction, grad, p_in=1.0, p_out=0.0, opts=None, per_component=0):
    """Adjoint d kappa_eff / d log kappa into `grad`; returns (kappa_eff, [info fwd, info adj])."""
    k = c_double()
    info = (EtcInfo * 2)()
    _check(load_library().etc_gradient(h, direction, p_in, p_out, byref(opts) if opts else None,
                                       per_component, _ptr(grad), byref(k), info), h)
    return k.value, [info[0], info[1]]


class Batch:
    """Full tensors of several RVEs in one CUDA graph (etc_batch_*)."""

    def __init__(self, rves, rtol=1e-8, maxit=5000, precision=ETC_PREC_FP64, true_residual=1,
                 queue=False, init=ETC_INIT_ZERO):
        lib = load_library()
        self.rves = list(rves)
        self.count = len(self.rves)
        hs = (c_void_p * self.count)(*[r.h.value for r in self.rves])
        self.opts = make_opts(rtol, maxit, precision, true_residual, int(bool(queue)), init)
        self.b = c_void_p()
        _check(lib.etc_batch_create(self.count, hs, byref(self.opts), byref(self.b)),
               thread_reason=True)

    def run(self):
        """Returns (K as a list of 9-lists, info dicts per solve, batch ms, status)."""
        lib = load_library()
        K = (c_double * (9 * self.count))()
        info = (EtcInfo * (3 * self.count))()
        ms = c_double()
        st = lib.etc_batch_run(self.b, K, info, byref(ms))
        _check(st, ok=(ETC_OK, ETC_ENOCONV, ETC_EBREAKDOWN))
        Ks = [[K[9 * i + j] for j in range(9)] for i in range(self.count)]
        return Ks, [info[i].as_dict() for i in range(3 * self.count)], ms.value, st

    def queued(self):
        """Handles whose solves run in work-queue loops."""
        return int(load_library().etc_batch_queued(self.b))

    def close(self):
        if getattr(self, "b", None) and self.b.value:
            load_library().etc_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def etc_kernel_launches():
    return int(load_library().etc_kernel_launches())


# -------------------------------------------------------------- tensor wrapper
class RVE:
    """One voxel RVE on the current CUDA device (Sec. 2.2 arrays kappa^{x,y,z})."""

    def __init__(self, kx, ky=None, kz=None, lengths=(1.0, 1.0, 1.0), stream=None):
        import torch
        if kx.dim() != 3:
            raise ValueError("kappa must have shape (nz, ny, nx)")
        nz, ny, nx = kx.shape
        self.shape = (nz, ny, nx)
        self.lengths = tuple(float(v) for v in lengths)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self._keep = [kx, ky, kz]
        self.h = etc_create_rve(nx, ny, nz, *self.lengths, kx, ky, kz,
                                stream=self.stream.cuda_stream)

    def close(self):
        if getattr(self, "h", None):
            etc_destroy_rve(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def solve(self, direction, p_in=1.0, p_out=0.0, rtol=1e-8, maxit=5000,
              precision=ETC_PREC_FP64, true_residual=1, init=ETC_INIT_ZERO):
        opts = make_opts(rtol, maxit, precision, true_residual, init=init)
        st, k, info = etc_solve_direction(self.h, direction, p_in, p_out, opts)
        return k, info.as_dict()

    def tensor(self, rtol=1e-8, maxit=5000, precision=ETC_PREC_FP64, true_residual=1):
        opts = make_opts(rtol, maxit, precision, true_residual)
        st, K, infos = etc_effective_tensor(self.h, opts)
        return K, [i.as_dict() for i in infos], st

    def solution(self, direction, out=None):
        import torch
        if out is None:
            out = torch.empty(self.shape, dtype=torch.float64, device="cuda")
        etc_get_solution(self.h, direction, out)
        return out

    def gradient(self, direction, p_in=1.0, p_out=0.0, rtol=1e-10, maxit=5000,
                 per_component=False, precision=ETC_PREC_FP64):
        """(d kappa_eff / d log kappa as a CUDA tensor, kappa_eff, infos)."""
        import torch
        shape = ((3,) if per_component else ()) + self.shape
        out = torch.empty(shape, dtype=torch.float64, device="cuda")
        opts = make_opts(rtol, maxit, precision, 1)
        k, infos = etc_gradient(self.h, direction, out, p_in, p_out, opts, int(per_component))
        return out, k, [i.as_dict() for i in infos]

    def solve_general(self, direction, p_in_face=None, p_out_face=None, source=None, rtol=1e-8,
                      maxit=5000, precision=ETC_PREC_FP64):
        """General face data (loading-frame planes) and source (original layout)."""
        opts = make_opts(rtol, maxit, precision, 1)
        info = EtcInfo()
        st = load_library().etc_solve_general(self.h, direction, _ptr(p_in_face), _ptr(p_out_face),
                                              _ptr(source), byref(opts), byref(info))
        _check(st, self.h, ok=(ETC_OK, ETC_ENOCONV, ETC_EBREAKDOWN))
        return info.as_dict()

    def loading_dims(self, direction):
        return etc_loading_dims(self.h, direction)

    def history(self, cap=8192):
        """(first iteration, relative residuals) of the last solve (etc_residual_history)."""
        out = (c_double * cap)()
        first, count = c_int(), c_int()
        _check(load_library().etc_residual_history(self.h, out, cap, byref(first), byref(count)),
               self.h)
        return first.value, [out[i] for i in range(count.value)]

    def set_reference(self, direction, mode=ETC_REF_LP, kref=None):
        return etc_set_reference_params(self.h, direction, mode, kref)
