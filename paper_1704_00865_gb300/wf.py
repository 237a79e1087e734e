"""Thin ctypes binding of libwf.so (C ABI in include/wf.h).

Argument marshalling only: every step of the Wiener-filter iteration runs in
the library's CUDA kernels.  Arrays may be torch tensors (CUDA or CPU) or
numpy arrays; CPU arrays are handed to the library as host pointers and the
library stages them.  There is no fallback: if libwf.so is missing this
module raises.
"""

from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Sequence

import numpy as np

from . import build as _build

WF_OK, WF_EINVAL, WF_ENOTPD, WF_ENOCONV, WF_ETIMEOUT, WF_ECUDA, WF_ENOMEM, WF_EUNSUPPORTED, WF_ESTALL = range(9)
_FINISHED = (WF_OK, WF_ENOCONV, WF_ESTALL)
WF_PART_WHITE, WF_PART_1F, WF_PART_STRIPE = 1, 2, 4
WF_SCHED_FIXED, WF_SCHED_ADAPTIVE = 0, 1
WF_FIELD_S, WF_FIELD_T_2DF, WF_FIELD_D_2DF, WF_FIELD_T_RF, WF_FIELD_D_RF = range(5)

# every symbol include/wf.h declares
EXPORTS = ["wf_version", "wf_strerror", "wf_params_default", "wf_plan_create", "wf_plan_destroy",
           "wf_set_problem", "wf_run", "wf_iterate", "wf_residual", "wf_chi2_aug", "wf_get_field", "wf_solve",
           "wf_fft2", "wf_launch_count", "wf_time_passes", "wf_time_sweeps", "wf_get_trace", "wf_fft2_noalloc",
           "wf_batch_create", "wf_batch_destroy", "wf_batch_solve", "wf_batch_launch_count",
           "wf_fno_create", "wf_fno_destroy", "wf_fno_num_params", "wf_fno_forward", "wf_fno_gradient",
           "wf_fno_train_step", "wf_fno_get_params", "wf_fno_features", "wf_solve_warm", "wf_plan_shapes",
           "wf_inverse_noise"]


class wf_schedule(C.Structure):
    _fields_ = [("mode", C.c_int), ("lam", C.POINTER(C.c_double)), ("iters", C.POINTER(C.c_int)),
                ("nlevels", C.c_int), ("lam0", C.c_double), ("ratio", C.c_double),
                ("expo", C.c_double), ("snap", C.c_double)]


class wf_params(C.Structure):
    _fields_ = [("theta", C.c_double * 3), ("split_f", C.c_double), ("split_fp", C.c_double),
                ("split_w", C.c_double), ("tol_u_scale", C.c_double), ("residual_every", C.c_int), ("max_iters", C.c_int),
                ("check_every", C.c_int), ("merge_2df", C.c_int), ("refine", C.c_int),
                ("refine_tol_scale", C.c_double), ("refine_max_iters", C.c_int),
                ("refine_lam1_iters", C.c_int), ("stall_checks", C.c_int), ("autotune", C.c_int),
                ("dft_precision", C.c_int), ("refine_extra", C.c_int), ("sweep_kernel", C.c_int),
                ("trace", C.c_int), ("refine_accel", C.c_int)]


class wf_stats(C.Structure):
    _fields_ = [("iters", C.c_int), ("checkpoints", C.c_int), ("lam_final", C.c_double),
                ("rel_rho_u", C.c_double), ("rel_rho_m", C.c_double), ("tau", C.c_double * 3),
                ("status", C.c_int), ("parts", C.c_int)]

    def as_dict(self):
        return dict(iters=self.iters, checkpoints=self.checkpoints, lam_final=self.lam_final,
                    rel_rho_u=self.rel_rho_u, rel_rho_m=self.rel_rho_m, tau=list(self.tau),
                    status=self.status, parts=self.parts)


class wf_map(C.Structure):
    _fields_ = [("d", C.c_void_p), ("pixel_var", C.c_void_p), ("mask", C.c_void_p), ("C", C.c_void_p),
                ("P1f", C.c_void_p), ("Pst", C.c_void_p), ("stripe_amp2", C.c_void_p), ("s_out", C.c_void_p)]


class WFError(RuntimeError):
    def __init__(self, code, where=""):
        self.code = code
        super().__init__(f"{where}: {strerror(code)} (code {code})")


_LIB = None


def lib_path() -> str:
    return _build.LIB


def load(path: Optional[str] = None):
    """Load libwf.so (built in-tree by paper_1704_00865_gb300.build)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    p = path or lib_path()
    if not os.path.exists(p):
        raise RuntimeError(f"libwf.so not found at {p}: run paper_1704_00865_gb300.build.build()")
    L = C.CDLL(p)
    vp = C.c_void_p
    L.wf_version.restype = C.c_int
    L.wf_strerror.restype = C.c_char_p
    L.wf_strerror.argtypes = [C.c_int]
    L.wf_params_default.restype = None
    L.wf_params_default.argtypes = [C.POINTER(wf_params)]
    L.wf_plan_create.argtypes = [C.POINTER(vp), C.c_int, C.c_int, C.c_uint, C.POINTER(wf_params), vp]
    L.wf_plan_destroy.restype = None
    L.wf_plan_destroy.argtypes = [vp]
    L.wf_set_problem.argtypes = [vp] + [vp] * 7
    L.wf_run.argtypes = [vp, C.POINTER(wf_schedule), C.c_double, C.POINTER(wf_stats)]
    L.wf_iterate.argtypes = [vp, C.c_double, C.c_int]
    L.wf_residual.argtypes = [vp, C.POINTER(C.c_double), C.POINTER(C.c_double)]
    L.wf_chi2_aug.argtypes = [vp, C.POINTER(C.c_double)]
    L.wf_get_field.argtypes = [vp, C.c_int, vp]
    L.wf_solve.argtypes = [vp] + [vp] * 7 + [C.POINTER(wf_schedule), C.c_double, vp, C.POINTER(wf_stats)]
    L.wf_fft2.argtypes = [vp, vp, vp, C.c_int, C.c_int]
    L.wf_launch_count.argtypes = [vp]
    L.wf_time_passes.argtypes = [vp, C.c_double, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double)]
    L.wf_time_sweeps.argtypes = [vp, C.c_double, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_int)]
    L.wf_get_trace.argtypes = [vp, vp, C.c_int, C.POINTER(C.c_int)]
    L.wf_fft2_noalloc.argtypes = [C.c_int, C.c_int, vp, vp, C.c_int, vp]
    L.wf_batch_create.argtypes = [C.POINTER(vp), C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int), C.c_uint,
                                  C.POINTER(wf_params), C.c_int, vp]
    L.wf_batch_destroy.restype = None
    L.wf_batch_destroy.argtypes = [vp]
    L.wf_batch_solve.argtypes = [vp, C.POINTER(wf_map), C.POINTER(wf_schedule), C.c_double, C.POINTER(wf_stats)]
    L.wf_batch_launch_count.argtypes = [vp]
    L.wf_fno_create.argtypes = [C.POINTER(vp), C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, vp, vp]
    L.wf_fno_destroy.restype = None
    L.wf_fno_destroy.argtypes = [vp]
    L.wf_fno_num_params.argtypes = [vp]
    L.wf_fno_forward.argtypes = [vp, vp, vp, C.c_int]
    L.wf_fno_gradient.argtypes = [vp, vp, vp, C.c_int, vp, C.POINTER(C.c_double)]
    L.wf_fno_train_step.argtypes = [vp, vp, vp, C.c_int, C.c_double, C.POINTER(C.c_double)]
    L.wf_fno_get_params.argtypes = [vp, vp, C.c_int]
    L.wf_fno_features.argtypes = [C.c_int, C.c_int, vp, vp, vp, vp, vp, vp]
    L.wf_inverse_noise.argtypes = [vp] + [vp] * 6 + [C.c_double, C.POINTER(wf_schedule), C.c_double, vp,
                                                     C.POINTER(wf_stats)]
    L.wf_plan_shapes.argtypes = [vp, C.POINTER(C.c_int), C.POINTER(C.c_int)]
    L.wf_solve_warm.argtypes = [vp] + [vp] * 8 + [C.POINTER(wf_schedule), C.c_double, vp, C.POINTER(wf_stats)]
    for n in EXPORTS:
        if n not in ("wf_strerror", "wf_params_default", "wf_plan_destroy", "wf_launch_count",
                     "wf_batch_destroy", "wf_batch_launch_count", "wf_fno_destroy", "wf_fno_num_params"):
            getattr(L, n).restype = C.c_int
    L.wf_launch_count.restype = C.c_longlong
    L.wf_batch_launch_count.restype = C.c_longlong
    L.wf_fno_num_params.restype = C.c_longlong
    _LIB = L
    return L


def strerror(code: int) -> str:
    return load().wf_strerror(int(code)).decode()


def _check(code, where):
    if code != WF_OK:
        raise WFError(code, where)


def _ptr(a, dtype, n: Optional[int] = None, writable: bool = False):
    """(pointer, keepalive) for a torch tensor or numpy array."""
    if a is None:
        return None, None
    try:
        import torch
        if isinstance(a, torch.Tensor):
            tdt = {np.float32: torch.float32, np.uint8: torch.uint8}[dtype]
            if a.dtype != tdt or not a.is_contiguous():
                if writable:
                    raise ValueError("output tensor must be contiguous with the right dtype")
                a = a.to(tdt).contiguous()
            if n is not None and a.numel() != n:
                raise ValueError(f"expected {n} elements, got {a.numel()}")
            return C.c_void_p(a.data_ptr()), a
    except ImportError:  # pragma: no cover
        pass
    arr = np.asarray(a)
    if arr.dtype != dtype or not arr.flags.c_contiguous:
        if writable:
            raise ValueError("output array must be C-contiguous with the right dtype")
        arr = np.ascontiguousarray(arr, dtype=dtype)
    if n is not None and arr.size != n:
        raise ValueError(f"expected {n} elements, got {arr.size}")
    return C.c_void_p(arr.ctypes.data), arr


def wf_params_default() -> wf_params:
    p = wf_params()
    load().wf_params_default(C.byref(p))
    return p


def make_params(theta=None, split_f=None, split_w=None, residual_every=None, max_iters=None,
                check_every=None, merge_2df=None, tol_u_scale=None, split_fp=None,
                refine=None, refine_tol_scale=None, refine_max_iters=None,
                refine_lam1_iters=None, stall_checks=None, autotune=None,
                dft_precision=None, refine_extra=None, sweep_kernel=None, trace=None,
                refine_accel=None) -> wf_params:
    p = wf_params_default()
    if trace is not None:
        p.trace = int(trace)
    if refine_accel is not None:
        p.refine_accel = int(refine_accel)
    if sweep_kernel is not None:
        p.sweep_kernel = int(sweep_kernel)
    if refine_extra is not None:
        p.refine_extra = int(refine_extra)
    if dft_precision is not None:
        p.dft_precision = int(dft_precision)
    if autotune is not None:
        p.autotune = int(autotune)
    if stall_checks is not None:
        p.stall_checks = int(stall_checks)
    if refine_lam1_iters is not None:
        p.refine_lam1_iters = int(refine_lam1_iters)
    if refine_max_iters is not None:
        p.refine_max_iters = int(refine_max_iters)
    if refine_tol_scale is not None:
        p.refine_tol_scale = float(refine_tol_scale)
    if refine is not None:
        p.refine = int(refine)
    if split_fp is not None:
        p.split_fp = float(split_fp)
    if merge_2df is not None:
        p.merge_2df = int(bool(merge_2df))
    if tol_u_scale is not None:
        p.tol_u_scale = float(tol_u_scale)
    if theta is not None:
        for i in range(3):
            p.theta[i] = float(theta[i])
    if split_f is not None:
        p.split_f = float(split_f)
    if split_w is not None:
        p.split_w = float(split_w)
    if residual_every is not None:
        p.residual_every = int(residual_every)
    if max_iters is not None:
        p.max_iters = int(max_iters)
    if check_every is not None:
        p.check_every = int(check_every)
    return p


def make_schedule(mode="adaptive", lam: Sequence[float] = (), iters: Sequence[int] = (),
                  lam0=5e5, ratio=1e-2, expo=0.7, snap=1.01):
    s = wf_schedule()
    keep = []
    if mode in ("fixed", WF_SCHED_FIXED):
        la = (C.c_double * len(lam))(*lam)
        it = (C.c_int * len(iters))(*iters)
        keep = [la, it]
        s.mode = WF_SCHED_FIXED
        s.lam = C.cast(la, C.POINTER(C.c_double))
        s.iters = C.cast(it, C.POINTER(C.c_int))
        s.nlevels = len(lam)
    else:
        s.mode = WF_SCHED_ADAPTIVE
        s.lam0, s.ratio, s.expo, s.snap = lam0, ratio, expo, snap
    s._keep = keep
    return s


def _current_stream():
    try:
        import torch
        if torch.cuda.is_available():
            return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    except Exception:  # pragma: no cover
        pass
    return C.c_void_p(0)


def wf_plan_create(ny, nx, parts, params: Optional[wf_params] = None, stream=None):
    h = C.c_void_p()
    p = C.byref(params) if params is not None else None
    _check(load().wf_plan_create(C.byref(h), int(ny), int(nx), int(parts), p,
                                 stream if stream is not None else _current_stream()), "wf_plan_create")
    return h


class Plan:
    """A plan for ny x nx maps (see wf_plan_create in include/wf.h)."""

    def __init__(self, ny, nx, parts=WF_PART_WHITE | WF_PART_1F | WF_PART_STRIPE,
                 params: Optional[wf_params] = None, stream=None):
        self.ny, self.nx, self.parts = int(ny), int(nx), int(parts)
        self.params = params if params is not None else wf_params_default()
        self.h = wf_plan_create(ny, nx, parts, self.params, stream)
        self._keep = []

    def close(self):
        if self.h is not None and self.h.value:
            load().wf_plan_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- marshalling helpers
    def _problem_ptrs(self, d, pixel_var, mask, Cs, P1f, Pst, amp2):
        ny, nx = self.ny, self.nx
        nspec = ny * (nx // 2 + 1)
        out = [
            _ptr(d, np.float32, ny * nx), _ptr(pixel_var, np.float32, ny * nx),
            _ptr(mask, np.uint8, ny * nx), _ptr(Cs, np.float32, nspec),
            _ptr(P1f, np.float32, nspec), _ptr(Pst, np.float32, nx // 2 + 1),
            _ptr(amp2, np.float32, ny),
        ]
        self._keep = [k for _, k in out]
        return [p for p, _ in out]

    def set_problem(self, d, pixel_var, mask, Cs, P1f=None, Pst=None, stripe_amp2=None):
        ptrs = self._problem_ptrs(d, pixel_var, mask, Cs, P1f, Pst, stripe_amp2)
        _check(load().wf_set_problem(self.h, *ptrs), "wf_set_problem")

    def run(self, schedule, tol: float):
        st = wf_stats()
        rc = load().wf_run(self.h, C.byref(schedule), float(tol), C.byref(st))
        if rc not in _FINISHED:
            _check(rc, "wf_run")
        return st.as_dict()

    def iterate(self, lam: float, n: int):
        _check(load().wf_iterate(self.h, float(lam), int(n)), "wf_iterate")

    def residual(self):
        u, m = C.c_double(), C.c_double()
        _check(load().wf_residual(self.h, C.byref(u), C.byref(m)), "wf_residual")
        return u.value, m.value

    def chi2_aug(self) -> float:
        """Augmented objective of the current iterate (wf_chi2_aug)."""
        v = C.c_double()
        _check(load().wf_chi2_aug(self.h, C.byref(v)), "wf_chi2_aug")
        return v.value

    def get_field(self, field: int, out=None):
        if out is None:
            out = np.empty((self.ny, self.nx), np.float32)
        p, keep = _ptr(out, np.float32, self.ny * self.nx, writable=True)
        _check(load().wf_get_field(self.h, int(field), p), "wf_get_field")
        return out

    def solve(self, d, pixel_var, mask, Cs, P1f, Pst, stripe_amp2, schedule, tol, out=None):
        if out is None:
            out = np.empty((self.ny, self.nx), np.float32)
        ptrs = self._problem_ptrs(d, pixel_var, mask, Cs, P1f, Pst, stripe_amp2)
        po, keep = _ptr(out, np.float32, self.ny * self.nx, writable=True)
        st = wf_stats()
        rc = load().wf_solve(self.h, *ptrs, C.byref(schedule), float(tol), po, C.byref(st))
        if rc not in _FINISHED:
            _check(rc, "wf_solve")
        return out, st.as_dict()

    def inverse_noise(self, d, pixel_var, mask, P1f, Pst, stripe_amp2, alpha, schedule, tol, out=None):
        """Approximately N^-1 d through a Wiener filter with S = alpha I
        (see wf_inverse_noise)."""
        if out is None:
            out = np.empty((self.ny, self.nx), np.float32)
        ny, nx = self.ny, self.nx
        nspec = ny * (nx // 2 + 1)
        ptrs = [_ptr(d, np.float32, ny * nx), _ptr(pixel_var, np.float32, ny * nx), _ptr(mask, np.uint8, ny * nx),
                _ptr(P1f, np.float32, nspec), _ptr(Pst, np.float32, nx // 2 + 1), _ptr(stripe_amp2, np.float32, ny)]
        po, ko = _ptr(out, np.float32, ny * nx, writable=True)
        st = wf_stats()
        rc = load().wf_inverse_noise(self.h, *[p for p, _ in ptrs], float(alpha), C.byref(schedule), float(tol), po,
                                     C.byref(st))
        if rc not in _FINISHED:
            _check(rc, "wf_inverse_noise")
        return out, st.as_dict()

    def solve_warm(self, d, pixel_var, mask, Cs, P1f, Pst, stripe_amp2, s_init, schedule, tol, out=None):
        """wf_solve started from the estimate s_init (see wf_solve_warm)."""
        if out is None:
            out = np.empty((self.ny, self.nx), np.float32)
        ptrs = self._problem_ptrs(d, pixel_var, mask, Cs, P1f, Pst, stripe_amp2)
        pi, ki = _ptr(s_init, np.float32, self.ny * self.nx)
        po, keep = _ptr(out, np.float32, self.ny * self.nx, writable=True)
        st = wf_stats()
        rc = load().wf_solve_warm(self.h, *ptrs, pi, C.byref(schedule), float(tol), po, C.byref(st))
        if rc not in _FINISHED:
            _check(rc, "wf_solve_warm")
        return out, st.as_dict()

    def fft2(self, x, inverse=False, rows_only=False, out=None):
        n = self.ny * self.nx
        if out is None:
            out = np.empty(n, np.float32)
        pi, ki = _ptr(x, np.float32, n)
        po, ko = _ptr(out, np.float32, n, writable=True)
        _check(load().wf_fft2(self.h, pi, po, int(bool(inverse)), int(bool(rows_only))), "wf_fft2")
        return out


    def launch_count(self) -> int:
        return int(load().wf_launch_count(self.h))

    def shapes(self):
        """(values per thread of the row pass, of the column pass)."""
        r, c = C.c_int(), C.c_int()
        _check(load().wf_plan_shapes(self.h, C.byref(r), C.byref(c)), "wf_plan_shapes")
        return r.value, c.value

    def trace(self):
        """Per-checkpoint records of the runs since the last load (wf_get_trace):
        a list of dicts with sweeps, lam, rel_rho_u, rel_rho_m, chi2_aug, run."""
        n = C.c_int()
        _check(load().wf_get_trace(self.h, None, 0, C.byref(n)), "wf_get_trace")
        buf = np.empty((max(n.value, 1), 6), np.float64)
        _check(load().wf_get_trace(self.h, C.c_void_p(buf.ctypes.data), n.value, C.byref(n)), "wf_get_trace")
        keys = ("sweeps", "lam", "rel_rho_u", "rel_rho_m", "chi2_aug", "run")
        return [{k: (int(v) if k in ("sweeps", "run") else float(v)) for k, v in zip(keys, row)}
                for row in buf[:n.value]]

    def time_sweeps(self, lam: float, n: int):
        """Mean CUDA-event time (us) of one sweep as the plan launches it, and
        whether that is the one-launch form."""
        us, one = C.c_double(), C.c_int()
        _check(load().wf_time_sweeps(self.h, float(lam), int(n), C.byref(us), C.byref(one)), "wf_time_sweeps")
        return us.value, bool(one.value)

    def time_passes(self, lam: float, n: int):
        """Mean CUDA-event time (us) of the row pass and of the column pass."""
        r, c = C.c_double(), C.c_double()
        _check(load().wf_time_passes(self.h, float(lam), int(n), C.byref(r), C.byref(c)), "wf_time_passes")
        return r.value, c.value


def wf_fft2_noalloc(ny: int, nx: int, x, out, inverse: bool = False, stream=None):
    """The 2D transform without a plan or any device allocation (device
    tensors in and out; see include/wf.h).  Returns after launching.  x must
    already be a contiguous float32 tensor: a converted copy would be a
    temporary allocation that could be freed while the transform, queued on
    `stream`, still reads it."""
    import torch
    if not (isinstance(x, torch.Tensor) and x.dtype == torch.float32 and x.is_contiguous()):
        raise ValueError("wf_fft2_noalloc: x must be a contiguous float32 tensor")
    pi, ki = _ptr(x, np.float32, ny * nx)
    po, ko = _ptr(out, np.float32, ny * nx, writable=True)
    _check(load().wf_fft2_noalloc(int(ny), int(nx), pi, po, int(bool(inverse)),
                                  stream if stream is not None else _current_stream()), "wf_fft2_noalloc")
    return out


class Batch:
    """Plans for many independent maps of uneven sizes solved together
    (see wf_batch_create / wf_batch_solve in include/wf.h)."""

    def __init__(self, shapes, parts=WF_PART_WHITE | WF_PART_1F | WF_PART_STRIPE,
                 params: Optional[wf_params] = None, lanes: int = 8, stream=None):
        self.shapes = [(int(a), int(b)) for a, b in shapes]
        n = len(self.shapes)
        ny = (C.c_int * max(n, 1))(*[a for a, _ in self.shapes])
        nx = (C.c_int * max(n, 1))(*[b for _, b in self.shapes])
        self.params = params if params is not None else wf_params_default()
        self.h = C.c_void_p()
        _check(load().wf_batch_create(C.byref(self.h), n, ny, nx, int(parts), C.byref(self.params), int(lanes),
                                      stream if stream is not None else _current_stream()), "wf_batch_create")

    def close(self):
        if self.h is not None and self.h.value:
            load().wf_batch_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def solve(self, problems, schedule, tol, outs):
        """problems: sequence of (d, pixel_var, mask, C, P1f, Pst, stripe_amp2)
        in the batch's map order; outs: one output per map.  Returns (status,
        list of stats dicts)."""
        n = len(self.shapes)
        if len(problems) != n or len(outs) != n:
            raise ValueError("one problem and one output per map")
        maps = (wf_map * n)()
        keep = []
        for i, ((ny, nx), pr, out) in enumerate(zip(self.shapes, problems, outs)):
            d, pv, mask, Cs, P1f, Pst, amp2 = pr
            nspec = ny * (nx // 2 + 1)
            ptrs = [_ptr(d, np.float32, ny * nx), _ptr(pv, np.float32, ny * nx), _ptr(mask, np.uint8, ny * nx),
                    _ptr(Cs, np.float32, nspec), _ptr(P1f, np.float32, nspec), _ptr(Pst, np.float32, nx // 2 + 1),
                    _ptr(amp2, np.float32, ny), _ptr(out, np.float32, ny * nx, writable=True)]
            keep.extend(k for _, k in ptrs)
            for f, (pp, _) in zip(("d", "pixel_var", "mask", "C", "P1f", "Pst", "stripe_amp2", "s_out"), ptrs):
                setattr(maps[i], f, pp)
        stats = (wf_stats * n)()
        rc = load().wf_batch_solve(self.h, maps, C.byref(schedule), float(tol), stats)
        if rc not in _FINISHED:
            _check(rc, "wf_batch_solve")
        return rc, [s.as_dict() for s in stats]

    def launch_count(self) -> int:
        return int(load().wf_batch_launch_count(self.h))


class FNO:
    """The warm-start network and its training state (wf_fno_* in include/wf.h).
    Arrays passed to forward / gradient / train_step are CUDA tensors."""

    def __init__(self, n, batch, params, width=32, mx=16, my=16, layers=4, stream=None):
        self.n, self.batch, self.width, self.mx, self.my, self.layers = n, batch, width, mx, my, layers
        pp, keep = _ptr(params, np.float32)
        self.h = C.c_void_p()
        _check(load().wf_fno_create(C.byref(self.h), int(n), int(batch), int(width), int(mx), int(my), int(layers),
                                    pp, stream if stream is not None else _current_stream()), "wf_fno_create")
        self.num_params = int(load().wf_fno_num_params(self.h))

    def close(self):
        if self.h is not None and self.h.value:
            load().wf_fno_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def forward(self, x, y, nb):
        px, kx = _ptr(x, np.float32)
        py, ky = _ptr(y, np.float32, writable=True)
        _check(load().wf_fno_forward(self.h, px, py, int(nb)), "wf_fno_forward")
        return y

    def gradient(self, x, t, nb):
        g = np.empty(self.num_params, np.float32)
        px, kx = _ptr(x, np.float32)
        pt, kt = _ptr(t, np.float32)
        l = C.c_double()
        _check(load().wf_fno_gradient(self.h, px, pt, int(nb), C.c_void_p(g.ctypes.data), C.byref(l)),
               "wf_fno_gradient")
        return l.value, g

    def train_step(self, x, t, nb, lr):
        px, kx = _ptr(x, np.float32)
        pt, kt = _ptr(t, np.float32)
        l = C.c_double()
        _check(load().wf_fno_train_step(self.h, px, pt, int(nb), float(lr), C.byref(l)), "wf_fno_train_step")
        return l.value

    def params(self, rounded=False):
        out = np.empty(self.num_params, np.float32)
        _check(load().wf_fno_get_params(self.h, C.c_void_p(out.ctypes.data), int(bool(rounded))), "wf_fno_get_params")
        return out


def fno_features(d, pixel_var, mask, x_out, sigma_out, stream=None):
    """Network input of one map into x_out [2, ny, nx] and sigma into
    sigma_out (CUDA tensors; see wf_fno_features)."""
    ny, nx = d.shape
    pd, kd = _ptr(d, np.float32)
    pv, kv = _ptr(pixel_var, np.float32)
    pm, km = _ptr(mask, np.uint8)
    px, kx = _ptr(x_out, np.float32, writable=True)
    ps, ks = _ptr(sigma_out, np.float32, writable=True)
    _check(load().wf_fno_features(int(ny), int(nx), pd, pv, pm, px, ps,
                                  stream if stream is not None else _current_stream()), "wf_fno_features")
    return x_out


def parts_of(prob) -> int:
    """Parts bit mask for a synth.Problem."""
    p = WF_PART_WHITE
    if prob.P1f is not None:
        p |= WF_PART_1F
    if prob.Pst is not None:
        p |= WF_PART_STRIPE
    return p
