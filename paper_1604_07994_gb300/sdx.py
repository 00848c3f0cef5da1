"""Thin ctypes binding of libsdx.so (C ABI in include/sdx.h).

Argument marshalling only: every operation runs in the library's CUDA kernels.  Device
vectors are passed as torch CUDA tensors (float64, contiguous, 4*(n+1)^3 elements, SoA
u_x, u_y, u_z, p) or raw integer device pointers; the stream defaults to torch's current
stream.  The library must have been built (``paper_1604_07994_gb300.build.build()``); there
is no fallback of any kind when it is missing.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_lib", "libsdx.so")

OK, EINVAL, ENOMEM, ENONFINITE, ENOCONV, ECUDA, ESINGULAR = 0, -1, -2, -3, -4, -5, -6
FACE_DIRICHLET, FACE_FREESLIP, FACE_TRACTION = 0, 1, 2
FORM_DECOUPLED, FORM_STRAIN, FORM_GRADIENT = 0, 1, 2
FORMS = {"tr": FORM_DECOUPLED, "decoupled": FORM_DECOUPLED, "sym": FORM_STRAIN,
         "strain": FORM_STRAIN, "grad": FORM_GRADIENT, "gradient": FORM_GRADIENT}
PREC_FP64, PREC_FP32_REFINED = 0, 1
OUTER_VCYCLE, OUTER_FGMRES = 0, 1
NOALLOC_MAX_ROWS = 65536

EXPORTED = ("sdx_create", "sdx_destroy", "sdx_levels", "sdx_level_size", "sdx_constraint_mask",
            "sdx_interface_mask", "sdx_apply", "sdx_residual", "sdx_rhs", "sdx_uzawa", "sdx_smooth_pass",
            "sdx_kernel_launches", "sdx_smooth_pass_noalloc", "sdx_apply_f32", "sdx_smooth_pass_f32",
            "sdx_restrict", "sdx_prolong_add", "sdx_vcycle", "sdx_solve", "sdx_solve_host",
            "sdx_last_error", "sdx_strerror")


class SdxError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"sdx error {code}: {msg}")
        self.code = code


class sdx_desc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("n_coarse", ctypes.c_int),
                ("cell_id", ctypes.POINTER(ctypes.c_uint8)), ("mu", ctypes.POINTER(ctypes.c_double)),
                ("n_mu", ctypes.c_int), ("face", ctypes.c_int * 6), ("form", ctypes.c_int),
                ("coarse_form", ctypes.c_int), ("prec", ctypes.c_int), ("pspg_beta", ctypes.c_double)]


class sdx_stats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("restarts", ctypes.c_int), ("res0", ctypes.c_double),
                ("res", ctypes.c_double), ("bnorm", ctypes.c_double), ("status", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def load() -> ctypes.CDLL:
    """Load libsdx.so (once).  Raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_1604_07994_gb300.build.build()")
    lib = ctypes.CDLL(LIB_PATH)
    P, I, D, L = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_int64
    sig = {
        "sdx_create": [ctypes.POINTER(sdx_desc), ctypes.POINTER(P)],
        "sdx_destroy": [P],
        "sdx_levels": [P, ctypes.POINTER(I)],
        "sdx_level_size": [P, I, ctypes.POINTER(I), ctypes.POINTER(L), ctypes.POINTER(L)],
        "sdx_constraint_mask": [P, I, P],
        "sdx_interface_mask": [P, I, P],
        "sdx_apply": [P, I, P, P, P],
        "sdx_residual": [P, I, P, P, P, P],
        "sdx_rhs": [P, P, P, P],
        "sdx_uzawa": [P, I, P, P, P],
        "sdx_smooth_pass": [P, I, I, I, P, P, P],
        "sdx_smooth_pass_noalloc": [P, I, I, P, P, P],
        "sdx_apply_f32": [P, I, P, P, P],
        "sdx_smooth_pass_f32": [P, I, I, I, P, P, P],
        "sdx_restrict": [P, I, P, P, P],
        "sdx_prolong_add": [P, I, P, P, P],
        "sdx_vcycle": [P, P, P, P],
        "sdx_solve": [P, P, P, D, I, I, I, ctypes.POINTER(sdx_stats), P],
        "sdx_solve_host": [P, P, P, D, I, I, I, ctypes.POINTER(sdx_stats), P],
    }
    for name, args in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int
    lib.sdx_kernel_launches.argtypes = []
    lib.sdx_kernel_launches.restype = ctypes.c_int64
    lib.sdx_last_error.argtypes = []
    lib.sdx_last_error.restype = ctypes.c_char_p
    lib.sdx_strerror.argtypes = [ctypes.c_int]
    lib.sdx_strerror.restype = ctypes.c_char_p
    _lib = lib
    return lib


def _check(code: int, allow=(OK,)) -> int:
    if code not in allow:
        raise SdxError(code, load().sdx_last_error().decode())
    return code


def _ptr(t, itemsize: int = 8) -> int:
    if t is None:
        return None
    if isinstance(t, int):
        return t
    if t.dtype.itemsize != itemsize or not t.is_contiguous() or not t.is_cuda:
        raise ValueError(f"vectors must be contiguous {8 * itemsize}-bit float CUDA tensors")
    return t.data_ptr()


def _stream(stream) -> Optional[int]:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


class Hierarchy:
    """A grid hierarchy built by sdx_create (owned; freed by close() or on deletion)."""

    def __init__(self, n: int, n_coarse: int, cell_id: np.ndarray, mu: Sequence[float],
                 face: Sequence[int], form="tr", coarse_form=None, prec=PREC_FP64,
                 beta: float = 1.0 / 12.0):
        lib = load()
        self._cell = np.ascontiguousarray(np.asarray(cell_id, dtype=np.uint8).ravel())
        self._mu = np.ascontiguousarray(np.asarray(mu, dtype=np.float64))
        d = sdx_desc()
        d.n, d.n_coarse = int(n), int(n_coarse)
        d.cell_id = self._cell.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))
        d.mu = self._mu.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        d.n_mu = int(self._mu.size)
        for f in range(6):
            d.face[f] = int(face[f])
        d.form = FORMS[form] if isinstance(form, str) else int(form)
        if coarse_form is None:
            d.coarse_form = -1
        else:
            d.coarse_form = FORMS[coarse_form] if isinstance(coarse_form, str) else int(coarse_form)
        d.prec = int(prec)
        d.pspg_beta = float(beta)
        h = ctypes.c_void_p()
        _check(lib.sdx_create(ctypes.byref(d), ctypes.byref(h)))
        self._h = h
        self.n = int(n)
        self.nn = (self.n + 1) ** 3

    @classmethod
    def from_problem(cls, problem, form="tr", coarse_form=None, prec=PREC_FP64, beta=1.0 / 12.0):
        return cls(problem.n, problem.n_coarse, problem.cell_id, problem.mu, problem.face, form,
                   coarse_form, prec, beta)

    def close(self):
        if getattr(self, "_h", None):
            load().sdx_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---------------------------------------------------------------- queries
    def sdx_levels(self) -> int:
        v = ctypes.c_int()
        _check(load().sdx_levels(self._h, ctypes.byref(v)))
        return v.value

    def sdx_level_size(self, level: int):
        n, nodes, free = ctypes.c_int(), ctypes.c_int64(), ctypes.c_int64()
        _check(load().sdx_level_size(self._h, level, ctypes.byref(n), ctypes.byref(nodes), ctypes.byref(free)))
        return n.value, nodes.value, free.value

    def sdx_constraint_mask(self, level: int = 0) -> np.ndarray:
        _, nodes, _ = self.sdx_level_size(level)
        m = np.zeros(4 * nodes, dtype=np.uint8)
        _check(load().sdx_constraint_mask(self._h, level, m.ctypes.data))
        return m.astype(bool)

    def sdx_interface_mask(self, level: int = 0) -> np.ndarray:
        _, nodes, _ = self.sdx_level_size(level)
        m = np.zeros(nodes, dtype=np.uint8)
        _check(load().sdx_interface_mask(self._h, level, m.ctypes.data))
        return m.astype(bool)

    # ---------------------------------------------------------------- operations
    def sdx_apply(self, level, x, y, stream=None):
        _check(load().sdx_apply(self._h, level, _ptr(x), _ptr(y), _stream(stream)))

    def sdx_residual(self, level, b, x, r, stream=None):
        _check(load().sdx_residual(self._h, level, _ptr(b), _ptr(x), _ptr(r), _stream(stream)))

    def sdx_rhs(self, f, b, stream=None):
        _check(load().sdx_rhs(self._h, _ptr(f), _ptr(b), _stream(stream)))

    def sdx_uzawa(self, level, b, x, stream=None):
        _check(load().sdx_uzawa(self._h, level, _ptr(b), _ptr(x), _stream(stream)))

    def sdx_smooth_pass(self, level, which, colour, b, x, stream=None):
        _check(load().sdx_smooth_pass(self._h, level, which, colour, _ptr(b), _ptr(x), _stream(stream)))

    def sdx_apply_f32(self, level, x, y, stream=None):
        _check(load().sdx_apply_f32(self._h, level, _ptr(x, 4), _ptr(y, 4), _stream(stream)))

    def sdx_smooth_pass_f32(self, level, which, colour, b, x, stream=None):
        _check(load().sdx_smooth_pass_f32(self._h, level, which, colour, _ptr(b, 4), _ptr(x, 4), _stream(stream)))

    def sdx_smooth_pass_noalloc(self, level, colour, b, x, stream=None):
        _check(load().sdx_smooth_pass_noalloc(self._h, level, colour, _ptr(b), _ptr(x), _stream(stream)))

    def sdx_restrict(self, level, r_fine, b_coarse, stream=None):
        _check(load().sdx_restrict(self._h, level, _ptr(r_fine), _ptr(b_coarse), _stream(stream)))

    def sdx_prolong_add(self, level, e_coarse, x_fine, stream=None):
        _check(load().sdx_prolong_add(self._h, level, _ptr(e_coarse), _ptr(x_fine), _stream(stream)))

    def sdx_vcycle(self, b, x, stream=None):
        _check(load().sdx_vcycle(self._h, _ptr(b), _ptr(x), _stream(stream)))

    def sdx_solve(self, b, x, rtol=1e-8, maxit=100, outer=OUTER_FGMRES, restart=30, stream=None,
                  allow_noconv=False) -> dict:
        st = sdx_stats()
        allow = (OK, ENOCONV) if allow_noconv else (OK,)
        _check(load().sdx_solve(self._h, _ptr(b), _ptr(x), float(rtol), int(maxit), int(outer),
                                int(restart), ctypes.byref(st), _stream(stream)), allow)
        return st.as_dict()

    def sdx_solve_host(self, b_host: np.ndarray, x_host: np.ndarray, rtol=1e-8, maxit=100,
                       outer=OUTER_FGMRES, restart=30, stream=None, allow_noconv=False) -> dict:
        for a in (b_host, x_host):
            if a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"] or a.size != 4 * self.nn:
                raise ValueError("host vectors must be contiguous float64 of 4*(n+1)^3 entries")
        st = sdx_stats()
        allow = (OK, ENOCONV) if allow_noconv else (OK,)
        _check(load().sdx_solve_host(self._h, b_host.ctypes.data, x_host.ctypes.data, float(rtol),
                                     int(maxit), int(outer), int(restart), ctypes.byref(st),
                                     _stream(stream)), allow)
        return st.as_dict()


def sdx_kernel_launches() -> int:
    return int(load().sdx_kernel_launches())
