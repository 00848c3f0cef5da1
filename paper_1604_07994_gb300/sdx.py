"""Thin ctypes binding of libsdx.so (C ABI in include/sdx.h).

Argument marshalling only: every operation runs in the library's CUDA kernels.  Device
vectors are passed as torch CUDA tensors (float64, contiguous, 4*(n+1)^3 elements, SoA
u_x, u_y, u_z, p) or raw integer device pointers; the stream defaults to torch's current
stream.  A tensor argument must have exactly the entries of its grid level (checked here,
before the call, since the library receives bare pointers); raw pointers are the caller's
responsibility.  The library must have been built (``paper_1604_07994_gb300.build.build()``); there
is no fallback of any kind when it is missing.
"""
from __future__ import annotations

import ctypes
import os
import threading
from typing import Optional, Sequence

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_lib", "libsdx.so")

OK, EINVAL, ENOMEM, ENONFINITE, ENOCONV, ECUDA, ESINGULAR, ETIMEOUT = 0, -1, -2, -3, -4, -5, -6, -7
FACE_DIRICHLET, FACE_FREESLIP, FACE_TRACTION = 0, 1, 2
FORM_DECOUPLED, FORM_STRAIN, FORM_GRADIENT = 0, 1, 2
FORMS = {"tr": FORM_DECOUPLED, "decoupled": FORM_DECOUPLED, "sym": FORM_STRAIN,
         "strain": FORM_STRAIN, "grad": FORM_GRADIENT, "gradient": FORM_GRADIENT}
PREC_FP64, PREC_FP32_REFINED = 0, 1
OUTER_VCYCLE, OUTER_FGMRES = 0, 1
# P1-P1 stabilisation constant beta of tau_T = beta h^2 / mu_T (not printed in the paper; 1/24
# gives the depth-independent decoupled multigrid rates that its Sec. 5 table reports)
PSPG_BETA = 1.0 / 24.0
NOALLOC_MAX_ROWS = 65536

EXPORTED = ("sdx_create", "sdx_destroy", "sdx_levels", "sdx_level_size", "sdx_constraint_mask",
            "sdx_interface_mask", "sdx_apply", "sdx_residual", "sdx_rhs", "sdx_uzawa", "sdx_smooth_pass",
            "sdx_kernel_launches", "sdx_smooth_pass_noalloc", "sdx_apply_f32", "sdx_smooth_pass_f32",
            "sdx_uzawa_f32", "sdx_p0_create", "sdx_p0_destroy", "sdx_p0_size", "sdx_p0_apply",
            "sdx_p0_residual", "sdx_p0_rhs", "sdx_p0_uzawa", "sdx_p0_vcycle", "sdx_p0_solve", "sdx_p0_fluxes",
            "sdx_restrict", "sdx_prolong_add", "sdx_vcycle", "sdx_solve", "sdx_solve_host",
            "sdx_batch_create", "sdx_batch_destroy", "sdx_batch_size", "sdx_batch_shape", "sdx_batch_instance",
            "sdx_batch_vcycle", "sdx_batch_solve", "sdx_net_param_count", "sdx_net_create",
            "sdx_net_destroy", "sdx_net_get_params", "sdx_net_set_params", "sdx_net_forward",
            "sdx_net_loss_grad", "sdx_net_train", "sdx_conv3", "sdx_conv3_wgrad", "sdx_conv3_dgrad",
            "sdx_guess_features",
            "sdx_guess_target", "sdx_guess_predict", "sdx_guess_refine", "sdx_last_error", "sdx_strerror")


class SdxError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"sdx error {code}: {msg}")
        self.code = code


class sdx_desc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("n_coarse", ctypes.c_int),
                ("cell_id", ctypes.POINTER(ctypes.c_uint8)), ("mu", ctypes.POINTER(ctypes.c_double)),
                ("n_mu", ctypes.c_int), ("face", ctypes.c_int * 6), ("form", ctypes.c_int),
                ("coarse_form", ctypes.c_int), ("prec", ctypes.c_int), ("pspg_beta", ctypes.c_double),
                ("coarsest_form", ctypes.c_int), ("coarse_correction", ctypes.c_int),
                ("coarsening", ctypes.c_int)]


class sdx_stats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("restarts", ctypes.c_int), ("res0", ctypes.c_double),
                ("res", ctypes.c_double), ("bnorm", ctypes.c_double), ("status", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None
_load_lock = threading.Lock()


def load() -> ctypes.CDLL:
    """Load libsdx.so (once, thread-safe).  Raises if it has not been built."""
    if _lib is not None:
        return _lib
    with _load_lock:
        return _lib if _lib is not None else _load_locked()


def _load_locked() -> ctypes.CDLL:
    global _lib
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
        "sdx_uzawa_f32": [P, I, P, P, I, P],
        "sdx_p0_create": [ctypes.POINTER(sdx_desc), D, ctypes.POINTER(P)],
        "sdx_p0_destroy": [P],
        "sdx_p0_size": [P, I, ctypes.POINTER(I), ctypes.POINTER(L), ctypes.POINTER(L), ctypes.POINTER(L)],
        "sdx_p0_apply": [P, I, P, P, P],
        "sdx_p0_residual": [P, I, P, P, P, P],
        "sdx_p0_rhs": [P, P, P, P],
        "sdx_p0_uzawa": [P, I, P, P, P],
        "sdx_p0_vcycle": [P, P, P, P],
        "sdx_p0_solve": [P, P, P, D, I, I, I, ctypes.POINTER(sdx_stats), P],
        "sdx_p0_fluxes": [P, P, P, P, P],
        "sdx_restrict": [P, I, P, P, P],
        "sdx_prolong_add": [P, I, P, P, P],
        "sdx_vcycle": [P, P, P, P],
        "sdx_solve": [P, P, P, D, I, I, I, ctypes.POINTER(sdx_stats), P],
        "sdx_solve_host": [P, P, P, D, I, I, I, ctypes.POINTER(sdx_stats), P],
        "sdx_batch_create": [ctypes.POINTER(sdx_desc), I, I, ctypes.POINTER(P)],
        "sdx_batch_destroy": [P],
        "sdx_batch_size": [P, I, ctypes.POINTER(I), ctypes.POINTER(L), ctypes.POINTER(L)],
        "sdx_batch_shape": [P, I, ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(I)],
        "sdx_batch_vcycle": [P, P, P, P],
        "sdx_batch_instance": [P, I, ctypes.POINTER(P)],
        "sdx_batch_solve": [P, P, P, D, I, I, ctypes.POINTER(sdx_stats), P],
        "sdx_net_create": [ctypes.c_uint64, ctypes.POINTER(P)],
        "sdx_net_destroy": [P],
        "sdx_net_get_params": [P, P],
        "sdx_net_set_params": [P, P],
        "sdx_net_forward": [P, I, P, P, P],
        "sdx_net_loss_grad": [P, I, P, P, ctypes.POINTER(D), P, P],
        "sdx_net_train": [P, I, I, P, P, I, I, ctypes.c_float, ctypes.c_uint64, P, P],
        "sdx_conv3": [I, I, I, P, P, P, I, P, P],
        "sdx_conv3_wgrad": [I, I, I, P, P, P, P],
        "sdx_conv3_dgrad": [I, I, I, P, P, P, P],
        "sdx_guess_features": [P, P, P, ctypes.POINTER(D), P],
        "sdx_guess_target": [P, P, D, P, P],
        "sdx_guess_predict": [P, P, P, P, P],
        "sdx_guess_refine": [P, P, P, I, P],
    }
    for name, args in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int
    lib.sdx_net_param_count.argtypes = []
    lib.sdx_net_param_count.restype = ctypes.c_int64
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
        raise ValueError(f"tensors must be contiguous CUDA tensors of {8 * itemsize}-bit elements")
    return t.data_ptr()


def _check_len(t, count: int) -> None:
    """The C ABI takes bare pointers, so a tensor shorter than its grid would let the kernels
    run past its end: check the length.  Raw integer pointers are not checked (their extent is
    the caller's promise)."""
    if t is not None and not isinstance(t, int) and t.numel() != count:
        raise ValueError(f"vector has {t.numel()} elements where {count} are needed")


def _vecs(*pairs, itemsize: int = 8):
    """Device pointers of several (tensor, length) arguments; every length is checked before
    any pointer is taken."""
    for t, m in pairs:
        _check_len(t, m)
    return [_ptr(t, itemsize) for t, _ in pairs]


def _stream(stream) -> Optional[int]:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _form(f):
    if f is None:
        return -1
    return FORMS[f] if isinstance(f, str) else int(f)


COARSENING = {"resolved": 0, "majority": 1}


def _make_desc(n, n_coarse, cell_id, mu, face, form, coarse_form, prec, beta, coarsest_form=None,
               coarse_correction=False, coarsening="resolved"):
    """An sdx_desc for the arguments, plus the host arrays it points into (keep them alive)."""
    cell = np.ascontiguousarray(np.asarray(cell_id, dtype=np.uint8).ravel())
    mu_a = np.ascontiguousarray(np.asarray(mu, dtype=np.float64))
    d = sdx_desc()
    d.n, d.n_coarse = int(n), int(n_coarse)
    d.cell_id = cell.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))
    d.mu = mu_a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    d.n_mu = int(mu_a.size)
    for f in range(6):
        d.face[f] = int(face[f])
    d.form = FORMS[form] if isinstance(form, str) else int(form)
    if coarse_form is None:
        d.coarse_form = -1
    else:
        d.coarse_form = FORMS[coarse_form] if isinstance(coarse_form, str) else int(coarse_form)
    d.prec = int(prec)
    d.pspg_beta = float(beta)
    d.coarsest_form = _form(coarsest_form)
    d.coarse_correction = 1 if coarse_correction else 0
    d.coarsening = COARSENING[coarsening] if isinstance(coarsening, str) else int(coarsening)
    return d, (cell, mu_a)


class Hierarchy:
    """A grid hierarchy built by sdx_create (owned; freed by close() or on deletion)."""

    def __init__(self, n: int, n_coarse: int, cell_id: np.ndarray, mu: Sequence[float],
                 face: Sequence[int], form="tr", coarse_form=None, prec=PREC_FP64,
                 beta: float = PSPG_BETA, coarsest_form=None, coarse_correction: bool = False,
                 coarsening="resolved"):
        lib = load()
        d, self._keep = _make_desc(n, n_coarse, cell_id, mu, face, form, coarse_form, prec, beta,
                                   coarsest_form, coarse_correction, coarsening)
        h = ctypes.c_void_p()
        _check(lib.sdx_create(ctypes.byref(d), ctypes.byref(h)))
        self._h = h
        self.n = int(n)
        self.nn = (self.n + 1) ** 3

    @classmethod
    def from_problem(cls, problem, form="tr", coarse_form=None, prec=PREC_FP64, beta=PSPG_BETA,
                     coarsest_form=None, coarse_correction=False, coarsening="resolved"):
        return cls(problem.n, problem.n_coarse, problem.cell_id, problem.mu, problem.face, form,
                   coarse_form, prec, beta, coarsest_form, coarse_correction, coarsening)

    @classmethod
    def paper_coarse_variant(cls, problem, prec=PREC_FP64, beta=PSPG_BETA):
        """The coarse-grid variant of Sec. 5: decoupled form a_tr on every level but the
        coarsest, which takes a_sym with the corrected momentum right-hand side."""
        return cls.from_problem(problem, form="tr", coarse_form="tr", prec=prec, beta=beta,
                                coarsest_form="sym", coarse_correction=True)

    def close(self):
        if getattr(self, "_borrowed", False):
            self._h = None
            return
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

    def _len(self, level: int, comps: int = 4) -> int:
        """Entries of a vector of `comps` components on grid level `level`."""
        if level == 0:
            return comps * self.nn
        cache = self.__dict__.setdefault("_level_nodes", {})
        if level not in cache:
            cache[level] = self.sdx_level_size(level)[1]
        return comps * cache[level]

    # ---------------------------------------------------------------- operations
    def sdx_apply(self, level, x, y, stream=None):
        m = self._len(level)
        px, py = _vecs((x, m), (y, m))
        _check(load().sdx_apply(self._h, level, px, py, _stream(stream)))

    def sdx_residual(self, level, b, x, r, stream=None):
        m = self._len(level)
        pb, px, pr = _vecs((b, m), (x, m), (r, m))
        _check(load().sdx_residual(self._h, level, pb, px, pr, _stream(stream)))

    def sdx_rhs(self, f, b, stream=None):
        pf, pb = _vecs((f, self._len(0, 3)), (b, self._len(0)))
        _check(load().sdx_rhs(self._h, pf, pb, _stream(stream)))

    def sdx_uzawa(self, level, b, x, stream=None):
        m = self._len(level)
        pb, px = _vecs((b, m), (x, m))
        _check(load().sdx_uzawa(self._h, level, pb, px, _stream(stream)))

    def sdx_smooth_pass(self, level, which, colour, b, x, stream=None):
        m = self._len(level)
        pb, px = _vecs((b, m), (x, m))
        _check(load().sdx_smooth_pass(self._h, level, which, colour, pb, px, _stream(stream)))

    def sdx_apply_f32(self, level, x, y, stream=None):
        m = self._len(level)
        px, py = _vecs((x, m), (y, m), itemsize=4)
        _check(load().sdx_apply_f32(self._h, level, px, py, _stream(stream)))

    def sdx_smooth_pass_f32(self, level, which, colour, b, x, stream=None):
        m = self._len(level)
        pb, px = _vecs((b, m), (x, m), itemsize=4)
        _check(load().sdx_smooth_pass_f32(self._h, level, which, colour, pb, px, _stream(stream)))

    def sdx_uzawa_f32(self, level, b, x, steps=1, stream=None):
        m = self._len(level)
        pb, px = _vecs((b, m), (x, m), itemsize=4)
        _check(load().sdx_uzawa_f32(self._h, level, pb, px, int(steps), _stream(stream)))

    def sdx_smooth_pass_noalloc(self, level, colour, b, x, stream=None):
        m = self._len(level)
        pb, px = _vecs((b, m), (x, m))
        _check(load().sdx_smooth_pass_noalloc(self._h, level, colour, pb, px, _stream(stream)))

    def sdx_restrict(self, level, r_fine, b_coarse, stream=None):
        pr, pb = _vecs((r_fine, self._len(level)), (b_coarse, self._len(level + 1)))
        _check(load().sdx_restrict(self._h, level, pr, pb, _stream(stream)))

    def sdx_prolong_add(self, level, e_coarse, x_fine, stream=None):
        pe, px = _vecs((e_coarse, self._len(level + 1)), (x_fine, self._len(level)))
        _check(load().sdx_prolong_add(self._h, level, pe, px, _stream(stream)))

    def sdx_vcycle(self, b, x, stream=None):
        m = self._len(0)
        pb, px = _vecs((b, m), (x, m))
        _check(load().sdx_vcycle(self._h, pb, px, _stream(stream)))

    def sdx_solve(self, b, x, rtol=1e-8, maxit=100, outer=OUTER_FGMRES, restart=30, stream=None,
                  allow_noconv=False) -> dict:
        st = sdx_stats()
        allow = (OK, ENOCONV) if allow_noconv else (OK,)
        m = self._len(0)
        pb, px = _vecs((b, m), (x, m))
        _check(load().sdx_solve(self._h, pb, px, float(rtol), int(maxit), int(outer),
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


class P1P0:
    """A hierarchy of the P1-P0 scheme (sdx_p0_*; owned, freed by close() or on deletion).
    Vectors: 3 (n+1)^3 velocities then 6 n^3 pressures (tetrahedron s of cell c at s n^3 + c)."""

    def __init__(self, problem, form="tr", coarse_form=None, gamma: float = 1.0, coarsening="resolved"):
        lib = load()
        d, self._keep = _make_desc(problem.n, problem.n_coarse, problem.cell_id, problem.mu, problem.face, form,
                                   coarse_form, PREC_FP64, PSPG_BETA, None, False, coarsening)
        h = ctypes.c_void_p()
        _check(lib.sdx_p0_create(ctypes.byref(d), float(gamma), ctypes.byref(h)))
        self._h = h
        self.n = int(problem.n)

    def close(self):
        if getattr(self, "_h", None):
            load().sdx_p0_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def size(self, level: int = 0):
        n, nodes, tets, free = ctypes.c_int(), ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        _check(load().sdx_p0_size(self._h, level, ctypes.byref(n), ctypes.byref(nodes), ctypes.byref(tets),
                                  ctypes.byref(free)))
        return n.value, nodes.value, tets.value, free.value

    def _len(self, level: int) -> int:
        _, nodes, tets, _ = self.size(level)
        return 3 * nodes + tets

    def apply(self, level, x, y, stream=None):
        m = self._len(level)
        px, py = _vecs((x, m), (y, m))
        _check(load().sdx_p0_apply(self._h, level, px, py, _stream(stream)))

    def residual(self, level, b, x, r, stream=None):
        m = self._len(level)
        pb, px, pr = _vecs((b, m), (x, m), (r, m))
        _check(load().sdx_p0_residual(self._h, level, pb, px, pr, _stream(stream)))

    def rhs(self, f, b, stream=None):
        _, nodes, _, _ = self.size(0)
        pf, pb = _vecs((f, 3 * nodes), (b, self._len(0)))
        _check(load().sdx_p0_rhs(self._h, pf, pb, _stream(stream)))

    def uzawa(self, level, b, x, stream=None):
        m = self._len(level)
        pb, px = _vecs((b, m), (x, m))
        _check(load().sdx_p0_uzawa(self._h, level, pb, px, _stream(stream)))

    def vcycle(self, b, x, stream=None):
        m = self._len(0)
        pb, px = _vecs((b, m), (x, m))
        _check(load().sdx_p0_vcycle(self._h, pb, px, _stream(stream)))

    def solve(self, b, x, rtol=1e-8, maxit=100, outer=OUTER_FGMRES, restart=30, stream=None) -> dict:
        st = sdx_stats()
        m = self._len(0)
        pb, px = _vecs((b, m), (x, m))
        _check(load().sdx_p0_solve(self._h, pb, px, float(rtol), int(maxit), int(outer), int(restart),
                                   ctypes.byref(st), _stream(stream)))
        return st.as_dict()

    def fluxes(self, x, flux, balance, stream=None):
        _, _, tets, _ = self.size(0)
        px, pf, pbal = _vecs((x, self._len(0)), (flux, 4 * tets), (balance, tets))
        _check(load().sdx_p0_fluxes(self._h, px, pf, pbal, _stream(stream)))


def _ptr_array(vectors, itemsize=8):
    arr = (ctypes.c_void_p * len(vectors))()
    for i, v in enumerate(vectors):
        arr[i] = _ptr(v, itemsize)
    return arr


class Batch:
    """Independent problems solved together by sdx_batch_* (owned; freed by close())."""

    def __init__(self, problems, form="tr", coarse_form=None, prec=PREC_FP32_REFINED,
                 beta: float = PSPG_BETA, autotune: bool = True, coarsening="resolved"):
        lib = load()
        descs = (sdx_desc * len(problems))()
        self._keep = []
        for i, p in enumerate(problems):
            d, keep = _make_desc(p.n, p.n_coarse, p.cell_id, p.mu, p.face, form, coarse_form, prec, beta,
                                 coarsening=coarsening)
            descs[i] = d
            self._keep.append(keep)
        h = ctypes.c_void_p()
        _check(lib.sdx_batch_create(descs, len(problems), 1 if autotune else 0, ctypes.byref(h)))
        self._h = h
        self.count = len(problems)
        self._lens = [4 * self.sdx_batch_size(i)[1] for i in range(self.count)]

    def close(self):
        if getattr(self, "_h", None):
            load().sdx_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def sdx_batch_size(self, instance: int):
        n, nodes, free = ctypes.c_int(), ctypes.c_int64(), ctypes.c_int64()
        _check(load().sdx_batch_size(self._h, instance, ctypes.byref(n), ctypes.byref(nodes), ctypes.byref(free)))
        return n.value, nodes.value, free.value

    def instance(self, i: int) -> "Hierarchy":
        """The batch-owned hierarchy of instance i (queries, sdx_rhs, apply, sdx_guess_*)."""
        h = ctypes.c_void_p()
        _check(load().sdx_batch_instance(self._h, int(i), ctypes.byref(h)))
        view = Hierarchy.__new__(Hierarchy)
        view._h = h
        view._owner = self  # keeps the batch alive; close() must not destroy it
        view._borrowed = True
        n, nodes, _ = self.sdx_batch_size(i)
        view.n, view.nn = n, nodes
        return view

    def _ptr_arrays(self, *lists):
        """Pointer arrays of per-instance vector lists: one vector per instance, each of its
        instance's length, all checked before any pointer is taken."""
        for lst in lists:
            if len(lst) != self.count:
                raise ValueError(f"{len(lst)} vectors for a batch of {self.count} instances")
            for t, m in zip(lst, self._lens):
                _check_len(t, m)
        return [_ptr_array(lst) for lst in lists]

    def sdx_batch_shape(self, level: int):
        v = [ctypes.c_int() for _ in range(4)]
        _check(load().sdx_batch_shape(self._h, level, *[ctypes.byref(x) for x in v]))
        return {"tpb_pass": v[0].value, "grid_pass": v[1].value, "tpb_residual": v[2].value,
                "grid_residual": v[3].value}

    def sdx_batch_vcycle(self, b_list, x_list, stream=None):
        pb, px = self._ptr_arrays(b_list, x_list)
        _check(load().sdx_batch_vcycle(self._h, pb, px, _stream(stream)))

    def sdx_batch_solve(self, b_list, x_list, rtol=1e-8, maxit=200, restart=30, stream=None,
                        allow_noconv=False, allow_codes=()):
        """Per-instance stats; a return code outside (OK, ENOCONV if allow_noconv, allow_codes)
        raises SdxError (each instance's own code is in its stats' "status")."""
        st = (sdx_stats * self.count)()
        allow = ((OK, ENOCONV) if allow_noconv else (OK,)) + tuple(allow_codes)
        pb, px = self._ptr_arrays(b_list, x_list)
        _check(load().sdx_batch_solve(self._h, pb, px, float(rtol),
                                      int(maxit), int(restart), st, _stream(stream)), allow)
        return [st[i].as_dict() for i in range(self.count)]


class Net:
    """The learned-initial-guess network (sdx_net_*; owned, freed by close())."""

    def __init__(self, seed: int = 0):
        h = ctypes.c_void_p()
        _check(load().sdx_net_create(int(seed), ctypes.byref(h)))
        self._h = h
        self.param_count = int(load().sdx_net_param_count())

    def close(self):
        if getattr(self, "_h", None):
            load().sdx_net_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def get_params(self) -> np.ndarray:
        out = np.zeros(self.param_count, dtype=np.float32)
        _check(load().sdx_net_get_params(self._h, out.ctypes.data))
        return out

    def set_params(self, params: np.ndarray):
        p = np.ascontiguousarray(params, dtype=np.float32)
        if p.size != self.param_count:
            raise ValueError("wrong parameter count")
        _check(load().sdx_net_set_params(self._h, p.ctypes.data))

    def forward(self, n, x_bf16, y_f32, stream=None):
        _check(load().sdx_net_forward(self._h, int(n), _ptr(x_bf16, 2), _ptr(y_f32, 4), _stream(stream)))

    def loss_grad(self, n, x_bf16, target_f32, stream=None):
        loss = ctypes.c_double()
        g = np.zeros(self.param_count, dtype=np.float32)
        _check(load().sdx_net_loss_grad(self._h, int(n), _ptr(x_bf16, 2), _ptr(target_f32, 4),
                                        ctypes.byref(loss), g.ctypes.data, _stream(stream)))
        return loss.value, g

    def train(self, n, count, x_bf16, target_f32, epochs, batch, lr, seed=0, stream=None):
        hist = np.zeros(epochs, dtype=np.float64)
        _check(load().sdx_net_train(self._h, int(n), int(count), _ptr(x_bf16, 2), _ptr(target_f32, 4),
                                    int(epochs), int(batch), float(lr), int(seed), hist.ctypes.data,
                                    _stream(stream)))
        return hist

    def predict(self, hier: "Hierarchy", f_nodal, x0, stream=None):
        _check(load().sdx_guess_predict(hier._h, self._h, _ptr(f_nodal), _ptr(x0), _stream(stream)))


def sdx_conv3(n, cin, cout, x_bf16, w_bf16, bias_f32, relu, y_f32, stream=None):
    _check(load().sdx_conv3(int(n), int(cin), int(cout), _ptr(x_bf16, 2), _ptr(w_bf16, 2),
                            _ptr(bias_f32, 4), int(relu), _ptr(y_f32, 4), _stream(stream)))


def sdx_conv3_dgrad(n, cin, cout, dz_bf16, w_f32, dx_f32, stream=None):
    _check(load().sdx_conv3_dgrad(int(n), int(cin), int(cout), _ptr(dz_bf16, 2), _ptr(w_f32, 4),
                                  _ptr(dx_f32, 4), _stream(stream)))


def sdx_conv3_wgrad(n, cin, cout, x_bf16, dz_bf16, dw_f32, stream=None):
    _check(load().sdx_conv3_wgrad(int(n), int(cin), int(cout), _ptr(x_bf16, 2), _ptr(dz_bf16, 2),
                                  _ptr(dw_f32, 4), _stream(stream)))


def sdx_guess_features(hier: "Hierarchy", f_nodal, x_bf16, stream=None) -> float:
    fs = ctypes.c_double()
    _check(load().sdx_guess_features(hier._h, _ptr(f_nodal), _ptr(x_bf16, 2), ctypes.byref(fs), _stream(stream)))
    return fs.value


def sdx_guess_refine(hier: "Hierarchy", b, x, steps, stream=None):
    _check(load().sdx_guess_refine(hier._h, _ptr(b), _ptr(x), int(steps), _stream(stream)))


def sdx_guess_target(hier: "Hierarchy", x_solution, fscale, target_f32, stream=None):
    _check(load().sdx_guess_target(hier._h, _ptr(x_solution), float(fscale), _ptr(target_f32, 4), _stream(stream)))


def sdx_kernel_launches() -> int:
    return int(load().sdx_kernel_launches())
