"""The C-ABI library builds, loads, and exports every entry point include/sdx.h declares
(no GPU needed: nothing here launches a kernel)."""
import ctypes
import os
import re
import subprocess

import numpy as np

from tests._lib import ensure_built

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    text = open(os.path.join(ROOT, "include", "sdx.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sdx_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_documented_entry_points():
    names = _declared()
    for n in ("sdx_create", "sdx_destroy", "sdx_apply", "sdx_vcycle", "sdx_solve", "sdx_strerror"):
        assert n in names


def test_library_exports_every_declared_symbol():
    lib = ensure_built()
    for name in _declared():
        assert hasattr(lib, name), name
    from paper_1604_07994_gb300 import sdx
    assert set(sdx.EXPORTED) == set(_declared())


def test_exports_are_plain_c_symbols():
    from paper_1604_07994_gb300 import sdx
    ensure_built()
    out = subprocess.run(["nm", "-D", "--defined-only", sdx.LIB_PATH], capture_output=True, text=True).stdout
    syms = {line.split()[-1] for line in out.splitlines() if line.strip()}
    for name in _declared():
        assert name in syms, name  # unmangled: extern "C"


def test_strerror_and_argument_validation_without_a_device():
    from paper_1604_07994_gb300 import sdx
    lib = ensure_built()
    assert lib.sdx_strerror(sdx.EINVAL) == b"invalid argument"
    assert lib.sdx_strerror(12345) == b"unknown error"
    # a null descriptor is rejected before any CUDA call
    h = ctypes.c_void_p()
    assert lib.sdx_create(None, ctypes.byref(h)) == sdx.EINVAL
    assert h.value is None
    # host-side validation: n not n_coarse * 2^k, bad viscosity, out-of-range id
    cells = np.zeros(6 ** 3, dtype=np.uint8)
    mu = np.array([1.0, -2.0])
    d = sdx.sdx_desc()
    d.n, d.n_coarse = 6, 4
    d.cell_id = cells.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))
    d.mu = mu.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    d.n_mu = 1
    d.form, d.coarse_form, d.prec, d.pspg_beta = 0, -1, 0, 1.0 / 12
    assert lib.sdx_create(ctypes.byref(d), ctypes.byref(h)) == sdx.EINVAL
    assert b"n_coarse" in lib.sdx_last_error()
    d.n, d.n_coarse = 2048, 8  # beyond the 32-bit node indices of the special-row lists
    assert lib.sdx_create(ctypes.byref(d), ctypes.byref(h)) == sdx.EINVAL
    assert b"1024" in lib.sdx_last_error()
    d.n, d.n_coarse = 6, 4
    d.n, d.n_coarse, d.n_mu = 8, 4, 2
    cells8 = np.zeros(8 ** 3, dtype=np.uint8)
    d.cell_id = cells8.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))
    assert lib.sdx_create(ctypes.byref(d), ctypes.byref(h)) == sdx.EINVAL
    assert b"viscosit" in lib.sdx_last_error()
    mu_ok = np.array([1.0])
    d.mu = mu_ok.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    d.n_mu = 1
    cells8[5] = 3
    assert lib.sdx_create(ctypes.byref(d), ctypes.byref(h)) == sdx.EINVAL
    assert b"cell id" in lib.sdx_last_error()
    cells8[5] = 0
    # the Sec. 5 coarse-grid correction needs a coarser level with the strain form
    d.coarsest_form, d.coarse_correction = sdx.FORM_DECOUPLED, 1
    assert lib.sdx_create(ctypes.byref(d), ctypes.byref(h)) == sdx.EINVAL
    assert b"coarse_correction" in lib.sdx_last_error()
    d.coarsest_form, d.n_coarse = sdx.FORM_STRAIN, 8  # a single level
    assert lib.sdx_create(ctypes.byref(d), ctypes.byref(h)) == sdx.EINVAL
    assert b"coarse_correction" in lib.sdx_last_error()
    d.coarse_correction, d.coarsest_form = 2, -1
    assert lib.sdx_create(ctypes.byref(d), ctypes.byref(h)) == sdx.EINVAL
    assert h.value is None
    # null hierarchy handles
    assert lib.sdx_apply(None, 0, None, None, None) == sdx.EINVAL
    assert lib.sdx_destroy(None) == sdx.OK



def test_batch_validation_without_a_device():
    """sdx_batch_create refuses bad arguments before any CUDA call: no descriptors, a count
    out of range, and instances that disagree on the form."""
    from paper_1604_07994_gb300 import sdx
    lib = ensure_built()
    h = ctypes.c_void_p()
    assert lib.sdx_batch_create(None, 1, 0, ctypes.byref(h)) == sdx.EINVAL
    assert h.value is None
    cells = np.zeros(8 ** 3, dtype=np.uint8)
    mu = np.array([1.0])
    descs = (sdx.sdx_desc * 2)()
    for i, form in enumerate((sdx.FORM_DECOUPLED, sdx.FORM_STRAIN)):
        d = descs[i]
        d.n, d.n_coarse = 8, 2
        d.cell_id = cells.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))
        d.mu = mu.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        d.n_mu = 1
        d.form, d.coarse_form, d.prec, d.pspg_beta = form, -1, 1, 1.0 / 12
    assert lib.sdx_batch_create(descs, 0, 0, ctypes.byref(h)) == sdx.EINVAL
    assert lib.sdx_batch_create(descs, 2, 0, ctypes.byref(h)) == sdx.EINVAL
    assert b"same form" in lib.sdx_last_error()
    assert h.value is None
    assert lib.sdx_batch_destroy(None) == sdx.OK
    assert lib.sdx_batch_solve(None, None, None, 1e-8, 10, 10, None, None) == sdx.EINVAL


def test_p1p0_argument_validation_without_a_device():
    """The P1-P0 entry points reject bad arguments on the host, before any CUDA call: a
    non-positive or non-finite penalty gamma, a null descriptor, FP32 cycles (the scheme runs in
    FP64), the P1-P1 coarse-grid correction, the descriptor's own host checks, null handles
    and vectors."""
    from paper_1604_07994_gb300 import sdx
    lib = ensure_built()
    h = ctypes.c_void_p()
    cells = np.zeros(8 ** 3, dtype=np.uint8)
    mu = np.array([1.0])
    d = sdx.sdx_desc()
    d.n, d.n_coarse, d.n_mu = 8, 4, 1
    d.cell_id = cells.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))
    d.mu = mu.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    d.form, d.coarse_form, d.prec, d.pspg_beta = 0, -1, 0, sdx.PSPG_BETA
    d.coarsest_form = -1
    for gamma in (0.0, -1.0, float("nan"), float("inf")):
        assert lib.sdx_p0_create(ctypes.byref(d), ctypes.c_double(gamma), ctypes.byref(h)) == sdx.EINVAL
        assert b"gamma" in lib.sdx_last_error()
    assert lib.sdx_p0_create(None, ctypes.c_double(1.0), ctypes.byref(h)) == sdx.EINVAL
    assert lib.sdx_p0_create(ctypes.byref(d), ctypes.c_double(1.0), None) == sdx.EINVAL
    d.prec = 1
    assert lib.sdx_p0_create(ctypes.byref(d), ctypes.c_double(1.0), ctypes.byref(h)) == sdx.EINVAL
    assert b"FP64" in lib.sdx_last_error()
    d.prec, d.coarse_correction = 0, 1
    assert lib.sdx_p0_create(ctypes.byref(d), ctypes.c_double(1.0), ctypes.byref(h)) == sdx.EINVAL
    assert b"coarse_correction" in lib.sdx_last_error()
    d.coarse_correction, d.n_coarse = 0, 3  # 8 is not 3 * 2^k
    assert lib.sdx_p0_create(ctypes.byref(d), ctypes.c_double(1.0), ctypes.byref(h)) == sdx.EINVAL
    assert b"n_coarse" in lib.sdx_last_error()
    assert h.value is None
    assert lib.sdx_p0_apply(None, 0, None, None, None) == sdx.EINVAL
    assert lib.sdx_p0_solve(None, None, None, ctypes.c_double(1e-8), 10, 1, 30, None, None) == sdx.EINVAL
    assert lib.sdx_p0_fluxes(None, None, None, None, None) == sdx.EINVAL
    assert lib.sdx_p0_destroy(None) == sdx.OK
