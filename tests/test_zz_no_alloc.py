"""The allocation-free velocity pass agrees with the standard one.

sdx_smooth_pass_noalloc serves callers that cannot allocate device memory when they call it
(for example a phase of their program where cudaMalloc is forbidden because it would
synchronise the device, or where device memory was budgeted up front): it stages the new
values of the boundary and interface rows in a fixed array compiled into the library
instead of a scratch buffer of the hierarchy.  It must give what sdx_smooth_pass gives, call
after call.  This file is named so that pytest collects it last.
"""
import numpy as np
import pytest

from tests._lib import ensure_built

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1604_07994_gb300 import workloads as W  # noqa: E402

TOL = 1e-13  # the per-operation tolerance of the FP64 parity tests


@pytest.fixture(scope="module")
def sdx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ensure_built()
    from paper_1604_07994_gb300 import sdx as mod
    return mod


def _vectors(H, n, seed):
    con = torch.from_numpy(H.sdx_constraint_mask(0)).cuda()
    x = torch.from_numpy(W.random_vector(n, seed).ravel()).cuda()
    b = torch.from_numpy(W.random_vector(n, seed + 1).ravel()).cuda()
    x[con] = 0.0
    b[con] = 0.0
    return x, b


@pytest.mark.parametrize("case,form", [("cube", "tr"), ("layer", "tr"), ("layer", "grad"), ("columns", "tr")])
def test_noalloc_pass_matches_standard_pass_twice(sdx, case, form):
    p = {"cube": W.cube_inclusion(16, 4), "layer": W.top_layer(32, 8),
         "columns": W.viscosity_columns(32, 4)}[case]
    H = sdx.Hierarchy.from_problem(p, form=form)
    x0, b = _vectors(H, p.n, 3)
    xa, xb = x0.clone(), x0.clone()
    for _call in range(2):  # two calls in a row on each colour: the shared array is reused
        for colour in (0, 1):
            H.sdx_smooth_pass(0, 0, colour, b, xa)
            H.sdx_smooth_pass_noalloc(0, colour, b, xb)
            torch.cuda.synchronize()
            err = float((xb - xa).abs().max() / xa.abs().max())
            assert err <= TOL, (case, form, colour, err)
    assert float((xa - x0).abs().max()) > 0.0  # the pass did change the iterate


def test_noalloc_pass_rejects_what_it_cannot_do(sdx):
    # strain form: needs a full-grid scratch vector
    p = W.cube_inclusion(16, 4)
    H = sdx.Hierarchy.from_problem(p, form="sym")
    x, b = _vectors(H, p.n, 5)
    with pytest.raises(sdx.SdxError) as e:
        H.sdx_smooth_pass_noalloc(0, 0, b, x)
    assert e.value.code == sdx.EINVAL and "strain" in str(e.value)
    # more boundary rows in one colour than the fixed array holds (free-slip box, 160^3)
    n = 160
    big = W.Problem(n=n, n_coarse=5, cell_id=np.zeros((n, n, n), dtype=np.uint8), mu=np.array([1.0]),
                    face=(W.FREESLIP,) * 6, forcing=None, name="freeslip_160")
    Hb = sdx.Hierarchy.from_problem(big, form="tr")
    xb = torch.zeros(4 * (n + 1) ** 3, dtype=torch.float64, device="cuda")
    with pytest.raises(sdx.SdxError) as e:
        Hb.sdx_smooth_pass_noalloc(0, 0, xb, xb.clone())
    assert e.value.code == sdx.EINVAL and str(sdx.NOALLOC_MAX_ROWS) in str(e.value)
