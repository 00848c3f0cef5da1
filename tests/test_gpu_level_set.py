"""GPU parity for interfaces the coarse grids do not resolve (Sec. 2.2, closing remark): a
stiff sphere given by a level set cuts the cells of every coarser grid.  The finest operator
(interface rows classified per node from the cells around it) must equal the oracle's assembly
at 1e-13; the hierarchy coarsens the viscosity by the majority rule (coarsening = 1), and its
V-cycles must equal the oracle's with the same rule at 1e-10; solves reach the direct solution
at 1e-8."""
import numpy as np
import pytest

from tests._lib import ensure_built

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle.forms import Discretisation, masked  # noqa: E402
from oracle.solvers import Hierarchy as OracleHierarchy  # noqa: E402
from paper_1604_07994_gb300 import workloads as W  # noqa: E402


@pytest.fixture(scope="module")
def sdx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ensure_built()
    from paper_1604_07994_gb300 import sdx as mod
    return mod


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def _host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def test_unresolved_interface_needs_majority_coarsening(sdx):
    p = W.level_set_sphere(16, 4)
    with pytest.raises(sdx.SdxError) as e:
        sdx.Hierarchy.from_problem(p)
    assert e.value.code == sdx.EINVAL and "coarsening" in str(e.value)


@pytest.mark.parametrize("form", ["tr", "sym"])
@pytest.mark.parametrize("n", [16, 32])
def test_level_set_masks_and_apply_match_oracle(sdx, n, form):
    p = W.level_set_sphere(n, 4)
    d = Discretisation(p.n, p.cell_mu().ravel(), p.face)
    H = sdx.Hierarchy.from_problem(p, form=form, coarsening="majority")
    assert np.array_equal(H.sdx_constraint_mask(0), d.constrained())
    iface = H.sdx_interface_mask(0)
    assert np.array_equal(iface, d.interface_nodes())
    assert iface.sum() > 0
    K = masked(d.saddle(form), d.constrained())
    x = W.random_vector(p.n, 5).ravel()
    x[d.constrained()] = 0.0
    y = _dev(np.zeros_like(x))
    H.sdx_apply(0, _dev(x), y)
    ref = K @ x
    assert np.abs(_host(y) - ref).max() <= 1e-13 * np.abs(ref).max()


@pytest.mark.parametrize("coarse_form", [None, "sym"])
@pytest.mark.parametrize("n", [16, 32])
def test_level_set_vcycle_matches_oracle(sdx, n, coarse_form):
    """Two V_var cycles from zero on the majority-coarsened hierarchy (coarse grids 8^3 and 4^3
    do not resolve the sphere)."""
    p = W.level_set_sphere(n, 4)
    OH = OracleHierarchy(p.n, p.n_coarse, p.cell_mu().ravel(), p.face, "tr", coarse_form=coarse_form,
                         coarsening="majority")
    b = OH.levels[0].disc.rhs(p.nodal_forcing())
    H = sdx.Hierarchy.from_problem(p, form="tr", coarse_form=coarse_form, coarsening="majority")
    for l, L in enumerate(OH.levels):
        assert H.sdx_level_size(l)[2] == int(L.free.sum())
    xd, bd = _dev(np.zeros_like(b)), _dev(b)
    xo = np.zeros_like(b)
    for _ in range(2):
        H.sdx_vcycle(bd, xd)
        OH.vcycle(xo, b)
        assert np.linalg.norm(_host(xd) - xo) <= 1e-10 * np.linalg.norm(xo)


@pytest.mark.parametrize("prec", [0, 1])
def test_level_set_solve_matches_direct_solution(sdx, prec):
    p = W.level_set_sphere(16, 4)
    L = OracleHierarchy(p.n, p.n, p.cell_mu().ravel(), p.face, "tr").levels[0]
    b = L.disc.rhs(p.nodal_forcing())
    xo = L.direct(b)
    H = sdx.Hierarchy.from_problem(p, form="tr", coarse_form="sym", prec=prec, coarsening="majority")
    xd = _dev(np.zeros_like(b))
    st = H.sdx_solve(_dev(b), xd, rtol=1e-12, maxit=300, outer=sdx.OUTER_FGMRES, restart=40)
    assert st["res"] <= 1e-12 * st["bnorm"]
    x = _host(xd)
    w = L.disc.pressure_weights()
    x[3 * L.nn:] -= np.dot(w, x[3 * L.nn:]) / w.sum()
    assert np.linalg.norm(x - xo) <= 1e-8 * np.linalg.norm(xo)
