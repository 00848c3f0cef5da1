"""The paper's columns error tables (Sec. 4.2.4) computed on the GPU path against the oracle:
the strain, decoupled and gradient forms solved by the CUDA multigrid, then the relative
differences to the strain solution in the norms of Sec. 3, at levels 2 and 3 (16^3, 32^3)."""
import numpy as np
import pytest

from tests._lib import ensure_built

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import bench  # noqa: E402
from oracle.solvers import Hierarchy as OracleHierarchy, fgmres, vcycle_preconditioner  # noqa: E402
from paper_1604_07994_gb300 import workloads as W  # noqa: E402


@pytest.fixture(scope="module")
def sdx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ensure_built()
    from paper_1604_07994_gb300 import sdx as mod
    return mod


def _oracle_differences(n):
    p = W.viscosity_columns(n, 4)
    sols = {}
    for form in ("sym", "tr", "grad"):
        H = OracleHierarchy(n, 4, p.cell_mu().ravel(), p.face, form)
        L = H.levels[0]
        b = L.disc.rhs(p.nodal_forcing())
        x, hist = fgmres(L.K, vcycle_preconditioner(H), b, L.free, rtol=1e-12, restart=40, maxit=200)
        assert hist[-1] <= 1e-12 * np.linalg.norm(b[L.free])
        w = L.disc.pressure_weights()
        x[3 * L.nn:] -= np.dot(w, x[3 * L.nn:]) / w.sum()
        sols[form] = x
    d = L.disc
    U = sols["sym"]
    base = d.paper_norms(U)
    return {"decoupled": d.paper_norms(sols["tr"] - U) / base,
            "gradient": d.paper_norms(sols["grad"] - U) / base}


def test_columns_tables_match_the_oracle(sdx):
    """GPU solves to 1e-10: the table entries agree with the oracle's to 1e-6 relative (the
    smallest entry, the decoupled L2 difference, is 2e-3 of the solution)."""
    out = bench.run_paper_tables(None, sdx, torch, levels=(2, 3))
    for lvl, n in ((2, 16), (3, 32)):
        got = out[f"L{lvl}"]
        assert "error" not in got, got
        for s in got["solves"].values():
            assert s["final_rel_res"] <= 1e-10
        ref = _oracle_differences(n)
        for k in ("decoupled", "gradient"):
            g = np.array(got["relative_differences"][k])
            assert np.all(np.abs(g / ref[k] - 1.0) <= 1e-6), (lvl, k, g, ref[k])
