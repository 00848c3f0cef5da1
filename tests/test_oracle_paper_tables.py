"""The oracle against the paper's printed error tables for the viscosity-layers and
viscosity-columns problems (Sec. 4.2.3, 4.2.4): relative differences between the discrete
solutions of the gradient form or the decoupled form and the strain form, in the norms of
Sec. 3 (no GPU).

Two facts in those tables do not depend on the element pair or on the pressure
stabilisation, so they pin this oracle's P1-P1 PSPG scheme:

* the gradient form converges to a different solution: its relative difference to the strain
  form tends to a fixed, problem-dependent value (columns: about 2.0e-2 / 4.2e-2 / 6.6e-2;
  layers: about 0.31 / 0.52 / 0.26), which both of the paper's discretisations approach and
  which is a property of the continuous problems;
* the decoupled form is consistent: its difference to the strain form vanishes under
  refinement, at second order in ||.||_0 and first order in ||.||_V and ||.||_Q.

The size of the decoupled form's difference on a given mesh is a discretisation error and
depends on the stabilisation, so it is not compared value by value."""
from pathlib import Path

import numpy as np
import pytest

from oracle.solvers import Hierarchy, fgmres, vcycle_preconditioner
from paper_1604_07994_gb300 import workloads as W

GOLDEN = Path(__file__).parent / "golden" / "relative_differences_layers_columns.txt"
RTOL = 1e-11


def _paper():
    """{(problem, form, element, level): [velocity_L2, velocity_V, pressure_Q]}."""
    out = {}
    for line in GOLDEN.read_text().splitlines():
        if not line.strip() or line.startswith("#"):
            continue
        prob, form, elem, lvl, *vals = line.split()
        out[(prob, form, elem, int(lvl))] = np.array([float(v) for v in vals])
    return out


def _solve(prob, form):
    """The discrete solution of one form, FGMRES + V-cycle to 1e-11, pressure normalised by
    the weights of the discrete constraint int p / mu = 0 (free-slip faces everywhere)."""
    H = Hierarchy(prob.n, 4, prob.cell_mu().ravel(), prob.face, form)
    L = H.levels[0]
    b = L.disc.rhs(prob.nodal_forcing())
    x, hist = fgmres(L.K, vcycle_preconditioner(H), b, L.free, rtol=RTOL, restart=40, maxit=200)
    assert hist[-1] <= RTOL * np.linalg.norm(b[L.free])
    w = L.disc.pressure_weights()
    x[3 * L.nn:] -= np.dot(w, x[3 * L.nn:]) / w.sum()
    return x, L.disc


@pytest.fixture(scope="module", params=["layers", "columns"])
def differences(request):
    """Relative differences to the strain form at level 2 (16^3 cells) and level 3 (32^3)."""
    make = W.viscosity_layers if request.param == "layers" else W.viscosity_columns
    out = {}
    for level, n in ((2, 16), (3, 32)):
        prob = make(n, 4)
        sol = {f: _solve(prob, f) for f in ("sym", "tr", "grad")}
        U, d = sol["sym"]
        ref = d.paper_norms(U)
        for f in ("tr", "grad"):
            out[(f, level)] = d.paper_norms(sol[f][0] - U) / ref
    return request.param, out


def test_golden_file_is_complete():
    t = _paper()
    assert len(t) == 30
    for prob in ("layers", "columns"):
        for form in ("grad", "tr"):
            assert all((prob, form, "P1P0", l) in t for l in range(5))
    for form in ("grad", "tr"):
        assert all(("columns", form, "P1P1", l) in t for l in range(2, 7))


def test_gradient_form_difference_matches_the_papers_value(differences):
    """At level 3 the gradient form's relative difference agrees with the paper's level-3
    P1-P0 entry within 5 % in all three norms; on the columns problem it also agrees with the
    paper's finest P1-P1 entry (level 6, 256^3) within 6 %."""
    prob, got = differences
    t = _paper()
    g3 = got[("grad", 3)]
    ref = t[(prob, "grad", "P1P0", 3)]
    assert np.all(np.abs(g3 / ref - 1.0) <= 0.05), (prob, g3, ref)
    if prob == "columns":
        fine = t[("columns", "grad", "P1P1", 6)]
        assert np.all(np.abs(g3 / fine - 1.0) <= 0.06), (g3, fine)


def test_gradient_form_difference_does_not_vanish(differences):
    """The gradient form's error to the strain form stays (the paper's rates are 0.00-0.08 at
    these levels on the columns problem and not displayed, being negative, on the layers)."""
    prob, got = differences
    assert np.all(got[("grad", 3)] >= 0.85 * got[("grad", 2)]), (prob, got)


def test_decoupled_form_difference_vanishes_at_the_papers_rates(differences):
    """The decoupled form converges to the strain form's limit: from level 2 to 3 the
    relative difference falls at a rate of at least 1.6 in ||.||_0, 0.7 in ||.||_V and 0.6 in
    ||.||_Q (the paper's tables: 1.43-1.97, 0.94-1.21 and 0.72-1.44 at levels 2-4), and at level
    3 it is below 0.3 of the gradient form's difference in every norm."""
    prob, got = differences
    t2, t3 = got[("tr", 2)], got[("tr", 3)]
    rate = np.log2(t2 / t3)
    assert rate[0] >= 1.6 and rate[1] >= 0.7 and rate[2] >= 0.6, (prob, rate)
    assert np.all(t3 > 0.0)
    assert np.all(t3 <= 0.3 * got[("grad", 3)]), (prob, t3, got[("grad", 3)])
