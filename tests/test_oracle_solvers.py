"""Pins for the oracle's solvers (no GPU): convergence to exact solutions, the paper's
qualitative results, and algebraic properties of the smoother, V-cycle and FGMRES."""
import os

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import solvers as S
from oracle.forms import DIRICHLET, Discretisation
from oracle.solvers import Hierarchy, Level, fgmres, vcycle_preconditioner
from paper_1604_07994_gb300 import workloads as W


def _layer(n):
    """A stiff layer z > 1/2 (mu = 10 over mu = 1), no-slip walls, manufactured solution."""
    return W.inclusion_problem(n, 4, [((0.0, 1.0), (0.0, 1.0), (0.5, 1.0))], 10.0, 1.0, seed=0)


def _nodal_exact_velocity(p, xyz):
    n = p.n
    cm = p.cell_mu()
    idx = np.minimum((xyz * n).astype(int), n - 1)
    mu_at = cm[idx[:, 2], idx[:, 1], idx[:, 0]]
    return np.stack(p.exact(xyz[:, 0], xyz[:, 1], xyz[:, 2], mu_at)[:3])


@pytest.mark.parametrize("form", ["tr", "sym", "grad"])
def test_manufactured_velocity_converges_at_second_order(form):
    """O(h^2) velocity L2 convergence on a manufactured piecewise solution satisfying the
    interface conditions (the paper's tables report rates near 2 for consistent forms).  The
    exact velocity has zero gradient on the interface, so all three forms are consistent.
    Between 8^3 and 16^3 the rate is still pre-asymptotic: with the stabilisation constant
    beta = 1/24 the strain form gives 1.78 there and 1.95 between 16^3 and 32^3 (a 32^3 direct
    solve takes minutes, too long for this suite), so the bound is 1.7; a first-order mistake
    (a dropped term, a wrong coefficient) gives 1.1 or less."""
    errs = []
    for n in (8, 16):
        p = _layer(n)
        H = Hierarchy(n, 4, p.cell_mu().ravel(), p.face, form)
        L = H.levels[0]
        b = L.disc.rhs(p.nodal_forcing())
        x = L.direct(b)
        ue = _nodal_exact_velocity(p, L.disc.xyz)
        m = L.disc.lumped_mass()
        uh = x[: 3 * L.nn].reshape(3, -1)
        errs.append(np.sqrt(np.sum(m * (uh - ue) ** 2) / np.sum(m * ue ** 2)))
    rate = np.log2(errs[0] / errs[1])
    assert rate >= 1.7, (form, errs, rate)


def _couette_error(n, form, mu1=1.0, mu2=1e-3):
    """Couette flow of Sec. 4.2.2 shifted to the unit cube (interface y = 1/2):
    u = (1/2 (1 - x^2), x (y - 1/2), 0), f = (3 mu, 0, 0), exact Dirichlet data."""
    c = (np.arange(n) + 0.5) / n
    _, Y, _ = np.meshgrid(c, c, c, indexing="ij")
    cmu = np.where(Y < 0.5, mu1, mu2).ravel()
    d = Discretisation(n, cmu, (DIRICHLET,) * 6)
    fc = np.zeros((3, n ** 3))
    fc[0] = 3.0 * cmu
    b = d.rhs(f_cell=fc)
    x, y, _ = d.xyz.T
    ue = np.stack([0.5 * (1.0 - x ** 2), x * (y - 0.5), 0.0 * x])
    con = d.constrained()
    xD = np.zeros(4 * d.nn)
    xD[: 3 * d.nn] = ue.ravel()
    xD[~con] = 0.0
    L = Level(n, cmu, (DIRICHLET,) * 6, form)
    rhs = b - d.saddle(form) @ xD
    rhs[con] = 0.0
    xs = L.direct(rhs) + xD
    m = d.lumped_mass()
    uh = xs[: 3 * d.nn].reshape(3, -1)
    return np.sqrt(np.sum(m * (uh - ue) ** 2) / np.sum(m * ue ** 2))


def test_couette_consistent_forms_converge_gradient_form_stalls():
    """Sec. 4.2.2 / Tables 2-7: a_tr and a_sym converge to the exact interface solution while
    the gradient form converges to a different one (its error stops decreasing).  With a
    continuous P1 pressure the jump [p] = 2x[mu] is not representable, so the consistent forms
    converge below second order here; the pin is on the qualitative split."""
    e = {f: [_couette_error(n, f) for n in (8, 16)] for f in ("tr", "sym", "grad")}
    for f in ("tr", "sym"):
        assert np.log2(e[f][0] / e[f][1]) >= 1.2, (f, e[f])
    assert np.log2(e["grad"][0] / e["grad"][1]) <= 0.6, e["grad"]
    assert e["grad"][1] > 2.0 * e["tr"][1]


def test_dense_and_sparse_direct_solves_agree(monkeypatch):
    p = W.cube_inclusion(8, 4)
    L1 = Level(8, p.cell_mu().ravel(), p.face, "tr")
    b = L1.disc.rhs(p.nodal_forcing())
    x1 = L1.direct(b)
    monkeypatch.setattr(S, "DENSE_LIMIT", 10)
    L2 = Level(8, p.cell_mu().ravel(), p.face, "tr")
    x2 = L2.direct(b)
    assert np.linalg.norm(x1 - x2) <= 1e-10 * np.linalg.norm(x1)
    r = L1.residual(x1, b)
    assert np.linalg.norm(r[L1.free]) <= 1e-12 * np.linalg.norm(b)
    w = L1.disc.pressure_weights()
    assert abs(np.dot(w, x1[3 * L1.nn:])) <= 1e-12 * np.abs(x1).max()


def test_single_level_cycle_is_the_direct_solve():
    p = W.cube_inclusion(4, 4)
    H = Hierarchy(4, 4, p.cell_mu().ravel(), p.face, "tr")
    b = H.levels[0].disc.rhs(p.nodal_forcing())
    x = H.vcycle(np.zeros_like(b), b)
    assert np.array_equal(x, H.levels[0].direct(b))


@pytest.mark.parametrize("form", ["tr", "sym"])
def test_discrete_solution_is_a_fixed_point_of_the_smoother(form):
    """Eq. (Uzawa_smooth) is consistent: both updates vanish at the discrete solution."""
    p = W.cube_inclusion(8, 4)
    L = Level(8, p.cell_mu().ravel(), p.face, form)
    b = L.disc.rhs(p.nodal_forcing())
    x = L.direct(b)
    y = x.copy()
    L.uzawa(y, b)
    assert np.abs(y - x).max() <= 1e-9 * np.abs(x).max()


@pytest.mark.parametrize("form", ["tr", "grad"])
def test_colour_passes_are_exact_block_gauss_seidel_when_isoviscous(form):
    """With one viscosity and no-slip walls there are no interface rows, so the a_tr and
    gradient-form velocity blocks are the 7-point Laplacian per component (eq.
    equivalence-stencil), and C is the constant-tau 7-point Laplacian: a node couples only to
    nodes of the other colour.  One colour of the velocity pass is then an exact block solve
    (the momentum residual vanishes on that colour's free rows, while the other colour's rows
    still carry one), and one colour of the pressure pass scales that colour's pressure
    residual by exactly 1 - omega.  A dropped term, a wrong colour or a wrong relaxation in a
    pass fails this."""
    n = 8
    p = W.Problem(n=n, n_coarse=4, cell_id=np.zeros((n, n, n), dtype=np.uint8), mu=np.array([2.5]),
                  face=(DIRICHLET,) * 6, forcing=W.gaussian_blobs(1))
    L = Level(n, p.cell_mu().ravel(), p.face, form)
    nn = L.nn
    x = W.random_vector(n, 11).ravel()
    x[L.con] = 0.0
    b = W.random_vector(n, 12).ravel()
    b[L.con] = 0.0
    u, pr = x[: 3 * nn], x[3 * nn:]
    f, g = b[: 3 * nn], b[3 * nn:]
    free_v = L.free[: 3 * nn]
    for red in (True, False):
        col = np.tile(L.red if red else ~L.red, 3) & free_v
        r0 = f - L.BT @ pr - L.A @ u
        L.velocity_pass(u, pr, f, red)
        r1 = f - L.BT @ pr - L.A @ u
        assert np.abs(r1[col]).max() <= 1e-12 * np.abs(r0).max(), (form, red)
        assert np.abs(r1[free_v & ~col]).max() > 1e-3 * np.abs(r0).max()  # the other colour moved
        pc = L.red if red else ~L.red
        s0 = (L.B @ u - g) - L.C @ pr
        L.pressure_pass(u, pr, g, red)
        s1 = (L.B @ u - g) - L.C @ pr
        assert np.abs(s1[pc] - (1.0 - S.OMEGA) * s0[pc]).max() <= 1e-12 * np.abs(s0).max(), (form, red)


@pytest.mark.parametrize("form", ["tr", "sym"])
def test_vcycle_contracts_on_the_papers_columns_problem(form):
    """Sec. 5 runs the V_var(3,3) Uzawa multigrid on the viscosity-columns problem and
    measures asymptotic rates of 0.24 to 0.30 (Table timeANDconv).  Here, at n = 16 with a
    4^3 coarsest grid, the rate stays well below one as well."""
    p = W.viscosity_columns(16, 4)
    H = Hierarchy(16, 4, p.cell_mu().ravel(), p.face, form)
    b = H.levels[0].disc.rhs(p.nodal_forcing())
    x, hist = H.solve(b, rtol=1e-10, maxit=30)
    rho = (hist[-1] / hist[-4]) ** (1.0 / 3.0)
    assert hist[-1] <= 1e-10 * np.linalg.norm(b[H.levels[0].free])
    assert rho < 0.5, rho


@pytest.mark.parametrize("coarse_form", [None, "sym"])
def test_fgmres_vcycle_reaches_the_direct_solution_at_high_contrast(coarse_form):
    """Floating stiff boxes (mu ratio 1e4): a_tr is indefinite (Sec. 3) and plain Uzawa
    multigrid diverges, but FGMRES preconditioned by the V-cycle reaches the direct solution."""
    p = W.three_boxes(16, 8, contrast=1e4)
    H = Hierarchy(16, 8, p.cell_mu().ravel(), p.face, "tr", coarse_form=coarse_form)
    L = H.levels[0]
    b = L.disc.rhs(p.nodal_forcing())
    x, hist = fgmres(L.K, vcycle_preconditioner(H), b, L.free, rtol=1e-12, restart=60, maxit=120)
    assert hist[-1] <= 1e-12 * np.linalg.norm(b[L.free])
    xd = L.direct(b)
    w = L.disc.pressure_weights()
    x[3 * L.nn:] -= np.dot(w, x[3 * L.nn:]) / w.sum()
    assert np.linalg.norm(x - xd) <= 1e-8 * np.linalg.norm(xd)


def test_fgmres_solves_a_small_system_exactly():
    """With restart >= dimension, (F)GMRES terminates with the exact solution; checked against
    numpy's dense solve on a nonsymmetric system with a Jacobi preconditioner."""
    rng = np.random.Generator(np.random.PCG64(7))
    n = 40
    A = sp.csr_matrix(rng.standard_normal((n, n)) + 8.0 * np.eye(n))
    b = rng.standard_normal(n)
    d = A.diagonal()
    x, hist = fgmres(A, lambda v: v / d, b, np.ones(n, dtype=bool), rtol=1e-13, restart=n)
    assert np.linalg.norm(x - np.linalg.solve(A.toarray(), b)) <= 1e-11 * np.linalg.norm(x)


def test_tight_fgmres_reference_equals_direct_solution():
    """The GPU solve tests use the oracle's FGMRES at rtol 1e-14 as reference where sparse LU is
    too slow; on a case where both are affordable they agree to 1e-10."""
    p = W.cube_inclusion(16, 4)
    H = Hierarchy(16, 4, p.cell_mu().ravel(), p.face, "sym")
    L = H.levels[0]
    b = L.disc.rhs(p.nodal_forcing())
    x, hist = fgmres(L.K, vcycle_preconditioner(H), b, L.free, rtol=1e-14, restart=60, maxit=600)
    w = L.disc.pressure_weights()
    x[3 * L.nn:] -= np.dot(w, x[3 * L.nn:]) / w.sum()
    xd = L.direct(b)
    assert np.linalg.norm(x - xd) <= 1e-10 * np.linalg.norm(xd)


# Sec. 5, Table timeANDconv: asymptotic rates of the V_var(3,3) cycle on the columns problem at
# levels 5-8, per form (cited fixture); the pins use each form's printed range
def _paper_rates():
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "vvar33_rates_columns.txt")
    rows = {}
    for line in open(path):
        if line.strip() and not line.startswith("#"):
            form, *vals = line.split()
            rows[form] = tuple(float(v) for v in vals)
    return rows


PAPER_RHO = {form: (min(v), max(v)) for form, v in _paper_rates().items()}


def _asymptotic_rate(H, cycles=25, last=8, seed=77):
    """Plain V-cycles on K x = 0 from a seeded random start, the pressure constant (kernel of K
    on an all-free-slip cube) projected out and the iterate renormalised to a unit residual
    after every cycle; geometric mean of the last reductions."""
    L = H.levels[0]
    nn = L.nn
    w = L.disc.pressure_weights()
    x = W.random_vector(L.n, seed).ravel()
    x[L.con] = 0.0
    zero = np.zeros_like(x)
    x[3 * nn:] -= np.dot(w, x[3 * nn:]) / w.sum()
    prev = np.linalg.norm(L.residual(x, zero))
    rates = []
    for _ in range(cycles):
        H.vcycle(x, zero)
        x[3 * nn:] -= np.dot(w, x[3 * nn:]) / w.sum()
        cur = np.linalg.norm(L.residual(x, zero))
        rates.append(cur / prev)
        x /= cur
        prev = 1.0
    return float(np.exp(np.mean(np.log(rates[-last:])))), rates


@pytest.mark.parametrize("form", ["tr", "sym", "grad"])
def test_asymptotic_rate_matches_the_papers_table(form):
    """At 16^3 (coarsest 4^3) the oracle's V_var(3,3) Uzawa cycle contracts at the paper's
    rates and has settled (the last reductions agree to 2 %).  The paper does not print its
    stabilisation constant; with beta = 1/24 the three forms contract at 0.217-0.222 here, flat
    with depth as in the paper's table (0.222 at 64^3), up to 15 % faster than the printed
    ranges (strain 0.255-0.296), so the band is 0.8 to 1.1 times the printed range.  A wrong
    smoother, transfer or coarse solve gives 0.4 or more, or diverges."""
    p = W.viscosity_columns(16, 4)
    H = Hierarchy(16, 4, p.cell_mu().ravel(), p.face, form)
    rho, rates = _asymptotic_rate(H)
    lo, hi = PAPER_RHO[form]
    assert 0.8 * lo <= rho <= 1.1 * hi, (form, rho)
    assert max(rates[-4:]) / min(rates[-4:]) <= 1.02, rates[-4:]


def test_corrected_coarse_swap_contracts_at_the_papers_rate():
    """Sec. 5: a_sym on the coarsest grid with the corrected momentum right-hand side
    r1 + B^T D r2 (sign and weight from the saddle matrix of Sec. 5) keeps the decoupled
    cycle at the paper's rate for the modified stencil form (0.241-0.244) on the columns
    problem; the printed sign (0.47 here) or the correction without mu (0.38) do not."""
    p = W.viscosity_columns(16, 4)
    H = Hierarchy(16, 4, p.cell_mu().ravel(), p.face, "tr", coarse_correction=True)
    assert H.levels[-1].form == "sym" and H.levels[0].form == "tr" and H.levels[1].form == "tr"
    rho, rates = _asymptotic_rate(H)
    lo, hi = PAPER_RHO["tr"]
    assert 0.9 * lo <= rho <= 1.1 * hi, rho
    # the correction acts through the pressure rows only
    b = W.random_vector(4, 3).ravel()
    Lc = H.levels[-1]
    b[Lc.con] = 0.0
    b0 = b.copy()
    b0[3 * Lc.nn:] = 0.0
    assert np.array_equal(H.coarse_rhs(b0), b0)
    assert not np.array_equal(H.coarse_rhs(b), b)
    with pytest.raises(ValueError):
        Hierarchy(16, 4, p.cell_mu().ravel(), p.face, "sym", coarse_correction=True)


@pytest.mark.parametrize("case,form", [("columns", "sym"), ("columns", "grad"), ("layer", "tr"), ("boxes", "sym")])
def test_block_minres_reaches_the_direct_solution(case, form):
    """Sec. 5's coarse solver (MINRES, block-diagonal preconditioner: Jacobi-CG on the
    velocity block, 1/mu-weighted lumped pressure mass) converges to the direct solution where
    the velocity block is positive definite."""
    p = {"columns": W.viscosity_columns(8, 4), "layer": W.top_layer(8, 8),
         "boxes": W.three_boxes(8, 8, contrast=1e2)}[case]
    L = S.Level(8, p.cell_mu().ravel(), p.face, form)
    b = L.disc.rhs(p.nodal_forcing())
    x = S.block_minres(L, b, rtol=1e-14)  # preconditioned-residual test; contrast adds conditioning
    xd = L.direct(b)
    assert np.linalg.norm(x - xd) <= 1e-9 * np.linalg.norm(xd)


def test_block_minres_refuses_the_indefinite_decoupled_block():
    """Sec. 5: the block preconditioner cannot be applied to a_tr where its velocity block is
    indefinite (the columns problem); MINRES stops instead of returning a wrong solution."""
    p = W.viscosity_columns(8, 4)
    L = S.Level(8, p.cell_mu().ravel(), p.face, "tr")
    with pytest.raises(RuntimeError):
        S.block_minres(L, L.disc.rhs(p.nodal_forcing()), rtol=1e-12)


def test_papers_coarse_variant_with_minres_keeps_the_rate():
    """The paper's whole coarse-grid variant - a_sym on the coarsest grid, corrected right-hand
    side, MINRES to 1e-8 - contracts like the same cycle with a direct coarsest solve."""
    p = W.viscosity_columns(16, 4)
    cm = p.cell_mu().ravel()
    Hd = Hierarchy(16, 4, cm, p.face, "tr", coarse_correction=True)
    Hm = Hierarchy(16, 4, cm, p.face, "tr", coarse_correction=True, coarse_solver="minres", coarse_rtol=1e-8)
    rd, _ = _asymptotic_rate(Hd)
    rm, _ = _asymptotic_rate(Hm)
    assert abs(rm - rd) <= 0.01 * rd, (rm, rd)
