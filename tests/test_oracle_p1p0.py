"""Pins for the P1-P0 oracle (Sec. 3.1-3.2: P0 pressure, interior-penalty stabilisation eq.
(stabc) with gamma = 1, local flux post-process) against the paper's printed P1-P0 results and
exact identities.  A dropped facet, a wrong weight, sign or normal, or a transposed divergence
fails one of them."""
import os

import numpy as np
import pytest
import scipy.sparse as sp

from oracle.forms import DIRICHLET, FREESLIP
from oracle.mesh import kuhn_tets, node_xyz
from oracle.p1p0 import GAMMA, P1P0, P1P0Hierarchy, p0_parent
from oracle.solvers import fgmres
from oracle.transfer import prolongation
from paper_1604_07994_gb300 import workloads as W

HERE = os.path.dirname(os.path.abspath(__file__))
GOLDEN = os.path.join(HERE, "golden", "relative_differences_layers_columns.txt")
# Sec. 4.2.2, table couette-results-1e3 (P1-P0, mu1/mu2 = 1e3): rows (level, ||u - u_h||_0,
# ||u - u_h||_V, ||p - p_h||_Q), read from the cited fixture
COUETTE_GOLDEN = os.path.join(HERE, "golden", "couette_p1p0_errors_1e3.txt")
COUETTE = [tuple(float(v) for v in line.split()) for line in open(COUETTE_GOLDEN)
           if line.strip() and not line.startswith("#")]


def _golden(problem, form, element):
    rows = {}
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        pr, fo, el, lv, *vals = line.split()
        if (pr, fo, el) == (problem, form, element):
            rows[int(lv)] = np.array([float(v) for v in vals])
    return rows


def test_facets_and_penalty_weights():
    """12 n^3 - 6 n^2 interior facets (4 faces per tetrahedron, 12 n^2 on the boundary); every
    tetrahedron has at least its two in-cube facets; equal tetrahedra give w = gamma h^3/(24 mu)."""
    n, mu = 3, 2.5
    P = P1P0(n, np.full(n ** 3, mu), (DIRICHLET,) * 6)
    assert P.f_t1.size == 12 * n ** 3 - 6 * n ** 2
    deg = np.bincount(np.concatenate([P.f_t1, P.f_t2]), minlength=P.nT)
    assert deg.min() >= 2 and deg.max() == 4
    assert np.allclose(P.penalty_weights(), GAMMA * (1.0 / n) ** 3 / (24 * mu), rtol=1e-14, atol=0)
    assert np.allclose(P.f_area[:, None] * P.f_normal @ np.ones(3) * 0 + P.f_area, P.f_area)


def test_stabilisation_structure():
    """C0 symmetric positive semi-definite, C0 1 = 0, and no coupling across the viscosity
    interface or the domain boundary (eq. stabc excludes the facets of the subdomain boundaries)."""
    p = W.cube_inclusion(4, 4)
    P = P1P0(4, p.cell_mu().ravel(), p.face)
    C = P.stabilisation()
    assert abs(C - C.T).max() == 0.0
    assert np.abs(C @ np.ones(P.nT)).max() <= 1e-18
    assert np.linalg.eigvalsh(C.toarray()).min() >= -1e-15
    Cc = sp.coo_matrix(C)
    off = (Cc.row != Cc.col) & (Cc.data != 0.0)
    assert np.all(P.mu_T[Cc.row[off]] == P.mu_T[Cc.col[off]])
    assert np.count_nonzero(~P.f_inner) > 0  # the inclusion's facets exist and are excluded


def test_divergence_of_linear_fields():
    """B0 I(u) = -|T| div u exactly for a linear u, on every tetrahedron."""
    P = P1P0(3, np.ones(27), (FREESLIP,) * 6)
    x = node_xyz(3)
    u = np.stack([2 * x[:, 0] - x[:, 1], 0.5 * x[:, 1] + x[:, 2], -3 * x[:, 2] + x[:, 0]]).ravel()
    assert np.abs(P.divergence() @ u + P.vol * (2 + 0.5 - 3)).max() <= 1e-15


def test_p0_parents_are_nested():
    """Every coarse tetrahedron is the union of exactly eight fine ones: the children's volumes add
    up and their centroids lie inside the parent (barycentric coordinates >= 0)."""
    nf = 4
    par = p0_parent(nf)
    tc, _ = kuhn_tets(nf // 2)
    tf, _ = kuhn_tets(nf)
    assert np.all(np.bincount(par, minlength=tc.shape[0]) == 8)
    xf, xc = node_xyz(nf), node_xyz(nf // 2)
    cen = xf[tf].mean(axis=1)
    V = xc[tc[par]]
    M = np.concatenate([np.ones((par.size, 4, 1)), V], axis=2)
    rhs = np.concatenate([np.ones((par.size, 1)), cen], axis=1)[:, :, None]
    lam = np.linalg.solve(np.transpose(M, (0, 2, 1)), rhs)[:, :, 0]
    assert lam.min() > 0.0


def test_nested_galerkin_identity_for_b():
    """P_p^T B0_h P_u = B0_2h: the divergence form is h-independent on nested spaces."""
    mu = np.ones(64)
    Pf, Pc = P1P0(4, mu, (DIRICHLET,) * 6), P1P0(2, np.ones(8), (DIRICHLET,) * 6)
    Pu = prolongation(2)
    P3 = sp.block_diag([Pu, Pu, Pu], format="csr")
    par = p0_parent(4)
    Pp = sp.coo_matrix((np.ones(Pf.nT), (np.arange(Pf.nT), par)), shape=(Pf.nT, Pc.nT)).tocsr()
    G = (Pp.T @ Pf.divergence() @ P3).toarray()
    assert np.abs(G - Pc.divergence().toarray()).max() <= 1e-15


def _couette(n, mu1=1.0, mu2=1e-3):
    c = (np.arange(n) + 0.5) / n
    _, Y, _ = np.meshgrid(c, c, c, indexing="ij")
    cmu = np.where(Y < 0.5, mu1, mu2).ravel()
    P = P1P0(n, cmu, (DIRICHLET,) * 6)
    fc = np.zeros((3, n ** 3))
    fc[0] = 3.0 * cmu
    x, y, _ = P.disc.xyz.T
    xD = np.concatenate([np.stack([0.5 * (1 - x ** 2), x * (y - 0.5), 0 * x]).ravel(), np.zeros(P.nT)])
    sol = P.solve(P.rhs(f_cell=fc), "tr", xD)
    ph = sol[3 * P.nn:]
    ph -= np.sum(P.vol * ph) / P.vol.sum()  # the exact pressure has zero mean

    def ue(X):
        x, y, _ = X
        g = np.zeros((3, 3) + x.shape)
        g[0, 0], g[1, 0], g[1, 1] = -x, y - 0.5, x
        return np.stack([0.5 * (1 - x ** 2), x * (y - 0.5), 0 * x]), g
    errs = P.errors(sol, ue, lambda X: 2 * X[0] * P.mu_T - 0.5 * (mu1 + mu2), P.mu_T)
    return np.array(errs), np.abs(P.element_balance(sol)).max()


def test_couette_against_the_papers_table():
    """Sec. 4.2.2, P1-P0, gamma = 1: the velocity L2 errors within 6 % of the printed values at
    levels 0-1 (same Kuhn mesh; level 2 matches to 4 % but its direct solve takes minutes on a
    CPU), the rates of all three norms within 0.25 of the printed ones, and exact element-wise
    mass balance of the post-processed fluxes."""
    res = [_couette(n) for n in (4, 8)]
    errs = np.array([r[0] for r in res])
    ref = np.array([row[1:] for row in COUETTE[:2]])
    assert np.all(np.abs(errs[:, 0] / ref[:, 0] - 1) <= 0.06), errs[:, 0]
    rates, rref = np.log2(errs[:-1] / errs[1:]), np.log2(ref[:-1] / ref[1:])
    assert np.all(np.abs(rates - rref) <= 0.25), (rates, rref)
    assert max(r[1] for r in res) <= 1e-13


@pytest.mark.parametrize("problem", ["layers", "columns"])
def test_gradient_form_differences_against_the_papers_tables(problem):
    """The gradient form's relative difference to the strain form (a difference of the two
    continuous problems, Sec. 4.2.3-4.2.4) within 12 % of the printed P1-P0 entries, in ||.||_0,
    ||.||_V and ||.||_Q: levels 0 and 1 of the layers problem, level 1 of the columns problem
    (at level 0, 4^3 cells, the columns' corner singularities are not yet resolved: 10-13 %)."""
    gold = _golden(problem, "grad", "P1P0")
    for lvl, n in (((0, 4), (1, 8)) if problem == "layers" else ((1, 8),)):
        p = (W.viscosity_layers if problem == "layers" else W.viscosity_columns)(n, 4)
        P = P1P0(n, p.cell_mu().ravel(), p.face)
        b = P.rhs(p.nodal_forcing())
        xs, xg = P.solve(b, "sym"), P.solve(b, "grad")
        rel = P.norms(xg - xs) / P.norms(xs)
        assert np.all(np.abs(rel / gold[lvl] - 1) <= 0.12), (lvl, rel, gold[lvl])


def test_flux_balance_and_multigrid_solution():
    """On a stiff inclusion: the post-processed fluxes balance on every element for the direct
    solution, and FGMRES preconditioned by the P1-P0 V-cycle reaches that solution."""
    p = W.cube_inclusion(8, 4)
    H = P1P0Hierarchy(p.n, p.n_coarse, p.cell_mu().ravel(), p.face, "tr")
    L = H.levels[0]
    b = L.sp.rhs(p.nodal_forcing())
    xd = L.sp.solve(b, "tr")
    bal = L.sp.element_balance(xd)
    assert np.abs(bal).max() <= 1e-12 * np.abs(L.sp.facet_fluxes(xd)).max()
    x, hist = fgmres(L.K, lambda v: H.vcycle(np.zeros_like(v), v.copy()), b, L.free, rtol=1e-12, restart=40,
                     maxit=100)
    w = np.zeros_like(x)
    w[3 * L.nn:] = L.mp
    x[3 * L.nn:] -= np.dot(w, x) / L.mp.sum()
    assert np.linalg.norm(x - xd) <= 1e-8 * np.linalg.norm(xd)


@pytest.mark.parametrize("form", ["tr", "sym"])
def test_sampled_rows_equal_the_assembled_saddle_matrix(form):
    """The locally assembled rows of sampled_rows_p1p0 (used at sizes too large to assemble)
    equal the rows of the globally assembled saddle matrix [[A, B0^T], [B0, -C0]] (facets found
    there by sorting vertex triples, here by a local search) on random states, constrained
    velocity entries zero: every node's velocity rows and every ninth tetrahedron's pressure row
    (all six permutations, interior, boundary and interface cells) at 1e-13."""
    from oracle.p1p0 import sampled_rows_p1p0
    for p in (W.viscosity_columns(8, 4), W.cube_inclusion(8, 4)):
        n = p.n
        O = P1P0(n, p.cell_mu().ravel(), p.face)
        con = O.constrained()
        rng = np.random.Generator(np.random.PCG64(17))
        x = rng.uniform(-1, 1, 3 * O.nn + O.nT)
        x[con] = 0.0
        y = O.saddle(form) @ x
        y[con] = 0.0
        nodes = np.arange(O.nn)
        T = np.arange(0, O.nT, 9)
        s, r = np.divmod(T, n ** 3)
        ci, r = np.divmod(r, n * n)
        cj, ck = np.divmod(r, n)
        vel, pre = sampled_rows_p1p0(n, p.cell_mu().ravel(), p.face, form, x[: 3 * O.nn].reshape(3, -1),
                                     x[3 * O.nn:], nodes, list(zip(s, ci, cj, ck)))
        scale = np.abs(y).max()
        assert np.abs(vel.ravel() - y[: 3 * O.nn]).max() <= 1e-13 * scale
        assert np.abs(pre - y[3 * O.nn + T]).max() <= 1e-13 * scale
