"""Pins for interfaces the coarse grids do not resolve (Sec. 2.2, closing remark: a level-set
interface cutting the cells).  The finest operator is the plain assembly (pinned elsewhere);
what is new is the coarsening rule of the viscosity (the coarse levels only precondition) and
the workload.  Checked here against brute force on tiny inputs and against the direct solve."""
import numpy as np
import pytest

from oracle.solvers import Hierarchy, coarsen_cell_mu, fgmres, vcycle_preconditioner
from paper_1604_07994_gb300 import workloads as W


def _one_coarse_cell(children):
    """A 2^3 grid whose 8 cells carry `children` in x-fastest order."""
    return np.asarray(children, dtype=np.float64)


@pytest.mark.parametrize("children,expected", [
    ([1, 1, 1, 1, 1, 2, 2, 2], 1.0),    # plain majority
    ([1, 1, 1, 1, 2, 2, 2, 2], 2.0),    # 4:4 tie goes to the larger viscosity
    ([3, 3, 1, 1, 2, 2, 5, 7], 3.0),    # three-way tie of pairs: the largest of the tied values
    ([7, 7, 7, 7, 7, 7, 7, 7], 7.0),    # agreeing children: the resolved value
    ([0.1, 9, 9, 0.1, 0.1, 5, 5, 5], 5.0),  # 3 x 0.1 and 3 x 5 tie, 5 is larger
])
def test_majority_rule_brute_force(children, expected):
    assert coarsen_cell_mu(2, _one_coarse_cell(children), "majority")[0] == expected


def test_majority_rule_cell_placement():
    """Each coarse cell takes its own 8 children (x-fastest ordering of both grids)."""
    rng = np.random.Generator(np.random.PCG64(3))
    fine = rng.choice([1.0, 10.0, 100.0], size=(4, 4, 4))
    coarse = coarsen_cell_mu(4, fine.ravel(), "majority").reshape(2, 2, 2)
    for K in range(2):
        for J in range(2):
            for I in range(2):
                kids = fine[2 * K:2 * K + 2, 2 * J:2 * J + 2, 2 * I:2 * I + 2].ravel()
                vals, counts = np.unique(kids, return_counts=True)
                assert coarse[K, J, I] == vals[counts == counts.max()].max()


def test_resolved_rule_refuses_a_level_set():
    """The sphere cuts the cells of the coarser grids: the resolved rule refuses it, the
    majority rule coarsens it to a non-empty stiff core down to the coarsest grid."""
    p = W.level_set_sphere(32, 4)
    mu = p.cell_mu().ravel()
    with pytest.raises(ValueError):
        coarsen_cell_mu(32, mu, "resolved")
    m, n = mu, 32
    while n > 4:
        m = coarsen_cell_mu(n, m, "majority")
        n //= 2
    assert 0 < np.count_nonzero(m == p.mu[1]) < m.size


def test_level_set_workload_is_a_sphere():
    """Cell ids are the sign of |x - c| - r at the cell centres: the stiff volume approaches
    4/3 pi r^3 and the ids are those of a ball (convex: every row of cells inside is one
    contiguous run)."""
    p = W.level_set_sphere(64, 4)
    ids = p.cell_id
    frac = ids.mean()
    rng = np.random.Generator(np.random.PCG64(6))
    rng.uniform(0.4, 0.6, 3)
    r = rng.uniform(0.17, 0.27)
    assert abs(frac - 4.0 / 3.0 * np.pi * r ** 3) <= 0.02 * frac
    for k in range(64):
        for j in range(64):
            row = np.flatnonzero(ids[k, j])
            if row.size:
                assert row[-1] - row[0] + 1 == row.size


def test_majority_hierarchy_solves_to_the_direct_solution():
    """With the majority-coarsened levels as preconditioner, FGMRES reaches the direct solution
    of the finest system (the coarsening changes the preconditioner only)."""
    p = W.level_set_sphere(16, 4)
    H = Hierarchy(p.n, p.n_coarse, p.cell_mu().ravel(), p.face, "tr", coarse_form="sym",
                  coarsening="majority")
    L = H.levels[0]
    b = L.disc.rhs(p.nodal_forcing())
    x, hist = fgmres(L.K, vcycle_preconditioner(H), b, L.free, rtol=1e-12, restart=40, maxit=200)
    xd = L.direct(b)
    w = L.disc.pressure_weights()
    x[3 * L.nn:] -= np.dot(w, x[3 * L.nn:]) / w.sum()
    assert np.linalg.norm(x - xd) <= 1e-8 * np.linalg.norm(xd)
    assert len(hist) <= 3  # converged within the first restart cycles
