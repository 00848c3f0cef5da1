"""Pins for the oracle's assembly (no GPU): closed forms and identities from the paper.

Each test checks the oracle against something other than itself: an identity or closed form
stated in the paper, an exact property of P1 finite elements, or a textbook eigenvalue
formula.  A dropped term, wrong sign or transposed index in oracle/forms.py breaks one of them.
"""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle.forms import DIRICHLET, FREESLIP, TRACTION, Discretisation
from oracle.solvers import coarsen_cell_mu
from oracle.transfer import prolongation
from paper_1604_07994_gb300 import workloads as W


def _disc(n, cell_mu, face=(DIRICHLET,) * 6):
    return Discretisation(n, np.asarray(cell_mu, dtype=np.float64).ravel(), face)


def _field(d, fun):
    """Nodal interpolant of a vector field as a [3nn] SoA vector."""
    x = d.xyz
    v = fun(x[:, 0], x[:, 1], x[:, 2])
    return np.concatenate([np.broadcast_to(c, (d.nn,)) for c in v]).astype(np.float64)


def _random_piecewise_mu(n, seed, lattice=None):
    rng = np.random.Generator(np.random.PCG64(seed))
    if lattice is None:
        return 10.0 ** rng.uniform(-2, 2, n ** 3)
    c = 10.0 ** rng.uniform(-2, 2, lattice ** 3).reshape(lattice, lattice, lattice)
    r = n // lattice
    return np.repeat(np.repeat(np.repeat(c, r, 0), r, 1), r, 2).ravel()


RIGID = [
    lambda x, y, z: (1.0, 0.0, 0.0),
    lambda x, y, z: (0.0, 1.0, 0.0),
    lambda x, y, z: (0.0, 0.0, 1.0),
    lambda x, y, z: (0.0 * x, -z, y),      # e_x cross x
    lambda x, y, z: (z, 0.0 * x, -x),      # e_y cross x
    lambda x, y, z: (-y, x, 0.0 * x),      # e_z cross x
]


@pytest.mark.parametrize("form", ["tr", "sym", "dev"])
def test_rigid_motions_have_zero_energy(form):
    """a_sym, a_dev and a_tr vanish on rigid motions (sym grad r = 0, div r = 0), for any
    piecewise viscosity: the unconstrained matrices annihilate their interpolants."""
    d = _disc(4, _random_piecewise_mu(4, 1))
    A = d.velocity_block(form)
    scale = abs(A).max()
    for r in RIGID:
        y = A @ _field(d, r)
        assert np.abs(y).max() <= 1e-13 * scale


def test_gradient_form_is_not_objective():
    """The gradient form (mu grad u, grad v) does not annihilate rotations once mu jumps:
    the objectivity failure noted in Sec. 1 after eq. (aint)."""
    p = W.cube_inclusion(8, 4)
    d = _disc(8, p.cell_mu())
    A = d.velocity_block("grad")
    y = A @ _field(d, RIGID[5])
    iface = d.interface_nodes()
    yi = y.reshape(3, d.nn)[:, iface]
    assert np.abs(yi).max() > 1e-3 * abs(A).max()
    # away from the interface and the boundary the rows are pure Laplacian rows: zero
    i, j, k = d.node_ijk()
    inner = (i > 0) & (i < 8) & (j > 0) & (j < 8) & (k > 0) & (k < 8) & ~iface
    assert np.abs(y.reshape(3, d.nn)[:, inner]).max() <= 1e-13 * abs(A).max()


def test_quadratic_forms_of_identity_field():
    """Sec. 3: for v = x, a_dev(v,v) = 0 and a_tr(v,v) = -3 sum_i mu_i |Omega_i|; also
    a_sym(x,x) = 6 sum mu|Omega| (sym grad x = I) and (mu grad x, grad x) = 3 sum mu|Omega|."""
    n = 4
    mu = _random_piecewise_mu(n, 2)
    d = _disc(n, mu)
    X = _field(d, lambda x, y, z: (x, y, z))
    s = np.sum(mu) / n ** 3  # sum_i mu_i |Omega_i| with cell volume 1/n^3
    expect = {"tr": -3.0 * s, "sym": 6.0 * s, "dev": 0.0, "grad": 3.0 * s}
    for form, val in expect.items():
        got = X @ (d.velocity_block(form) @ X)
        assert abs(got - val) <= 1e-12 * 6.0 * s, (form, got, val)


def test_newbil_relations_between_three_forms():
    """Eq. (newbil): a_tr = a_sym - (mu div, div) = a_dev - (1/3)(mu div, div) in 3D.  The
    three forms are assembled from independent tensor definitions, so
    A_sym - A_tr = (3/2)(A_sym - A_dev), and that difference is positive semi-definite."""
    n = 3
    d = _disc(n, _random_piecewise_mu(n, 3))
    As, At, Ad = (d.velocity_block(f).toarray() for f in ("sym", "tr", "dev"))
    D = As - At
    assert np.abs(D - 1.5 * (As - Ad)).max() <= 1e-13 * np.abs(As).max()
    ev = np.linalg.eigvalsh(D)
    assert ev.min() >= -1e-12 * ev.max()


@pytest.mark.parametrize("case", ["cube", "layer_traction", "columns_freeslip"])
def test_decoupling_outside_interface_rows(case):
    """Sec. 2.2, eq. (equivalence-stencil): rows of test functions in H^1_0 of one isoviscous
    subdomain are pure mu-Laplacian rows, so the velocity cross-blocks of A_tr vanish on every
    free row outside the interface set and are present on it; the diagonal blocks of A_tr
    equal those of the gradient form on all rows (the two extra terms cancel for i = j)."""
    if case == "cube":
        p = W.cube_inclusion(8, 4)
    elif case == "layer_traction":
        p = W.top_layer(8, 8)
    else:
        p = W.viscosity_columns(8)
    d = Discretisation(p.n, p.cell_mu().ravel(), p.face)
    nn = d.nn
    con = d.constrained()
    dm = sp.diags((~con[: 3 * nn]).astype(float))
    At = (dm @ d.velocity_block("tr") @ dm).tocsr()
    Ag = (dm @ d.velocity_block("grad") @ dm).tocsr()
    scale = abs(At).max()
    iface = d.interface_nodes()
    cross_on_iface = 0.0
    for j in range(3):
        for i in range(3):
            blk = At[j * nn:(j + 1) * nn, i * nn:(i + 1) * nn]
            if i == j:
                g = Ag[j * nn:(j + 1) * nn, i * nn:(i + 1) * nn]
                assert abs(blk - g).max() <= 1e-14 * scale
                continue
            rowmax = np.asarray(abs(blk).max(axis=1).todense()).ravel()
            assert rowmax[~iface].max() <= 1e-14 * scale, (case, j, i)
            cross_on_iface = max(cross_on_iface, rowmax[iface].max())
    assert cross_on_iface > 1e-3 * scale


def test_interface_set_size_cube_inclusion():
    """For the box [1/4, 3/4]^3 at n = 16 the interface nodes are the surface nodes of a
    9 x 9 x 9 node block: 9^3 - 7^3 = 386."""
    p = W.cube_inclusion(16, 4)
    d = Discretisation(16, p.cell_mu().ravel(), p.face)
    assert int(d.interface_nodes().sum()) == 9 ** 3 - 7 ** 3


def test_isoviscous_block_is_vector_laplacian_with_known_spectrum():
    """mu1 = mu2: with homogeneous Dirichlet data the free A_tr block equals the gradient form
    (three decoupled mu-Laplacians).  On the Kuhn mesh the P1 Laplacian is the 7-point stencil
    mu h (6, -1), whose Dirichlet eigenvalues are mu h sum_k 4 sin^2(pi m_k / (2n)),
    m_k = 1..n-1, each with multiplicity 3 here."""
    n, mu = 4, 2.5
    d = _disc(n, np.full(n ** 3, mu))
    free = np.flatnonzero(~d.constrained()[: 3 * d.nn])
    At = d.velocity_block("tr")[free][:, free].toarray()
    Ag = d.velocity_block("grad")[free][:, free].toarray()
    assert np.abs(At - Ag).max() <= 1e-14 * np.abs(At).max()
    m = np.arange(1, n)
    s = 4.0 * np.sin(np.pi * m / (2 * n)) ** 2
    lam = (s[:, None, None] + s[None, :, None] + s[None, None, :]).ravel()
    expect = np.sort(np.tile(mu * lam / n, 3))
    got = np.linalg.eigvalsh(At)
    assert np.abs(got - expect).max() <= 1e-12 * expect.max()


@pytest.mark.parametrize("form", ["tr", "sym", "grad"])
def test_saddle_matrix_is_symmetric(form):
    p = W.top_layer(4, 4)
    d = Discretisation(4, p.cell_mu().ravel(), p.face)
    K = d.saddle(form)
    assert abs(K - K.T).max() == 0.0


def test_nested_spaces_galerkin_identity():
    """Nested P1 spaces with h-independent bilinear forms: P^T A_h P = A_2h and
    P^T B_h P = B_2h exactly when the viscosity is resolved on the coarse grid.  (C is not
    included: its weight tau depends on h.)"""
    nc = 2
    mu_f = _random_piecewise_mu(4, 4, lattice=2)
    df = _disc(4, mu_f)
    dc = _disc(2, coarsen_cell_mu(4, mu_f))
    P = prolongation(nc)
    P3 = sp.block_diag([P] * 3, format="csr")
    for form in ("tr", "sym", "grad"):
        Af, Ac = df.velocity_block(form), dc.velocity_block(form)
        assert abs(P3.T @ Af @ P3 - Ac).max() <= 1e-13 * abs(Ac).max()
    Bf, Bc = df.divergence(), dc.divergence()
    assert abs(P.T @ Bf @ P3 - Bc).max() <= 1e-13 * abs(Bc).max()


def test_divergence_and_stabilisation_consistency():
    """b(v, lambda_b) = -(div v, lambda_b): for a linear field (constant divergence) B I(u)
    equals -div(u) times the lumped mass at every node; C annihilates constants; and for
    all-Dirichlet or free-slip walls B^T 1 = 0 on free rows (int div v = 0)."""
    p = W.cube_inclusion(4, 4)
    for face in [(DIRICHLET,) * 6, (FREESLIP,) * 6]:
        d = Discretisation(4, p.cell_mu().ravel(), face)
        B = d.divergence()
        u = _field(d, lambda x, y, z: (2.0 * x + y, 3.0 * y - z, -0.5 * z + x))  # div = 4.5
        assert np.abs(B @ u + 4.5 * d.lumped_mass()).max() <= 1e-14
        assert np.abs(d.stabilisation() @ np.ones(d.nn)).max() <= 1e-15
        bt1 = B.T @ np.ones(d.nn)
        free = ~d.constrained()[: 3 * d.nn]
        assert np.abs(bt1[free]).max() <= 1e-15


@pytest.mark.parametrize("n,seed", [(4, 21), (6, 22), (8, 23)])
def test_stabilisation_energy_of_linear_pressure_closed_form(n, seed):
    """For a linear pressure q = a + g.x the gradient is exact and constant, so
    q^T C q = sum_T tau_T |T| |g|^2 = |g|^2 beta h^2 sum_cells h^3 / mu_cell
    (six tetrahedra of volume h^3/6 per cell, tau_T = beta h^2 / mu_T).  With a viscosity that
    varies cell by cell this pins the power of h and of mu in tau_T and the volume factor |T|,
    which C 1 = 0 cannot see (a wrong exponent or a missing |T| keeps C 1 = 0)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    mu = _random_piecewise_mu(n, seed)
    d = _disc(n, mu)
    g = rng.normal(size=3)
    x = d.xyz
    q = 0.7 + x @ g
    exact = float(g @ g) * d.beta * d.h ** 2 * np.sum(d.h ** 3 / mu)
    assert abs(q @ (d.stabilisation() @ q) - exact) <= 1e-13 * exact
    # the same energy with beta doubled: C is linear in beta
    d2 = Discretisation(n, mu, (DIRICHLET,) * 6, beta=2.0 * d.beta)
    assert abs(q @ (d2.stabilisation() @ q) - 2.0 * exact) <= 1e-13 * exact


def test_mass_and_pressure_weights():
    p = W.three_boxes(8, 8, contrast=1e4)
    d = Discretisation(8, p.cell_mu().ravel(), p.face)
    assert abs(d.lumped_mass().sum() - 1.0) <= 1e-14
    mu = p.cell_mu().ravel()
    assert abs(d.pressure_weights().sum() - np.sum(1.0 / mu) / 8 ** 3) <= 1e-14


def test_pspg_rhs_closed_form_for_constant_forcing():
    """g_b = -tau int f . grad lambda_b.  For f = e_z and constant mu the divergence theorem
    gives -tau int_{dOmega} lambda_b n_z: zero at interior nodes, -tau h^2 at nodes interior
    to the top face and +tau h^2 on the bottom face (a face node's hat function integrates to
    h^2 over the triangulated face)."""
    n, mu = 6, 3.0
    d = _disc(n, np.full(n ** 3, mu), face=(TRACTION,) * 6)
    f = np.zeros((3, d.nn))
    f[2] = 1.0
    g = d.rhs(f).reshape(4, d.nn)[3]
    tau = d.beta * d.h ** 2 / mu
    i, j, k = d.node_ijk()
    inner_xy = (i > 0) & (i < n) & (j > 0) & (j < n)
    interior = inner_xy & (k > 0) & (k < n)
    assert np.abs(g[interior]).max() <= 1e-15
    assert np.allclose(g[inner_xy & (k == n)], -tau * d.h ** 2, rtol=1e-12, atol=0)
    assert np.allclose(g[inner_xy & (k == 0)], tau * d.h ** 2, rtol=1e-12, atol=0)


def test_prolongation_reproduces_linear_functions():
    nc = 3
    P = prolongation(nc)
    from oracle.mesh import node_xyz
    xc, xf = node_xyz(nc), node_xyz(2 * nc)
    lin = lambda X: 1.0 + 2.0 * X[:, 0] - 3.0 * X[:, 1] + 0.5 * X[:, 2]
    assert np.abs(P @ lin(xc) - lin(xf)).max() <= 1e-14
    assert np.all(np.asarray(P.sum(axis=1)).ravel() == 1.0)


def test_consistent_mass_integrates_linear_fields_exactly():
    """A linear field is its own P1 interpolant, so l^T M l is the exact integral of l^2 over
    the unit cube: a^2 + (b^2+c^2+d^2)/3 + a(b+c+d) + (bc+bd+cd)/2 for l = a+bx+cy+dz.  The row
    sums of M are the lumped masses; with the weight 1/(2 mu_T) the total is int 1/(2 mu)."""
    n = 4
    mu = _random_piecewise_mu(n, 5, lattice=2)
    d = _disc(n, mu)
    a, b, c, e = 1.0, 2.0, -3.0, 0.5
    lin = a + b * d.xyz[:, 0] + c * d.xyz[:, 1] + e * d.xyz[:, 2]
    exact = a * a + (b * b + c * c + e * e) / 3.0 + a * (b + c + e) + (b * c + b * e + c * e) / 2.0
    M = d.mass_matrix()
    assert abs(lin @ (M @ lin) - exact) <= 1e-13 * exact
    assert np.abs(np.asarray(M.sum(axis=1)).ravel() - d.lumped_mass()).max() <= 1e-16
    Mq = d.mass_matrix(1.0 / (2.0 * d.mu_T))
    one = np.ones(d.nn)
    assert abs(one @ (Mq @ one) - np.sum(1.0 / (2.0 * mu)) / n ** 3) <= 1e-13 * np.sum(1.0 / mu) / n ** 3


def test_paper_norms_of_closed_form_fields():
    """The norms of Sec. 3 on u = x (identity field) and a linear pressure, constant mu:
    ||u||_0^2 = int |x|^2 = 1, ||u||_V^2 = a_sym(x, x) = 6 mu (sym grad x = I), and
    ||p||_Q^2 = int p^2 / (2 mu)."""
    n, mu = 4, 2.5
    d = _disc(n, np.full(n ** 3, mu))
    X = _field(d, lambda x, y, z: (x, y, z))
    p = 1.0 - d.xyz[:, 0]
    l0, lv, lq = d.paper_norms(np.concatenate([X, p]))
    assert abs(l0 ** 2 - 1.0) <= 1e-13
    assert abs(lv ** 2 - 6.0 * mu) <= 1e-12 * 6.0 * mu
    # int (1 - x)^2 over the unit cube = 1/3
    assert abs(lq ** 2 - (1.0 / 3.0) / (2.0 * mu)) <= 1e-13



def test_decoupled_block_is_indefinite_on_the_columns_problem():
    """Sec. 3: a_tr is not positive semi-definite.  On the paper's columns problem (free-slip
    faces) its constrained velocity block has negative eigenvalues - the planar dilation
    (x, y, 0) has zero a_tr energy and satisfies the free-slip conditions inside a column
    that touches the faces x = 0 and y = 0 - while the strain and gradient blocks are
    positive definite."""
    from oracle.forms import masked
    p = W.viscosity_columns(8, 4)
    d = Discretisation(8, p.cell_mu().ravel(), p.face)
    free = np.flatnonzero(~d.constrained()[: 3 * d.nn])
    low = {}
    for form in ("tr", "sym", "grad"):
        A = d.velocity_block(form)[free][:, free].toarray()
        s = 1.0 / np.sqrt(np.diag(A))
        low[form] = np.linalg.eigvalsh(s[:, None] * A * s[None, :])[:5]
    assert np.count_nonzero(low["tr"] < -1e-3) == 4, low["tr"]
    assert low["sym"][0] > 1e-2 and low["grad"][0] > 1e-2, (low["sym"], low["grad"])
    X = _field(d, lambda x, y, z: (x, y, 0.0 * x))
    assert abs(X @ (d.velocity_block("tr") @ X)) <= 1e-13 * np.abs(X @ (d.velocity_block("sym") @ X))


def test_divergence_weights_lump_the_div_div_form_exactly_for_constant_divergence():
    """D_b = mu_b / m_b makes (B u)^T diag(D) (B u) the mass-lumped (mu div u, div u); for a
    field of constant divergence the lumping is exact: (B u)_b = -div(u) m_b, so the sum is
    div^2 sum_T mu_T |T| = div^2 sum_i mu_i |Omega_i| (piecewise mu)."""
    n = 4
    mu = _random_piecewise_mu(n, 6, lattice=2)
    d = _disc(n, mu)
    B = d.divergence()
    D = d.divergence_weights()
    s = np.sum(mu) / n ** 3
    for field, div in ((lambda x, y, z: (x, y, z), 3.0), (lambda x, y, z: (x, 0.0 * x, 0.0 * x), 1.0),
                       (lambda x, y, z: (0.0 * x, 2.0 * y, -z), 1.0)):
        Bu = B @ _field(d, field)
        assert np.allclose(Bu, -div * d.lumped_mass(), rtol=1e-12, atol=1e-15)
        assert abs(Bu @ (D * Bu) - div ** 2 * s) <= 1e-12 * div ** 2 * s
