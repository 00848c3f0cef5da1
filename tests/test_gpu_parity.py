"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle on the same seeded
inputs.  Tolerances: 1e-13 relative max-norm per FP64 operator apply and 1e-8 relative L2 per
solve (the accuracy targets of this work); smoother, transfer and cycle steps, which add
divisions and a dense coarse inverse, use 1e-12 / 1e-10 as stated in each test."""
import numpy as np
import pytest

from tests._lib import ensure_built

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle.forms import Discretisation, masked, sampled_rows  # noqa: E402
from oracle.solvers import Hierarchy as OracleHierarchy  # noqa: E402
from paper_1604_07994_gb300 import workloads as W  # noqa: E402

APPLY_TOL = 1e-13
SOLVE_TOL = 1e-8


@pytest.fixture(scope="module")
def sdx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ensure_built()
    from paper_1604_07994_gb300 import sdx as mod
    return mod


def _problems():
    rng = np.random.Generator(np.random.PCG64(11))
    # 48 cells per side, coarse lattice 6 (not a power of two), three viscosity ids
    ids = rng.integers(0, 3, (6, 6, 6)).astype(np.uint8)
    ids = np.repeat(np.repeat(np.repeat(ids, 8, 0), 8, 1), 8, 2)
    mixed = W.Problem(n=48, n_coarse=6, cell_id=ids, mu=np.array([1.0, 30.0, 0.05]),
                      face=(0, 1, 2, 1, 0, 2), forcing=W.gaussian_blobs(5), name="mixed_48")
    return {
        "cube16": W.cube_inclusion(16, 4),
        "boxes16": W.three_boxes(16, 8, contrast=1e4),
        "layer16": W.top_layer(16, 8),
        "columns16": W.viscosity_columns(16, 4),
        "layers16": W.viscosity_layers(16, 4),
        "mixed48": mixed,
        "tiny2": W.Problem(n=2, n_coarse=2, cell_id=np.array([[[0, 1], [1, 0]], [[1, 1], [0, 0]]], dtype=np.uint8),
                           mu=np.array([1.0, 7.0]), face=(2, 0, 1, 2, 0, 1), forcing=W.gaussian_blobs(1), name="tiny2"),
    }


PROBLEMS = _problems()


def _masked_random(d, seed):
    x = W.random_vector(d.n, seed).ravel()
    x[d.constrained()] = 0.0
    return x


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def _host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def _relmax(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.mark.parametrize("form", ["tr", "sym", "grad"])
@pytest.mark.parametrize("name", list(PROBLEMS))
def test_apply_matches_oracle(sdx, name, form):
    p = PROBLEMS[name]
    d = Discretisation(p.n, p.cell_mu().ravel(), p.face)
    K = masked(d.saddle(form), d.constrained())
    H = sdx.Hierarchy.from_problem(p, form=form)
    for seed in (1, 2):
        x = _masked_random(d, seed)
        y = _dev(np.zeros_like(x))
        H.sdx_apply(0, _dev(x), y)
        assert _relmax(_host(y), K @ x) <= APPLY_TOL


@pytest.mark.parametrize("name", ["cube16", "layer16", "mixed48", "tiny2"])
def test_masks_match_oracle(sdx, name):
    p = PROBLEMS[name]
    d = Discretisation(p.n, p.cell_mu().ravel(), p.face)
    H = sdx.Hierarchy.from_problem(p)
    assert np.array_equal(H.sdx_constraint_mask(0), d.constrained())
    assert np.array_equal(H.sdx_interface_mask(0), d.interface_nodes())
    n, nodes, free = H.sdx_level_size(0)
    assert (n, nodes, free) == (p.n, d.nn, int((~d.constrained()).sum()))


@pytest.mark.parametrize("name", ["cube16", "layer16", "mixed48"])
def test_residual_and_rhs_match_oracle(sdx, name):
    p = PROBLEMS[name]
    d = Discretisation(p.n, p.cell_mu().ravel(), p.face)
    K = masked(d.saddle("tr"), d.constrained())
    H = sdx.Hierarchy.from_problem(p)
    f = p.nodal_forcing()
    b = _dev(np.zeros(4 * d.nn))
    H.sdx_rhs(_dev(f.ravel()), b)
    bo = d.rhs(f)
    assert _relmax(_host(b), bo) <= APPLY_TOL
    x = _masked_random(d, 4)
    r = _dev(np.zeros_like(x))
    H.sdx_residual(0, _dev(bo), _dev(x), r)
    assert _relmax(_host(r), bo - K @ x) <= APPLY_TOL


@pytest.mark.parametrize("form", ["tr", "sym"])
@pytest.mark.parametrize("name", ["cube16", "boxes16", "layer16", "mixed48", "tiny2"])
def test_uzawa_step_matches_oracle(sdx, name, form):
    """One smoothing step (eq. Uzawa_smooth) from a random state, same colour order."""
    p = PROBLEMS[name]
    OH = OracleHierarchy(p.n, p.n, p.cell_mu().ravel(), p.face, form)
    L = OH.levels[0]
    H = sdx.Hierarchy.from_problem(p, form=form)
    x = _masked_random(L.disc, 7)
    b = _masked_random(L.disc, 8)
    xd = _dev(x)
    H.sdx_uzawa(0, _dev(b), xd)
    L.uzawa(x, b)
    assert _relmax(_host(xd), x) <= 1e-12


@pytest.mark.parametrize("name", ["cube16", "layer16", "mixed48"])
def test_transfers_match_oracle(sdx, name):
    p = PROBLEMS[name]
    OH = OracleHierarchy(p.n, p.n // 2, p.cell_mu().ravel(), p.face, "tr")
    H = sdx.Hierarchy.from_problem(p)  # level 1 of the full hierarchy is the grid n/2
    fine, coarse = OH.levels
    rf = _masked_random(fine.disc, 9)
    bc = _dev(np.zeros(4 * coarse.nn))
    H.sdx_restrict(0, _dev(rf), bc)
    assert _relmax(_host(bc), OH.P[0].T @ rf) <= APPLY_TOL
    ec = _masked_random(coarse.disc, 10)
    xf0 = _masked_random(fine.disc, 11)
    xf = _dev(xf0)
    H.sdx_prolong_add(0, _dev(ec), xf)
    assert _relmax(_host(xf), xf0 + OH.P[0] @ ec) <= APPLY_TOL


@pytest.mark.parametrize("form,coarse_form", [("tr", None), ("sym", None), ("tr", "sym")])
@pytest.mark.parametrize("name", ["cube16", "columns16", "boxes16", "layer16", "mixed48"])
def test_vcycle_matches_oracle(sdx, name, form, coarse_form):
    """Two consecutive V_var cycles from zero: smoother, residual, restriction, coarse solve
    (dense inverse vs. LU: 1e-10), prolongation and post-smoothing in the oracle's order.
    The second cycle checks that no level keeps state from the first."""
    p = PROBLEMS[name]
    OH = OracleHierarchy(p.n, p.n_coarse, p.cell_mu().ravel(), p.face, form, coarse_form=coarse_form)
    d = OH.levels[0].disc
    b = d.rhs(p.nodal_forcing())
    H = sdx.Hierarchy.from_problem(p, form=form, coarse_form=coarse_form)
    xd = _dev(np.zeros_like(b))
    bd = _dev(b)
    xo = np.zeros_like(b)
    for _ in range(2):
        H.sdx_vcycle(bd, xd)
        OH.vcycle(xo, b)
        assert np.linalg.norm(_host(xd) - xo) <= 1e-10 * np.linalg.norm(xo)


def _reference_solution(OH, b):
    """Oracle solution: direct LU when the system is small, otherwise the oracle's FGMRES +
    V-cycle driven to a 1e-13 relative residual, near FP64's attainable accuracy (sparse LU
    with partial pivoting fills in badly on the high-contrast strain systems)."""
    from oracle import solvers as S
    L = OH.levels[0]
    if int(L.free.sum()) <= S.DENSE_LIMIT:
        return L.direct(b)
    x, hist = S.fgmres(L.K, S.vcycle_preconditioner(OH), b, L.free, rtol=1e-13, restart=60, maxit=600)
    assert hist[-1] <= 3e-13 * np.linalg.norm(b[L.free])
    return _project(x, L.disc) if L.nullspace else x


def _project(x, d):
    w = d.pressure_weights()
    x = x.copy()
    x[3 * d.nn:] -= np.dot(w, x[3 * d.nn:]) / w.sum()
    return x


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("name,form,outer", [("cube16", "tr", 0), ("cube16", "sym", 0), ("boxes16", "tr", 1),
                                             ("boxes16", "sym", 1), ("layer16", "tr", 1), ("columns16", "tr", 0)])
def test_solve_matches_direct_solution(sdx, name, form, outer, prec):
    p = PROBLEMS[name]
    OH = OracleHierarchy(p.n, p.n_coarse, p.cell_mu().ravel(), p.face, form)
    L = OH.levels[0]
    b = L.disc.rhs(p.nodal_forcing())
    xo = _reference_solution(OH, b)
    H = sdx.Hierarchy.from_problem(p, form=form, prec=prec)
    xd = _dev(np.zeros_like(b))
    st = H.sdx_solve(_dev(b), xd, rtol=1e-12, maxit=300, outer=outer, restart=40)
    assert st["res"] <= 1e-12 * st["bnorm"]
    x = _host(xd)
    if L.nullspace:
        x = _project(x, L.disc)
    assert np.linalg.norm(x - xo) <= SOLVE_TOL * np.linalg.norm(xo)


def test_solve_host_matches_device_solve(sdx):
    p = PROBLEMS["cube16"]
    d = Discretisation(p.n, p.cell_mu().ravel(), p.face)
    b = d.rhs(p.nodal_forcing())
    H = sdx.Hierarchy.from_problem(p)
    xd = _dev(np.zeros_like(b))
    st1 = H.sdx_solve(_dev(b), xd, rtol=1e-9, outer=0)
    xh = np.zeros_like(b)
    st2 = H.sdx_solve_host(np.ascontiguousarray(b), xh, rtol=1e-9, outer=0)
    assert st1["iterations"] == st2["iterations"]
    assert np.array_equal(_host(xd), xh)  # deterministic: same bits from the same inputs


def test_full_size_apply_sampled_rows(sdx):
    """128^3 cells, three boxes with mu ratio 1e4 (the benchmark workload): sampled rows
    of the GPU apply against the oracle's patch-wise row evaluation."""
    p = W.three_boxes(128, 8, contrast=1e4)
    cm = p.cell_mu().ravel()
    nn = p.nodes
    rng = np.random.Generator(np.random.PCG64(21))
    H = sdx.Hierarchy.from_problem(p)
    con = H.sdx_constraint_mask(0)
    iface = np.flatnonzero(H.sdx_interface_mask(0))
    x = W.random_vector(p.n, 12).ravel()
    x[con] = 0.0
    y = _dev(np.zeros_like(x))
    H.sdx_apply(0, _dev(x), y)
    yh = _host(y).reshape(4, nn)
    nodes = np.concatenate([rng.integers(0, nn, 300), rng.choice(iface, 200), np.arange(0, 129 * 3)])
    for form in ("tr",):
        ys = sampled_rows(p.n, cm, p.face, form, x, nodes)
        assert np.abs(ys - yh[:, nodes]).max() <= APPLY_TOL * np.abs(yh).max()


def test_oversized_coarsest_grid_is_rejected(sdx):
    """The dense coarse solve takes at most 12000 unknowns: a 24^3 coarsest grid is refused
    with SDX_EINVAL instead of attempting a 60k x 60k inverse."""
    p = W.Problem(n=24, n_coarse=24, cell_id=np.zeros((24, 24, 24), dtype=np.uint8), mu=np.array([1.0]),
                  face=(0,) * 6, forcing=None)
    with pytest.raises(sdx.SdxError) as e:
        sdx.Hierarchy.from_problem(p)
    assert e.value.code == sdx.EINVAL and "coarsest grid" in str(e.value)


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("name", ["cube16", "mixed48", "boxes16"])
def test_fused_smoothing_launches_match_per_pass_kernels(sdx, name, prec, monkeypatch):
    """The fused smoothing launches (grid-wide cooperative, single cluster) run the same
    per-node code in the same dependency order as the per-pass kernels: V-cycles agree bit for
    bit.  Which path a hierarchy takes is fixed when it is created, from the environment."""
    p = PROBLEMS[name]
    d = Discretisation(p.n, p.cell_mu().ravel(), p.face)
    b = _dev(d.rhs(p.nodal_forcing()))
    out = {}
    for tag, env in (("per_pass", {"SDX_NO_COOP": "1"}),
                     ("fused", {"SDX_COOP_MAX_NODES": "200000", "SDX_CLUSTER_MAX_NODES": "10000"})):
        for k in ("SDX_NO_COOP", "SDX_COOP_MAX_NODES", "SDX_CLUSTER_MAX_NODES"):
            monkeypatch.delenv(k, raising=False)
        for k, v in env.items():
            monkeypatch.setenv(k, v)
        H = sdx.Hierarchy.from_problem(p, form="tr", coarse_form="sym", prec=prec)
        x = _dev(np.zeros(4 * p.nodes))
        for _ in range(2):
            H.sdx_vcycle(b, x)
        out[tag] = _host(x)
        H.close()
    assert np.array_equal(out["per_pass"], out["fused"])


def test_stuck_grid_barrier_times_out_and_reports(sdx, monkeypatch):
    """A grid barrier of the cooperative smoother that cannot complete (it waits for one more
    block than the grid has: a flag that nothing sets) gives up after its bounded wait, the
    solve returns SDX_ETIMEOUT, and the device stays usable for the next hierarchy."""
    p = PROBLEMS["cube16"]
    d = Discretisation(p.n, p.cell_mu().ravel(), p.face)
    b = _dev(d.rhs(p.nodal_forcing()))
    for k in ("SDX_NO_COOP", "SDX_CLUSTER_MAX_NODES"):
        monkeypatch.delenv(k, raising=False)
    monkeypatch.setenv("SDX_COOP_MAX_NODES", "200000")
    monkeypatch.setenv("SDX_TEST_BARRIER_EXTRA", "1")
    H = sdx.Hierarchy.from_problem(p, form="tr", prec=0)
    x = _dev(np.zeros(4 * p.nodes))
    with pytest.raises(sdx.SdxError) as e:
        H.sdx_solve(b, x, rtol=1e-8, maxit=5, outer=sdx.OUTER_VCYCLE)
    assert e.value.code == sdx.ETIMEOUT
    H.close()
    monkeypatch.delenv("SDX_TEST_BARRIER_EXTRA")
    H = sdx.Hierarchy.from_problem(p, form="tr", prec=0)
    x = _dev(np.zeros(4 * p.nodes))
    st = H.sdx_solve(b, x, rtol=1e-8, maxit=100, outer=sdx.OUTER_FGMRES)
    assert st["res"] <= 1e-8 * st["bnorm"]


def test_nonfinite_rhs_and_iteration_cap_are_reported(sdx):
    """A NaN planted in the right-hand side on the host is caught by the norm kernel
    (SDX_ENONFINITE); a solve stopped by maxit returns SDX_ENOCONV with its statistics filled
    and the last iterate in x (its residual below the initial one)."""
    p = PROBLEMS["cube16"]
    d = Discretisation(p.n, p.cell_mu().ravel(), p.face)
    b = d.rhs(p.nodal_forcing())
    H = sdx.Hierarchy.from_problem(p)
    bad = b.copy()
    bad[np.flatnonzero(~d.constrained())[10]] = np.nan
    x = _dev(np.zeros_like(b))
    with pytest.raises(sdx.SdxError) as e:
        H.sdx_solve(_dev(bad), x, rtol=1e-8, maxit=10, outer=sdx.OUTER_FGMRES)
    assert e.value.code == sdx.ENONFINITE
    x = _dev(np.zeros_like(b))
    st = H.sdx_solve(_dev(b), x, rtol=1e-14, maxit=2, outer=sdx.OUTER_VCYCLE, allow_noconv=True)
    assert st["status"] == sdx.ENOCONV and st["iterations"] == 2 and st["res"] < 0.5 * st["res0"]
    r = torch.empty_like(x)
    H.sdx_residual(0, _dev(b), x, r)
    assert abs(float(torch.linalg.norm(r)) - st["res"]) <= 1e-12 * st["res0"]


def test_full_size_top_layer_256(sdx):
    """256^3 cells, top layer of viscosity 1e3, traction-free top, free-slip sides, no-slip
    bottom (the mixed-precision workload): sampled rows of the FP64 apply against the oracle's
    row evaluation (interior, layer interface, traction and free-slip faces), and the
    FP32-refined solve, whose final residual recomputed in FP64 meets 1e-8."""
    p = W.top_layer(256, 8)
    cm = p.cell_mu().ravel()
    nn = p.nodes
    n1 = p.n + 1
    H = sdx.Hierarchy.from_problem(p, form="tr", coarse_form="sym", prec=1)
    con = H.sdx_constraint_mask(0)
    x = W.random_vector(p.n, 31).ravel()
    x[con] = 0.0
    y = _dev(np.zeros_like(x))
    H.sdx_apply(0, _dev(x), y)
    yh = _host(y).reshape(4, nn)
    rng = np.random.Generator(np.random.PCG64(32))
    i, j = rng.integers(0, n1, 100), rng.integers(0, n1, 100)
    top = i + n1 * (j + n1 * p.n)                       # traction face
    iface = i + n1 * (j + n1 * (7 * p.n // 8))          # viscosity interface plane
    side = 0 + n1 * (j + n1 * rng.integers(0, n1, 100))  # free-slip face x = 0
    nodes = np.concatenate([rng.integers(0, nn, 200), top, iface, side])
    ys = sampled_rows(p.n, cm, p.face, "tr", x, nodes)
    assert np.abs(ys - yh[:, nodes]).max() <= APPLY_TOL * np.abs(yh).max()
    f = _dev(p.nodal_forcing().ravel())
    b = torch.zeros(4 * nn, dtype=torch.float64, device="cuda")
    H.sdx_rhs(f, b)
    xs = torch.zeros_like(b)
    st = H.sdx_solve(b, xs, rtol=1e-8, maxit=200, outer=sdx.OUTER_FGMRES, restart=30)
    r = torch.empty_like(b)
    H.sdx_residual(0, b, xs, r)
    assert st["status"] == 0 and float(torch.linalg.norm(r)) <= SOLVE_TOL * float(torch.linalg.norm(b))
