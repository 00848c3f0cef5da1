"""GPU parity of the single smoother passes and of the FP32 kernels against the CPU oracle.

FP64: one colour pass of the Uzawa smoother (Sec. 5, eq. Uzawa_smooth) - the velocity
Gauss-Seidel pass on A u = f - B^T p or the relaxed pressure pass on C p = B u - g, for one
colour - through sdx_smooth_pass, against the oracle's pass of the same colour from the same
state (oracle.solvers.Level.velocity_pass / pressure_pass), at 1e-13 relative max-norm.

FP32: sdx_apply_f32, sdx_smooth_pass_f32 and sdx_uzawa_f32 (the arithmetic of the FP32
multigrid cycle) against the FP64 oracle on the same inputs (FP32 values widened exactly).
Tolerances follow from FP32 rounding, unit roundoff u = 2^-24:

* one row of y = K x is a sum of at most 60 products (a 15-point stencil over 4 components);
  the kernels evaluate it in a regrouped order (shared differences of the Kuhn stencil) whose
  coefficients are at most 3 times the matrix entries in absolute value, plus rounding of each
  coefficient to FP32.  The standard bound for a computed sum of products then gives
  |y32 - y|_row <= 64 u (|K| |x|)_row well inside its constant (the evaluation has about 20
  rounded operations per row);
* a velocity update u + (f - row) / diag adds a few roundings on top of the row:
  |u32 - u|_row <= 64 u (|u| + (|f| + (|A| |u| + |B^T| |p|)_row) / diag); the pressure update
  likewise with omega / diag(C);
* over several Uzawa steps the perturbations of the passes do not grow (Gauss-Seidel
  contracts them; an FP32 emulation of the oracle's steps on the CPU stays at 1e-7 relative
  after 1-5 steps), so 1e-5 relative max-norm leaves a margin of about 100 while a wrong
  coefficient or index shows up at 1e-3 or more.
"""
import numpy as np
import pytest
import scipy.sparse as sp

from tests._lib import ensure_built

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle.solvers import OMEGA  # noqa: E402
from oracle.solvers import Hierarchy as OracleHierarchy  # noqa: E402
from paper_1604_07994_gb300 import workloads as W  # noqa: E402

PASS_TOL = 1e-13
U32 = 2.0 ** -24
ROW_FACTOR = 64
STEPS_TOL = 1e-5


@pytest.fixture(scope="module")
def sdx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ensure_built()
    from paper_1604_07994_gb300 import sdx as mod
    return mod


def _mixed48():
    rng = np.random.Generator(np.random.PCG64(11))
    ids = rng.integers(0, 3, (6, 6, 6)).astype(np.uint8)
    ids = np.repeat(np.repeat(np.repeat(ids, 8, 0), 8, 1), 8, 2)
    return W.Problem(n=48, n_coarse=6, cell_id=ids, mu=np.array([1.0, 30.0, 0.05]),
                     face=(0, 1, 2, 1, 0, 2), forcing=W.gaussian_blobs(5), name="mixed_48")


PROBLEMS = {
    "cube16": lambda: W.cube_inclusion(16, 4),
    "boxes16": lambda: W.three_boxes(16, 8, contrast=1e4),
    "layer16": lambda: W.top_layer(16, 8),
    "columns16": lambda: W.viscosity_columns(16, 4),
    "mixed48": _mixed48,
    "tiny2": lambda: W.Problem(n=2, n_coarse=2,
                               cell_id=np.array([[[0, 1], [1, 0]], [[1, 1], [0, 0]]], dtype=np.uint8),
                               mu=np.array([1.0, 7.0]), face=(2, 0, 1, 2, 0, 1),
                               forcing=W.gaussian_blobs(1), name="tiny2"),
}

_oracle_cache = {}


def _oracle_level(name, form, level=0, coarse_form=None):
    """Oracle level `level` of the problem's hierarchy (the finest takes `form`, the coarser
    ones `coarse_form`, as the library's hierarchy does)."""
    key = (name, form, coarse_form)
    if key not in _oracle_cache:
        p = PROBLEMS[name]()
        _oracle_cache[key] = (p, OracleHierarchy(p.n, p.n_coarse, p.cell_mu().ravel(), p.face, form,
                                                 coarse_form=coarse_form))
    p, OH = _oracle_cache[key]
    return p, OH.levels[level]


def _state(L, seed, dtype=np.float64):
    """Random (x, b) of the level, constrained entries zero, exactly representable in dtype."""
    x = W.random_vector(L.n, seed).ravel().astype(dtype).astype(np.float64)
    b = W.random_vector(L.n, seed + 1).ravel().astype(dtype).astype(np.float64)
    x[L.con] = 0.0
    b[L.con] = 0.0
    return x, b


def _dev(a, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dtype).cuda()


def _host(t):
    torch.cuda.synchronize()
    return t.double().cpu().numpy()


def _relmax(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def _oracle_pass(L, x, b, which, colour):
    nn = L.nn
    x = x.copy()
    u, p = x[: 3 * nn], x[3 * nn:]
    if which == 0:
        L.velocity_pass(u, p, b[: 3 * nn], colour == 0)
    else:
        L.pressure_pass(u, p, b[3 * nn:], colour == 0)
    return x


# ---------------------------------------------------------------------------------- FP64
@pytest.mark.parametrize("form", ["tr", "sym", "grad"])
@pytest.mark.parametrize("name", list(PROBLEMS))
def test_single_colour_pass_matches_oracle(sdx, name, form):
    """Each of the four passes (velocity / pressure, colour 0 / 1) from the same random state,
    and the five passes of one Uzawa step chained, pass by pass, at 1e-13."""
    p, L = _oracle_level(name, form)
    H = sdx.Hierarchy.from_problem(p, form=form)
    for which in (0, 1):
        for colour in (0, 1):
            x, b = _state(L, 40 + 2 * which + colour)
            xd = _dev(x)
            H.sdx_smooth_pass(0, which, colour, _dev(b), xd)
            ref = _oracle_pass(L, x, b, which, colour)
            err = _relmax(_host(xd), ref)
            assert err <= PASS_TOL, (name, form, which, colour, err)
            assert np.abs(ref - x).max() > 0.0  # the pass changed something
    # chained: velocity 0, 1, 0 then pressure 0, 1, compared after every pass
    x, b = _state(L, 50)
    xd, bd = _dev(x), _dev(b)
    for which, colour in ((0, 0), (0, 1), (0, 0), (1, 0), (1, 1)):
        H.sdx_smooth_pass(0, which, colour, bd, xd)
        x = _oracle_pass(L, x, b, which, colour)
        err = _relmax(_host(xd), x)
        assert err <= PASS_TOL, (name, form, "chained", which, colour, err)


# ---------------------------------------------------------------------------------- FP32
def _abs(M):
    return abs(M).tocsr() if sp.issparse(M) else np.abs(M)


@pytest.mark.parametrize("form", ["tr", "sym", "grad"])
@pytest.mark.parametrize("name", ["cube16", "boxes16", "layer16", "mixed48", "tiny2"])
def test_fp32_apply_within_rounding_bound(sdx, name, form):
    p, L = _oracle_level(name, form)
    H = sdx.Hierarchy.from_problem(p, form=form, prec=1)
    absK = _abs(L.K)
    for seed in (60, 61):
        x, _ = _state(L, seed, np.float32)
        y = _dev(np.zeros_like(x), torch.float32)
        H.sdx_apply_f32(0, _dev(x, torch.float32), y)
        yg = _host(y)
        ref = L.K @ x
        bound = ROW_FACTOR * U32 * (absK @ np.abs(x))
        excess = np.abs(yg - ref) - bound
        assert excess.max() <= 0.0, (name, form, float((np.abs(yg - ref) / np.maximum(bound, 1e-300)).max()))
        assert np.all(yg[L.con] == 0.0)


@pytest.mark.parametrize("form", ["tr", "sym", "grad"])
@pytest.mark.parametrize("name", ["cube16", "boxes16", "layer16", "mixed48", "tiny2"])
def test_fp32_single_pass_within_rounding_bound(sdx, name, form):
    p, L = _oracle_level(name, form)
    H = sdx.Hierarchy.from_problem(p, form=form, prec=1)
    nn = L.nn
    absA, absBT, absB, absC = _abs(L.A), _abs(L.BT), _abs(L.B), _abs(L.C)
    for which in (0, 1):
        for colour in (0, 1):
            x, b = _state(L, 70 + 2 * which + colour, np.float32)
            xd = _dev(x, torch.float32)
            H.sdx_smooth_pass_f32(0, which, colour, _dev(b, torch.float32), xd)
            xg = _host(xd)
            ref = _oracle_pass(L, x, b, which, colour)
            changed = ref != x
            u, pr = np.abs(x[: 3 * nn]), np.abs(x[3 * nn:])
            if which == 0:
                dA = np.where(L.diagA != 0, np.abs(L.diagA), 1.0)
                scale = np.concatenate([u + (np.abs(b[: 3 * nn]) + absA @ u + absBT @ pr) / dA, pr])
            else:
                dC = np.where(L.diagC != 0, np.abs(L.diagC), 1.0)
                scale = np.concatenate([u, pr + OMEGA * (absB @ u + np.abs(b[3 * nn:]) + absC @ pr) / dC])
            bound = ROW_FACTOR * U32 * scale
            assert np.all(xg[~changed] == x[~changed]), (name, form, which, colour)  # untouched entries
            ratio = float((np.abs(xg - ref)[changed] / bound[changed]).max())
            assert ratio <= 1.0, (name, form, which, colour, ratio)


@pytest.mark.parametrize("steps", [1, 3])
@pytest.mark.parametrize("name,form,coarse_form,level", [
    ("cube16", "tr", None, 0), ("cube16", "sym", None, 0), ("boxes16", "tr", None, 0),
    ("layer16", "tr", "sym", 0), ("layer16", "tr", "sym", 1), ("columns16", "grad", None, 0),
    ("mixed48", "tr", "sym", 1), ("mixed48", "tr", "sym", 2), ("mixed48", "tr", None, 2)])
@pytest.mark.parametrize("cluster", [False, True])
def test_fp32_uzawa_steps_match_oracle(sdx, name, form, coarse_form, level, steps, cluster, monkeypatch):
    """`steps` FP32 Uzawa steps through the launches of the FP32 V-cycle: one launch per pass,
    or (cluster=True: SDX_CLUSTER_MAX_NODES=10000 when the hierarchy is created) all steps of a
    level of at most 10000 nodes in one thread-block cluster (one launch, checked with the
    launch counter).  Against the oracle's FP64 steps at 1e-5."""
    p, L = _oracle_level(name, form, level, coarse_form)
    for k in ("SDX_NO_COOP", "SDX_COOP_MAX_NODES", "SDX_CLUSTER_MAX_NODES"):
        monkeypatch.delenv(k, raising=False)
    if cluster:
        monkeypatch.setenv("SDX_CLUSTER_MAX_NODES", "10000")
    H = sdx.Hierarchy.from_problem(p, form=form, coarse_form=coarse_form, prec=1)
    x, b = _state(L, 80 + level, np.float32)
    xd, bd = _dev(x, torch.float32), _dev(b, torch.float32)
    torch.cuda.synchronize()
    before = sdx.sdx_kernel_launches()
    H.sdx_uzawa_f32(level, bd, xd, steps)
    launches = sdx.sdx_kernel_launches() - before
    for _ in range(steps):
        L.uzawa(x, b)
    err = _relmax(_host(xd), x)
    assert err <= STEPS_TOL, (name, form, level, steps, err)
    if cluster and L.nn <= 10000:
        assert launches == 1  # the single-cluster path
    else:
        assert launches >= 5 * steps


def test_full_size_smoother_passes_sampled_rows(sdx):
    """The benchmark's passes at the benchmark's size (128^3 three boxes, mu ratio 1e4, decoupled
    form, FP64): one red velocity pass and one red pressure pass from a random state, checked at
    sampled nodes (interface rows, rows next to the walls, uniform interior rows, both colours)
    against the oracle's locally assembled rows (oracle.forms.sampled_rows): a red node takes
    u + (f - A u - B^T p) / diag(A) on its free components and p + omega (B u - C p - g) /
    diag(C) respectively, with the diagonals probed by unit vectors; black nodes keep their values
    to the bit.  1e-13 of the largest sampled value."""
    from oracle.forms import sampled_rows
    p = W.three_boxes(128, 8, contrast=1e4)
    n = p.n
    n1 = n + 1
    nn = n1 ** 3
    cm = p.cell_mu().ravel()
    H = sdx.Hierarchy.from_problem(p, form="tr", coarse_form="sym", prec=sdx.PREC_FP64)
    con = H.sdx_constraint_mask(0)
    iface = np.flatnonzero(H.sdx_interface_mask(0))
    rng = np.random.Generator(np.random.PCG64(93))
    x = W.random_vector(n, 91).ravel()
    b = W.random_vector(n, 92).ravel()
    x[con] = 0.0
    b[con] = 0.0
    picks = [(1, 1, 1), (2, 1, 1), (64, 64, 64), (65, 64, 64), (127, 126, 127), (126, 127, 127), (1, 77, 33)]
    nodes = [i + n1 * (j + n1 * k) for i, j, k in picks]
    nodes += list(rng.choice(iface, 8, replace=False)) + list(rng.integers(0, nn, 6))
    nodes = np.array(sorted(set(int(v) for v in nodes)))
    ijk = np.stack([nodes % n1, (nodes // n1) % n1, nodes // (n1 * n1)])
    red = (ijk.sum(axis=0) % 2) == 0
    assert red.any() and (~red).any() and np.isin(iface, nodes).any()
    rows = sampled_rows(n, cm, p.face, "tr", x, nodes)  # [4, len(nodes)]: A u + B^T p ; B u - C p
    diagA = np.zeros((3, len(nodes)))
    diagC = np.zeros(len(nodes))
    for t, v in enumerate(nodes):
        for c in range(4):
            e = np.zeros(4 * nn)
            if c < 3 and con[c * nn + v]:
                continue
            e[c * nn + v] = 1.0
            r = sampled_rows(n, cm, p.face, "tr", e, np.array([v]))[:, 0]
            if c < 3:
                diagA[c, t] = r[c]
            else:
                diagC[t] = -r[3]
    # velocity pass, colour 0
    xd = _dev(x)
    H.sdx_smooth_pass(0, 0, 0, _dev(b), xd)
    xg = _host(xd)
    for t, v in enumerate(nodes):
        for c in range(3):
            old = x[c * nn + v]
            got = xg[c * nn + v]
            if not red[t] or con[c * nn + v]:
                assert got == old, (v, c)
            else:
                want = old + (b[c * nn + v] - rows[c, t]) / diagA[c, t]
                assert abs(got - want) <= 1e-13 * max(1.0, abs(want)), (v, c, got, want)
    # pressure pass, colour 0, from the same state
    xd = _dev(x)
    H.sdx_smooth_pass(0, 1, 0, _dev(b), xd)
    xg = _host(xd)
    for t, v in enumerate(nodes):
        old = x[3 * nn + v]
        got = xg[3 * nn + v]
        if not red[t]:
            assert got == old, v
        else:
            want = old + OMEGA * (rows[3, t] - b[3 * nn + v]) / diagC[t]
            assert abs(got - want) <= 1e-13 * max(1.0, abs(want)), (v, got, want)
