"""GPU parity of the batched driver (sdx_batch_*): many independent problems of uneven sizes,
depths, viscosity layouts and boundary faces.  sdx_batch_solve runs every instance's FGMRES in
one persistent launch over a device work queue (default) or, with SDX_BATCH_LOCKSTEP=1, one
launch per phase with the instances' Krylov steps in lock step; both are tested.

* One batched V-cycle equals, instance by instance, the single-hierarchy sdx_vcycle (FP64:
  to 1e-14 relative, i.e. roundoff of the same arithmetic; FP32 cycles: 1e-5, since the
  FP32 input scaling uses a norm summed in another order), and the oracle's cycle from the
  same start (FP64 1e-10, FP32 1e-4).
* Batched FGMRES solves match the oracle's direct solutions to 1e-8 relative L2 (the solve
  tolerance of this work), each instance converging on its own schedule.
* At the benchmark's sizes ({32,48,64,96}^3, contrasts up to 1e6, FP32 cycles) every
  instance's final residual, recomputed by the single-hierarchy sdx_residual, meets 1e-8.
"""
import numpy as np
import pytest

from tests._lib import ensure_built

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle.forms import Discretisation  # noqa: E402
from oracle.solvers import Hierarchy as OracleHierarchy  # noqa: E402
from paper_1604_07994_gb300 import workloads as W  # noqa: E402

SOLVE_TOL = 1e-8


@pytest.fixture(scope="module")
def sdx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ensure_built()
    from paper_1604_07994_gb300 import sdx as mod
    return mod


def _small_batch():
    """Uneven sizes and depths (1 to 3 levels), all face types, up to three viscosities."""
    rng = np.random.Generator(np.random.PCG64(5))
    ids = rng.integers(0, 3, (3, 3, 3)).astype(np.uint8)
    ids = np.repeat(np.repeat(np.repeat(ids, 4, 0), 4, 1), 4, 2)
    mixed = W.Problem(n=12, n_coarse=3, cell_id=ids, mu=np.array([1.0, 30.0, 0.05]),
                      face=(0, 1, 2, 1, 0, 2), forcing=W.gaussian_blobs(5), name="mixed_12")
    tiny = W.Problem(n=2, n_coarse=2, cell_id=np.array([[[0, 1], [1, 0]], [[1, 1], [0, 0]]], dtype=np.uint8),
                     mu=np.array([1.0, 7.0]), face=(2, 0, 1, 2, 0, 1), forcing=W.gaussian_blobs(1), name="tiny2")
    # contrasts up to 1e4: with 1e6 the direct solution itself is only good to ~1e-7 relative
    return [W.cube_inclusion(16, 4), W.random_instance(8, 2, 3, 2, log10_contrast=(0, 4)), mixed,
            W.top_layer(16, 8), W.random_instance(16, 4, 7, 4, log10_contrast=(0, 4)), tiny,
            W.viscosity_columns(8, 4)]


def _rhs(p):
    d = Discretisation(p.n, p.cell_mu().ravel(), p.face)
    return d.rhs(p.nodal_forcing()), d


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def _host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def _project(x, d):
    w = d.pressure_weights()
    x = x.copy()
    x[3 * d.nn:] -= np.dot(w, x[3 * d.nn:]) / w.sum()
    return x


@pytest.mark.parametrize("form,coarse_form,prec", [("tr", None, 0), ("sym", None, 0), ("tr", "sym", 0),
                                                   ("grad", None, 0), ("tr", None, 1), ("tr", "sym", 1)])
def test_batch_vcycle_matches_single_vcycles(sdx, form, coarse_form, prec):
    probs = _small_batch()
    B = sdx.Batch(probs, form=form, coarse_form=coarse_form, prec=prec, autotune=True)
    bs, xs_b, xs_s, hs = [], [], [], []
    for k, p in enumerate(probs):
        b, _ = _rhs(p)
        H = sdx.Hierarchy.from_problem(p, form=form, coarse_form=coarse_form, prec=prec)
        con = H.sdx_constraint_mask(0)
        x0 = W.random_vector(p.n, 40 + k).ravel() * 1e-3
        x0[con] = 0.0
        bs.append(_dev(b))
        xs_b.append(_dev(x0))
        xs_s.append(_dev(x0))
        hs.append(H)
    # the oracle's cycle from the same start: 1e-10 for FP64 cycles (as the single-hierarchy
    # V-cycle tests); 1e-4 for FP32 cycles: FP32 rounding (u = 6e-8) of the scaled residual and of
    # every pass and transfer, amplified by the viscosity contrast (1e3 to 1e4 in this batch;
    # measured up to 2.4e-5 on the top-layer instance), while a wrong coefficient or index shows
    # at 1e-3 or more
    ohs = [OracleHierarchy(p.n, p.n_coarse, p.cell_mu().ravel(), p.face, form, coarse_form=coarse_form)
           for p in probs]
    xo = [_host(x).copy() for x in xs_b]
    bo = [_host(b) for b in bs]
    for _ in range(2):  # the second cycle checks that no level keeps state from the first
        B.sdx_batch_vcycle(bs, xs_b)
        for H, b, x in zip(hs, bs, xs_s):
            H.sdx_vcycle(b, x)
        for k in range(len(probs)):
            ohs[k].vcycle(xo[k], bo[k])
            xb, xs = _host(xs_b[k]), _host(xs_s[k])
            err = np.linalg.norm(xb - xs) / np.linalg.norm(xs)
            assert err <= (1e-14 if prec == 0 else 1e-5), (probs[k].name, err)
            err_o = np.linalg.norm(xb - xo[k]) / np.linalg.norm(xo[k])
            assert err_o <= (1e-10 if prec == 0 else 1e-4), (probs[k].name, "oracle", err_o)


@pytest.fixture(params=["queue", "lockstep"])
def solver(request, monkeypatch):
    """The batch solver under test (read by sdx_batch_solve at every call)."""
    if request.param == "lockstep":
        monkeypatch.setenv("SDX_BATCH_LOCKSTEP", "1")
    else:
        monkeypatch.delenv("SDX_BATCH_LOCKSTEP", raising=False)
    return request.param


@pytest.mark.parametrize("form,coarse_form,prec", [("tr", None, 0), ("tr", None, 1), ("tr", "sym", 1), ("sym", None, 1),
                                                   ("grad", "sym", 0)])
def test_batch_solve_matches_direct_solutions(sdx, form, coarse_form, prec, solver):
    probs = _small_batch()
    B = sdx.Batch(probs, form=form, coarse_form=coarse_form, prec=prec)
    bs, xs, refs = [], [], []
    for p in probs:
        b, d = _rhs(p)
        OH = OracleHierarchy(p.n, p.n_coarse, p.cell_mu().ravel(), p.face, form)
        L = OH.levels[0]
        xo = L.direct(b)
        refs.append((xo, d, L.nullspace))
        bs.append(_dev(b))
        xs.append(_dev(np.zeros_like(b)))
    stats = B.sdx_batch_solve(bs, xs, rtol=1e-12, maxit=300, restart=30)
    its = set()
    for k, (st, (xo, d, ns)) in enumerate(zip(stats, refs)):
        assert st["status"] == 0 and st["res"] <= 1e-12 * st["bnorm"], (probs[k].name, st)
        x = _host(xs[k])
        if ns:
            x = _project(x, d)
        assert np.linalg.norm(x - xo) <= SOLVE_TOL * np.linalg.norm(xo), probs[k].name
        its.add(st["iterations"])
    assert len(its) > 1  # instances converged on their own schedules inside one batch


def test_batch_edge_cases(sdx, solver):
    """A zero right-hand side converges at once (x stays 0) while the others iterate, and a
    one-instance batch gives the same bits as the same instance inside a larger batch."""
    probs = [W.cube_inclusion(8, 4), W.random_instance(12, 3, 9, 3, log10_contrast=(0, 4))]
    B = sdx.Batch(probs, prec=1)
    b0, _ = _rhs(probs[0])
    b1, _ = _rhs(probs[1])
    bs = [_dev(np.zeros_like(b0)), _dev(b1)]
    xs = [_dev(np.zeros_like(b0)), _dev(np.zeros_like(b1))]
    st = B.sdx_batch_solve(bs, xs, rtol=1e-10, maxit=100)
    assert st[0]["iterations"] == 0 and np.all(_host(xs[0]) == 0.0)
    assert st[1]["iterations"] > 0 and st[1]["res"] <= 1e-10 * st[1]["bnorm"]
    one = sdx.Batch(probs[1:], prec=1, autotune=False)
    x1 = _dev(np.zeros_like(b1))
    st1 = one.sdx_batch_solve([bs[1]], [x1], rtol=1e-10, maxit=100)
    assert st1[0]["iterations"] == st[1]["iterations"]
    assert np.array_equal(_host(x1), _host(xs[1]))  # instances do not influence each other
    # a batch-owned hierarchy serves queries and the operator, not the solver calls
    H = B.instance(1)
    r = torch.empty_like(bs[1])
    H.sdx_residual(0, bs[1], xs[1], r)
    assert float(torch.linalg.norm(r)) <= 1e-10 * float(torch.linalg.norm(bs[1]))
    with pytest.raises(sdx.SdxError) as e:
        H.sdx_vcycle(bs[1], xs[1])
    assert e.value.code == sdx.EINVAL


def test_batch_benchmark_sizes_reach_tolerance(sdx, solver):
    """Instances of the benchmark family ({32,48,64,96}^3 cells, 1-4 boxes, contrast
    log-uniform in [1, 1e6], FP32 cycles in FP64 refinement): every instance's residual,
    recomputed in FP64 by the single-hierarchy sdx_residual, meets 1e-8."""
    sizes = [32, 48, 64, 96, 48, 32]
    probs = [W.random_instance(n, n // 8, 100 + k, n // 8, forcing="blobs") for k, n in enumerate(sizes)]
    B = sdx.Batch(probs, prec=1, coarse_form="sym")
    bs, xs = [], []
    for p in probs:
        H = sdx.Hierarchy.from_problem(p)
        f = _dev(p.nodal_forcing().ravel())
        b = torch.zeros(4 * p.nodes, dtype=torch.float64, device="cuda")
        H.sdx_rhs(f, b)
        bs.append(b)
        xs.append(torch.zeros_like(b))
        H.close()
    stats = B.sdx_batch_solve(bs, xs, rtol=1e-8, maxit=300, restart=30)
    for p, b, x, st in zip(probs, bs, xs, stats):
        H = sdx.Hierarchy.from_problem(p)
        r = torch.empty_like(b)
        H.sdx_residual(0, b, x, r)
        rel = float(torch.linalg.norm(r) / torch.linalg.norm(b))
        assert st["status"] == 0 and rel <= SOLVE_TOL, (p.name, rel, st)
        H.close()


def test_batch_statuses_are_per_instance(sdx, solver):
    """A NaN in one instance's right-hand side marks that instance SDX_ENONFINITE (and the call
    returns it) while the other instance still converges in the same batch."""
    probs = [W.cube_inclusion(8, 4), W.random_instance(12, 3, 9, 3, log10_contrast=(0, 4))]
    B = sdx.Batch(probs, prec=1, autotune=False)
    b0, d0 = _rhs(probs[0])
    b1, _ = _rhs(probs[1])
    b0[np.flatnonzero(~d0.constrained())[5]] = np.inf
    bs = [_dev(b0), _dev(b1)]
    xs = [_dev(np.zeros_like(b0)), _dev(np.zeros_like(b1))]
    st = B.sdx_batch_solve(bs, xs, rtol=1e-10, maxit=100, allow_codes=(sdx.ENONFINITE,))
    assert st[0]["status"] == sdx.ENONFINITE
    assert st[1]["status"] == 0 and st[1]["res"] <= 1e-10 * st[1]["bnorm"]


def test_destroy_refuses_a_batch_owned_hierarchy(sdx):
    """sdx_destroy on an instance handle of a batch returns SDX_EINVAL instead of freeing what
    the batch still owns; the batch and its instance stay usable."""
    probs = [W.cube_inclusion(8, 4)]
    B = sdx.Batch(probs, prec=1, autotune=False)
    H = B.instance(0)
    assert sdx.load().sdx_destroy(H._h) == sdx.EINVAL
    assert "batch" in sdx.load().sdx_last_error().decode()
    b, _ = _rhs(probs[0])
    x = _dev(np.zeros_like(b))
    st = B.sdx_batch_solve([_dev(b)], [x], rtol=1e-8, maxit=100)
    assert st[0]["res"] <= 1e-8 * st[0]["bnorm"]
    B.close()


def test_queue_solver_is_deterministic_and_matches_lockstep_iterations(sdx, monkeypatch):
    """The persistent solver gives the same bits on a repeated call (which CTA runs which tile
    does not change any sum), and each instance needs the same number of FGMRES iterations as
    in the lock-step solver (same preconditioner; the Gram-Schmidt arithmetic differs only in
    rounding), give or take one."""
    probs = _small_batch()
    B = sdx.Batch(probs, form="tr", coarse_form="sym", prec=1)
    bs = [_dev(_rhs(p)[0]) for p in probs]
    runs = []
    for env in ("0", "0", "1"):
        monkeypatch.setenv("SDX_BATCH_LOCKSTEP", env)
        xs = [torch.zeros_like(b) for b in bs]
        st = B.sdx_batch_solve(bs, xs, rtol=1e-10, maxit=300, restart=30)
        runs.append(([_host(x) for x in xs], [s["iterations"] for s in st]))
    for a, b in zip(runs[0][0], runs[1][0]):
        assert np.array_equal(a, b)
    assert runs[0][1] == runs[1][1]
    for iq, il in zip(runs[0][1], runs[2][1]):
        assert abs(iq - il) <= 1


def test_queue_solver_stall_times_out_and_batch_recovers(sdx, monkeypatch):
    """A test hook (SDX_TEST_QUEUE_STALL) clears every instance's work word after
    initialisation, so no CTA of the persistent launch ever finds a tile: each waits without
    progress until its bounded wait (about 4e9 clock cycles) ends, the solve returns
    SDX_ETIMEOUT, and the next solve on the same batch converges."""
    monkeypatch.delenv("SDX_BATCH_LOCKSTEP", raising=False)
    probs = _small_batch()[:3]
    B = sdx.Batch(probs, form="tr", coarse_form="sym", prec=0)
    bs = [_dev(_rhs(p)[0]) for p in probs]
    xs = [torch.zeros_like(b) for b in bs]
    monkeypatch.setenv("SDX_TEST_QUEUE_STALL", "1")
    with pytest.raises(sdx.SdxError) as e:
        B.sdx_batch_solve(bs, xs, rtol=1e-8, maxit=100, restart=30)
    assert e.value.code == sdx.ETIMEOUT
    monkeypatch.delenv("SDX_TEST_QUEUE_STALL")
    xs = [torch.zeros_like(b) for b in bs]
    st = B.sdx_batch_solve(bs, xs, rtol=1e-8, maxit=100, restart=30)
    for s in st:
        assert s["res"] <= 1e-8 * s["bnorm"]
    B.close()
