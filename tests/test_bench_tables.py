"""The benchmark's error-table norms (torch, device-independent) against the oracle's, on CPU
tensors (no GPU): the consistent-mass L2 norm, the a_sym energy norm, the 1/(2 mu)-weighted
pressure norm (Sec. 3) and the pressure normalisation weights."""
import numpy as np
import torch

import bench
from oracle.forms import Discretisation, masked
from oracle.solvers import Level
from paper_1604_07994_gb300 import workloads as W


def _setup(n):
    p = W.viscosity_columns(n, 4)
    d = Discretisation(n, p.cell_mu().ravel(), p.face)
    Ks = masked(d.saddle("sym"), d.constrained())
    cell_mu = torch.from_numpy(np.ascontiguousarray(p.cell_mu(), dtype=np.float64))
    return p, d, Ks, cell_mu, (lambda v: torch.from_numpy(Ks @ v.numpy()))


def test_kuhn_offsets_cover_each_cube_with_six_tetrahedra():
    offs = bench._kuhn_vertex_offsets()
    assert len(offs) == 6 and len({tuple(v) for v in offs}) == 6
    for v in offs:
        assert v[0] == (0, 0, 0) and v[3] == (1, 1, 1)
        # consecutive vertices differ by one unit step along one axis
        for a, b in zip(v[:-1], v[1:]):
            assert sorted(np.subtract(b, a).tolist()) == [0, 0, 1]


def test_table_norms_match_the_oracle():
    n = 8
    p, d, Ks, cell_mu, apply_sym = _setup(n)
    for seed in (3, 4):
        x = W.random_vector(n, seed).ravel()
        x[d.constrained()] = 0.0
        got = bench.table_norms(torch, torch.from_numpy(x.copy()), n, cell_mu, apply_sym)
        ref = d.paper_norms(x)
        assert np.all(np.abs(got / ref - 1.0) <= 1e-12), (got, ref)


def test_pressure_weights_match_the_oracle():
    n = 8
    p, d, Ks, cell_mu, _ = _setup(n)
    w = bench.pressure_weights_t(torch, n, cell_mu).numpy()
    assert np.abs(w - d.pressure_weights()).max() <= 1e-15 * 8 ** 3


def test_relative_differences_match_the_oracle():
    """Direct solutions of the three forms on the columns problem at 8^3: the benchmark's
    table entries equal the oracle's computation from the same solutions."""
    n = 8
    p, d, Ks, cell_mu, apply_sym = _setup(n)
    sols = {}
    for name, form in (("strain", "sym"), ("decoupled", "tr"), ("gradient", "grad")):
        L = Level(n, p.cell_mu().ravel(), p.face, form)
        x = L.direct(L.disc.rhs(p.nodal_forcing()))
        x[3 * d.nn:] += 0.37 * (1 + "sdg".index(name[0]))  # arbitrary pressure constants
        sols[name] = x
    got = bench.relative_differences(torch, {k: torch.from_numpy(v.copy()) for k, v in sols.items()},
                                     n, cell_mu, apply_sym)
    w = d.pressure_weights()
    for v in sols.values():
        v[3 * d.nn:] -= np.dot(w, v[3 * d.nn:]) / w.sum()
    U = sols["strain"]
    for k in ("decoupled", "gradient"):
        ref = d.paper_norms(sols[k] - U) / d.paper_norms(U)
        assert np.all(np.abs(np.array(got[k]) / ref - 1.0) <= 1e-10), (k, got[k], ref)


def test_vcycle_rate_helper_reproduces_the_oracle_rate():
    """bench.vcycle_rate (the GPU benchmark's rate measurement, torch) driven by the oracle's
    V-cycle gives the rate of the oracle's own measurement, and that rate is the paper's
    (within 10 %: decoupled form 0.241-0.244 in Table timeANDconv)."""
    from oracle.solvers import Hierarchy
    from test_oracle_solvers import PAPER_RHO, _asymptotic_rate
    n = 16
    p = W.viscosity_columns(n, 4)
    H = Hierarchy(n, 4, p.cell_mu().ravel(), p.face, "tr")
    L = H.levels[0]
    rho_ref, _ = _asymptotic_rate(H)
    x = W.random_vector(n, 77).ravel()
    x[L.con] = 0.0
    xt = torch.from_numpy(x)
    zero = np.zeros_like(x)
    cell_mu = torch.from_numpy(np.ascontiguousarray(p.cell_mu(), dtype=np.float64))
    w = bench.pressure_weights_t(torch, n, cell_mu)

    def vcycle(v):
        v.copy_(torch.from_numpy(H.vcycle(v.numpy().copy(), zero)))

    def residual(v):
        return torch.from_numpy(L.residual(v.numpy(), zero))

    rho, rates = bench.vcycle_rate(torch, vcycle, residual, xt, L.nn, w, cycles=25, last=8)
    assert abs(rho - rho_ref) <= 1e-10 * rho_ref, (rho, rho_ref)
    lo, hi = PAPER_RHO["tr"]
    assert 0.9 * lo <= rho <= 1.1 * hi
