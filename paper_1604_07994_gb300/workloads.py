"""Seeded synthetic problem definitions shared by the CUDA path's tests and the oracle.

This module describes *problems*, never the method: viscosity layouts (cell ids and a
viscosity table), boundary-face types, forcing functions evaluated at grid nodes, exact
manufactured solutions and random test vectors.  It contains no finite-element, stencil or
multigrid arithmetic, so both sides of every parity check can draw their inputs from it
without sharing any of the computation they are compared on.

Geometry conventions (paper Sec. 4.2.2: unit cube, 4^3 base cubes split into 6 tetrahedra and
refined uniformly): the finest grid has N^3 hexahedral cells, h = 1/N, and (N+1)^3 nodes.
Node (i, j, k) sits at h*(i, j, k) and has flat index i + (N+1)*(j + (N+1)*k); cell (i, j, k)
spans [ih,(i+1)h]x[jh,(j+1)h]x[kh,(k+1)h] and has flat index i + N*(j + N*k).  Numpy arrays
are shaped [k, j, i] (x fastest).

Face order everywhere: -x, +x, -y, +y, -z, +z.  Face types: 0 Dirichlet (no-slip), 1
free-slip, 2 traction-free (paper Sec. 1, eq. (boundary)).
"""
from __future__ import annotations

import dataclasses
from typing import Callable, List, Optional, Sequence, Tuple

import numpy as np

DIRICHLET, FREESLIP, TRACTION = 0, 1, 2


@dataclasses.dataclass
class Problem:
    """One Stokes interface problem on the unit cube.

    n          : cells per side on the finest grid (n = n_coarse * 2**k)
    n_coarse   : cells per side on the coarsest multigrid level; every viscosity interface
                 lies on a plane of that grid
    cell_id    : uint8 array [n, n, n] ([k, j, i]) of subdomain ids
    mu         : float64 viscosity table indexed by cell id, all > 0
    face       : six face types (-x, +x, -y, +y, -z, +z)
    forcing    : callable (x, y, z) -> (fx, fy, fz) evaluated on node coordinates
    exact      : optional callable (x, y, z, cell_mu_at_point) -> (ux, uy, uz, p)
    """

    n: int
    n_coarse: int
    cell_id: np.ndarray
    mu: np.ndarray
    face: Tuple[int, int, int, int, int, int]
    forcing: Callable
    exact: Optional[Callable] = None
    name: str = ""

    @property
    def nodes(self) -> int:
        return (self.n + 1) ** 3

    def cell_mu(self) -> np.ndarray:
        return self.mu[self.cell_id]

    def nodal_forcing(self) -> np.ndarray:
        """Forcing f evaluated at every node, shape (3, (n+1)^3), x-fastest."""
        x, y, z = node_coords(self.n)
        fx, fy, fz = self.forcing(x, y, z)
        out = np.empty((3, self.nodes))
        out[0] = np.broadcast_to(fx, x.shape).ravel()
        out[1] = np.broadcast_to(fy, x.shape).ravel()
        out[2] = np.broadcast_to(fz, x.shape).ravel()
        return out


def node_coords(n: int):
    """Node coordinates as three [n+1, n+1, n+1] arrays (index [k, j, i])."""
    t = np.arange(n + 1, dtype=np.float64) / n
    z, y, x = np.meshgrid(t, t, t, indexing="ij")
    return x, y, z


def box_cell_ids(n: int, boxes: Sequence[Tuple[Tuple[float, float], ...]]) -> np.ndarray:
    """Cell ids: 1 inside the union of axis-aligned boxes ((x0,x1),(y0,y1),(z0,z1)), else 0.

    A cell belongs to a box when its centre does."""
    c = (np.arange(n, dtype=np.float64) + 0.5) / n
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    ids = np.zeros((n, n, n), dtype=np.uint8)
    for (x0, x1), (y0, y1), (z0, z1) in boxes:
        inside = (x > x0) & (x < x1) & (y > y0) & (y < y1) & (z > z0) & (z < z1)
        ids[inside] = 1
    return ids


def box_planes(boxes) -> List[List[float]]:
    """Distinct interior interface planes per axis spanned by the faces of the boxes."""
    planes: List[List[float]] = [[], [], []]
    for b in boxes:
        for ax in range(3):
            for c in b[ax]:
                if 0.0 < c < 1.0 and all(abs(c - o) > 1e-12 for o in planes[ax]):
                    planes[ax].append(float(c))
    return [sorted(p) for p in planes]


class Manufactured:
    """Piecewise manufactured solution satisfying the interface jump conditions.

    q(x) = prod_k qk(x_k),  qk(t) = [t(1-t)]^2 * prod_{c in planes_k} (t - c)^3, scaled to
    max|q| ~ 1.  With Phi = cvec * q, the velocity is u = curl(Phi) / mu (piecewise), which is
    solenoidal in every subdomain, zero on the boundary, and zero together with its gradient on
    every interface plane (cubic zero), so [u] = 0 and [sigma n] = 0 there (paper Sec. 1, eq.
    stokes-strong-interface).  The pressure is a seeded quadratic.  Because mu is constant in
    each subdomain, the forcing f = -Laplace(curl Phi) + grad p is one global polynomial.
    """

    def __init__(self, planes: Sequence[Sequence[float]], seed: int):
        P = np.polynomial.Polynomial
        rng = np.random.Generator(np.random.PCG64(seed))
        self.cvec = rng.standard_normal(3)
        # p = a0 + a.x + x^T S x (S symmetric), drawn once
        self.pa0 = rng.standard_normal()
        self.pa = rng.standard_normal(3)
        s = rng.standard_normal((3, 3))
        self.pS = 0.5 * (s + s.T)
        self.q = []
        for ax in range(3):
            poly = P([0.0, 1.0, -1.0]) ** 2  # [t(1-t)]^2
            for c in planes[ax]:
                poly = poly * P([-c, 1.0]) ** 3
            self.q.append(poly)
        # normalise max|q| on a fine sample
        t = np.linspace(0.0, 1.0, 2001)
        scale = 1.0
        for ax in range(3):
            scale *= np.max(np.abs(self.q[ax](t)))
        self.scale = scale if scale > 0 else 1.0
        self.dq = [[self.q[ax].deriv(m) if m else self.q[ax] for m in range(4)] for ax in range(3)]

    def _qd(self, x, y, z, mx, my, mz):
        X = (x, y, z)
        m = (mx, my, mz)
        out = 1.0 / self.scale
        for ax in range(3):
            out = out * self.dq[ax][m[ax]](X[ax])
        return out

    def grad_q(self, x, y, z):
        return (self._qd(x, y, z, 1, 0, 0), self._qd(x, y, z, 0, 1, 0), self._qd(x, y, z, 0, 0, 1))

    def grad_lap_q(self, x, y, z):
        # d/dx_i (q_xx + q_yy + q_zz)
        out = []
        for i in range(3):
            tot = 0.0
            for l in range(3):
                m = [0, 0, 0]
                m[l] += 2
                m[i] += 1
                tot = tot + self._qd(x, y, z, *m)
            out.append(tot)
        return tuple(out)

    def pressure(self, x, y, z):
        X = (x, y, z)
        p = self.pa0 + sum(self.pa[i] * X[i] for i in range(3))
        for i in range(3):
            for j in range(3):
                p = p + self.pS[i, j] * X[i] * X[j]
        return p

    def grad_p(self, x, y, z):
        X = (x, y, z)
        return tuple(self.pa[i] + 2.0 * sum(self.pS[i, j] * X[j] for j in range(3)) for i in range(3))

    @staticmethod
    def _cross(a, c):
        return (a[1] * c[2] - a[2] * c[1], a[2] * c[0] - a[0] * c[2], a[0] * c[1] - a[1] * c[0])

    def curl_phi(self, x, y, z):
        return self._cross(self.grad_q(x, y, z), self.cvec)

    def forcing(self, x, y, z):
        lap_curl = self._cross(self.grad_lap_q(x, y, z), self.cvec)
        gp = self.grad_p(x, y, z)
        return tuple(-lap_curl[i] + gp[i] for i in range(3))

    def exact(self, x, y, z, mu_at):
        cp = self.curl_phi(x, y, z)
        return (cp[0] / mu_at, cp[1] / mu_at, cp[2] / mu_at, self.pressure(x, y, z))


def gaussian_blobs(seed: int, count: int = 8):
    """Buoyancy-like forcing f = (0, 0, -sum_k A_k exp(-|x-c_k|^2 / (2 s_k^2)))."""
    rng = np.random.Generator(np.random.PCG64(seed))
    A = rng.uniform(-1.0, 1.0, count)
    C = rng.uniform(0.1, 0.9, (count, 3))
    S = rng.uniform(0.03, 0.1, count)

    def f(x, y, z):
        fz = 0.0
        for k in range(count):
            r2 = (x - C[k, 0]) ** 2 + (y - C[k, 1]) ** 2 + (z - C[k, 2]) ** 2
            fz = fz - A[k] * np.exp(-r2 / (2.0 * S[k] ** 2))
        zero = np.zeros_like(np.asarray(x, dtype=np.float64))
        return (zero, zero, zero + fz)

    return f


def random_boxes(rng: np.random.Generator, count: int, lattice: int):
    """`count` boxes with corners on the 1/lattice grid, lo < hi on every axis."""
    boxes = []
    for _ in range(count):
        b = []
        for _ax in range(3):
            lo, hi = sorted(rng.choice(np.arange(lattice + 1), size=2, replace=False))
            b.append((lo / lattice, hi / lattice))
        boxes.append(tuple(b))
    return boxes


def inclusion_problem(n: int, n_coarse: int, boxes, mu_in: float, mu_out: float, seed: int,
                      face=(DIRICHLET,) * 6, name="") -> Problem:
    """Box inclusions (id 1, viscosity mu_in) in a matrix (id 0, mu_out), manufactured forcing."""
    ids = box_cell_ids(n, boxes)
    man = Manufactured(box_planes(boxes), seed)
    return Problem(n=n, n_coarse=n_coarse, cell_id=ids, mu=np.array([mu_out, mu_in]),
                   face=tuple(face), forcing=man.forcing, exact=man.exact, name=name)


def cube_inclusion(n: int = 16, n_coarse: int = 4, seed: int = 0) -> Problem:
    """16^3 cells, inclusion [0.25,0.75]^3 with mu=10 in a mu=1 matrix, no-slip walls."""
    boxes = [((0.25, 0.75),) * 3]
    return inclusion_problem(n, n_coarse, boxes, 10.0, 1.0, seed, name=f"cube_inclusion_{n}")


def three_boxes(n: int = 128, n_coarse: int = 8, seed: int = 1, contrast: float = 1e4) -> Problem:
    """Three seeded boxes on the 1/8 lattice (union: mu = contrast), mu = 1 elsewhere."""
    rng = np.random.Generator(np.random.PCG64(seed))
    boxes = random_boxes(rng, 3, 8)
    return inclusion_problem(n, n_coarse, boxes, contrast, 1.0, seed, name=f"three_boxes_{n}")


def top_layer(n: int = 256, n_coarse: int = 8, seed: int = 3, mu_top: float = 1e3) -> Problem:
    """Layer z >= 7/8 with mu = mu_top over mu = 1; traction-free top, free-slip sides,
    no-slip bottom; seeded Gaussian-blob buoyancy forcing."""
    c = (np.arange(n, dtype=np.float64) + 0.5) / n
    z = np.broadcast_to(c[:, None, None], (n, n, n))
    ids = (z > 7.0 / 8.0).astype(np.uint8)
    face = (FREESLIP, FREESLIP, FREESLIP, FREESLIP, DIRICHLET, TRACTION)
    return Problem(n=n, n_coarse=n_coarse, cell_id=np.ascontiguousarray(ids), mu=np.array([1.0, mu_top]),
                   face=face, forcing=gaussian_blobs(seed), name=f"top_layer_{n}")


def viscosity_columns(n: int, n_coarse: int = 4) -> Problem:
    """Paper Sec. 4.2.4 'viscosity columns': mu = 10 in (0,1/4)^2x(0,1) and (3/4,1)^2x(0,1),
    mu = 1 elsewhere; free-slip on every face; f = (0, 0, -cos(2 pi x) cos(2 pi y) sin(pi z))."""
    c = (np.arange(n, dtype=np.float64) + 0.5) / n
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    col = ((x < 0.25) & (y < 0.25)) | ((x > 0.75) & (y > 0.75))
    ids = col.astype(np.uint8)

    def f(x, y, z):
        zero = np.zeros_like(np.asarray(x, dtype=np.float64))
        return (zero, zero, -np.cos(2 * np.pi * x) * np.cos(2 * np.pi * y) * np.sin(np.pi * z))

    return Problem(n=n, n_coarse=n_coarse, cell_id=ids, mu=np.array([1.0, 10.0]),
                   face=(FREESLIP,) * 6, forcing=f, name=f"columns_{n}")


def viscosity_layers(n: int, n_coarse: int = 4) -> Problem:
    """Paper Sec. 4.2.3 'viscosity layers': four layers (0,1)^2 x (i/4,(i+1)/4) with
    mu_i = 10^i, free-slip on every face, same forcing as the columns problem."""
    c = (np.arange(n, dtype=np.float64) + 0.5) / n
    z = np.broadcast_to(c[:, None, None], (n, n, n))
    ids = np.minimum((z * 4).astype(np.int64), 3).astype(np.uint8)
    base = viscosity_columns(n, n_coarse)
    return Problem(n=n, n_coarse=n_coarse, cell_id=np.ascontiguousarray(ids),
                   mu=np.array([1.0, 10.0, 100.0, 1000.0]), face=(FREESLIP,) * 6,
                   forcing=base.forcing, name=f"layers_{n}")


def level_set_cell_ids(n: int, phi: Callable) -> np.ndarray:
    """Cell ids of a level-set interface that the grid does not resolve: 1 where the level-set
    function phi(x, y, z) is negative at the cell centre, else 0 ([n, n, n], [k, j, i])."""
    c = (np.arange(n, dtype=np.float64) + 0.5) / n
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    return (np.asarray(phi(x, y, z)) < 0.0).astype(np.uint8)


def level_set_sphere(n: int = 32, n_coarse: int = 4, seed: int = 6, mu_in: float = 1e3,
                     mu_out: float = 1.0) -> Problem:
    """A stiff sphere whose surface cuts the cells (phi = |x - c| - r, c and r seeded, the
    sphere inside the cube): not aligned with any grid plane, so the coarser grids do not
    resolve it.  No-slip walls, Gaussian-blob forcing."""
    rng = np.random.Generator(np.random.PCG64(seed))
    centre = rng.uniform(0.4, 0.6, 3)
    radius = rng.uniform(0.17, 0.27)
    ids = level_set_cell_ids(n, lambda x, y, z: np.sqrt((x - centre[0]) ** 2 + (y - centre[1]) ** 2
                                                         + (z - centre[2]) ** 2) - radius)
    return Problem(n=n, n_coarse=n_coarse, cell_id=ids, mu=np.array([mu_out, mu_in]),
                   face=(DIRICHLET,) * 6, forcing=gaussian_blobs(seed), name=f"sphere_{n}")


def random_vector(n: int, seed: int, dtype=np.float64) -> np.ndarray:
    """A seeded random SoA vector [4, (n+1)^3] (u_x, u_y, u_z, p), entries ~ U[-1, 1]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.uniform(-1.0, 1.0, (4, (n + 1) ** 3)).astype(dtype)


def random_instance(n: int, n_coarse: int, seed: int, lattice: int, max_boxes: int = 4,
                    log10_contrast=(0.0, 6.0), forcing: str = "manufactured") -> Problem:
    """One instance of a batched/training family: 1..max_boxes boxes on the 1/lattice grid,
    inclusion viscosity 10^U[log10_contrast], matrix viscosity 1, no-slip walls."""
    rng = np.random.Generator(np.random.PCG64(seed))
    count = int(rng.integers(1, max_boxes + 1))
    boxes = random_boxes(rng, count, lattice)
    contrast = float(10.0 ** rng.uniform(*log10_contrast))
    if forcing == "manufactured":
        return inclusion_problem(n, n_coarse, boxes, contrast, 1.0, seed, name=f"instance_{seed}_{n}")
    ids = box_cell_ids(n, boxes)
    return Problem(n=n, n_coarse=n_coarse, cell_id=ids, mu=np.array([1.0, contrast]),
                   face=(DIRICHLET,) * 6, forcing=gaussian_blobs(seed), name=f"instance_{seed}_{n}")


def batched_instances(count: int = 48, seed: int = 2024, sizes=(32, 48, 64, 96)) -> List[Problem]:
    """The batched workload: `count` independent instances, grid size drawn uniformly from
    `sizes` (cells per side), coarsest grid n/8 (so every instance has four levels), 1-4
    seeded boxes on that coarsest lattice, contrast log-uniform in [1, 1e6], no-slip walls,
    Gaussian-blob forcing."""
    rng = np.random.Generator(np.random.PCG64(seed))
    ns = rng.choice(np.asarray(sizes), size=count)
    return [random_instance(int(n), int(n) // 8, seed * 1000 + k, int(n) // 8, forcing="blobs")
            for k, n in enumerate(ns)]
