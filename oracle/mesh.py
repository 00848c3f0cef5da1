"""Kuhn (Freudenthal) tetrahedral mesh of the unit cube and generic P1 element geometry.

Paper Sec. 4.2.3 builds the coarsest mesh from 4^3 cubes, each subdivided into six
tetrahedra, and refines it uniformly (Bey's refinement, remark in Sec. 3.2).  The split of a
cube is not stated; we use the Kuhn split along the (1,1,1) diagonal: for every permutation
s of the axes, the tetrahedron with vertices c, c+e_s1, c+e_s1+e_s2, c+(1,1,1).  Its uniform
refinement is again a Kuhn mesh, so the P1 spaces of consecutive levels are nested.

The element geometry here is computed generically (inverse of the 4x4 vertex matrix), not
from the Kuhn shape, so that the oracle does not rely on any hand-derived stencil.

Test infrastructure: only tests/, the entry module's smoke check and the benchmark's CPU legs
import it; it shares no code with the CUDA library.
"""
from __future__ import annotations

import itertools

import numpy as np

PERMS = list(itertools.permutations(range(3)))


def node_index(n: int, i, j, k):
    return i + (n + 1) * (j + (n + 1) * k)


def kuhn_tets(n: int):
    """All 6 n^3 tetrahedra.

    Returns (tets, cell): tets is int64 [6 n^3, 4] of node indices, cell is int64 [6 n^3]
    of the flat index of the hexahedral cell that contains each tetrahedron.
    """
    ci, cj, ck = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    ci, cj, ck = ci.ravel(), cj.ravel(), ck.ravel()
    cell = ci + n * (cj + n * ck)
    tets = []
    cells = []
    for s in PERMS:
        verts = []
        off = np.zeros(3, dtype=np.int64)
        verts.append(node_index(n, ci, cj, ck))
        for ax in s:
            off[ax] += 1
            verts.append(node_index(n, ci + off[0], cj + off[1], ck + off[2]))
        tets.append(np.stack(verts, axis=1))
        cells.append(cell)
    return np.concatenate(tets, axis=0), np.concatenate(cells, axis=0)


def node_xyz(n: int) -> np.ndarray:
    """Coordinates [(n+1)^3, 3] of the nodes, x fastest."""
    t = np.arange(n + 1, dtype=np.float64) / n
    k, j, i = np.meshgrid(t, t, t, indexing="ij")
    return np.stack([i.ravel(), j.ravel(), k.ravel()], axis=1)


def p1_geometry(xyz: np.ndarray, tets: np.ndarray):
    """Barycentric gradients and volumes of P1 tetrahedra.

    With M_T = [[1, x_a]]_{a=0..3} (rows), the barycentric coordinates are the columns of
    M_T^{-1}: lambda_a(x) = C[0,a] + C[1:,a].x.  Returns grad [nT, 4, 3] (grad[T, a] =
    grad lambda_a) and vol [nT] = |det M_T| / 6.
    """
    X = xyz[tets]  # [nT, 4, 3]
    M = np.concatenate([np.ones(X.shape[:2] + (1,)), X], axis=2)  # [nT, 4, 4]
    C = np.linalg.inv(M)
    grad = np.transpose(C[:, 1:, :], (0, 2, 1))  # [nT, a, d]
    vol = np.abs(np.linalg.det(M)) / 6.0
    return grad, vol
