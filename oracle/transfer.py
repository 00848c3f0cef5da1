"""Nested P1 prolongation between uniformly refined Kuhn meshes.

Paper Sec. 5 takes the standard restriction and prolongation operators.  For nested conforming
P1 spaces the standard prolongation is the natural embedding: a coarse P1 function is also a
fine P1 function, so its fine nodal values are its point values.  Every fine node is either a
coarse node or the midpoint of a coarse edge, where a linear function takes the mean of the
two end values.  Restriction is the transpose.

Test infrastructure: only tests/, the entry module's smoke check and the benchmark's CPU legs
import it; it shares no code with the CUDA library.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .mesh import kuhn_tets, node_xyz


def prolongation(n_coarse: int) -> sp.csr_matrix:
    """Scalar P [(2nc+1)^3, (nc+1)^3] from the coarse grid with n_coarse cells per side.

    Built from the coarse tetrahedra: each coarse vertex injects into the fine node at the
    same point, each coarse edge's midpoint takes 1/2 from both ends."""
    nc = n_coarse
    nf = 2 * nc
    tets, _ = kuhn_tets(nc)
    xc = node_xyz(nc)

    def fine_index(pt):
        ijk = np.rint(pt * nf).astype(np.int64)
        return ijk[..., 0] + (nf + 1) * (ijk[..., 1] + (nf + 1) * ijk[..., 2])

    # vertices
    va = np.arange(xc.shape[0])
    vrows = fine_index(xc)
    # edges of the coarse tetrahedra (deduplicated); each midpoint lies on exactly one edge
    pairs = np.concatenate([tets[:, [p, q]] for p in range(4) for q in range(p + 1, 4)])
    edges = np.unique(np.sort(pairs, axis=1), axis=0)
    erows = fine_index(0.5 * (xc[edges[:, 0]] + xc[edges[:, 1]]))
    rows = np.concatenate([vrows, erows, erows])
    cols = np.concatenate([va, edges[:, 0], edges[:, 1]])
    vals = np.concatenate([np.ones(va.size), np.full(2 * erows.size, 0.5)])
    P = sp.coo_matrix((vals, (rows, cols)), shape=((nf + 1) ** 3, (nc + 1) ** 3)).tocsr()
    assert P.nnz == rows.size, "a fine node was reached twice"
    return P


def system_prolongation(n_coarse: int, constrained_f: np.ndarray, constrained_c: np.ndarray):
    """P for the four-component SoA vector (u_x, u_y, u_z, p) with constrained DoFs of both
    levels removed (rows and columns zeroed)."""
    P = prolongation(n_coarse)
    P4 = sp.block_diag([P, P, P, P], format="csr")
    df = sp.diags((~constrained_f).astype(np.float64))
    dc = sp.diags((~constrained_c).astype(np.float64))
    return (df @ P4 @ dc).tocsr()
