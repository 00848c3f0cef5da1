"""Global sparse assembly of the P1-P1 PSPG-stabilised Stokes system on a Kuhn mesh.

Degrees of freedom are numbered component-major ("SoA"): index c*nn + node for component
c in (u_x, u_y, u_z, p), nn = (n+1)^3 nodes, node index x-fastest.

Paper passages followed here:

* a_sym(u,v) = (2 mu sym grad u, sym grad v)               Sec. 1, eq. (standard)
* a_tr(u,v)  = a_sym(u,v) - (mu div u, div v)                Sec. 2, eq. (newbil)
* a_dev(u,v) = (2 mu dev sym grad u, dev sym grad v)         Sec. 2, below eq. (newbil)
* gradient form (mu grad u, grad v)                         Sec. 4.1 / 4.2.3 (inconsistent)
* b(v,q) = -(div v, q)                                       Sec. 1, below eq. (weakma)
* saddle matrix [[A, B^T], [B, -C]]                          Sec. 5, first display
* C: PSPG / Brezzi-Pitkaranta pressure stabilisation. The paper states only that the
  equal-order P1-P1 scheme is stabilised (Sec. 4 intro, Sec. 5); we read it as
  C = sum_T tau_T (grad p, grad q)_T with tau_T = beta h^2 / mu_T (h the cube edge), the 1/mu
  scaling mirroring the 1/(2 mu_i) weight of eq. (stabc).  The paper does not print beta;
  beta = 1/24 is the value at which the decoupled cycle's rate is independent of depth, as the
  Sec. 5 table of rates reports (about 0.24 at every level; with 1/12 it grows with depth).  Its consistent
  right-hand side is g_q = -sum_T tau_T (f, grad q)_T.
* boundary conditions: Dirichlet (all components), free-slip (normal component), traction
  (natural) - Sec. 1, eq. (boundary)
* interface rows: test functions that are not in H^1_0 of one isoviscous subdomain, i.e. nodes
  on Gamma_12 or on a traction face - Sec. 2.2, eq. (equivalence-stencil)

Test infrastructure: only tests/, the entry module's smoke check and the benchmark's CPU legs
import it; it shares no code with the CUDA library.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .mesh import kuhn_tets, node_xyz, p1_geometry

FORMS = ("tr", "sym", "grad", "dev")
DIRICHLET, FREESLIP, TRACTION = 0, 1, 2
PSPG_BETA = 1.0 / 24.0


def _sym_basis(grad):
    """sym grad of the vector basis function lambda_a e_i: E[T, a, i] is a 3x3 tensor.

    grad(lambda_a e_i) has entries (e_i)_k (d_l lambda_a) at (k, l)."""
    nT = grad.shape[0]
    G = np.zeros((nT, 4, 3, 3, 3))  # [T, a, i, k, l]
    for i in range(3):
        G[:, :, i, i, :] = grad
    return 0.5 * (G + np.swapaxes(G, 3, 4)), G


class Discretisation:
    """All matrices of one grid level (unconstrained), plus constraint and interface sets.

    n      : cells per side; h = 1/n
    cell_mu: float64 [n^3] viscosity per hexahedral cell (flat index i + n*(j + n*k))
    face   : six face types (-x, +x, -y, +y, -z, +z)
    beta   : PSPG constant
    """

    def __init__(self, n: int, cell_mu: np.ndarray, face, beta: float = PSPG_BETA):
        self.n = n
        self.nn = (n + 1) ** 3
        self.h = 1.0 / n
        self.cell_mu = np.asarray(cell_mu, dtype=np.float64).ravel()
        assert self.cell_mu.size == n ** 3 and np.all(self.cell_mu > 0)
        self.face = tuple(int(f) for f in face)
        self.beta = beta
        self.xyz = node_xyz(n)
        self.tets, self.tet_cell = kuhn_tets(n)
        self.grad, self.vol = p1_geometry(self.xyz, self.tets)
        self.mu_T = self.cell_mu[self.tet_cell]
        self.tau_T = beta * self.h ** 2 / self.mu_T
        self._cache = {}

    # ------------------------------------------------------------------ element matrices
    def _assemble(self, vals, rows, cols, shape):
        return sp.coo_matrix((vals.ravel(), (rows.ravel(), cols.ravel())), shape=shape).tocsr()

    def velocity_block(self, form: str) -> sp.csr_matrix:
        """A for the chosen bilinear form, unconstrained, [3nn, 3nn], rows = test (b, j).

        Entries are integrals of products of constant element gradients, i.e. |T| times the
        integrand, written straight from the tensor definitions of the forms."""
        assert form in FORMS
        if form in self._cache:
            return self._cache[form]
        nn = self.nn
        E, G = _sym_basis(self.grad)
        w = self.mu_T * self.vol
        if form == "sym":
            # (2 mu sym grad u, sym grad v): u = lambda_a e_i (column), v = lambda_b e_j (row)
            ent = 2.0 * np.einsum("t,taikl,tbjkl->tbjai", w, E, E)
        elif form == "tr":
            div = self.grad  # div(lambda_a e_i) = d_i lambda_a
            ent = 2.0 * np.einsum("t,taikl,tbjkl->tbjai", w, E, E) - np.einsum(
                "t,tai,tbj->tbjai", w, div, div)
        elif form == "grad":
            ent = np.einsum("t,taikl,tbjkl->tbjai", w, G, G)
        else:  # dev
            D = E.copy()
            tr = np.einsum("taikk->tai", E) / 3.0
            for k in range(3):
                D[:, :, :, k, k] -= tr
            ent = 2.0 * np.einsum("t,taikl,tbjkl->tbjai", w, D, D)
        nT = self.tets.shape[0]
        node = self.tets
        comp = np.arange(3)
        rows = comp[None, None, :, None, None] * nn + node[:, :, None, None, None]
        cols = comp[None, None, None, None, :] * nn + node[:, None, None, :, None]
        rows = np.broadcast_to(rows, (nT, 4, 3, 4, 3))
        cols = np.broadcast_to(cols, (nT, 4, 3, 4, 3))
        A = self._assemble(ent, rows, cols, (3 * nn, 3 * nn))
        self._cache[form] = A
        return A

    def divergence(self) -> sp.csr_matrix:
        """B [nn, 3nn]: B[b, (a,i)] = b(lambda_a e_i, lambda_b) = -sum_T d_i lambda_a |T|/4."""
        nn = self.nn
        nT = self.tets.shape[0]
        ent = -np.einsum("t,tai->tai", self.vol / 4.0, self.grad)  # independent of b
        ent = np.broadcast_to(ent[:, None, :, :], (nT, 4, 4, 3))  # [T, b, a, i]
        rows = np.broadcast_to(self.tets[:, :, None, None], (nT, 4, 4, 3))
        cols = np.arange(3)[None, None, None, :] * nn + self.tets[:, None, :, None]
        cols = np.broadcast_to(cols, (nT, 4, 4, 3))
        return self._assemble(ent, rows, cols, (nn, 3 * nn))

    def stabilisation(self) -> sp.csr_matrix:
        """C [nn, nn] = sum_T tau_T |T| grad lambda_a . grad lambda_b."""
        ent = np.einsum("t,tad,tbd->tba", self.tau_T * self.vol, self.grad, self.grad)
        nT = self.tets.shape[0]
        rows = np.broadcast_to(self.tets[:, :, None], (nT, 4, 4))
        cols = np.broadcast_to(self.tets[:, None, :], (nT, 4, 4))
        return self._assemble(ent, rows, cols, (self.nn, self.nn))

    def lumped_mass(self) -> np.ndarray:
        """Row sums of the P1 mass matrix: m_b = sum_{T ni b} |T| / 4."""
        m = np.zeros(self.nn)
        np.add.at(m, self.tets.ravel(), np.repeat(self.vol / 4.0, 4))
        return m

    def mass_matrix(self, weight_T: np.ndarray = None) -> sp.csr_matrix:
        """Consistent P1 mass matrix [nn, nn]: M[b, a] = sum_T w_T int_T lambda_a lambda_b
        = sum_T w_T |T| (1 + delta_ab) / 20, with w_T = 1 unless a per-tetrahedron weight is
        given."""
        w = self.vol if weight_T is None else self.vol * np.asarray(weight_T, dtype=np.float64)
        nT = self.tets.shape[0]
        loc = (np.ones((4, 4)) + np.eye(4)) / 20.0
        ent = w[:, None, None] * loc[None, :, :]
        rows = np.broadcast_to(self.tets[:, :, None], (nT, 4, 4))
        cols = np.broadcast_to(self.tets[:, None, :], (nT, 4, 4))
        return self._assemble(ent, rows, cols, (self.nn, self.nn))

    def paper_norms(self, x: np.ndarray) -> np.ndarray:
        """The three norms of a discrete pair (u, p) (SoA [4nn]) used in the error tables of
        Sec. 4.2: ||u||_0 (L2 of the P1 velocity field), ||u||_V with ||v||_V^2 = a_sym(v, v)
        and ||p||_Q with ||q||_Q^2 = (q / (2 mu), q)_0, the norms defined in Sec. 3 before
        Lemma 3.  Returns [||u||_0, ||u||_V, ||p||_Q]."""
        nn = self.nn
        x = np.asarray(x, dtype=np.float64).ravel()
        u = x[: 3 * nn]
        p = x[3 * nn:]
        M = self.mass_matrix()
        l2 = np.sqrt(sum(u[c * nn:(c + 1) * nn] @ (M @ u[c * nn:(c + 1) * nn]) for c in range(3)))
        en = np.sqrt(u @ (self.velocity_block("sym") @ u))
        q = np.sqrt(p @ (self.mass_matrix(1.0 / (2.0 * self.mu_T)) @ p))
        return np.array([l2, en, q])

    def divergence_weights(self) -> np.ndarray:
        """D_b = mu_b / m_b with m_b the lumped mass and mu_b m_b = sum_{T ni b} mu_T |T| / 4, so
        that (B u)^T diag(D) (B v) is the mass-lumped (mu div u, div v): with b(v, q) = -(div v, q)
        (Sec. 1), (B u)_b = -int div(u) lambda_b ~ -m_b (div u)_b.  Used by the coarse-grid
        right-hand-side correction of Sec. 5 (A_tr ~ A_sym - B^T diag(D) B)."""
        mum = np.zeros(self.nn)
        np.add.at(mum, self.tets.ravel(), np.repeat(self.mu_T * self.vol / 4.0, 4))
        m = self.lumped_mass()
        return mum / (m * m)

    def pressure_weights(self) -> np.ndarray:
        """w_b = int lambda_b / mu = sum_{T ni b} |T| / (4 mu_T): the discrete form of the
        constraint int mu^{-1} q = 0 that fixes the pressure constant (Sec. 1, space Q)."""
        w = np.zeros(self.nn)
        np.add.at(w, self.tets.ravel(), np.repeat(self.vol / (4.0 * self.mu_T), 4))
        return w

    def saddle(self, form: str) -> sp.csr_matrix:
        """K = [[A, B^T], [B, -C]] unconstrained, [4nn, 4nn] (Sec. 5)."""
        A = self.velocity_block(form)
        B = self.divergence()
        C = self.stabilisation()
        return sp.bmat([[A, B.T], [B, -C]], format="csr")

    # ------------------------------------------------------------------ boundary data
    def node_ijk(self):
        n1 = self.n + 1
        idx = np.arange(self.nn)
        return idx % n1, (idx // n1) % n1, idx // (n1 * n1)

    def constrained(self) -> np.ndarray:
        """Boolean [4nn]: True for velocity components fixed to zero by the boundary
        conditions.  Dirichlet faces fix all components, free-slip faces the normal one;
        a node on several faces takes the union.  Pressure is never constrained."""
        i, j, k = self.node_ijk()
        on = [i == 0, i == self.n, j == 0, j == self.n, k == 0, k == self.n]
        mask = np.zeros((4, self.nn), dtype=bool)
        for f in range(6):
            axis = f // 2
            if self.face[f] == DIRICHLET:
                mask[:3, on[f]] = True
            elif self.face[f] == FREESLIP:
                mask[axis, on[f]] = True
        return mask.ravel()

    def has_pressure_nullspace(self) -> bool:
        """Without a traction face the constant pressure is in the kernel of [B^T; -C]."""
        return TRACTION not in self.face

    def interface_nodes(self) -> np.ndarray:
        """Boolean [nn]: nodes whose velocity test functions are not in H^1_0 of one
        isoviscous subdomain - nodes touching cells of two or more viscosities, or lying on a
        traction face - restricted to nodes with at least one free velocity component."""
        n = self.n
        mu = self.cell_mu.reshape(n, n, n)  # [k, j, i]
        lo = np.full((n + 1,) * 3, np.inf)
        hi = np.full((n + 1,) * 3, -np.inf)
        for dk in (0, 1):
            for dj in (0, 1):
                for di in (0, 1):
                    sl = (slice(dk, dk + n), slice(dj, dj + n), slice(di, di + n))
                    lo[sl] = np.minimum(lo[sl], mu)
                    hi[sl] = np.maximum(hi[sl], mu)
        iface = (hi > lo).ravel()
        i, j, k = self.node_ijk()
        on = [i == 0, i == n, j == 0, j == n, k == 0, k == n]
        for f in range(6):
            if self.face[f] == TRACTION:
                iface |= on[f]
        free = ~self.constrained().reshape(4, self.nn)[:3].all(axis=0)
        return iface & free

    def rhs(self, f_nodal: np.ndarray = None, f_cell: np.ndarray = None) -> np.ndarray:
        """Right-hand side [4nn] for a forcing given either at the nodes (f_nodal [3, nn])
        or as a constant per hexahedral cell (f_cell [3, n^3]).

        Nodal forcing: velocity rows are the lumped mass times the nodal value; the pressure
        rows take the PSPG term g_b = -sum_T tau_T int_T f_h . grad lambda_b with f_h the P1
        interpolant (exact integral: |T| times the vertex mean).  Cell forcing: velocity rows
        are the exact integrals sum_T f_T |T| / 4 and g_b = -sum_T tau_T |T| f_T . grad
        lambda_b.  Constrained rows are zero."""
        b = np.zeros((4, self.nn))
        if f_nodal is not None:
            f = np.asarray(f_nodal, dtype=np.float64).reshape(3, self.nn)
            b[:3] = self.lumped_mass()[None, :] * f
            fT = f[:, self.tets].mean(axis=2).T  # [T, 3]
        else:
            fc = np.asarray(f_cell, dtype=np.float64).reshape(3, -1)
            fT = fc[:, self.tet_cell].T
            for c in range(3):
                np.add.at(b[c], self.tets.ravel(), np.repeat(fT[:, c] * self.vol / 4.0, 4))
        contrib = -np.einsum("t,td,tbd->tb", self.tau_T * self.vol, fT, self.grad)
        np.add.at(b[3], self.tets.ravel(), contrib.ravel())
        b = b.ravel()
        b[self.constrained()] = 0.0
        return b


def sampled_rows(n, cell_mu, face, form, x, nodes, beta: float = PSPG_BETA):
    """(K x) at selected nodes only, for grids too large to assemble: the rows of the given
    nodes are summed over the tetrahedra of their patches with the same element integrals as
    the global assembly (generic P1 geometry), the constrained rows set to zero.

    cell_mu: [n^3] cell viscosities; x: [4 (n+1)^3] SoA vector (zero at constrained DoFs);
    nodes: node indices.  Returns [4, len(nodes)]."""
    n1 = n + 1
    nn = n1 ** 3
    cell_mu = np.asarray(cell_mu, dtype=np.float64).ravel()
    x = np.asarray(x, dtype=np.float64).reshape(4, nn)
    xyz_all = None
    out = np.zeros((4, len(nodes)))
    from .mesh import PERMS
    h = 1.0 / n
    for t, b in enumerate(nodes):
        bi, bj, bk = b % n1, (b // n1) % n1, b // (n1 * n1)
        tets, cells = [], []
        for dk in (-1, 0):
            for dj in (-1, 0):
                for di in (-1, 0):
                    ci, cj, ck = bi + di, bj + dj, bk + dk
                    if min(ci, cj, ck) < 0 or max(ci, cj, ck) >= n:
                        continue
                    for s in PERMS:
                        off = [0, 0, 0]
                        verts = [ci + n1 * (cj + n1 * ck)]
                        for ax in s:
                            off[ax] += 1
                            verts.append(ci + off[0] + n1 * (cj + off[1] + n1 * (ck + off[2])))
                        if b in verts:
                            tets.append(verts)
                            cells.append(ci + n * (cj + n * ck))
        tets = np.array(tets)
        cells = np.array(cells)
        ijk = np.stack([tets % n1, (tets // n1) % n1, tets // (n1 * n1)], axis=2)
        xyz = ijk * h
        M = np.concatenate([np.ones(xyz.shape[:2] + (1,)), xyz], axis=2)
        C = np.linalg.inv(M)
        grad = np.transpose(C[:, 1:, :], (0, 2, 1))
        vol = np.abs(np.linalg.det(M)) / 6.0
        mu_T = cell_mu[cells]
        tau_T = beta * h ** 2 / mu_T
        loc = np.array([list(tv).index(b) for tv in tets])  # b's vertex in each tet
        gb = grad[np.arange(len(tets)), loc]  # [T, 3]
        E, G = _sym_basis(grad)
        Eb = E[np.arange(len(tets)), loc]  # [T, j, k, l]
        Gb = G[np.arange(len(tets)), loc]
        U = x[:3][:, tets]  # [i, T, a]
        Pv = x[3][tets]  # [T, a]
        w = mu_T * vol
        # sym grad u_h and grad u_h per tet
        Gu = np.einsum("iTa,Tad->Tid", U, grad)  # d_d u_i
        Eu = 0.5 * (Gu + np.transpose(Gu, (0, 2, 1)))
        divu = np.einsum("Tii->T", Gu)
        if form == "sym":
            au = 2.0 * np.einsum("T,Tkl,Tjkl->j", w, Eu, Eb)
        elif form == "tr":
            au = 2.0 * np.einsum("T,Tkl,Tjkl->j", w, Eu, Eb) - np.einsum("T,T,Tj->j", w, divu, gb)
        elif form == "grad":
            au = np.einsum("T,Tkl,Tjkl->j", w, Gu, Gb)
        else:
            raise ValueError(form)
        btp = -np.einsum("T,Tj,T->j", vol / 4.0, gb, Pv.sum(axis=1))
        bu = -np.sum(vol / 4.0 * divu)
        gp = np.einsum("Ta,Tad->Td", Pv, grad)
        cp = np.sum(tau_T * vol * np.einsum("Td,Td->T", gp, gb))
        out[:3, t] = au + btp
        out[3, t] = bu - cp
    # constrained rows
    d = _BoundaryOnly(n, face)
    con = d.constrained_nodes(np.asarray(nodes))
    out[:3][con] = 0.0
    return out


class _BoundaryOnly:
    """Constraint flags of selected nodes without building the mesh (same rule as
    Discretisation.constrained)."""

    def __init__(self, n, face):
        self.n, self.face = n, tuple(int(f) for f in face)

    def constrained_nodes(self, nodes):
        n1 = self.n + 1
        i, j, k = nodes % n1, (nodes // n1) % n1, nodes // (n1 * n1)
        on = [i == 0, i == self.n, j == 0, j == self.n, k == 0, k == self.n]
        mask = np.zeros((3, nodes.size), dtype=bool)
        for f in range(6):
            if self.face[f] == DIRICHLET:
                mask[:, on[f]] = True
            elif self.face[f] == FREESLIP:
                mask[f // 2, on[f]] = True
        return mask


def masked(K: sp.spmatrix, constrained: np.ndarray) -> sp.csr_matrix:
    """D K D with D the diagonal 0/1 matrix of free DoFs: rows and columns of constrained
    DoFs set to zero, so K x on vectors that are zero at constrained DoFs gives the free
    rows of K_ff x_f and zeros elsewhere."""
    d = sp.diags((~constrained).astype(np.float64))
    return (d @ K @ d).tocsr()
