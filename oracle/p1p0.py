"""P1-P0 discretisation with interior-penalty pressure stabilisation and the local flux
post-process (test infrastructure: only tests/, the entry's smoke check and the benchmark's CPU
leg use it).

Paper passages followed:

* spaces: P1 velocity, P0 pressure (one value per tetrahedron)      Sec. 3.1 (stab-p1p0)
* saddle problem a(u, v) + b(v, p) = f(v), b(u, q) - c(p, q) = 0     Sec. 3.1, eq. (weakdis)
  with b(v, q) = -(div v, q)                                        Sec. 1
* c(p, q) = gamma sum_i 1/(2 mu_i) sum_{F in F_h(Omega_i)}
  |T1||T2| / (|T1| + |T2|) [p]_F [q]_F                              Sec. 3.2, eq. (stabc)
  over the interior facets of each isoviscous subdomain (facets on the interface or the domain
  boundary excluded), gamma = 1 (Sec. 4.2, "Interface problems")
* facet flux j_{F;T} = u_h . n_T + Delta j_{F;T},
  Delta j_{F;T} = gamma / (2 mu |F|) |T||T^F| / (|T| + |T^F|) (p_T - p_{T^F})
  on the facets of F_h(Omega_i); the fluxes of every element sum to zero   Sec. 3.2 (remark
  after eq. stabc)

The velocity block, constraints and load vector are those of oracle.forms (same mesh, same
forms a_tr / a_sym / gradient).  Pressure unknowns are numbered by tetrahedron in the order of
oracle.mesh.kuhn_tets.  Norms and errors are integrated with a collapsed-coordinate Gauss rule
that is exact for polynomials of degree 5 on every tetrahedron.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .forms import DIRICHLET, TRACTION, Discretisation, masked
from .solvers import DENSE_LIMIT

GAMMA = 1.0

# faces of a tetrahedron: the three vertices opposite vertex a
_FACE_VERTS = np.array([[1, 2, 3], [0, 2, 3], [0, 1, 3], [0, 1, 2]])


def _collapsed_gauss(q: int = 4):
    """Points (barycentric-free, reference tetrahedron x, y, z >= 0, x + y + z <= 1) and weights
    summing to 1/6 of a rule exact for degree 2q - 3: x = a, y = (1 - a) b, z = (1 - a)(1 - b) c
    with Gauss-Legendre nodes in a, b, c and the Jacobian (1 - a)^2 (1 - b)."""
    g, w = np.polynomial.legendre.leggauss(q)
    g = 0.5 * (g + 1.0)
    w = 0.5 * w
    A, Bb, Cc = np.meshgrid(g, g, g, indexing="ij")
    WA, WB, WC = np.meshgrid(w, w, w, indexing="ij")
    x = A
    y = (1.0 - A) * Bb
    z = (1.0 - A) * (1.0 - Bb) * Cc
    wt = WA * WB * WC * (1.0 - A) ** 2 * (1.0 - Bb)
    return np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1), wt.ravel()


class P1P0:
    """All matrices of one grid level of the P1-P0 scheme (unconstrained), its facets and the
    flux post-process."""

    def __init__(self, n: int, cell_mu: np.ndarray, face, gamma: float = GAMMA):
        self.disc = Discretisation(n, cell_mu, face)
        d = self.disc
        self.n, self.nn, self.gamma = n, d.nn, gamma
        self.nT = d.tets.shape[0]
        self.mu_T = d.mu_T
        self.vol = d.vol
        self._facets()

    # ------------------------------------------------------------------ facets
    def _facets(self):
        """Interior facets (pairs of tetrahedra sharing three vertices), their area and the
        unit normal pointing out of the first tetrahedron."""
        d = self.disc
        fv = np.sort(d.tets[:, _FACE_VERTS], axis=2).reshape(-1, 3)  # [4 nT, 3]
        owner = np.repeat(np.arange(self.nT), 4)
        opp = np.tile(np.arange(4), self.nT)  # local index of the vertex opposite the face
        key = (fv[:, 0] * (d.nn + 1) + fv[:, 1]) * (d.nn + 1) + fv[:, 2]
        order = np.argsort(key, kind="stable")
        ks = key[order]
        same = np.flatnonzero(ks[1:] == ks[:-1])
        i1, i2 = order[same], order[same + 1]
        self.f_t1, self.f_t2 = owner[i1], owner[i2]
        X = d.xyz[fv[i1]]  # [nF, 3, 3]
        nrm = np.cross(X[:, 1] - X[:, 0], X[:, 2] - X[:, 0])
        area = 0.5 * np.linalg.norm(nrm, axis=1)
        nrm = nrm / (2.0 * area[:, None])
        # orient out of T1: away from T1's vertex opposite the face
        xo = d.xyz[d.tets[self.f_t1, opp[i1]]]
        flip = np.einsum("fd,fd->f", xo - X[:, 0], nrm) > 0
        nrm[flip] *= -1.0
        self.f_area, self.f_normal = area, nrm
        self.f_centroid = X.mean(axis=1)
        self.f_nodes = fv[i1]
        # facets of F_h(Omega_i): both sides in one isoviscous subdomain
        self.f_inner = self.mu_T[self.f_t1] == self.mu_T[self.f_t2]

    def penalty_weights(self) -> np.ndarray:
        """w_F = gamma / (2 mu_i) |T1||T2| / (|T1| + |T2|) on facets of F_h(Omega_i), else 0."""
        v1, v2 = self.vol[self.f_t1], self.vol[self.f_t2]
        w = self.gamma / (2.0 * self.mu_T[self.f_t1]) * v1 * v2 / (v1 + v2)
        return np.where(self.f_inner, w, 0.0)

    # ------------------------------------------------------------------ matrices
    def divergence(self) -> sp.csr_matrix:
        """B0 [nT, 3nn]: B0[T, (a, i)] = b(lambda_a e_i, 1_T) = -|T| d_i lambda_a."""
        d = self.disc
        ent = -self.vol[:, None, None] * d.grad  # [T, a, i]
        rows = np.broadcast_to(np.arange(self.nT)[:, None, None], ent.shape)
        cols = np.arange(3)[None, None, :] * d.nn + d.tets[:, :, None]
        cols = np.broadcast_to(cols, ent.shape)
        return sp.coo_matrix((ent.ravel(), (rows.ravel(), cols.ravel())), shape=(self.nT, 3 * d.nn)).tocsr()

    def stabilisation(self) -> sp.csr_matrix:
        """C0 [nT, nT] of eq. (stabc): sum over facets of w_F (e_T1 - e_T2)(e_T1 - e_T2)^T."""
        w = self.penalty_weights()
        t1, t2 = self.f_t1, self.f_t2
        rows = np.concatenate([t1, t2, t1, t2])
        cols = np.concatenate([t1, t2, t2, t1])
        vals = np.concatenate([w, w, -w, -w])
        return sp.coo_matrix((vals, (rows, cols)), shape=(self.nT, self.nT)).tocsr()

    def saddle(self, form: str) -> sp.csr_matrix:
        A = self.disc.velocity_block(form)
        B = self.divergence()
        return sp.bmat([[A, B.T], [B, -self.stabilisation()]], format="csr")

    def constrained(self) -> np.ndarray:
        """[3nn + nT]: constrained velocity components (pressures are never constrained)."""
        return np.concatenate([self.disc.constrained()[: 3 * self.nn], np.zeros(self.nT, dtype=bool)])

    def pressure_weights(self) -> np.ndarray:
        """w_T = |T| / mu_T: the constraint int q / mu = 0 of the pressure constant."""
        return self.vol / self.mu_T

    def rhs(self, f_nodal=None, f_cell=None) -> np.ndarray:
        """Velocity rows as in the P1-P1 scheme (lumped nodal or exact cell-wise load); the
        pressure rows are zero (the interior-penalty form needs no consistent load)."""
        b4 = self.disc.rhs(f_nodal=f_nodal, f_cell=f_cell)
        return np.concatenate([b4[: 3 * self.nn], np.zeros(self.nT)])

    # ------------------------------------------------------------------ direct solve
    def solve(self, b: np.ndarray, form: str = "tr", x_dirichlet: np.ndarray = None) -> np.ndarray:
        """Solve K x = b on the free DoFs (x = x_dirichlet on the constrained ones, default 0);
        with a pressure null space (no traction face) the result satisfies sum_T w_T p_T = 0."""
        con = self.constrained()
        K = self.saddle(form)
        xD = np.zeros(3 * self.nn + self.nT) if x_dirichlet is None else np.asarray(x_dirichlet, float).copy()
        xD[~con] = 0.0
        rhs = b - K @ xD
        free = np.flatnonzero(~con)
        Kff = K[free][:, free].tocsc()
        r = rhs[free]
        nullspace = TRACTION not in self.disc.face
        w = np.zeros(3 * self.nn + self.nT)
        w[3 * self.nn:] = self.pressure_weights()
        wf = w[free]
        if free.size <= DENSE_LIMIT:
            # bordered [[K_ff, w], [w^T, 0]]: also right for a right-hand side with a component
            # along the constant pressure (lifted boundary data of non-zero discrete net flux)
            M = Kff.toarray()
            rr = r
            if nullspace:
                M = np.block([[M, wf[:, None]], [wf[None, :], np.zeros((1, 1))]])
                rr = np.concatenate([r, [0.0]])
            sol = sla.solve(M, rr)[: free.size]
        elif nullspace:
            # the constant pressure spans the null space: pin the last pressure DoF, then shift
            # the pressures to w.p = 0 (the bordered system's solution for a consistent b)
            keep = np.ones(free.size, dtype=bool)
            keep[-1] = False
            sol = np.zeros(free.size)
            sol[keep] = spla.splu(sp.csc_matrix(Kff[keep][:, keep])).solve(r[keep])
            pm = free >= 3 * self.nn
            sol[pm] -= np.dot(wf[pm], sol[pm]) / wf[pm].sum()
        else:
            sol = spla.splu(Kff).solve(r)
        x = xD.copy()
        x[free] = sol
        return x

    # ------------------------------------------------------------------ flux post-process
    def facet_fluxes(self, x: np.ndarray):
        """Post-processed fluxes int_F j_{F;T} ds of every interior facet, oriented out of its
        first tetrahedron: |F| u_h(centroid) . n + w_F (p_T1 - p_T2).  Returns (fluxes [nF],
        boundary fluxes int_F u_h . n_T of every boundary facet as (tet, value) arrays)."""
        nn = self.nn
        u = np.asarray(x[: 3 * nn]).reshape(3, nn)
        p = np.asarray(x[3 * nn:])
        uc = u[:, self.f_nodes].mean(axis=2).T  # P1 field at the facet centroid
        flux = self.f_area * np.einsum("fd,fd->f", uc, self.f_normal)
        flux = flux + self.penalty_weights() * (p[self.f_t1] - p[self.f_t2])
        return flux

    def element_balance(self, x: np.ndarray) -> np.ndarray:
        """Sum over the facets of every tetrahedron of its outward post-processed fluxes
        (interior facets from facet_fluxes, boundary facets int_F u_h . n): zero for a solution
        of the discrete problem (local mass conservation)."""
        d = self.disc
        nn = self.nn
        u = np.asarray(x[: 3 * nn]).reshape(3, nn)
        bal = np.zeros(self.nT)
        fl = self.facet_fluxes(x)
        np.add.at(bal, self.f_t1, fl)
        np.add.at(bal, self.f_t2, -fl)
        # boundary facets: all faces of all tets minus the interior ones
        total_div = self.vol * np.einsum("tai,ita->t", d.grad, u[:, d.tets])  # |T| div u_h = sum of all face fluxes
        inner_u = self.f_area * np.einsum("fd,fd->f", u[:, self.f_nodes].mean(axis=2).T, self.f_normal)
        interior_u = np.zeros(self.nT)
        np.add.at(interior_u, self.f_t1, inner_u)
        np.add.at(interior_u, self.f_t2, -inner_u)
        return bal + (total_div - interior_u)

    # ------------------------------------------------------------------ norms
    def errors(self, x: np.ndarray, u_exact, p_exact, mu_at):
        """||u - u_h||_0, ||u - u_h||_V (V norm: a_sym energy, 2 mu |sym grad|^2) and
        ||p - p_h||_Q ((p/(2 mu), p)_0) by quadrature exact to degree 5 on each tetrahedron.
        u_exact(X) -> [3, P], grad_u_exact(X) through finite differences is avoided: u_exact
        must be a callable returning (u [3, P], grad u [3, 3, P]); p_exact(X) -> [P]; mu_at is
        the per-tetrahedron viscosity."""
        d = self.disc
        nn = self.nn
        pts, wts = _collapsed_gauss(4)
        X0 = d.xyz[d.tets[:, 0]]
        E = np.stack([d.xyz[d.tets[:, a]] - X0 for a in (1, 2, 3)], axis=2)  # [T, d, 3]
        lam = np.concatenate([1.0 - pts.sum(axis=1, keepdims=True), pts], axis=1)  # [Q, 4]
        uh = np.asarray(x[: 3 * nn]).reshape(3, nn)
        ph = np.asarray(x[3 * nn:])
        e0 = ev = ep = 0.0
        for q in range(pts.shape[0]):
            Xq = X0 + np.einsum("tdk,k->td", E, pts[q])
            ue, gue = u_exact(Xq.T)
            uq = np.einsum("ita,a->it", uh[:, d.tets], lam[q])
            gh = np.einsum("ita,tad->tid", uh[:, d.tets], d.grad)  # [T, i, d]
            w = wts[q] * 6.0 * self.vol
            e0 += np.sum(w * np.sum((ue - uq) ** 2, axis=0))
            G = np.transpose(gue, (2, 0, 1)) - gh  # [T, i, d]
            S = 0.5 * (G + np.transpose(G, (0, 2, 1)))
            ev += np.sum(w * 2.0 * mu_at * np.einsum("tij,tij->t", S, S))
            ep += np.sum(w * (p_exact(Xq.T) - ph) ** 2 / (2.0 * mu_at))
        return np.sqrt(e0), np.sqrt(ev), np.sqrt(ep)

    def norms(self, x: np.ndarray):
        """||u_h||_0 (consistent mass), ||u_h||_V (a_sym energy) and ||p_h||_Q for the relative
        differences of the paper's tables."""
        nn = self.nn
        u = np.asarray(x[: 3 * nn])
        p = np.asarray(x[3 * nn:])
        M = self.disc.mass_matrix()
        l2 = np.sqrt(sum(u[c * nn:(c + 1) * nn] @ (M @ u[c * nn:(c + 1) * nn]) for c in range(3)))
        en = np.sqrt(u @ (self.disc.velocity_block("sym") @ u))
        q = np.sqrt(np.sum(self.vol * p ** 2 / (2.0 * self.mu_T)))
        return np.array([l2, en, q])


def _cell_tets(n, ci, cj, ck):
    """The six Kuhn tetrahedra of cell (ci, cj, ck) as (oracle index, [4] node indices): the
    path c, c + e_s1, c + e_s1 + e_s2, c + (1, 1, 1) for each axis permutation s of PERMS; the
    index numbers tetrahedra permutation by permutation, cells i-major inside (kuhn_tets)."""
    from .mesh import PERMS
    n1 = n + 1
    out = []
    for si, s in enumerate(PERMS):
        off = [0, 0, 0]
        verts = [ci + n1 * (cj + n1 * ck)]
        for ax in s:
            off[ax] += 1
            verts.append(ci + off[0] + n1 * (cj + off[1] + n1 * (ck + off[2])))
        out.append((si * n ** 3 + (ci * n + cj) * n + ck, verts))
    return out


def _tet_geometry(n, verts):
    """Barycentric gradients [4, 3] and volume of the tetrahedron with these node indices."""
    n1 = n + 1
    v = np.asarray(verts)
    xyz = np.stack([v % n1, (v // n1) % n1, v // (n1 * n1)], axis=1) / n
    M = np.concatenate([np.ones((4, 1)), xyz], axis=1)
    return np.linalg.inv(M)[1:, :].T, abs(np.linalg.det(M)) / 6.0


def sampled_rows_p1p0(n, cell_mu, face, form, u, p, nodes, tets, gamma: float = GAMMA):
    """Rows of K x at selected velocity nodes and tetrahedra, for grids too large to assemble
    (the full-size parity test).  Velocity rows: A u from oracle.forms.sampled_rows plus the
    P0 gradient sum over the tetrahedra T around the node of -|T| grad lambda_b p_T; pressure
    rows: (B0 u)_T = -|T| div u_h on T minus (C0 p)_T = sum over the facets F of T shared with a
    tetrahedron T' of the same viscosity of gamma / (2 mu) |T||T'| / (|T| + |T'|) (p_T - p_T'),
    the facet neighbours found by shared vertices among the tetrahedra of the 27 cells around
    T's cell.  u: [3, (n+1)^3] (zero at constrained DoFs); p: [6 n^3] in the oracle's order;
    nodes: node indices; tets: (permutation index, ci, cj, ck) tuples.  Returns ([3, len(nodes)]
    velocity rows, constrained components zero; [len(tets)] pressure rows)."""
    from .forms import sampled_rows, _BoundaryOnly
    n1 = n + 1
    nn = n1 ** 3
    cell_mu = np.asarray(cell_mu, dtype=np.float64).ravel()
    mu_cell = lambda ci, cj, ck: cell_mu[ci + n * (cj + n * ck)]  # noqa: E731
    nodes = np.asarray(nodes)
    x4 = np.concatenate([np.asarray(u, dtype=np.float64).reshape(3, nn), np.zeros((1, nn))])
    vel = sampled_rows(n, cell_mu, face, form, x4.ravel(), nodes)[:3].copy()
    for t, b in enumerate(nodes):
        bi, bj, bk = b % n1, (b // n1) % n1, b // (n1 * n1)
        for ck in (bk - 1, bk):
            for cj in (bj - 1, bj):
                for ci in (bi - 1, bi):
                    if min(ci, cj, ck) < 0 or max(ci, cj, ck) >= n:
                        continue
                    for idx, verts in _cell_tets(n, ci, cj, ck):
                        if b not in verts:
                            continue
                        grad, vol = _tet_geometry(n, verts)
                        vel[:, t] += -vol * grad[verts.index(b)] * p[idx]
    vel[_BoundaryOnly(n, face).constrained_nodes(nodes)] = 0.0
    pre = np.zeros(len(tets))
    for t, (si, ci, cj, ck) in enumerate(tets):
        own = dict(_cell_tets(n, ci, cj, ck))
        idx = si * n ** 3 + (ci * n + cj) * n + ck
        verts = own[idx]
        grad, vol = _tet_geometry(n, verts)
        divu = sum(u[i][verts[a]] * grad[a, i] for a in range(4) for i in range(3))
        row = -vol * divu
        mu = mu_cell(ci, cj, ck)
        vs = set(verts)
        for dk in (-1, 0, 1):
            for dj in (-1, 0, 1):
                for di in (-1, 0, 1):
                    cc = (ci + di, cj + dj, ck + dk)
                    if min(cc) < 0 or max(cc) >= n:
                        continue
                    for idx2, v2 in _cell_tets(n, *cc):
                        if idx2 == idx or len(vs.intersection(v2)) != 3:
                            continue
                        if mu_cell(*cc) != mu:
                            continue  # a facet on the viscosity interface carries no penalty
                        _, vol2 = _tet_geometry(n, v2)
                        w = gamma / (2.0 * mu) * vol * vol2 / (vol + vol2)
                        row -= w * (p[idx] - p[idx2])
        pre[t] = row
    return vel, pre


def masked_p1p0(K: sp.spmatrix, con: np.ndarray) -> sp.csr_matrix:
    """The saddle matrix with constrained rows and columns replaced by identity rows."""
    return masked(K, con)


# ---------------------------------------------------------------------- multigrid
# The paper's solver (Sec. 5) is written for the P1-P1 scheme; for P1-P0 this oracle uses the
# same all-at-once Uzawa V_var cycle with two changes forced by the element pair: the pressure
# lives on tetrahedra, so its smoother is a relaxed Jacobi step on the Schur-complement
# approximation M_mu = diag(|T| / mu_T) (the 1/mu-weighted P0 mass; C alone is too weak: it
# vanishes on pressures constant across facets), and the pressure transfers are the natural
# embedding of the coarse P0 space into the fine one (every coarse tetrahedron is the union of
# eight fine ones) and its transpose.
OMEGA_P = 0.6


def tet_perm_index(n: int) -> np.ndarray:
    """Permutation index (0..5, order of oracle.mesh.PERMS) of every tetrahedron."""
    return np.repeat(np.arange(6), n ** 3)


def p0_parent(n_fine: int) -> np.ndarray:
    """Coarse tetrahedron containing each fine tetrahedron: the coarse cell of the fine cell,
    and the Kuhn permutation that orders the fine centroid's local coordinates in that coarse
    cell decreasingly (tetrahedron s of a cube is {t_s1 >= t_s2 >= t_s3})."""
    from .mesh import PERMS, kuhn_tets, node_xyz
    nf, nc = n_fine, n_fine // 2
    tets, cell = kuhn_tets(nf)
    cen = node_xyz(nf)[tets].mean(axis=1)
    ci, cj, ck = cell % nf // 2, cell // nf % nf // 2, cell // (nf * nf) // 2
    t = np.stack([cen[:, 0] * nc - ci, cen[:, 1] * nc - cj, cen[:, 2] * nc - ck], axis=1)
    order = np.argsort(-t, axis=1, kind="stable")
    pidx = {p: q for q, p in enumerate(PERMS)}
    s = np.array([pidx[tuple(o)] for o in order])
    # coarse numbering as kuhn_tets(nc): permutation block, then the (i, j, k) meshgrid order
    return s * nc ** 3 + (ci * nc * nc + cj * nc + ck)


class P1P0Level:
    """Matrices and smoother of one level of the P1-P0 hierarchy (constrained DoFs masked)."""

    def __init__(self, n, cell_mu, face, form="tr", gamma=GAMMA):
        self.sp = P1P0(n, cell_mu, face, gamma)
        s = self.sp
        self.n, self.nn, self.nT = n, s.nn, s.nT
        self.con = s.constrained()
        self.free = ~self.con
        K = masked(s.saddle(form), self.con)
        nn3 = 3 * s.nn
        self.K = K
        self.A = K[:nn3, :nn3].tocsr()
        self.BT = K[:nn3, nn3:].tocsr()
        self.B = K[nn3:, :nn3].tocsr()
        self.C = (-K[nn3:, nn3:]).tocsr()
        self.diagA = self.A.diagonal()
        self.mp = s.vol / s.mu_T
        i, j, k = s.disc.node_ijk()
        self.red = (i + j + k) % 2 == 0
        self.nullspace = TRACTION not in s.disc.face
        self._lu = None

    def velocity_pass(self, u, p, f, red):
        r = f - self.BT @ p - self.A @ u
        sel = np.tile(self.red if red else ~self.red, 3) & self.free[: 3 * self.nn]
        u[sel] += r[sel] / self.diagA[sel]

    def pressure_pass(self, u, p, g):
        p += OMEGA_P * ((self.B @ u - g) - self.C @ p) / self.mp

    def uzawa(self, x, b):
        nn3 = 3 * self.nn
        u, p = x[:nn3], x[nn3:]
        for red in (True, False, True):
            self.velocity_pass(u, p, b[:nn3], red)
        self.pressure_pass(u, p, b[nn3:])

    def residual(self, x, b):
        return b - self.K @ x

    def direct(self, b):
        if self._lu is None:
            free = np.flatnonzero(self.free)
            M = self.K[free][:, free].toarray()
            if self.nullspace:
                w = np.zeros(3 * self.nn + self.nT)
                w[3 * self.nn:] = self.mp
                wf = w[free]
                M = np.block([[M, wf[:, None]], [wf[None, :], np.zeros((1, 1))]])
            import scipy.linalg as sla
            self._lu = (free, sla.lu_factor(M))
        free, lu = self._lu
        import scipy.linalg as sla
        r = b[free]
        if self.nullspace:
            r = np.concatenate([r, [0.0]])
        sol = sla.lu_solve(lu, r)[: free.size]
        x = np.zeros_like(b)
        x[free] = sol
        return x


class P1P0Hierarchy:
    """Levels n, n/2, ..., n_coarse of the P1-P0 scheme with rediscretised operators, V_var
    cycle with nu = 3 + 2k Uzawa steps k levels below the finest, direct coarsest solve."""

    def __init__(self, n, n_coarse, cell_mu, face, form="tr", coarse_form=None, gamma=GAMMA,
                 coarsening="resolved"):
        """coarsening: how coarse cells take their viscosity ("resolved": the interfaces must be
        resolved by every coarse grid; "majority": the majority rule of
        oracle.solvers.coarsen_cell_mu for interfaces the coarse grids do not resolve)."""
        from .solvers import coarsen_cell_mu
        from .transfer import prolongation
        self.levels, self.P = [], []
        mu = np.asarray(cell_mu, dtype=np.float64).ravel()
        m = n
        while True:
            f = form if (m == n or coarse_form is None) else coarse_form
            self.levels.append(P1P0Level(m, mu, face, f, gamma))
            if m == n_coarse:
                break
            mu = coarsen_cell_mu(m, mu, coarsening)
            m //= 2
        for l in range(len(self.levels) - 1):
            fL, cL = self.levels[l], self.levels[l + 1]
            Pu = prolongation(cL.n)
            P3 = sp.block_diag([Pu, Pu, Pu], format="csr")
            par = p0_parent(fL.n)
            Pp = sp.coo_matrix((np.ones(fL.nT), (np.arange(fL.nT), par)), shape=(fL.nT, cL.nT)).tocsr()
            Pfull = sp.block_diag([P3, Pp], format="csr")
            df = sp.diags(fL.free.astype(np.float64))
            dc = sp.diags(cL.free.astype(np.float64))
            self.P.append((df @ Pfull @ dc).tocsr())

    def vcycle(self, x, b, l=0):
        L = self.levels[l]
        if l == len(self.levels) - 1:
            x[:] = L.direct(b)
            return x
        nu = 3 + 2 * l
        for _ in range(nu):
            L.uzawa(x, b)
        rc = self.P[l].T @ L.residual(x, b)
        ec = self.vcycle(np.zeros_like(rc), rc, l + 1)
        x += self.P[l] @ ec
        for _ in range(nu):
            L.uzawa(x, b)
        return x
