"""Reference solvers: sparse direct solve, Uzawa smoother and variable V-cycle.

Paper Sec. 5: an all-at-once multigrid V_var(3,3) cycle with Uzawa-type smoothing (eq.
Uzawa_smooth)

    u_{k+1} = u_k + Ahat^{-1} (f - A u_k - B^T p_k)
    p_{k+1} = p_k + Shat^{-1} (B u_{k+1} - C p_k - g)

with Ahat a symmetric red-black Gauss-Seidel on A and Shat a forward Gauss-Seidel on C
under-relaxed by omega = 0.3, standard transfers, and a direct coarse-grid solve (which the
paper notes is unproblematic for a_tr).

Readings of points the paper leaves open (each one is also listed in the design notes):

* colours: node (i, j, k) is red when i+j+k is even.  The diagonal blocks of A (for a_tr and
  a_sym alike) and C couple only along cube edges, so each colour is internally decoupled in
  them.  Couplings between different velocity components at nodes of the same colour (the
  interface rows of a_tr, every row of a_sym) are taken Jacobi-style inside one colour
  pass ("hybrid" Gauss-Seidel).  The symmetric sweep is the colour sequence red, black, red.
* the pressure sweep is an in-place Gauss-Seidel on C p = B u - g with relaxation omega,
  red then black, i.e. Shat = D_C / omega + L_C.
* "variable" V-cycle: nu = 3 + 2k pre- and post-smoothing steps on the level k below the
  finest; one step is one velocity sweep followed by one pressure sweep.
* the residual norm is the Euclidean norm over all free DoFs (velocity and pressure
  stacked); the stopping test is ||b - K x|| <= rtol ||b||.
* with no traction face the pressure constant is fixed by the border row
  sum_b w_b p_b = 0, w_b = int lambda_b / mu (the discrete form of int q/mu = 0).
* coarse levels may use the strain form a_sym instead of a_tr (Sec. 5 swaps a_tr for a_sym
  on the coarsest grid; here the swap can cover every level below the finest).  That swapped
  cycle is only used as a preconditioner, so no right-hand-side correction is applied.
* the coarsest solve is direct, or (coarse_solver="minres") the block-preconditioned MINRES
  iteration of Sec. 5 (block_minres) stopped at a relative tolerance.
* alternatively (coarse_correction=True) only the coarsest level takes a_sym, with the
  momentum right-hand side corrected as Sec. 5 describes so that the a_sym system approximates
  the a_tr one.  Sign and weight follow from the saddle matrix of Sec. 5: lumping the
  divergence, (mu div u, div v) ~ (B u)^T D (B v), D = diag(mu_b / m_b), hence
  A_tr ~ A_sym - B^T D B, and with B z = r2 + C q the a_sym system takes r1 + B^T D r2 (the term
  B^T D C q is dropped).  The paper prints the correction with the opposite sign and without
  mu; the form above is the one the consistency argument gives.
* outer iteration: either plain repeated V-cycles (Sec. 5) or flexible GMRES(m)
  (Saad 1993), right-preconditioned by one V-cycle with zero initial guess.  GMRES is an
  addition of this implementation: with a floating stiff inclusion the a_tr Schur
  complement has negative directions (Sec. 3, kernel of dev sym grad) and plain Uzawa
  multigrid diverges.

Test infrastructure: only tests/, the entry module's smoke check and the benchmark's CPU legs
import it; it shares no code with the CUDA library.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.linalg as sla
import scipy.sparse.linalg as spla

from .forms import PSPG_BETA, Discretisation, masked
from .transfer import system_prolongation

OMEGA = 0.3
DENSE_LIMIT = 7000


def coarsen_cell_mu(n: int, cell_mu: np.ndarray, rule: str = "resolved") -> np.ndarray:
    """Viscosity of the cells of the next coarser grid; each coarse cell is the union of 8 fine
    cells.  rule "resolved": the 8 must share one viscosity (interfaces resolved on every
    level).  rule "majority" (interfaces the coarse grids do not resolve, e.g. a level set, Sec.
    2.2 closing remark): the viscosity that most of the 8 children have, a tie going to the
    larger viscosity.  The coarse levels only precondition; the finest operator is exact."""
    m = np.asarray(cell_mu).reshape(n, n, n)
    c = m[0::2, 0::2, 0::2]
    kids = [m[dk::2, dj::2, di::2] for dk in (0, 1) for dj in (0, 1) for di in (0, 1)]
    if rule == "resolved":
        for k in kids:
            if not np.array_equal(k, c):
                raise ValueError("viscosity interface not resolved on the coarser grid")
        return np.ascontiguousarray(c).ravel()
    if rule != "majority":
        raise ValueError("rule is 'resolved' or 'majority'")
    stack = np.stack([k.ravel() for k in kids])          # [8, cells]
    out = np.empty(stack.shape[1])
    for cell in range(stack.shape[1]):
        vals, counts = np.unique(stack[:, cell], return_counts=True)
        best = counts.max()
        out[cell] = vals[counts == best].max()
    return out


class Level:
    """Matrices of one multigrid level with constrained DoFs masked out."""

    def __init__(self, n, cell_mu, face, form="tr", beta=PSPG_BETA):
        self.n = n
        self.disc = Discretisation(n, cell_mu, face, beta)
        d = self.disc
        self.nn = d.nn
        self.con = d.constrained()
        self.free = ~self.con
        self.form = form
        self.K = masked(d.saddle(form), self.con)
        nn = self.nn
        K = self.K
        self.A = K[: 3 * nn, : 3 * nn].tocsr()
        self.BT = K[: 3 * nn, 3 * nn:].tocsr()
        self.B = K[3 * nn:, : 3 * nn].tocsr()
        self.C = (-K[3 * nn:, 3 * nn:]).tocsr()
        self.diagA = self.A.diagonal()
        self.diagC = self.C.diagonal()
        i, j, k = d.node_ijk()
        self.red = (i + j + k) % 2 == 0
        self.nullspace = d.has_pressure_nullspace()
        self._lu = None

    # ------------------------------------------------------------------ direct solve
    def _factor(self):
        """Factor the free system.  Small systems (the coarsest multigrid grids): dense LU of
        the bordered matrix [[K_ff, w], [w^T, 0]] when the pressure has a null space.  Large
        systems: sparse LU with one pressure DoF pinned to zero, the result then shifted to
        w.p = 0; for a consistent right-hand side both give the same solution."""
        free = np.flatnonzero(self.free)
        Kff = self.K[free][:, free]
        w = np.zeros(4 * self.nn)
        w[3 * self.nn:] = self.disc.pressure_weights()
        wf = w[free]
        if free.size <= DENSE_LIMIT:
            M = Kff.toarray()
            if self.nullspace:
                M = np.block([[M, wf[:, None]], [wf[None, :], np.zeros((1, 1))]])
            self._lu = ("dense", free, wf, sla.lu_factor(M))
        else:
            keep = np.ones(free.size, dtype=bool)
            if self.nullspace:
                keep[-1] = False  # the last free DoF is the last pressure node
            lu = spla.splu(sp.csc_matrix(Kff[keep][:, keep]))
            self._lu = ("sparse", free, wf, (keep, lu))

    def direct(self, b: np.ndarray) -> np.ndarray:
        """Solve K x = b on the free DoFs; with a pressure null space the result satisfies
        sum_b w_b p_b = 0."""
        if self._lu is None:
            self._factor()
        kind, free, wf, fac = self._lu
        rhs = b[free]
        if kind == "dense":
            if self.nullspace:
                rhs = np.concatenate([rhs, [0.0]])
            sol = sla.lu_solve(fac, rhs)[: free.size]
        else:
            keep, lu = fac
            sol = np.zeros(free.size)
            sol[keep] = lu.solve(rhs[keep])
            if self.nullspace:
                npf = int(np.count_nonzero(free >= 3 * self.nn))
                pw = wf[-npf:]
                sol[-npf:] -= np.dot(pw, sol[-npf:]) / pw.sum()
        x = np.zeros(4 * self.nn)
        x[free] = sol
        return x

    # ------------------------------------------------------------------ smoother
    def velocity_pass(self, u, p, f, red):
        """One colour of the velocity Gauss-Seidel on A u = f - B^T p, in place on u: every
        free component of every node of the colour (red: i+j+k even) takes
        u += (f - B^T p - A u) / diag(A), all from the residual before the pass."""
        nn = self.nn
        r = f - self.BT @ p - self.A @ u
        sel = np.tile(self.red if red else ~self.red, 3) & self.free[: 3 * nn]
        u[sel] += r[sel] / self.diagA[sel]

    def pressure_pass(self, u, p, g, red):
        """One colour of the relaxed pressure Gauss-Seidel on C p = B u - g, in place on p:
        p += omega (B u - C p - g) / diag(C) at the nodes of the colour."""
        s = (self.B @ u - g) - self.C @ p
        sel = self.red if red else ~self.red
        p[sel] += OMEGA * s[sel] / self.diagC[sel]

    def velocity_sweep(self, u, p, f):
        """Symmetric hybrid red-black Gauss-Seidel for A u = f - B^T p: colours R, B, R,
        all free components of the colour updated from the same residual."""
        for red in (True, False, True):
            self.velocity_pass(u, p, f, red)

    def pressure_sweep(self, u, p, g):
        """Forward red-black Gauss-Seidel on C p = B u - g with relaxation omega."""
        for red in (True, False):
            self.pressure_pass(u, p, g, red)

    def uzawa(self, x, b):
        """One Uzawa smoothing step (eq. Uzawa_smooth) on x = (u, p) in place."""
        nn = self.nn
        u, p = x[: 3 * nn], x[3 * nn:]
        f, g = b[: 3 * nn], b[3 * nn:]
        self.velocity_sweep(u, p, f)
        self.pressure_sweep(u, p, g)

    def residual(self, x, b):
        return b - self.K @ x


class Hierarchy:
    """Levels n, n/2, ..., n_coarse of one problem with rediscretised operators."""

    def __init__(self, n, n_coarse, cell_mu, face, form="tr", beta=PSPG_BETA, coarse_form=None,
                 coarse_correction=False, coarse_solver="direct", coarse_rtol=1e-8,
                 coarsening="resolved"):
        if coarse_correction and (form != "tr" or coarse_form is not None or n == n_coarse):
            raise ValueError("coarse_correction swaps a_tr for a_sym on the coarsest level only")
        if coarse_solver not in ("direct", "minres"):
            raise ValueError("coarse_solver is 'direct' or 'minres'")
        self.coarse_solver, self.coarse_rtol = coarse_solver, coarse_rtol
        self.levels = []
        self.P = []
        self.correction = None
        mu = np.asarray(cell_mu, dtype=np.float64).ravel()
        m = n
        while True:
            lf = form if (m == n or coarse_form is None) else coarse_form
            if coarse_correction and m == n_coarse:
                lf = "sym"
            self.levels.append(Level(m, mu, face, lf, beta))
            if m == n_coarse:
                break
            if m % 2 or m // 2 < n_coarse:
                raise ValueError("n must be n_coarse * 2^k")
            mu = coarsen_cell_mu(m, mu, coarsening)
            m //= 2
        for l in range(len(self.levels) - 1):
            f, c = self.levels[l], self.levels[l + 1]
            self.P.append(system_prolongation(c.n, f.con, c.con))
        if coarse_correction:
            self.correction = self.levels[-1].disc.divergence_weights()

    def coarse_rhs(self, b):
        """Right-hand side of the coarsest solve: b itself, or with coarse_correction the
        momentum rows r1 + B^T D r2 of the a_sym swap (Sec. 5; sign and weight as derived in the
        module notes), constrained rows zero."""
        if self.correction is None:
            return b
        L = self.levels[-1]
        nn = L.nn
        out = b.copy()
        out[: 3 * nn] += L.BT @ (self.correction * b[3 * nn:])
        out[L.con] = 0.0
        return out

    def vcycle(self, x, b, l=0):
        """Variable V-cycle on level l, x updated in place and returned."""
        L = self.levels[l]
        if l == len(self.levels) - 1:
            rhs = self.coarse_rhs(b)
            if self.coarse_solver == "minres":
                x[:] = block_minres(L, rhs, rtol=self.coarse_rtol)
            else:
                x[:] = L.direct(rhs)
            return x
        nu = 3 + 2 * l
        for _ in range(nu):
            L.uzawa(x, b)
        r = L.residual(x, b)
        rc = self.P[l].T @ r
        ec = self.vcycle(np.zeros_like(rc), rc, l + 1)
        x += self.P[l] @ ec
        for _ in range(nu):
            L.uzawa(x, b)
        return x

    def solve(self, b, rtol=1e-8, maxit=100, x0=None):
        """Repeat V-cycles until ||b - K x|| <= rtol ||b|| (norms over free DoFs).
        Returns (x, history of residual norms)."""
        L = self.levels[0]
        x = np.zeros_like(b) if x0 is None else x0.copy()
        bn = np.linalg.norm(b[L.free])
        hist = [np.linalg.norm(L.residual(x, b)[L.free])]
        for _ in range(maxit):
            if hist[-1] <= rtol * bn:
                break
            self.vcycle(x, b)
            hist.append(np.linalg.norm(L.residual(x, b)[L.free]))
        return x, np.array(hist)


def block_minres(L, b, rtol=1e-10, maxit=1000, inner_rtol=1e-12):
    """The coarse-grid solver of Sec. 5: MINRES on the level's saddle system (free DoFs),
    preconditioned block-diagonally by the velocity block A, applied through a
    Jacobi-preconditioned CG iteration, and the lumped pressure mass matrix.  The pressure
    mass is weighted by 1/mu (w_b = int lambda_b / mu, the Schur complement of a variable
    viscosity scaling like that); MINRES needs the preconditioner symmetric positive
    definite, which holds for a_sym and the gradient form but not for a_tr (Sec. 5 swaps the
    form for this reason).  Scipy's MINRES and CG serve as the two iterations.  With a pressure
    null space the result is shifted to sum_b w_b p_b = 0.  Returns the full-size solution."""
    free = np.flatnonzero(L.free)
    nn = L.nn
    Kff = L.K[free][:, free].tocsr()
    nu = int(np.count_nonzero(free < 3 * nn))
    A = Kff[:nu, :nu].tocsr()
    dA = A.diagonal()
    w = L.disc.pressure_weights()
    wp = w[free[nu:] - 3 * nn]

    def apply_prec(r):
        z = np.empty_like(r)
        zu, info = spla.cg(A, r[:nu], rtol=inner_rtol, atol=0.0, maxiter=10 * nu,
                           M=spla.LinearOperator(A.shape, matvec=lambda v: v / dA))
        if info != 0:
            raise RuntimeError("inner CG did not converge (velocity block not positive definite?)")
        z[:nu] = zu
        z[nu:] = r[nu:] / wp
        return z

    M = spla.LinearOperator(Kff.shape, matvec=apply_prec)
    try:
        sol, info = spla.minres(Kff, b[free], M=M, rtol=rtol, maxiter=maxit)
    except ValueError as e:  # scipy's check that the preconditioned operator is symmetric
        raise RuntimeError(f"MINRES cannot run with this preconditioner: {e}") from e
    if info != 0:
        raise RuntimeError(f"MINRES did not converge (info {info})")
    x = np.zeros(4 * nn)
    x[free] = sol
    if L.nullspace:
        x[3 * nn:] -= np.dot(w, x[3 * nn:]) / w.sum()
    return x


def fgmres(K, precond, b, free, rtol=1e-8, restart=30, maxit=200, x0=None):
    """Flexible GMRES(restart) with right preconditioning (Saad, SIAM J. Sci. Comput. 14,
    1993), modified Gram-Schmidt, Givens rotations.  Vectors are full-size with zeros at
    constrained DoFs; inner products run over the free DoFs.  Stops when the true residual
    ||b - K x|| <= rtol ||b||.  Returns (x, list of true residual norms, one at the start of
    every restart cycle plus the final one)."""
    x = np.zeros_like(b) if x0 is None else x0.copy()
    bn = np.linalg.norm(b[free])
    hist = []
    its = 0
    while its < maxit:
        r = b - K @ x
        r[~free] = 0.0
        beta = np.linalg.norm(r)
        hist.append(beta)
        if beta <= rtol * bn:
            break
        V = [r / beta]
        Z = []
        H = np.zeros((restart + 1, restart))
        cs = np.zeros(restart)
        sn = np.zeros(restart)
        g = np.zeros(restart + 1)
        g[0] = beta
        j = 0
        for j in range(restart):
            z = precond(V[j])
            z[~free] = 0.0
            Z.append(z)
            w = K @ z
            w[~free] = 0.0
            for i in range(j + 1):
                H[i, j] = np.dot(w, V[i])
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            V.append(w / H[j + 1, j] if H[j + 1, j] > 0 else w)
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            d = np.hypot(H[j, j], H[j + 1, j])
            cs[j], sn[j] = H[j, j] / d, H[j + 1, j] / d
            H[j, j] = d
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            its += 1
            if abs(g[j + 1]) <= rtol * bn or its >= maxit:
                break
        k = j + 1
        y = np.linalg.solve(np.triu(H[:k, :k]), g[:k])
        for i in range(k):
            x += y[i] * Z[i]
    return x, hist


def vcycle_preconditioner(hier):
    """z = V(0; v): one V-cycle with zero initial guess applied to v."""
    def apply(v):
        return hier.vcycle(np.zeros_like(v), v.copy())
    return apply
