"""Oracle, part 3: Schur complements, the BDDC preconditioner and PCG.

TEST INFRASTRUCTURE ONLY (see oracle/fe.py).

Follows Section 2 of the paper:
  * the reduced (interface) problem, eq. (reduced-problem): interiors are
    eliminated per substructure, S_i = A_GG - A_GI A_II^{-1} A_IG, and PCG runs
    on  sum_i R_i^T S_i R_i u = g,  g = F_G - sum_i R_i^T A_GI A_II^{-1} F_I;
  * the preconditioner of Lemma 2.1, eqs. (BDDC-prec)-(BDDC-Dc), written out
    literally on interface (discrete harmonic) functions: w_c in the space W^c
    continuous at corners solves the saddle-point system
        [A^c  D^cT] [w_c]   [R^cT E^T r]
        [D^c   0  ] [lam] = [    0     ]
    with A^c = R^cT diag(S_i) R^c, and M r = E R^c w_c.  (I - P)^T r is
    dropped because the residual vanishes in the interiors (the Remark after
    Lemma 2.1).  A glob constraint "c . w_i|G equal for all i sharing G"
    contributes the rows c.w_{i1} - c.w_{il}, l = 2..m (m - 1 rows).
  * PCG with x0 = 0 stopped at ||r_k|| <= tol ||r_0||; the condition number is
    estimated from the Lanczos tridiagonal built from the PCG coefficients
    (caption of Table 1: "from the Lanczos sequence in conjugate gradients"):
    diagonal 1/alpha_1, 1/alpha_j + beta_{j-1}/alpha_{j-1}; off-diagonal
    sqrt(beta_j)/alpha_j.
The sparse LU (scipy) and dense Cholesky (numpy) are library primitives used
as single steps.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .fe import element_matrices, assemble_global, Substructure
from .globs import Globs, weights


@dataclass
class GlobConstraint:
    """Rows c (m x len(dofs)) over the dofs of one glob, shared by ``subs``."""
    kind: str                 # "edge", "face" or "adaptive"
    nodes: np.ndarray
    subs: tuple
    rows: np.ndarray
    gdofs: np.ndarray = field(default=None)


class Model:
    """All oracle state for one substructured problem."""

    def __init__(self, prob, averages=()):
        self.prob = prob
        c = prob.ncomp
        self.ncomp = c
        self.Ke = element_matrices(prob)
        self.K, self.F, self.dofs = assemble_global(prob, self.Ke)
        self.subs = [Substructure(prob, i, self.Ke, self.dofs) for i in range(prob.nsub)]
        self.globs = Globs(prob)
        self.delta = weights(self.subs, self.dofs.n)
        n = self.dofs.n
        inode = np.array(self.globs.interface_nodes, dtype=np.int64)
        self.iface_gdof = np.sort(self.dofs.of_nodes(inode).ravel())
        self.nG = self.iface_gdof.size
        gidx = -np.ones(n, dtype=np.int64)
        gidx[self.iface_gdof] = np.arange(self.nG)
        self.gidx = gidx
        is_iface = np.zeros(prob.nn, dtype=bool)
        is_iface[inode] = True
        for i, s in enumerate(self.subs):
            lnode = np.repeat(s.free_nodes, c)
            iface = is_iface[lnode]
            s.I = np.nonzero(~iface)[0]
            s.G = np.nonzero(iface)[0]
            s.RG = gidx[s.gdof[s.G]]
            s.deltaG = self.delta[i][s.G]
            s.gposG = {int(g): k for k, g in enumerate(s.gdof[s.G])}
        self.constraints: list[GlobConstraint] = []
        for kind in averages:
            self.add_arithmetic_averages(kind)
        self._M = None

    # -- Schur complements (interior elimination) --------------------------
    def schur(self):
        for s in self.subs:
            A = s.A.toarray()
            AII = A[np.ix_(s.I, s.I)]
            AIG = A[np.ix_(s.I, s.G)]
            AGG = A[np.ix_(s.G, s.G)]
            if s.I.size:
                s.cII = sla.cho_factor(AII, lower=True)
                X = sla.cho_solve(s.cII, AIG)
                s.S = AGG - AIG.T @ X
            else:
                s.cII = None
                s.S = AGG.copy()
            s.S = 0.5 * (s.S + s.S.T)
            s.AIG = AIG
        return [s.S for s in self.subs]

    # -- constraints ---------------------------------------------------------
    def glob_gdofs(self, nodes):
        return self.dofs.of_nodes(np.asarray(nodes, dtype=np.int64)).ravel()

    def add_arithmetic_averages(self, kind):
        """One row per component: the plain sum of that component over the glob."""
        c = self.ncomp
        globs = self.globs.edges.items() if kind == "edge" else self.globs.faces.items()
        for key, nodes in globs:
            subs = tuple(sorted(key))
            nd = len(nodes)
            rows = np.zeros((c, nd * c))
            for comp in range(c):
                rows[comp, comp::c] = 1.0
            self.constraints.append(GlobConstraint(kind, np.array(nodes), subs, rows, self.glob_gdofs(nodes)))
        self._M = None

    def add_constraint(self, kind, nodes, subs, rows):
        self.constraints.append(GlobConstraint(kind, np.asarray(nodes), tuple(sorted(subs)), np.asarray(rows),
                                               self.glob_gdofs(nodes)))
        self._M = None

    def n_coarse(self):
        """Number of coarse degrees of freedom: corner dofs plus one per glob row."""
        return len(self.globs.corners) * self.ncomp + sum(g.rows.shape[0] for g in self.constraints)

    # -- the preconditioner of Lemma 2.1 -------------------------------------
    def build_preconditioner(self):
        c = self.ncomp
        corner_g = self.glob_gdofs(self.globs.corners) if self.globs.corners else np.zeros(0, np.int64)
        cidx = {int(g): k for k, g in enumerate(corner_g)}
        nwc = len(cidx)
        for s in self.subs:
            wc = np.empty(s.G.size, dtype=np.int64)
            for k, g in enumerate(s.gdof[s.G]):
                g = int(g)
                if g in cidx:
                    wc[k] = cidx[g]
                else:
                    wc[k] = nwc
                    nwc += 1
            s.wc = wc
        self.nwc = nwc
        rows, cols, vals = [], [], []
        for s in self.subs:
            r = np.repeat(s.wc, s.wc.size)
            cc = np.tile(s.wc, s.wc.size)
            rows.append(r)
            cols.append(cc)
            vals.append(s.S.ravel())
        Kc = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                           shape=(nwc, nwc)).tocsr()
        drows, dcols, dvals = [], [], []
        nd = 0
        for g in self.constraints:
            s1 = self.subs[g.subs[0]]
            w1 = s1.wc[[s1.gposG[int(x)] for x in g.gdofs]]
            for other in g.subs[1:]:
                so = self.subs[other]
                wl = so.wc[[so.gposG[int(x)] for x in g.gdofs]]
                for row in g.rows:
                    nz = np.nonzero(row)[0]
                    drows += [nd] * (2 * nz.size)
                    dcols += list(w1[nz]) + list(wl[nz])
                    dvals += list(row[nz]) + list(-row[nz])
                    nd += 1
        D = sp.coo_matrix((dvals, (drows, dcols)), shape=(nd, nwc)).tocsr()
        self.nD = nd
        Kfull = sp.bmat([[Kc, D.T], [D, None]], format="csc") if nd else Kc.tocsc()
        if Kfull.shape[0] <= 3000:
            self._saddle_dense = sla.lu_factor(Kfull.toarray())
            self._solve = lambda b: sla.lu_solve(self._saddle_dense, b)
        else:
            lu = spla.splu(Kfull, permc_spec="COLAMD")
            self._solve = lu.solve
        self._M = True

    def apply_M(self, r):
        if self._M is None:
            self.build_preconditioner()
        b = np.zeros(self.nwc + self.nD)
        for s in self.subs:
            np.add.at(b, s.wc, s.deltaG * r[s.RG])
        w = self._solve(b)[: self.nwc]
        u = np.zeros(self.nG)
        for s in self.subs:
            np.add.at(u, s.RG, s.deltaG * w[s.wc])
        return u

    def apply_S(self, x):
        y = np.zeros(self.nG)
        for s in self.subs:
            np.add.at(y, s.RG, s.S @ x[s.RG])
        return y

    # -- solve -----------------------------------------------------------------
    def condensed_rhs(self):
        g = self.F[self.iface_gdof].copy()
        for s in self.subs:
            if s.cII is not None:
                fI = self.F[s.gdof[s.I]]
                np.add.at(g, s.RG, -(s.AIG.T @ sla.cho_solve(s.cII, fI)))
        return g

    def recover(self, uG):
        u = np.zeros(self.dofs.n)
        u[self.iface_gdof] = uG
        for s in self.subs:
            if s.cII is not None:
                fI = self.F[s.gdof[s.I]]
                u[s.gdof[s.I]] = sla.cho_solve(s.cII, fI - s.AIG @ uG[s.RG])
        return u

    def solve(self, tol=1e-8, maxit=1000):
        if not hasattr(self.subs[0], "S"):
            self.schur()
        g = self.condensed_rhs()
        res = pcg(self.apply_S, self.apply_M, g, tol, maxit)
        res.u = self.recover(res.x)
        return res


@dataclass
class PCGResult:
    x: np.ndarray
    iters: int
    converged: bool
    alphas: list
    betas: list
    resnorms: list
    u: np.ndarray = None

    def condition(self):
        return lanczos_condition(self.alphas, self.betas)


def pcg(apply_A, apply_M, b, tol=1e-8, maxit=1000):
    """Preconditioned CG with x0 = 0; stops at the first k with ||r_k|| <= tol ||r_0||."""
    x = np.zeros_like(b)
    r = b.copy()
    r0 = np.linalg.norm(r)
    alphas, betas, norms = [], [], [r0]
    if r0 == 0.0:
        return PCGResult(x, 0, True, alphas, betas, norms)
    z = apply_M(r)
    p = z.copy()
    rz = r @ z
    for k in range(1, maxit + 1):
        q = apply_A(p)
        alpha = rz / (p @ q)
        alphas.append(alpha)
        x += alpha * p
        r -= alpha * q
        rn = np.linalg.norm(r)
        norms.append(rn)
        if rn <= tol * r0:
            return PCGResult(x, k, True, alphas, betas, norms)
        z = apply_M(r)
        rz_new = r @ z
        beta = rz_new / rz
        betas.append(beta)
        rz = rz_new
        p = z + beta * p
    return PCGResult(x, maxit, False, alphas, betas, norms)


def lanczos_tridiagonal(alphas, betas):
    k = len(alphas)
    T = np.zeros((k, k))
    for j in range(k):
        T[j, j] = 1.0 / alphas[j] + (betas[j - 1] / alphas[j - 1] if j > 0 else 0.0)
        if j + 1 < k:
            T[j, j + 1] = T[j + 1, j] = np.sqrt(betas[j]) / alphas[j]
    return T


def lanczos_condition(alphas, betas):
    """(theta_min, theta_max) of the Lanczos matrix T_k."""
    if not alphas:
        return 1.0, 1.0
    th = np.linalg.eigvalsh(lanczos_tridiagonal(alphas, betas))
    return th[0], th[-1]
