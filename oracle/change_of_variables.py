"""Oracle, part 5: the generalized change of variables (Section 5).

TEST INFRASTRUCTURE ONLY (see oracle/fe.py).

Follows Section 5 of the paper:
  * the averages of a glob, given as the rows of H^avg, are decomposed by QR with
    column pivoting, H^avg = Q [U V] K (eq. general-change-variables); the new
    variables are w_new = H w with H = [[U, V], [0, I]] K, so the k-th pivoted
    dof of the glob is replaced by the k-th transformed average;
  * w_new is in K order, as in the paper: its first r entries are the averages,
    then the unchanged dofs w[piv[r]], w[piv[r+1]], ...; a glob's new variable j sits
    at the glob's j-th dof position (column j of the glob's T);
  * the inverse change of variables is T = H^{-1} = K^{-1} [[U^{-1}, -U^{-1} V],
    [0, I]] (eq. T); rows of [U V] with a small diagonal entry of U are dropped as
    numerically redundant constraints;
  * with T = diag(T_i), A^c becomes R^cT T^T A T R^c and the constraint matrix
    becomes D-bar^c, whose rows each couple one explicit dof of two substructures
    with +1 and -1 (eq. BDDC-ch-var); the preconditioner is u = E T R^c w-bar;
  * the projected and regularised form of Section 4 (eqs. projection,
    BDDC-regular) with D-bar^c in place of D^c (eq. A-tilde), and the primal form
    of the Remark that closes Section 5 (the explicit dofs assembled like corners).

Reading: every dof lies in at most one glob (Section 4), so H_i^avg is block
diagonal over the globs of substructure i up to a row order, and its pivoted QR
is the QR of each glob's rows on their own.  The QR is therefore taken once per
glob, on the glob's dofs in increasing global order, which gives every
substructure sharing the glob the same [U V] and K: the explicit dofs of two
substructures then stand for the same average, as D-bar^c needs.  Rows are kept
while |U_kk| >= drop_rel |U_11| (|U_kk| does not increase along the pivoted
diagonal), the glob-relative drop of the dependent-row rule.

scipy's pivoted QR (LAPACK's DGEQP3, the routine the paper names), its
triangular solve, and dense / sparse LU are library primitives used as single
steps.  Nothing here is used by the CUDA library.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla


@dataclass
class GlobTransform:
    """The change of variables of one glob's averages (eqs. general-change-variables, T)."""
    U: np.ndarray          # r x r upper triangular, positive diagonal
    V: np.ndarray          # r x (n - r)
    piv: np.ndarray        # K: glob dof piv[j] becomes position j of K w
    r: int                 # kept (independent) averages

    def H(self):
        """H = [[U, V], [0, I]] K as a dense n x n matrix on the glob's dofs."""
        n = self.piv.size
        HK = np.eye(n)
        HK[: self.r, :] = np.hstack([self.U, self.V])
        Kmat = np.zeros((n, n))
        Kmat[np.arange(n), self.piv] = 1.0          # (K w)_j = w[piv[j]]
        return HK @ Kmat

    def T(self):
        """T = H^{-1} = K^{-1} [[U^{-1}, -U^{-1} V], [0, I]] (eq. T)."""
        n, r = self.piv.size, self.r
        Uinv = sla.solve_triangular(self.U, np.eye(r), lower=False)
        B = np.eye(n)
        B[:r, :r] = Uinv
        B[:r, r:] = -Uinv @ self.V
        Kinv = np.zeros((n, n))
        Kinv[self.piv, np.arange(n)] = 1.0          # K^{-1} = K^T
        return Kinv @ B


def glob_transform(Havg, drop_rel=1e-10):
    """Pivoted QR of the averages H^avg (m x n, m <= n), signs fixed so that the
    diagonal of U is positive, rows with |U_kk| < drop_rel |U_11| dropped."""
    Havg = np.atleast_2d(np.asarray(Havg, dtype=np.float64))
    m, n = Havg.shape
    _, R, piv = sla.qr(Havg, mode="economic", pivoting=True)   # Havg[:, piv] = Q R
    d = np.abs(np.diag(R))
    r = int(np.sum(d >= drop_rel * d[0])) if d.size and d[0] > 0 else 0
    R = R[:r, :]
    sgn = np.where(np.diag(R)[:r] < 0, -1.0, 1.0)
    R = sgn[:, None] * R                            # Q -> Q diag(sgn), [U V] -> diag(sgn) [U V]
    return GlobTransform(U=R[:, :r], V=R[:, r:], piv=np.asarray(piv, dtype=np.int64), r=r)


def glob_rows(model):
    """The averages of every glob, H^avg: the rows of all constraints on the same glob
    (an initial face average and the adaptive rows of that face, say) stacked over the
    glob's dofs in increasing global order.  Returns [(subs, gdofs, rows)]; every dof
    lies in at most one glob."""
    groups = {}
    for g in model.constraints:
        key = (tuple(g.subs), tuple(sorted(int(x) for x in g.gdofs)))
        order = np.argsort(g.gdofs)
        groups.setdefault(key, []).append(np.asarray(g.rows, dtype=np.float64)[:, order])
    out, seen = [], set()
    for (gsubs, gd), blocks in groups.items():
        assert not seen.intersection(gd), "two globs share a dof"
        seen.update(gd)
        out.append((gsubs, np.array(gd, dtype=np.int64), np.vstack(blocks)))
    return out


class TransformedBDDC:
    """The preconditioner of Lemma 2.1 after a change of variables T = diag(T_i).

    transform="qr":       T_i from the pivoted QR of each glob's averages (eq. T); the
                          constraint rows are D-bar^c: +1 / -1 on one explicit dof of
                          two substructures sharing the glob (eq. BDDC-ch-var).
    transform="identity": T_i = I and the rows of D^c as they are (Section 4's form).

    form="saddle":    the saddle-point system of eq. (BDDC-ch-var);
    form="projected": [Pi A Pi + t (I - Pi)] w = Pi R^cT T^T E^T r with the orthogonal
                      projection Pi onto null of the constraint rows (eqs. projection,
                      BDDC-regular, A-tilde), any t > 0;
    form="primal":    (transform="qr" only) every explicit dof assembled like a corner,
                      so that no constraint row is left (the Remark closing Section 5).

    In every form the result is u = E T R^c w (the residual vanishes in the interiors,
    so (I - P) is not applied, as in the Lemma 2.1 oracle).
    """

    def __init__(self, model, transform="qr", form="saddle", t=None, drop_rel=1e-10):
        if form == "primal" and transform != "qr":
            raise ValueError("the primal form needs the explicit dofs of the QR transform")
        m = model
        self.model, self.transform, self.form = m, transform, form
        subs = m.subs
        corner_g = m.glob_gdofs(m.globs.corners) if m.globs.corners else np.zeros(0, np.int64)
        cidx = {int(g): k for k, g in enumerate(corner_g)}
        # T_i, identity to start with
        self.T = [np.eye(s.G.size) for s in subs]
        # constraint rows: lists of (substructure, interface position, coefficient)
        rows = []
        # explicit dofs: (substructure, position) -> shared key, for the primal form
        explicit = {}
        self.n_explicit = 0
        self.glob_transforms = []
        for gi, (gsubs, gd, Cg) in enumerate(glob_rows(m)):
            assert not any(int(x) in cidx for x in gd), "a glob constraint on a corner dof"
            pos = {i: np.array([subs[i].gposG[int(x)] for x in gd], dtype=np.int64) for i in gsubs}
            if transform == "identity":
                C = Cg
                i1 = gsubs[0]
                for other in gsubs[1:]:
                    for c in C:
                        nz = np.nonzero(c)[0]
                        rows.append([(i1, int(p), float(v)) for p, v in zip(pos[i1][nz], c[nz])] +
                                    [(other, int(p), -float(v)) for p, v in zip(pos[other][nz], c[nz])])
                continue
            tr = glob_transform(Cg, drop_rel)
            self.glob_transforms.append(tr)
            Tg = tr.T()
            for i in gsubs:
                p = pos[i]
                self.T[i][np.ix_(p, p)] = Tg
                for k in range(tr.r):                  # w-bar = H w is in K order: average k at column k
                    explicit[(i, int(p[k]))] = (gi, k)
            self.n_explicit += tr.r
            i1 = gsubs[0]
            for other in gsubs[1:]:
                for k in range(tr.r):
                    rows.append([(i1, int(pos[i1][k]), 1.0), (other, int(pos[other][k]), -1.0)])
        # numbering of W-bar^c: corners shared; explicit dofs shared in the primal form
        nwc = len(cidx)
        shared = {}
        self.wc = []
        for i, s in enumerate(subs):
            wc = np.empty(s.G.size, dtype=np.int64)
            for k, gdf in enumerate(s.gdof[s.G]):
                gdf = int(gdf)
                key = explicit.get((i, k)) if form == "primal" else None
                if gdf in cidx:
                    wc[k] = cidx[gdf]
                elif key is not None and key in shared:
                    wc[k] = shared[key]
                else:
                    wc[k] = nwc
                    if key is not None:
                        shared[key] = nwc
                    nwc += 1
            self.wc.append(wc)
        self.nwc = nwc
        # A-bar^c = R^cT T^T A T R^c, assembled from T_i^T S_i T_i
        ri, ci, vi = [], [], []
        for i, s in enumerate(subs):
            Sb = self.T[i].T @ s.S @ self.T[i]
            w = self.wc[i]
            ri.append(np.repeat(w, w.size))
            ci.append(np.tile(w, w.size))
            vi.append(Sb.ravel())
        self.Abar = sp.coo_matrix((np.concatenate(vi), (np.concatenate(ri), np.concatenate(ci))),
                                  shape=(nwc, nwc)).tocsr()
        # constraint matrix in W-bar^c (none in the primal form)
        if form == "primal":
            rows = []
        dr, dc, dv = [], [], []
        for q, row in enumerate(rows):
            for (i, p, v) in row:
                dr.append(q)
                dc.append(self.wc[i][p])
                dv.append(v)
        self.D = sp.coo_matrix((dv, (dr, dc)), shape=(len(rows), nwc)).tocsr()
        self.nD = len(rows)
        if form == "projected":
            self._build_projected(t)
        elif form == "saddle" and self.nD:
            K = sp.bmat([[self.Abar, self.D.T], [self.D, None]], format="csc")
            self._lu = spla.splu(K, permc_spec="COLAMD")
        else:
            self._lu = spla.splu(self.Abar.tocsc(), permc_spec="COLAMD")

    def _build_projected(self, t):
        """Pi = I - D^T (D D^T)^{-1} D (eq. projection) and the regularised operator
        A-tilde = Pi A-bar Pi + t (I - Pi) (eqs. BDDC-regular, A-tilde)."""
        n = self.nwc
        I = sp.identity(n, format="csr")
        if self.nD:
            DDt = (self.D @ self.D.T).toarray()
            G = np.linalg.inv(DDt)
            G[np.abs(G) < 1e-15 * np.abs(G).max()] = 0.0   # block diagonal over the globs
            self.Pi = (I - self.D.T @ sp.csr_matrix(G) @ self.D).tocsr()
        else:
            self.Pi = I
        if t is None:                                      # "e.g. the maximal diagonal entry"
            t = float(self.Abar.diagonal().max())
        self.t = t
        self.Atilde = (self.Pi @ self.Abar @ self.Pi + t * (I - self.Pi)).tocsc()
        self._lu = spla.splu(self.Atilde, permc_spec="COLAMD")

    def apply(self, r):
        """u = M r for an assembled interface residual r."""
        m = self.model
        b = np.zeros(self.nwc)
        for i, s in enumerate(m.subs):
            np.add.at(b, self.wc[i], self.T[i].T @ (s.deltaG * r[s.RG]))
        if self.form == "projected":
            w = self._lu.solve(self.Pi @ b)
        elif self.form == "saddle" and self.nD:
            w = self._lu.solve(np.concatenate([b, np.zeros(self.nD)]))[: self.nwc]
        else:
            w = self._lu.solve(b)
        u = np.zeros(m.nG)
        for i, s in enumerate(m.subs):
            np.add.at(u, s.RG, s.deltaG * (self.T[i] @ w[self.wc[i]]))
        return u


def significant_nnz(A, rel=1e-13):
    """Entries of a sparse matrix above rel times its largest magnitude (the fill-in)."""
    A = sp.csr_matrix(A)
    v = np.abs(A.data)
    return int(np.sum(v > rel * v.max())) if v.size else 0
