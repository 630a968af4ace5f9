"""Oracle, part 4: adaptive face constraints (Section 3 of the paper).

TEST INFRASTRUCTURE ONLY (see oracle/fe.py).

For every pair of substructures (i, j) sharing a face, the pair eigenproblem
(eq. (eig-matrix))
    Pi (I - E_ij)^T S^c_ij (I - E_ij) Pi w = lambda Pi S^c_ij Pi w
is solved in the factorspace modulo null(Pi S^c_ij Pi) (eq. (eig-nullspace)),
and for every eigenvalue above tau (Algorithm 3.1: smallest k_ij with
lambda_{k_ij+1} <= tau) the row d = w^T Pi (I-E)^T S^c (I-E) Pi (eq. (d-def)) is
kept.  Its face part becomes a new weighted-average constraint (the edge
parts are dropped, Remark at the end of Section 3, unless adapt(keep_edges=...)
keeps them as edge rows).  omega_ij = lambda_1 and the indicator is
omega~ = max omega_ij (eq. (cond-ind)).

Steps, in the paper's notation:
  1. S^c_ij: diag(S_i, S_j) on the interface dofs of the pair, assembled at
     the corners shared by i and j.
  2. (I - E_ij) is non-zero only on s = the non-corner dofs shared by i and j
     (the face plus the edges containing both); E_ij averages with weights
     normalised over the pair, so on [w_i; w_j] restricted to s it is
     [d_j (w_i - w_j); d_i (w_j - w_i)].  Hence the left form is
     L = (I-E)^T diag(S_i,ss, S_j,ss) (I-E) on s, and for lambda != 0 the
     pencil condenses exactly onto s with the Schur complement S^ of S^c_ij.
  3. Pi: orthogonal projection onto null(D^c_ij), the initial glob rows on
     globs inside s (identity when there are none).  Q = orthonormal basis of
     range(Pi).
  4. Cyclic Jacobi on B = Q^T S^ Q; eigenvalues below 1e-12 max are the
     null space and are dropped (factorspace); C = L^-1/2 V^T Q^T L Q V L^-1/2
     is diagonalised by Jacobi again.
  5. Face rows are normalised and orthogonalised with row pivoting; a row
     whose pivot falls below 1e-10 (relative to the first) is dropped as
     linearly dependent (the rank drop of Section 5, applied per glob).
"""
from __future__ import annotations

from dataclasses import dataclass
import numpy as np

from .native import jacobi_eigh

NULL_REL = 1e-12
DROP_REL = 1e-10
TIE_REL = 1e-6


@dataclass
class PairResult:
    pair: tuple
    lam: np.ndarray            # all eigenvalues of the factorspace pencil, descending
    n_null: int                # dropped null directions of B
    selected: int              # number of lambda > tau
    face_rows: np.ndarray      # (selected, n_face_dofs) rows d restricted to the face on side i
    face_nodes: np.ndarray
    d_full: np.ndarray         # (selected, 2 n_s) full rows d on s (both sides)
    s_gdofs: np.ndarray
    face_mask: np.ndarray      # mask over s dofs: dof lies on the face
    ties: int
    W: np.ndarray = None
    L: np.ndarray = None
    Shat: np.ndarray = None
    Q: np.ndarray = None       # orthonormal basis of range(Pi) (2 n_s x dim)


def pair_data(model, i, j):
    """S^c_ij, the index sets and the weights of one face pair."""
    si, sj = model.subs[i], model.subs[j]
    sets = model.globs.sets
    c = model.ncomp
    corners = model.globs.corner_set
    ni = si.G.size
    gi = si.gdof[si.G]
    gj = sj.gdof[sj.G]
    nodes_i = si.free_nodes.repeat(c)[si.G]
    nodes_j = sj.free_nodes.repeat(c)[sj.G]
    idx_j = np.empty(gj.size, dtype=np.int64)
    nxt = ni
    for k, (g, nd) in enumerate(zip(gj, nodes_j)):
        if int(nd) in corners and int(g) in si.gposG:
            idx_j[k] = si.gposG[int(g)]
        else:
            idx_j[k] = nxt
            nxt += 1
    N = nxt
    Sc = np.zeros((N, N))
    Sc[:ni, :ni] += si.S
    Sc[np.ix_(idx_j, idx_j)] += sj.S
    # s: non-corner dofs whose node set contains both i and j
    pair = {i, j}
    s_mask_i = np.array([(int(nd) not in corners) and pair <= sets[int(nd)] for nd in nodes_i])
    s_g = np.sort(gi[s_mask_i])
    pos_i = np.array([si.gposG[int(g)] for g in s_g], dtype=np.int64)
    pos_j_loc = np.array([sj.gposG[int(g)] for g in s_g], dtype=np.int64)
    pos_j = idx_j[pos_j_loc]
    s_nodes = nodes_i[pos_i]
    face_mask = np.array([sets[int(nd)] == frozenset(pair) for nd in s_nodes])
    ai = si.A.diagonal()[si.G][pos_i]
    aj = sj.A.diagonal()[sj.G][pos_j_loc]
    di = ai / (ai + aj)
    dj = aj / (ai + aj)
    return dict(Sc=Sc, pos_i=pos_i, pos_j=pos_j, pos_i_loc=pos_i, pos_j_loc=pos_j_loc, s_g=s_g,
                s_nodes=s_nodes, face_mask=face_mask, di=di, dj=dj)


def initial_rows_on_s(model, i, j, s_g, include_adaptive=False):
    """Rows of D^c_ij: initial glob constraints on globs inside s (both i and j share them).
    include_adaptive: also the adaptive rows already added (the pair problem on the
    final space W~, whose largest eigenvalue is omega_ij after adaptation)."""
    ns = s_g.size
    pos = {int(g): k for k, g in enumerate(s_g)}
    rows = []
    for gc in model.constraints:
        if (gc.kind.startswith("adaptive") and not include_adaptive) or not ({i, j} <= set(gc.subs)):
            continue
        if not all(int(g) in pos for g in gc.gdofs):
            continue
        p = np.array([pos[int(g)] for g in gc.gdofs])
        for row in gc.rows:
            r = np.zeros(2 * ns)
            r[p] = row
            r[ns + p] = -row
            rows.append(r)
    return np.array(rows).reshape(-1, 2 * ns)


def pair_problem(model, i, j, tau, keep_matrices=False, n_fixed=None, include_adaptive=False):
    """tau: select lambda > tau (Algorithm 3.1).  n_fixed: instead select the n_fixed
    largest eigenvalues (all when there are fewer) -- the paper's "3eigv" constraints
    of Section 7, three dominant eigenvectors per face; ties then counts a boundary
    lambda_k ~ lambda_{k+1} (within TIE_REL), where the selected subspace is not unique."""
    pd = pair_data(model, i, j)
    Sc, pos_i, pos_j = pd["Sc"], pd["pos_i"], pd["pos_j"]
    ns = pos_i.size
    spos = np.concatenate([pos_i, pos_j])
    mask = np.ones(Sc.shape[0], dtype=bool)
    mask[spos] = False
    opos = np.nonzero(mask)[0]
    Sss = Sc[np.ix_(spos, spos)]
    if opos.size:
        Sso = Sc[np.ix_(spos, opos)]
        Soo = Sc[np.ix_(opos, opos)]
        Shat = Sss - Sso @ np.linalg.solve(Soo, Sso.T)
    else:
        Shat = Sss.copy()
    Shat = 0.5 * (Shat + Shat.T)
    si, sj = model.subs[i], model.subs[j]
    Sblk = np.zeros((2 * ns, 2 * ns))
    Sblk[:ns, :ns] = si.S[np.ix_(pd["pos_i_loc"], pd["pos_i_loc"])]
    Sblk[ns:, ns:] = sj.S[np.ix_(pd["pos_j_loc"], pd["pos_j_loc"])]
    di, dj = pd["di"], pd["dj"]
    IE = np.zeros((2 * ns, 2 * ns))
    k = np.arange(ns)
    IE[k, k] = dj
    IE[k, ns + k] = -dj
    IE[ns + k, k] = -di
    IE[ns + k, ns + k] = di
    L = IE.T @ Sblk @ IE
    L = 0.5 * (L + L.T)
    D = initial_rows_on_s(model, i, j, pd["s_g"], include_adaptive)
    if D.shape[0]:
        U, sv, Vt = np.linalg.svd(D)
        rank = int((sv > 1e-12 * sv[0]).sum())
        Q = Vt[rank:].T
        Pi = Q @ Q.T                      # I - D^T (D D^T)^{-1} D, also for dependent rows
    else:
        Pi = np.eye(2 * ns)
        Q = np.eye(2 * ns)
    B = Q.T @ Shat @ Q
    mu, V = jacobi_eigh(B)
    keep = mu > NULL_REL * mu.max()
    n_null = int((~keep).sum())
    Vk = V[:, keep] / np.sqrt(mu[keep])[None, :]
    C = Vk.T @ (Q.T @ L @ Q) @ Vk
    lam, Y = jacobi_eigh(C)
    lam, Y = lam[::-1], Y[:, ::-1]
    W = Q @ Vk @ Y
    PLP = Pi @ L @ Pi
    if n_fixed is None:
        sel = int((lam > tau).sum())
        ties = int((np.abs(lam / tau - 1.0) < TIE_REL).sum())
    else:
        sel = min(int(n_fixed), lam.size)
        ties = int(0 < sel < lam.size and abs(lam[sel] / lam[sel - 1] - 1.0) < TIE_REL)
    d = (PLP @ W[:, :sel]).T
    face_rows = d[:, :ns][:, pd["face_mask"]]
    res = PairResult((i, j), lam, n_null, sel, face_rows, np.unique(pd["s_nodes"][pd["face_mask"]]),
                     d, pd["s_g"], pd["face_mask"], ties)
    if keep_matrices:
        res.W, res.L, res.Shat, res.Q = W, L, Shat, Q
    return res


def row_pivots(rows):
    """The pivots of Gram-Schmidt with row pivoting on the normalised rows, relative to
    the first (non-increasing, as in a column-pivoted QR): the rows kept at a drop
    threshold t are those whose pivot is >= t."""
    if rows.shape[0] == 0:
        return np.zeros(0)
    R = rows / np.linalg.norm(rows, axis=1, keepdims=True)
    piv = []
    remaining = list(range(R.shape[0]))
    while remaining:
        norms = np.array([np.linalg.norm(R[k]) for k in remaining])
        kk = int(np.argmax(norms))
        p = norms[kk]
        piv.append(p)
        if p == 0.0:
            break
        q = R[remaining[kk]] / p
        remaining.pop(kk)
        for k in remaining:
            R[k] = R[k] - (R[k] @ q) * q
    piv = np.array(piv)
    return piv / piv[0]


def orthonormal_rows(rows, drop_rel=DROP_REL):
    """Normalise rows, then Gram-Schmidt with row pivoting; drop rows whose
    pivot is below drop_rel relative to the first pivot."""
    if rows.shape[0] == 0:
        return rows
    R = rows / np.linalg.norm(rows, axis=1, keepdims=True)
    out = []
    first = None
    remaining = list(range(R.shape[0]))
    while remaining:
        norms = np.array([np.linalg.norm(R[k]) for k in remaining])
        kk = int(np.argmax(norms))
        piv = norms[kk]
        if first is None:
            first = piv
        if piv < drop_rel * first:
            break
        q = R[remaining[kk]] / piv
        out.append(q)
        remaining.pop(kk)
        for k in remaining:
            R[k] = R[k] - (R[k] @ q) * q
    return np.array(out)


@dataclass
class AdaptResult:
    pairs: dict
    omega: float
    n_added: int
    per_face: dict


def edge_rows(model, res, orthonormal=True):
    """The edge parts of the rows d of one pair (Section 3, after Prop. 4.1: d split into
    one row on the face and one row per edge, so that every row stays on one glob).
    Returns [(edge nodes, rows)], the rows over the edge's dofs in global dof order; an
    edge part below DROP_REL of its whole row's norm carries no constraint and is left out."""
    ns = res.s_gdofs.size
    d_i = res.d_full[:, :ns]
    full = np.linalg.norm(res.d_full, axis=1)
    out = []
    for key, nodes in sorted(model.globs.edges.items(), key=lambda kv: kv[1][0]):
        if not set(res.pair) <= set(key):
            continue
        gd = model.glob_gdofs(nodes)
        pos = np.minimum(np.searchsorted(res.s_gdofs, gd), ns - 1)
        assert np.all(res.s_gdofs[pos] == gd), "an edge of the pair outside s"
        part = d_i[:, pos]
        keep = np.linalg.norm(part, axis=1) > DROP_REL * full
        if keep.any():
            rows = part[keep]
            out.append((np.asarray(nodes), orthonormal_rows(rows) if orthonormal else rows))
    return out


def adapt(model, tau, n_fixed=None, keep_edges=False, edge_drop_rel=DROP_REL):
    """Algorithm 3.1 on every face pair; the new face rows are added to the model.
    With n_fixed, the n_fixed dominant eigenvectors of every face are used instead of
    those above tau (Section 7, "3eigv").  keep_edges: the edge parts of the rows d are
    added too, instead of being dropped as in the paper's experiments (the Remark
    closing Section 3); then omega~ <= tau holds after adaptation.
      keep_edges=True:   the split rows of Section 3, each a constraint between the
                         pair's two substructures on one edge;
      keep_edges="glob": per edge, one orthonormal basis of the span of every pair's
                         edge rows on it, enforced on all substructures sharing the
                         edge (a stronger constraint set, whose rows stay independent
                         on every substructure, as a primal coarse space needs).
    edge_drop_rel: the rank rule of those per-edge bases (the rank drop of Section 5, as
    for the face rows); every edge's relative pivots are returned in edge_pivots."""
    pairs = {}
    for (i, j) in sorted(model.globs.faces):
        pairs[(i, j)] = pair_problem(model, i, j, tau, n_fixed=n_fixed)
    per_face = {}
    n_added = 0
    n_edge_rows = 0
    c = model.ncomp
    edge_stack = {}                # keep_edges="glob": edge nodes -> rows of every pair
    for (i, j), res in pairs.items():
        if res.selected == 0:
            per_face[(i, j)] = 0
            continue
        rows = orthonormal_rows(res.face_rows)
        # the face rows are over face dofs in s order (global dof order)
        nodes = np.array(model.globs.faces[(i, j)])
        model.add_constraint("adaptive", nodes, (i, j), rows)
        per_face[(i, j)] = rows.shape[0]
        n_added += rows.shape[0]
        if keep_edges == "glob":
            for enodes, erows in edge_rows(model, res, orthonormal=False):
                edge_stack.setdefault(tuple(int(v) for v in enodes), []).append(erows)
        elif keep_edges:
            for enodes, erows in edge_rows(model, res):
                model.add_constraint("adaptive_edge", enodes, (i, j), erows)
                n_edge_rows += erows.shape[0]
    edge_pivots = {}
    for key in sorted(edge_stack):
        stacked = np.vstack(edge_stack[key])
        edge_pivots[key] = row_pivots(stacked)
        rows = orthonormal_rows(stacked, edge_drop_rel)
        subs = sorted(model.globs.sets[key[0]])
        model.add_constraint("adaptive_edge", np.array(key), subs, rows)
        n_edge_rows += rows.shape[0]
    omega = max((r.lam[0] for r in pairs.values() if r.lam.size), default=0.0)
    out = AdaptResult(pairs, omega, n_added, per_face)
    out.n_edge_rows = n_edge_rows
    out.edge_pivots = edge_pivots
    return out


def indicator(model, tau=np.inf):
    """omega~ (eq. cond-ind) on the current space W~: the largest eigenvalue of every
    face pair's problem with all constraints in place, adaptive rows included."""
    return max((pair_problem(model, i, j, tau, include_adaptive=True).lam[:1].max(initial=0.0)
                for (i, j) in sorted(model.globs.faces)), default=0.0)
