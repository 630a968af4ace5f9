"""Oracle, part 6: LOBPCG for the pair eigenproblems (Section 3).

TEST INFRASTRUCTURE ONLY (see oracle/fe.py).

Section 3 notes that the dominant eigenpairs of the pair problem (eq. eig-matrix)
can be found by the subspace iteration LOBPCG of Knyazev, run in the factorspace
modulo null(Pi S^c Pi) (eq. eig-nullspace), and leaves its preconditioning for
later work (Section 8).  Here, on the pencil restricted to range(Pi) (an
orthonormal basis Q: A = Q^T L Q, B = Q^T S^ Q):
  * the factorspace is the orthogonal complement of null(B); the left operator
    vanishes on null(B) too (eq. eig-nullspace), so every iterate is kept there;
  * one LOBPCG block of k vectors: Rayleigh-Ritz on span[X, W, P] keeping the k
    largest Ritz pairs, W = T R the preconditioned residuals R = A X - B X Theta,
    P the previous step's direction (the part of the new X that is B-orthogonal
    to the old one); converged when every |r_j| <= tol (|A| + |theta_j| |B|) for
    B-normalised x_j (|.| the spectral norm);
  * T = I (plain) or T = B^+ (the pseudo-inverse on the factorspace): B^+ R =
    B^+ A X - X Theta is the step of subspace iteration with B^+ A, which favours
    the dominant end of the spectrum;
  * all eigenvalues above tau (Algorithm 3.1): blocks of k0 vectors, each
    B-orthogonal to the converged (locked) ones, until a block reaches tau; in a
    block only the pairs above tau and the largest one below it must converge.
The basis of the Rayleigh-Ritz step is B-orthonormalised through the eigen-
decomposition of its Gram matrix after scaling every column to unit B-norm
(directions below 1e-12 of the largest are dropped).  numpy's symmetric eigensolver is a library primitive used as a step.
"""
from __future__ import annotations

import numpy as np

from .adaptive import pair_problem, NULL_REL


def pair_pencil(model, i, j):
    """(A, B): the pair problem of faces pair (i, j) restricted to range(Pi)."""
    res = pair_problem(model, i, j, np.inf, keep_matrices=True)
    A = res.Q.T @ res.L @ res.Q
    B = res.Q.T @ res.Shat @ res.Q
    return 0.5 * (A + A.T), 0.5 * (B + B.T)


def _sym(M):
    return 0.5 * (M + M.T)


def _b_orthonormal(S, B, drop=1e-12):
    # columns scaled to unit B-norm first, then the Gram matrix's eigenbasis (SVQB)
    G = _sym(S.T @ B @ S)
    d = np.sqrt(np.maximum(np.diag(G), 1e-300))
    w, V = np.linalg.eigh(G / np.outer(d, d))
    keep = w > drop * w.max()
    return (S / d) @ (V[:, keep] / np.sqrt(w[keep]))


def lobpcg_block(A, B, k, precondition=True, Y=None, tol=1e-10, maxit=2000, seed=0, tau=-np.inf):
    """The k largest eigenpairs of A x = theta B x on the factorspace, B-orthogonal to
    the columns of Y.  Only the wanted pairs must converge: those with theta > tau and
    the largest one below it (which certifies the count above tau); the rest of the
    block only accelerates.  Returns (theta descending, X, iterations)."""
    n = A.shape[0]
    mu, V = np.linalg.eigh(B)
    fac = mu > NULL_REL * mu.max()
    N = V[:, ~fac]
    Bplus = (V[:, fac] / mu[fac]) @ V[:, fac].T
    Yl = np.zeros((n, 0)) if Y is None else Y

    def proj(X):
        X = X - N @ (N.T @ X)
        return X - Yl @ (Yl.T @ (B @ X))

    T = (lambda R: Bplus @ R) if precondition else (lambda R: R)
    nA, nB = np.linalg.norm(A, 2), np.linalg.norm(B, 2)
    rng = np.random.default_rng(seed)
    X = _b_orthonormal(proj(rng.standard_normal((n, k))), B)
    P = None
    for it in range(1, maxit + 1):
        th, C = np.linalg.eigh(_sym(X.T @ A @ X))
        th, C = th[::-1], C[:, ::-1]
        X = X @ C
        R = A @ X - (B @ X) * th
        want = min(int((th > tau).sum()) + 1, k)
        if np.all(np.linalg.norm(R[:, :want], axis=0) <= tol * (nA + np.abs(th[:want]) * nB)):
            return th, X, it
        W = proj(T(R))
        S = np.hstack([X, W] + ([P] if P is not None else []))
        S = _b_orthonormal(proj(S), B)
        ths, Cs = np.linalg.eigh(_sym(S.T @ A @ S))
        Xn = S @ Cs[:, ::-1][:, :k]
        P = proj(Xn - X @ (X.T @ (B @ Xn)))
        X = Xn
    raise RuntimeError("LOBPCG did not converge")


def eigs_above(A, B, tau, k0=8, precondition=True, tol=1e-10):
    """Every eigenvalue above tau (descending) with its eigenvectors, by blocks of k0
    locked in turn, and the total number of LOBPCG iterations."""
    n = A.shape[0]
    mu = np.linalg.eigvalsh(B)
    dim = int((mu > NULL_REL * mu.max()).sum())
    lam, vecs, iters = [], [], 0
    Y = np.zeros((n, 0))
    while Y.shape[1] < dim:
        k = min(k0, (dim - Y.shape[1]) // 3) or 1
        th, X, it = lobpcg_block(A, B, k, precondition, Y, tol, seed=Y.shape[1], tau=tau)
        iters += it
        above = th > tau
        lam += list(th[above])
        vecs.append(X[:, above])
        Y = np.hstack([Y, X])
        if not above.all():
            break
    return np.array(lam), np.hstack(vecs) if vecs else np.zeros((n, 0)), iters
