"""FP64 CPU oracle of adaptive BDDC in 3D (Mandel, Sousedik, Sistek).

TEST INFRASTRUCTURE ONLY.  Imported by tests/, by __graft_entry__.smoke() and
by the CPU-baseline leg of bench.py; the CUDA library and its binding never
import, call or link anything here, and nothing here imports them.

Modules: fe (Q1 elements, assembly), globs (faces/edges/corners, weights),
bddc (Schur complements, Lemma 2.1 preconditioner, PCG, Lanczos estimate),
adaptive (pair eigenproblems and face constraints, Algorithm 3.1),
change_of_variables (Section 5: pivoted-QR change of variables, the saddle,
projected and primal forms of the preconditioner in the new variables),
lobpcg (Section 3: LOBPCG on the pair pencil in the factorspace, plain or
preconditioned by B^+), native (the cyclic Jacobi helper in jacobi.c).
"""
from .bddc import Model, pcg, lanczos_condition, lanczos_tridiagonal
from .adaptive import adapt, pair_problem, orthonormal_rows


def run(prob, averages=(), tau=None, tol=1e-8, maxit=1000, n_fixed=None):
    """Setup (+ adapt when tau or n_fixed is given) + solve.  Returns (model, adapt_result,
    pcg_result).  n_fixed: the n_fixed dominant eigenvectors per face (Section 7, "3eigv")."""
    m = Model(prob, averages=averages)
    m.schur()
    ad = adapt(m, tau, n_fixed=n_fixed) if (tau is not None or n_fixed is not None) else None
    res = m.solve(tol=tol, maxit=maxit)
    return m, ad, res
