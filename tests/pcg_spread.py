"""Iteration-count spread of the oracle's PCG under rounding-level perturbations.

At condition numbers around 1e4 the number of PCG iterations needed for a
relative residual of 1e-8 moves by several units when every S_i is perturbed by
a symmetric relative 1e-13 (the size of the rounding error with which any
FP64 code forms S_i).  Iteration counts of another FP64-accurate implementation
are compared against that spread instead of a fixed +-1 there.  Test helper; it
uses the oracle only."""
import numpy as np


def perturbed_iteration_range(m, tol=1e-8, seeds=8, delta=1e-13):
    """(lo, hi) of the oracle's iteration count over the unperturbed run and
    `seeds` runs with S_i -> S_i + delta ||S_i|| E_i / ||E_i||, E_i symmetric
    Gaussian.  m: an oracle Model with its Schur complements formed."""
    S0 = [s.S.copy() for s in m.subs]
    m._M = None
    its = [m.solve(tol=tol).iters]
    try:
        for seed in range(seeds):
            rng = np.random.default_rng(seed)
            for s, S in zip(m.subs, S0):
                E = rng.standard_normal(S.shape)
                E = E + E.T
                s.S = S + delta * np.linalg.norm(S) / np.linalg.norm(E) * E
            m._M = None
            its.append(m.solve(tol=tol).iters)
    finally:
        for s, S in zip(m.subs, S0):
            s.S = S
        m._M = None
    return min(its), max(its)


def iterations_agree(it, m, kappa, tol=1e-8):
    """+-1 of the oracle where kappa <= 1e3.  Above, the oracle's own count moves
    over [lo, hi] when its S_i are perturbed at the rounding level (16 seeds);
    the count must lie in that range widened on both sides by its width (at
    least 1): another FP64-accurate implementation differs from the oracle by
    such perturbations, and 16 samples do not reach the ends of the range."""
    if kappa <= 1e3:
        lo, hi = perturbed_iteration_range(m, tol, seeds=0)
        return lo - 1 <= it <= hi + 1
    lo, hi = perturbed_iteration_range(m, tol, seeds=16, delta=1e-12)
    w = max(1, hi - lo)
    return lo - w <= it <= hi + w


def perturbed_rows_iteration_range(m, tol=1e-8, seeds=8, delta=1e-9):
    """(lo, hi) of the oracle's iteration count over the unperturbed run and `seeds` runs
    with every adaptive constraint row r -> r + delta |r| e / |e|, e Gaussian: the
    preconditioner then moves by ~delta, the size of the difference between two FP64
    implementations whose face eigenvectors agree to that level."""
    saved = [(g, g.rows.copy()) for g in m.constraints if g.kind.startswith("adaptive")]
    m._M = None
    its = [m.solve(tol=tol).iters]
    try:
        for seed in range(seeds):
            rng = np.random.default_rng(1000 + seed)
            for g, R in saved:
                E = rng.standard_normal(R.shape)
                g.rows = R + delta * (np.linalg.norm(R, axis=1, keepdims=True) * E
                                      / np.linalg.norm(E, axis=1, keepdims=True))
            m._M = None
            its.append(m.solve(tol=tol).iters)
    finally:
        for g, R in saved:
            g.rows = R
        m._M = None
    return min(its), max(its)
