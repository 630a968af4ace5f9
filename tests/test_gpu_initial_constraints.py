"""Adaptive constraints on top of initial averages (the c+e and c+e+f starts of
Section 7): the pair problems are restricted to jumps that satisfy the initial
glob constraints shared by the pair (the projection Pi_ij of Section 3, Pi != I),
and the face rows are d = w^T Pi L Pi.  Per-face eigenvalues, selected and kept
counts, the total, omega, iterations and kappa against the oracle."""
import numpy as np
import pytest

from paper_0910_5863_gb300 import problems as P
from paper_0910_5863_gb300 import bddc as B
import oracle

pytestmark = pytest.mark.gpu

TOL_LAM = 1e-6

CASES = {
    "poisson12_edge": (lambda: P.poisson_cube(12, 2, coef="random_high", seed=2), ("edge",), 2.0),
    "poisson12_edge_face": (lambda: P.poisson_cube(12, 2, coef="random_high", seed=2), ("edge", "face"), 2.0),
    "elast6_edge": (lambda: P.elasticity_cube(6, 2, channels=2, seed=3), ("edge",), 10.0),
}


@pytest.mark.parametrize("prec", [B.FP64, B.MIXED])
@pytest.mark.parametrize("case", sorted(CASES))
def test_adaptive_with_initial_averages(case, prec):
    make, av, tau = CASES[case]
    prob = make()
    m = oracle.Model(prob, averages=av)
    m.schur()
    ad = oracle.adapt(m, tau)
    res = m.solve(tol=1e-8)
    s = B.Solver(precision=prec)
    s.set_mesh_problem(prob)
    s.set_averages(edge="edge" in av, face="face" in av)
    s.setup()
    info = s.adapt(tau)
    assert info["n_ties"] == 0
    for f, key in enumerate(sorted(ad.pairs)):
        g = s.face_eigs(f)
        r = ad.pairs[key]
        assert g["pair"] == key
        assert g["selected"] == r.selected, (key, g["lam"][:4], r.lam[:4])
        assert g["kept"] == ad.per_face[key]
        n = min(len(g["lam"]), r.selected + 1)
        assert np.allclose(g["lam"][:n], r.lam[:n], rtol=TOL_LAM), (key, g["lam"][:n], r.lam[:n])
    assert info["n_added"] == ad.n_added
    assert abs(info["omega"] - ad.omega) <= TOL_LAM * ad.omega
    u, sinfo = s.solve(B.free_load_vector(prob))
    assert abs(sinfo["iters"] - res.iters) <= 1
    kr = res.condition()[1] / res.condition()[0]
    assert abs(sinfo["kappa"] - kr) <= 0.01 * kr
    assert np.linalg.norm(u - res.u) <= 1e-7 * np.linalg.norm(res.u)


CASES_FIXED = {
    # Section 7's "c+e+f (3eigv)": corners, arithmetic edge averages, three dominant
    # eigenvector constraints per face
    "elast6_edge_3eigv": (lambda: P.elasticity_cube(6, 2, channels=2, seed=3), ("edge",), 3),
    "poisson12_edge_3eigv": (lambda: P.poisson_cube(12, 2, coef="random_high", seed=2), ("edge",), 3),
    "poisson10_corners_2eigv": (lambda: P.poisson_cube(10, 2, coef="lognormal", seed=4), (), 2),
}


@pytest.mark.parametrize("prec", [B.FP64, B.MIXED])
@pytest.mark.parametrize("case", sorted(CASES_FIXED))
def test_fixed_number_of_eigenvectors_per_face(case, prec):
    make, av, k = CASES_FIXED[case]
    prob = make()
    m = oracle.Model(prob, averages=av)
    m.schur()
    ad = oracle.adapt(m, tau=None, n_fixed=k)
    res = m.solve(tol=1e-8)
    s = B.Solver(precision=prec)
    s.set_mesh_problem(prob)
    s.set_averages(edge="edge" in av, face="face" in av)
    s.setup()
    info = s.adapt_fixed(k)
    assert info["n_ties"] == 0 and all(r.ties == 0 for r in ad.pairs.values())
    for f, key in enumerate(sorted(ad.pairs)):
        g = s.face_eigs(f)
        r = ad.pairs[key]
        assert g["pair"] == key
        assert g["selected"] == r.selected == min(k, r.lam.size)
        assert g["kept"] == ad.per_face[key]
        n = min(len(g["lam"]), r.selected + 1)
        assert np.allclose(g["lam"][:n], r.lam[:n], rtol=TOL_LAM), (key, g["lam"][:n], r.lam[:n])
    assert info["n_added"] == ad.n_added
    assert abs(info["omega"] - ad.omega) <= TOL_LAM * ad.omega
    u, sinfo = s.solve(B.free_load_vector(prob))
    assert abs(sinfo["iters"] - res.iters) <= 1
    kr = res.condition()[1] / res.condition()[0]
    assert abs(sinfo["kappa"] - kr) <= 0.01 * kr
    assert np.linalg.norm(u - res.u) <= 1e-7 * np.linalg.norm(res.u)
