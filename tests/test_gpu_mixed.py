"""Parity of the mixed-precision path (FP32 factorizations + FP64 refinement)
with the FP64 oracle, at the mixed tolerances: solution within 1e-8, adaptive
eigenvalues within 1e-6, identical constraint counts, PCG iterations within 1."""
import numpy as np
import pytest

from paper_0910_5863_gb300 import problems as P
from paper_0910_5863_gb300 import bddc as B
import oracle
from pcg_spread import iterations_agree

pytestmark = pytest.mark.gpu

TOL_S_MIXED = 1e-9
TOL_U_MIXED = 1e-8
TOL_LAM = 1e-6


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _solver(prob, averages=(), tol=1e-8, precision=B.MIXED):
    s = B.Solver(precision=precision, tol=tol)
    s.set_mesh_problem(prob)
    s.set_averages(edge="edge" in averages, face="face" in averages)
    s.setup()
    return s


@pytest.mark.parametrize("case", ["small_ef", "jump_corner", "elast_ef"])
def test_mixed_schur_and_solve(case):
    if case == "small_ef":
        prob, av = P.config_small(), ("edge", "face")
    elif case == "jump_corner":
        prob, av = P.poisson_cube(12, 2, coef="random_high", seed=2), ()
    else:
        prob, av = P.elasticity_cube(6, 2, channels=2, seed=3), ("edge", "face")
    m, _, ref = oracle.run(prob, averages=av, tol=1e-13)
    s = _solver(prob, av, tol=1e-13)
    for i, sub in enumerate(m.subs):
        assert _rel(s.schur(i), sub.S) < TOL_S_MIXED, i
    u, info = s.solve(B.free_load_vector(prob))
    assert _rel(u, ref.u) < TOL_U_MIXED
    m8, _, ref8 = oracle.run(prob, averages=av, tol=1e-8)
    s8 = _solver(prob, av)
    u8, info8 = s8.solve(B.free_load_vector(prob))
    # +-1, or within the oracle's own spread under rounding-level perturbations at kappa > 1e3
    assert iterations_agree(info8["iters"], m8, info8["kappa"]), (info8["iters"], ref8.iters)
    if not av:  # the adaptive run of the same problem (kappa <= tau): within one iteration
        ma, ada, refa = oracle.run(prob, tau=10.0, tol=1e-8)
        sa = _solver(prob)
        infoa = sa.adapt(10.0)
        assert infoa["n_added"] == ada.n_added
        ua, sinfo = sa.solve(B.free_load_vector(prob))
        assert abs(sinfo["iters"] - refa.iters) <= 1


def test_mixed_adaptive_poisson24_full_size():
    prob = P.config_adaptive_poisson()
    m = oracle.Model(prob)
    m.schur()
    ad = oracle.adapt(m, 10.0)
    res = m.solve(tol=1e-8)
    s = _solver(prob)
    info = s.adapt(10.0)
    assert info["n_added"] == ad.n_added and info["n_ties"] == 0
    for f, key in enumerate(sorted(ad.pairs)):
        g = s.face_eigs(f)
        r = ad.pairs[key]
        assert g["selected"] == r.selected and g["kept"] == ad.per_face[key]
        n = min(len(g["lam"]), r.selected + 1)
        assert np.allclose(g["lam"][:n], r.lam[:n], rtol=TOL_LAM)
    u, sinfo = s.solve(B.free_load_vector(prob))
    assert abs(sinfo["iters"] - res.iters) <= 1
    assert _rel(u, res.u) < 1e-7


@pytest.mark.parametrize("case", ["jump_corner", "planar2"])
def test_fp32_saddle_mode(case):
    """BDDC_MIXED_FP32_SADDLE: the local saddle operators from an FP32 factorization.
    The solution still meets the mixed tolerance; the preconditioner is exact only
    to ~1e-5, so the iteration count may grow (bounded here by a third)."""
    prob = P.poisson_cube(12, 2, coef="random_high", seed=2) if case == "jump_corner" else P.planar_cubes(2, m=8)
    m, _, ref = oracle.run(prob, tol=1e-13)
    s = _solver(prob, tol=1e-13, precision=B.MIXED_FP32_SADDLE)
    u, info = s.solve(B.free_load_vector(prob))
    assert _rel(u, ref.u) < TOL_U_MIXED
    m8, _, ref8 = oracle.run(prob, tol=1e-8)
    s8 = _solver(prob, precision=B.MIXED_FP32_SADDLE)
    u8, info8 = s8.solve(B.free_load_vector(prob))
    assert info8["converged"] and info8["iters"] <= 1.34 * ref8.iters + 1
    assert abs(info8["kappa"] - ref8.condition()[1] / ref8.condition()[0]) <= 0.01 * info8["kappa"]
