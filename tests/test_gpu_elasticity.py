"""Elasticity at full size: 32^3 Q1 elements, 4x4x4 substructures, 8 stiff channels
(E = 1e6), clamped at z = 0, tau = 10, FP64 and mixed paths.  The oracle is
too slow for every face pair at this size, so parity is checked on sampled
faces (eigenvalues and constraint counts) and through properties that hold at
any size (global residual, FP64 vs mixed agreement, iteration counts)."""
import numpy as np
import pytest

from paper_0910_5863_gb300 import problems as P
from paper_0910_5863_gb300 import bddc as B
import oracle
from oracle.adaptive import pair_problem, orthonormal_rows

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def elast():
    prob = P.config_elasticity_channels()
    m = oracle.Model(prob)
    m.schur()
    runs = {}
    for prec in (B.FP64, B.MIXED):
        s = B.Solver(precision=prec, tol=1e-10)
        s.set_mesh_problem(prob)
        s.setup()
        info = s.adapt(10.0)
        u, sinfo = s.solve(B.free_load_vector(prob))
        runs[prec] = (s, info, u, sinfo)
    return prob, m, runs


def test_sizes(elast):
    prob, m, runs = elast
    sz = runs[B.FP64][0].sizes()
    assert (sz["n_corners"], sz["n_edges"], sz["n_faces"]) == m.globs.counts()
    assert sz["n_free"] == m.dofs.n == 104544


def test_global_residual_and_agreement(elast):
    prob, m, runs = elast
    F = m.F
    for prec, (s, info, u, sinfo) in runs.items():
        assert sinfo["converged"]
        assert np.linalg.norm(m.K @ u - F) <= 1e-7 * np.linalg.norm(F), prec
    u64, u32 = runs[B.FP64][2], runs[B.MIXED][2]
    assert np.linalg.norm(u64 - u32) <= 1e-8 * np.linalg.norm(u64)
    # kappa ~ 7.5e3 after adaptivity here (the face-only constraints do not bound the
    # channels crossing edges).  At that conditioning the count depends on the rounding of
    # the preconditioner: the oracle's own two forms of the same preconditioner need 108 and
    # 132 iterations to 1e-8 (tests/golden/elast32_forms.txt), 22% apart, while
    # rounding-level changes of the S_i move one form's count by 3 (tests/pcg_spread.py).
    # FP64 and mixed (double-float factorizations, 2^-48) are held to 10% of each other.
    it64, it32 = runs[B.FP64][3]["iters"], runs[B.MIXED][3]["iters"]
    assert abs(it64 - it32) <= max(3, round(0.1 * it64)), (it64, it32)
    assert runs[B.MIXED][3]["interior_fp32"]
    assert runs[B.FP64][1]["n_added"] == runs[B.MIXED][1]["n_added"]


@pytest.mark.parametrize("pick", [0, 71])
def test_sampled_face_eigs(elast, pick):
    prob, m, runs = elast
    keys = sorted(m.globs.faces)
    i, j = keys[pick]
    ref = pair_problem(m, i, j, 10.0)
    kept = orthonormal_rows(ref.face_rows).shape[0] if ref.selected else 0
    for prec, (s, info, u, sinfo) in runs.items():
        g = s.face_eigs(pick)
        assert g["pair"] == (i, j)
        assert g["selected"] == ref.selected and g["kept"] == kept
        n = min(len(g["lam"]), ref.selected + 1)
        assert np.allclose(g["lam"][:n], ref.lam[:n], rtol=1e-6), (prec, g["lam"][:n], ref.lam[:n])
