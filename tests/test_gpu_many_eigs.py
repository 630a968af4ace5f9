"""A face with more selected eigenvalues than the face kernel's first pass forms (48): the
library redoes such a face with room for all of them (Algorithm 3.1 keeps every eigenvector
above tau).  On the 8^3 elasticity problem with two stiff channels, tau = 1.001 selects 59
eigenvalues on one face (the next one down is 1.00072, so no eigenvalue lies within 1e-6 of
tau).  Every face's selected and kept counts, its eigenvalues (the selected ones and the next)
and its rows are checked against the oracle, and the solve with all these constraints still
converges."""
import numpy as np
import pytest

from paper_0910_5863_gb300 import problems as P
from paper_0910_5863_gb300 import bddc as B
import oracle
from test_gpu_parity import check_face_rows

pytestmark = pytest.mark.gpu

TAU = 1.001
TOL_LAM = 1e-6


@pytest.fixture(scope="module")
def ref():
    prob = P.elasticity_cube(8, 2, channels=2, seed=3)
    m = oracle.Model(prob)
    m.schur()
    ad = oracle.adapt(m, TAU)
    return prob, m, ad


@pytest.mark.parametrize("prec", [B.FP64, B.MIXED])
def test_more_than_48_selected_on_a_face(ref, prec):
    prob, m, ad = ref
    assert max(r.selected for r in ad.pairs.values()) > 48
    s = B.Solver(precision=prec, tol=1e-8)
    s.set_mesh_problem(prob)
    s.setup()
    info = s.adapt(TAU)
    assert info["n_ties"] == 0
    assert info["n_added"] == ad.n_added
    for f, key in enumerate(sorted(ad.pairs)):
        g = s.face_eigs(f)
        r = ad.pairs[key]
        assert g["pair"] == key
        assert g["selected"] == r.selected and g["kept"] == ad.per_face[key], (prec, key, g["selected"])
        n = min(len(g["lam"]), r.selected + 1)
        assert n == min(len(r.lam), r.selected + 1)
        assert np.allclose(g["lam"][:n], r.lam[:n], rtol=TOL_LAM), (prec, key)
        check_face_rows(s, f, r, m)
    u, sinfo = s.solve(B.free_load_vector(prob))
    assert sinfo["converged"] and sinfo["relres"] < 1.5e-8
