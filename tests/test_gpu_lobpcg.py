"""Batched LOBPCG for the large face-pair eigenproblems (Section 3 names LOBPCG for the
pair problems).  Faces whose reduced problem is larger than the eig_large_n option run
LOBPCG with a Cholesky certificate of the selected count; the rest run the dense kernel.

  * against the FP64 oracle (dense Jacobi on the 2 n_s pencil): every face of the 24^3
    Poisson jump problem and of a 12^3 elasticity channel problem forced onto LOBPCG
    (eig_large_n = 48), both precisions, with the oracle tolerances of the dense path;
  * against the library's dense kernel on the 48 x 48 x 24 irregular elasticity problem,
    with the faces above order 160 (up to ~1000 dofs) on LOBPCG."""
import numpy as np
import pytest

from paper_0910_5863_gb300 import problems as P
from paper_0910_5863_gb300 import bddc as B
import oracle
from test_gpu_parity import _check_adaptive

pytestmark = pytest.mark.gpu

TAU = 10.0
CASES = {
    "poisson24_jumps": P.config_adaptive_poisson,
    "elast12_channels_3x3x3": lambda: P.elasticity_cube(12, 3, channels=3, seed=1),
}


@pytest.fixture(scope="module")
def oracle_runs():
    out = {}
    for name, make in CASES.items():
        prob = make()
        m = oracle.Model(prob)
        m.schur()
        ad = oracle.adapt(m, TAU)
        res = m.solve(tol=1e-8)
        out[name] = (prob, m, ad, res)
    return out


@pytest.mark.parametrize("prec", [B.FP64, B.MIXED])
@pytest.mark.parametrize("case", sorted(CASES))
def test_lobpcg_faces_match_the_oracle(oracle_runs, case, prec):
    prob, m, ad, res = oracle_runs[case]
    s = B.Solver(precision=prec, tol=1e-8, eig_large_n=48)
    s.set_mesh_problem(prob)
    s.setup()
    info = s.adapt(TAU)
    # faces of order above 48 run LOBPCG (the trial space [X P R] of 3 x 16 columns)
    n_large = sum(1 for r in ad.pairs.values() if r.s_gdofs.size > 48)
    assert info["n_lobpcg"] == n_large > 0.5 * info["n_faces"]
    # a face whose iteration stalls or whose certificate fails goes to the dense kernel
    assert info["n_dense_fallback"] <= info["n_lobpcg"] // 4
    assert info["lobpcg_iters"] > 0
    _check_adaptive(m, ad, res, s, info, prob)


def _span_gap(a, b):
    if a.shape[0] == 0 and b.shape[0] == 0:
        return 0.0
    return np.linalg.norm(a.T @ a - b.T @ b, 2)


def test_irregular_lobpcg_against_the_dense_kernel():
    prob = P.config_irregular_elasticity()
    runs = {}
    for large_n in (160, -1):
        s = B.Solver(precision=B.FP64, tol=1e-8, eig_large_n=large_n)
        s.set_mesh_problem(prob)
        s.setup()
        runs[large_n] = (s, s.adapt(TAU))
    (sl, il), (sd, idn) = runs[160], runs[-1]
    assert il["n_lobpcg"] > 0 and il["n_dense_fallback"] <= il["n_lobpcg"] // 4 and idn["n_lobpcg"] == 0
    assert il["n_added"] == idn["n_added"] and il["n_ties"] == idn["n_ties"] == 0
    assert abs(il["omega"] - idn["omega"]) <= 1e-8 * idn["omega"]
    for f in range(il["n_faces"]):
        gl, gd = sl.face_eigs(f), sd.face_eigs(f)
        assert (gl["selected"], gl["kept"]) == (gd["selected"], gd["kept"]), f
        n = min(len(gl["lam"]), len(gd["lam"]))
        assert np.allclose(gl["lam"][:n], gd["lam"][:n], rtol=1e-8, atol=0.0), (f, gl["lam"][:n], gd["lam"][:n])
        assert _span_gap(sl.face_rows(f)[1], sd.face_rows(f)[1]) <= 1e-6, f
