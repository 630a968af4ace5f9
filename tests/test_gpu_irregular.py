"""Irregular substructures at full size: 48 x 48 x 24 elasticity split into 64
substructures by seeded region growing (rough interfaces, 424 face pairs, floating
substructures that need augmented corners), E in {1, 1e3} by z-layers of height 4,
clamped at z = 0, tau = 10, FP64 and mixed paths.  The oracle classifies the whole
mesh and solves sampled pair problems (its Schur complements of only the two
substructures involved); the rest is checked through properties that hold at any
size."""
import numpy as np
import pytest

from paper_0910_5863_gb300 import problems as P
from paper_0910_5863_gb300 import bddc as B
import oracle
from oracle.adaptive import pair_problem, orthonormal_rows
from test_gpu_parity import check_face_rows

pytestmark = pytest.mark.gpu

TAU = 10.0
# Eigenvalues (the selected ones and the next) and the spans of the face rows against the
# oracle, both paths at 1e-6 on every face.
TOL_LAM = {B.FP64: 1e-6, B.MIXED: 1e-6}
TOL_SPAN = {B.FP64: 1e-6, B.MIXED: 1e-6}


@pytest.fixture(scope="module")
def irregular():
    prob = P.config_irregular_elasticity()
    m = oracle.Model(prob)
    runs = {}
    for prec in (B.FP64, B.MIXED):
        s = B.Solver(precision=prec, tol=1e-8)
        s.set_mesh_problem(prob)
        s.setup()
        info = s.adapt(TAU)
        u, sinfo = s.solve(B.free_load_vector(prob))
        runs[prec] = (s, info, u, sinfo)
    return prob, m, runs


def test_classification(irregular):
    prob, m, runs = irregular
    for prec, (s, info, u, sinfo) in runs.items():
        sz = s.sizes()
        assert (sz["n_corners"], sz["n_edges"], sz["n_faces"]) == m.globs.counts()
        assert list(s.corners()) == m.globs.corners


def test_solution_and_agreement(irregular):
    prob, m, runs = irregular
    F = m.F
    for prec, (s, info, u, sinfo) in runs.items():
        assert sinfo["converged"]
        assert np.linalg.norm(m.K @ u - F) <= 1e-7 * np.linalg.norm(F), prec
    u64, u32 = runs[B.FP64][2], runs[B.MIXED][2]
    assert np.linalg.norm(u64 - u32) <= 1e-8 * np.linalg.norm(u64)
    assert runs[B.FP64][1]["n_added"] == runs[B.MIXED][1]["n_added"]
    assert abs(runs[B.FP64][3]["iters"] - runs[B.MIXED][3]["iters"]) <= 3


def test_face_rows_orthonormal_and_counts(irregular):
    """Every face's kept rows are orthonormal in both precisions, and both paths
    select and keep the same number of rows on every face."""
    prob, m, runs = irregular
    nf = runs[B.FP64][1]["n_faces"]
    for f in range(nf):
        counts = []
        for prec, (s, info, u, sinfo) in runs.items():
            g = s.face_eigs(f)
            gd, rows = s.face_rows(f)
            assert rows.shape[0] == g["kept"] <= gd.size
            if g["kept"]:
                assert np.abs(rows @ rows.T - np.eye(g["kept"])).max() < 1e-10, (prec, f)
            counts.append((g["selected"], g["kept"]))
        assert counts[0] == counts[1], (f, counts)


def _sampled_faces(m):
    """Faces at the 5/8, 1/2 and 1/8 quantiles of the face size: the oracle's dense
    Jacobi on the condensed 2 n_s pencil takes seconds there (the largest faces,
    2 n_s ~ 1700, take many minutes)."""
    keys = sorted(m.globs.faces)
    sizes = [len(m.globs.faces[k]) for k in keys]
    order = np.argsort(sizes, kind="stable")
    return [int(order[5 * len(order) // 8]), int(order[len(order) // 2]), int(order[len(order) // 8])]


def test_sampled_face_eigs(irregular):
    prob, m, runs = irregular
    keys = sorted(m.globs.faces)
    for f in _sampled_faces(m):
        i, j = keys[f]
        subs = m.subs
        m.subs = [subs[i], subs[j]]
        try:
            m.schur()
        finally:
            m.subs = subs
        ref = pair_problem(m, i, j, TAU)
        kept = orthonormal_rows(ref.face_rows).shape[0] if ref.selected else 0
        for prec, (s, info, u, sinfo) in runs.items():
            g = s.face_eigs(f)
            assert g["pair"] == (i, j)
            assert g["selected"] == ref.selected and g["kept"] == kept, (prec, f, g["lam"][:4], ref.lam[:4])
            n = min(len(g["lam"]), ref.selected + 1)
            assert np.allclose(g["lam"][:n], ref.lam[:n], rtol=TOL_LAM[prec]), (prec, f)
            check_face_rows(s, f, ref, m, tol_span=TOL_SPAN[prec])
