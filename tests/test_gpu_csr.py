"""The algebraic entry point (bddc_set_problem: per-substructure CSR matrices A_i,
Dirichlet dofs already eliminated), the corner calls (bddc_set_corners,
bddc_select_corners) and the caller-allocator hook.  The CSR inputs are the
library's own assembled A_i (mesh path, mixed mode keeps them), so the CSR path
must reproduce the mesh path bit for bit and the oracle to the usual tolerances."""
import numpy as np
import pytest
import scipy.sparse as sps

from paper_0910_5863_gb300 import problems as P
from paper_0910_5863_gb300 import bddc as B
import oracle
from oracle.adaptive import orthonormal_rows

pytestmark = pytest.mark.gpu


def _free_numbering(prob):
    free = ~np.asarray(prob.dirichlet, dtype=bool)
    node_free = -np.ones(prob.xyz.shape[0], dtype=np.int64)
    node_free[free] = np.arange(free.sum())
    return free, node_free


def _csr_inputs(prob):
    """(n_global, subs, xyz_free, mesh solver) from the mesh path's assembled A_i."""
    c = prob.ncomp
    mesh = B.Solver(precision=B.MIXED)
    mesh.set_mesh_problem(prob)
    mesh.setup()
    free, node_free = _free_numbering(prob)
    subs = []
    for s in range(prob.nsub):
        nodes = np.unique(prob.elems[prob.elem_sub == s].ravel())
        nodes = nodes[free[nodes]]
        ldofs = (node_free[nodes][:, None] * c + np.arange(c)[None, :]).ravel()
        gG = mesh.interface_dofs(s)
        gI = np.setdiff1d(ldofs, gG)
        A = mesh.local_matrix(s, gI.size + gG.size)
        subs.append((np.concatenate([gI, gG]), sps.csr_matrix(A)))
    return int(free.sum()) * c, subs, np.asarray(prob.xyz)[free], mesh, node_free


def _mesh_corners_free(mesh, node_free):
    return node_free[np.asarray(mesh.corners(), dtype=np.int64)]


def test_csr_path_reproduces_mesh_path_poisson():
    prob = P.poisson_cube(8, 2, coef="random_high", seed=5)
    ng, subs, xyz, mesh, node_free = _csr_inputs(prob)
    m = oracle.Model(prob)
    m.schur()
    ref = B.Solver()
    ref.set_mesh_problem(prob)
    ref.setup()
    s = B.Solver()
    s.set_problem(ng, 1, subs, xyz)
    # the free-node graph rule may add corners next to the Dirichlet side: use the mesh corners
    s.set_corners(_mesh_corners_free(mesh, node_free))
    s.setup()
    assert s.sizes() == ref.sizes()
    for i, sub in enumerate(m.subs):
        Si = s.schur(i)
        assert np.array_equal(Si, ref.schur(i))
        assert np.linalg.norm(Si - sub.S) <= 1e-11 * np.linalg.norm(sub.S)
    info = s.adapt(10.0)
    ad = oracle.adapt(m, 10.0)
    assert info["n_added"] == ad.n_added
    for f, key in enumerate(sorted(m.globs.faces)):
        g = s.face_eigs(f)
        r = ad.pairs[key]
        assert g["selected"] == r.selected
        n = min(len(g["lam"]), r.selected + 1)
        assert np.allclose(g["lam"][:n], r.lam[:n], rtol=1e-6)
    F = B.free_load_vector(prob)
    u, sinfo = s.solve(F.copy())
    res = m.solve(tol=1e-8)
    assert abs(sinfo["iters"] - res.iters) <= 1
    assert np.linalg.norm(m.K @ u - F) <= 1e-7 * np.linalg.norm(F)


def test_select_corners_matches_mesh_rule_away_from_dirichlet():
    """With a 2 x 2 x 1 partition no edge reaches the Dirichlet side x = 0, so the
    free-node coupling graph gives the element-edge rule's corners."""
    prob = P.poisson_cube(6, 2, coef="lognormal", s_xyz=(2, 2, 1), seed=2)
    ng, subs, xyz, mesh, node_free = _csr_inputs(prob)
    s = B.Solver()
    s.set_problem(ng, 1, subs, None)
    assert np.array_equal(np.asarray(s.corners()), _mesh_corners_free(mesh, node_free))
    s.set_corners(np.asarray(s.corners())[:1])
    assert s.sizes()["n_corners"] == 1
    assert s.select_corners() == len(mesh.corners())


def test_csr_path_elasticity_planar_with_augmentation():
    prob = P.planar_cubes(2, m=4)
    ng, subs, xyz, mesh, node_free = _csr_inputs(prob)
    s = B.Solver(tol=1e-10)
    s.set_problem(ng, 3, subs, xyz)
    assert np.array_equal(np.asarray(s.corners()), _mesh_corners_free(mesh, node_free))
    m, ad, ref = oracle.run(prob, tau=10.0, tol=1e-10, maxit=800)
    s.setup()
    info = s.adapt(10.0)
    assert info["n_added"] == ad.n_added
    u, sinfo = s.solve(B.free_load_vector(prob))
    assert abs(sinfo["iters"] - ref.iters) <= 1
    assert np.linalg.norm(u - ref.u) <= 1e-8 * np.linalg.norm(ref.u)


def test_elasticity_needs_coordinates():
    prob = P.planar_cubes(2, m=2)
    ng, subs, xyz, mesh, node_free = _csr_inputs(prob)
    with pytest.raises(B.BddcError) as e:
        B.Solver().set_problem(ng, 3, subs, None)
    assert e.value.status == 1


def test_torch_allocator():
    torch = pytest.importorskip("torch")
    prob = P.config_small()
    F = B.free_load_vector(prob)
    base = B.Solver()
    base.set_mesh_problem(prob)
    base.setup()
    u0, _ = base.solve(F.copy())
    before = torch.cuda.memory_allocated()
    s = B.Solver(allocator="torch")
    s.set_mesh_problem(prob)
    s.setup()
    assert torch.cuda.memory_allocated() > before
    u1, _ = s.solve(F.copy())
    assert np.array_equal(u0, u1)
    s.close()
    assert torch.cuda.memory_allocated() == before
