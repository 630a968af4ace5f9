"""Parity of the CUDA library (through the C ABI) with the FP64 CPU oracle."""
import numpy as np
import pytest

from paper_0910_5863_gb300 import problems as P
from paper_0910_5863_gb300 import bddc as B
import oracle
from oracle.adaptive import orthonormal_rows

pytestmark = pytest.mark.gpu

TOL_S = 1e-11        # Schur complements, FP64 path
TOL_U = 1e-10        # solution with PCG driven to 1e-13 (FP64 path)
TOL_LAM = 1e-6       # adaptive eigenvalues, relative


def _solver(prob, averages=(), tol=1e-8):
    s = B.Solver(tol=tol)
    s.set_mesh_problem(prob)
    s.set_averages(edge="edge" in averages, face="face" in averages)
    s.setup()
    return s


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.fixture(scope="module")
def small():
    prob = P.config_small()
    m = oracle.Model(prob, averages=("edge", "face"))
    m.schur()
    return prob, m


def test_classification_matches(small):
    prob, m = small
    s = _solver(prob, ("edge", "face"))
    sz = s.sizes()
    assert (sz["n_corners"], sz["n_edges"], sz["n_faces"]) == m.globs.counts()
    assert sz["n_interface"] == m.nG and sz["n_free"] == m.dofs.n
    assert list(s.corners()) == list(m.globs.corners)
    assert sz["n_coarse"] == m.n_coarse()


def test_schur_complements(small):
    prob, m = small
    s = _solver(prob, ("edge", "face"))
    for i, sub in enumerate(m.subs):
        assert np.array_equal(s.interface_dofs(i), sub.gdof[sub.G])
        assert _rel(s.schur(i), sub.S) < TOL_S


def test_operators(small):
    prob, m = small
    s = _solver(prob, ("edge", "face"))
    rng = np.random.default_rng(0)
    for _ in range(3):
        x = rng.standard_normal(m.nG)
        assert _rel(s.apply_schur(x), m.apply_S(x)) < 1e-12
        assert _rel(s.apply_preconditioner(x), m.apply_M(x)) < 1e-10


@pytest.mark.parametrize("case", ["small_ef", "small_corner_lognormal", "elast_ef"])
def test_solve(case):
    if case == "small_ef":
        prob, av = P.config_small(), ("edge", "face")
    elif case == "small_corner_lognormal":
        prob, av = P.poisson_cube(10, 2, coef="lognormal", seed=4), ()
    else:
        prob, av = P.elasticity_cube(6, 2), ("edge", "face")
    m, _, ref = oracle.run(prob, averages=av, tol=1e-13)
    s = _solver(prob, av, tol=1e-13)
    u, info = s.solve(B.free_load_vector(prob))
    assert _rel(u, ref.u) < TOL_U
    m8, _, ref8 = oracle.run(prob, averages=av, tol=1e-8)
    s8 = _solver(prob, av, tol=1e-8)
    u8, info8 = s8.solve(B.free_load_vector(prob))
    assert abs(info8["iters"] - ref8.iters) <= 1
    k_ref = ref8.condition()[1] / ref8.condition()[0]
    assert abs(info8["kappa"] - k_ref) <= 0.01 * k_ref


@pytest.mark.parametrize("prec", [B.FP64, B.MIXED])
def test_zero_load_gives_zero_solution(prec):
    """The degenerate right-hand side f = 0: the solution of K u = 0 is u = 0, PCG stops
    before its first iteration (r_0 = 0) and reports a zero residual; with no Lanczos
    coefficients the condition estimate is 1."""
    prob = P.config_small()
    s = B.Solver(precision=prec, tol=1e-8)
    s.set_mesh_problem(prob)
    s.setup()
    s.adapt(10.0)
    f = B.free_load_vector(prob)
    u = np.full_like(f, np.nan)            # every entry must be written by the solve
    u, info = s.solve(np.zeros_like(f), u=u)
    assert np.all(u == 0.0)
    assert info["converged"] and info["iters"] == 0
    assert info["relres"] == 0.0 and info["kappa"] == 1.0
    # the handle solves a nonzero load normally afterwards
    u1, info1 = s.solve(f)
    assert info1["converged"] and info1["iters"] > 0 and np.linalg.norm(u1) > 0


@pytest.mark.parametrize("prec,tol_u", [(B.FP64, 1e-8), (B.MIXED, 1e-6)])
def test_iteration_limit_returns_the_iterate(prec, tol_u):
    """PCG stopped by its iteration limit: BDDC_ENOCONV, and the solution returned is the one
    recovered from the third iterate, as the oracle's PCG stopped after three steps gives it.
    The iterate is about as sensitive as the operators (perturbing the oracle's S and M by
    eps moves it by ~eps), so the bounds are 100x the operators' accuracy on each path."""
    prob = P.config_small()
    av = ("edge", "face")
    m, _, ref = oracle.run(prob, averages=av, tol=1e-14, maxit=3)
    assert not ref.converged and ref.iters == 3
    s = B.Solver(precision=prec, tol=1e-14, maxit=3)
    s.set_mesh_problem(prob)
    s.set_averages(edge=True, face=True)
    s.setup()
    u, info = s.solve(B.free_load_vector(prob), check=False)
    assert info["status"] == "ENOCONV" and not info["converged"] and info["iters"] == 3
    assert _rel(u, ref.u) < tol_u
    with pytest.raises(B.BddcError) as e:
        s.solve(B.free_load_vector(prob))
    assert e.value.status == 5


@pytest.mark.parametrize("prec", [B.FP64, B.MIXED])
def test_non_finite_load_is_a_bad_argument(prec):
    """A NaN or an infinity in the load gives BDDC_EINVAL (not a zero residual), and the handle
    then solves a finite load as before."""
    prob = P.config_small()
    s = B.Solver(precision=prec, tol=1e-8)
    s.set_mesh_problem(prob)
    s.setup()
    f = B.free_load_vector(prob)
    for bad in (np.nan, np.inf):
        g = f.copy()
        g[len(g) // 2] = bad
        with pytest.raises(B.BddcError) as e:
            s.solve(g)
        assert e.value.status == 1
    u, info = s.solve(f)
    assert info["converged"] and np.all(np.isfinite(u))


def _adaptive_case(prob, tau=10.0):
    m = oracle.Model(prob)
    m.schur()
    ad = oracle.adapt(m, tau)
    res = m.solve(tol=1e-8)
    s = _solver(prob)
    info = s.adapt(tau)
    return m, ad, res, s, info


@pytest.mark.parametrize("case", ["poisson12_jump", "elast6"])
def test_adaptive_small(case):
    if case == "poisson12_jump":
        prob = P.poisson_cube(12, 2, coef="random_high", seed=2)
    else:
        prob = P.elasticity_cube(6, 2, channels=2, seed=3)
    m, ad, res, s, info = _adaptive_case(prob)
    _check_adaptive(m, ad, res, s, info, prob)


def _check_adaptive(m, ad, res, s, info, prob):
    assert info["n_faces"] == len(ad.pairs)
    assert info["n_ties"] == 0
    for f, key in enumerate(sorted(ad.pairs)):
        g = s.face_eigs(f)
        r = ad.pairs[key]
        assert g["pair"] == key
        assert g["selected"] == r.selected, (key, g, r.lam[:6])
        assert g["kept"] == ad.per_face[key]
        n = min(len(g["lam"]), r.selected + 1)
        assert np.allclose(g["lam"][:n], r.lam[:n], rtol=TOL_LAM), (key, g["lam"][:n], r.lam[:n])
        check_face_rows(s, f, r, m)
    assert info["n_added"] == ad.n_added
    assert abs(info["omega"] - ad.omega) <= TOL_LAM * ad.omega
    u, sinfo = s.solve(B.free_load_vector(prob))
    assert abs(sinfo["iters"] - res.iters) <= 1
    kr = res.condition()[1] / res.condition()[0]
    assert abs(sinfo["kappa"] - kr) <= 0.01 * kr
    assert _rel(u, res.u) < 1e-7


def check_face_rows(s, f, r, m, tol_span=1e-6):
    """The kept rows of face f are orthonormal, live on the oracle's face dofs and
    span the oracle's row space.  The span is as well determined as the normalised
    face rows are independent, so its tolerance is divided by their smallest
    singular value."""
    gd, rows = s.face_rows(f)
    if r.selected == 0:
        assert rows.shape[0] == 0
        return
    face_g = np.sort(m.dofs.of_nodes(np.asarray(r.face_nodes)).ravel())
    assert np.array_equal(gd, face_g)
    assert np.abs(rows @ rows.T - np.eye(rows.shape[0])).max() < 1e-10
    ref = orthonormal_rows(r.face_rows)
    assert rows.shape[0] == ref.shape[0]
    nrm = r.face_rows / np.linalg.norm(r.face_rows, axis=1, keepdims=True)
    sv = np.linalg.svd(nrm, compute_uv=False)
    smin = sv[ref.shape[0] - 1]
    gap = np.linalg.norm(rows.T @ rows - ref.T @ ref, 2)
    assert gap <= tol_span / smin, (f, gap, smin)


def test_adaptive_poisson24_full_size():
    """The 24^3, 27-substructure jump problem timed by the benchmark."""
    prob = P.config_adaptive_poisson()
    m, ad, res, s, info = _adaptive_case(prob)
    _check_adaptive(m, ad, res, s, info, prob)


def test_errors_are_statuses():
    prob = P.poisson_cube(4, 2, s_xyz=(2, 1, 1))
    prob.dirichlet[:] = False
    s = B.Solver()
    s.set_mesh_problem(prob)           # the augmentation gives the floating pair a corner
    assert s.sizes()["n_corners"] == 1
    with pytest.raises(B.BddcError) as e:
        s.set_corners([])              # floating substructures without corners
    assert e.value.status == 4
    s2 = B.Solver()
    with pytest.raises(B.BddcError) as e:
        s2.solve(np.zeros(3))
    assert e.value.status == 8
