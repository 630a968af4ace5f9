"""Pins of the oracle's generalized change of variables (Section 5) against what the
paper and the mathematics fix: the paper's worked example of T for one unit average
(eq. TB-example-general), the defining identities of H and T (eqs.
general-change-variables, T), the +1 / -1 structure of D-bar^c, the invariance of the
BDDC operator under the change of basis (the same constrained space and energy, so the
same M as the Lemma 2.1 saddle-point oracle), the independence of the regularisation t
(eq. BDDC-regular) and the lower fill-in of the projected operator."""
import numpy as np
import pytest

from paper_0910_5863_gb300 import problems as P
import oracle
from oracle.change_of_variables import TransformedBDDC, glob_transform, glob_rows, significant_nnz

EPS = np.finfo(float).eps


def _model(which):
    """(model, coefficient contrast) with S_i formed and the constraints in place."""
    if which == "small_cef":
        m = oracle.Model(P.config_small(), averages=("edge", "face"))
        m.schur()
        return m, 1.0
    if which == "poisson_adaptive_face":
        m = oracle.Model(P.poisson_cube(6, 2, coef="random_high", seed=5), averages=("face",))
        m.schur()
        oracle.adapt(m, 10.0)
        return m, 1e4
    if which == "elast_adaptive_edge":
        m = oracle.Model(P.elasticity_cube(4, 2, channels=1, seed=3), averages=("edge",))
        m.schur()
        oracle.adapt(m, 10.0)
        return m, 1e6
    raise ValueError(which)


def test_T_of_one_unit_average_is_the_papers_example():
    """One average with unit weights: U = [1], K = I, H = [[1, 1, ..., 1], [0, I]] and
    T = [[1, -1, ..., -1], [0, I]] (eq. TB-example-general)."""
    n = 6
    g = glob_transform(np.ones((1, n)))
    assert g.r == 1 and list(g.piv) == list(range(n))
    H = np.eye(n)
    H[0, :] = 1.0
    T = np.eye(n)
    T[0, 1:] = -1.0
    assert np.array_equal(g.H(), H)
    assert np.array_equal(g.T(), T)


def test_H_T_identity_and_averages_on_the_explicit_dofs_only():
    """T is the inverse of H, and in the new variables every average (also a dependent
    one, dropped by the rank rule) depends on the r explicit dofs only:
    H^avg T = Q [I, 0] by eqs. (general-change-variables) and (T)."""
    rng = np.random.default_rng(7)
    n = 11
    A = rng.standard_normal((2, n))
    Havg = np.vstack([A, 0.3 * A[0] - 2.0 * A[1], rng.standard_normal((1, n))])  # rank 3 of 4
    g = glob_transform(Havg)
    assert g.r == 3
    T = g.T()
    assert np.allclose(g.H() @ T, np.eye(n), atol=1e-12)
    assert np.all(np.diag(g.U) > 0)
    HT = Havg @ T
    assert np.abs(HT[:, g.r:]).max() < 1e-12 * np.abs(Havg).max()
    # the explicit part is Q: orthonormal columns spanning the rows' coefficient space
    Qr = HT[:, : g.r]
    assert np.allclose(Qr.T @ Qr, np.eye(g.r), atol=1e-12)


@pytest.mark.parametrize("which", ["small_cef", "poisson_adaptive_face", "elast_adaptive_edge"])
def test_every_form_equals_the_lemma21_preconditioner(which):
    """The change of basis keeps the constrained space and the energy, so the saddle
    form (eq. BDDC-ch-var), the projected form (eq. A-tilde) and the primal form (the
    Remark closing Section 5) give the Lemma 2.1 operator M.  Tolerance: rounding
    amplified by the coefficient contrast, 10 eps x contrast, at least 1e-12."""
    m, contrast = _model(which)
    tol = max(1e-12, 10 * EPS * contrast)
    rng = np.random.default_rng(3)
    R = rng.standard_normal((m.nG, 3))
    ref = np.column_stack([m.apply_M(R[:, k]) for k in range(3)])
    for tr, form in [("qr", "saddle"), ("qr", "projected"), ("qr", "primal"), ("identity", "projected")]:
        M = TransformedBDDC(m, transform=tr, form=form)
        got = np.column_stack([M.apply(R[:, k]) for k in range(3)])
        err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert err < tol, (which, tr, form, err)


def test_constraints_after_the_change_couple_two_explicit_dofs():
    """Each row of D-bar^c has one +1 and one -1, both on explicit dofs, and T maps
    the null space of D-bar^c into the null space of D^c (Section 5)."""
    m, _ = _model("poisson_adaptive_face")
    qr = TransformedBDDC(m, transform="qr", form="projected")
    ident = TransformedBDDC(m, transform="identity", form="projected")
    D = qr.D.tocsr()
    for q in range(D.shape[0]):
        vals = sorted(D.data[D.indptr[q]:D.indptr[q + 1]])
        assert vals == [-1.0, 1.0]
    # the two forms number W^c alike: corners shared, every other dof per substructure
    assert all(np.array_equal(a, b) for a, b in zip(qr.wc, ident.wc))
    rng = np.random.default_rng(5)
    wbar = qr.Pi @ rng.standard_normal(qr.nwc)          # a vector of null(D-bar)
    assert np.abs(D @ wbar).max() < 1e-12 * np.abs(wbar).max()
    w = np.zeros(qr.nwc)
    for i in range(len(m.subs)):
        w[qr.wc[i]] = qr.T[i] @ wbar[qr.wc[i]]          # T R^c w-bar (T_i = I on corners)
    assert np.abs(ident.D @ w).max() < 1e-11 * np.abs(w).max()


def test_dependent_averages_are_dropped():
    """Every face average given twice: the pivoted QR keeps one row per face, and M is
    unchanged (the dependent-row rule)."""
    prob = P.config_small()
    a = oracle.Model(prob, averages=("face",))
    b = oracle.Model(prob, averages=("face", "face"))
    a.schur()
    b.schur()
    assert sum(C.shape[0] for _, _, C in glob_rows(b)) == 2 * sum(C.shape[0] for _, _, C in glob_rows(a))
    Ma, Mb = TransformedBDDC(a, form="primal"), TransformedBDDC(b, form="primal")
    assert Ma.n_explicit == Mb.n_explicit == len(a.globs.faces)
    r = np.random.default_rng(2).standard_normal(a.nG)
    assert np.linalg.norm(Ma.apply(r) - Mb.apply(r)) < 1e-12 * np.linalg.norm(Ma.apply(r))


def test_projected_form_does_not_depend_on_t():
    """Any t > 0 gives the same solution of eq. (BDDC-regular)."""
    m, _ = _model("small_cef")
    r = np.random.default_rng(4).standard_normal(m.nG)
    u1 = TransformedBDDC(m, form="projected", t=1.0).apply(r)
    u2 = TransformedBDDC(m, form="projected").apply(r)          # t = max diag(A^c)
    assert np.linalg.norm(u1 - u2) < 1e-11 * np.linalg.norm(u2)


def test_change_of_variables_lowers_the_fill_in():
    """With corners and edge and face averages, the projected operator after the
    change of variables has far fewer entries than Pi A^c Pi + t (I - Pi) in the
    original variables (Section 5, Figure of the projected matrices)."""
    m, _ = _model("small_cef")
    nnz_cov = significant_nnz(TransformedBDDC(m, transform="qr", form="projected").Atilde)
    nnz_plain = significant_nnz(TransformedBDDC(m, transform="identity", form="projected").Atilde)
    assert nnz_cov < 0.5 * nnz_plain, (nnz_cov, nnz_plain)
