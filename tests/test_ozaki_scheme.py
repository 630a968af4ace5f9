"""The numerical scheme of the tensor-core trailing updates C -= L L^T of the double-float
factorizations (exact digit slicing, after Ozaki, Ogita, Oishi and Rump), emulated in NumPy on
the CPU so that the design's arithmetic claims are checked independently of the kernel:

  * each row of a 128-column block is scaled by 2^-e (e from the row's largest entry, so the
    scaled row lies in (-1, 1)) and written as sum_{p <= 7} d_p 2^-7p with integer digits,
    |d_1| <= 128 and |d_p| <= 64 after it, so every digit is exact in bf16;
  * a product of two digit planes summed over 128 columns stays below 2^24, so the FP32
    accumulators of the tensor cores hold it exactly whatever the summation order;
  * keeping the products with p + q <= 8 leaves an error below 2^-40 2^(e_i + e_j) per entry;
  * the row exponent from the row's own maximum keeps the update accurate relative to |L||L|^T
    on the 32^3 channel problem (E contrast 1e6), where exponents from the Cholesky bound
    |L_ij| <= sqrt(a_ii) would lose about three digits of that componentwise accuracy.
The kernel itself is checked against the oracle through the GPU parity tests."""
import numpy as np

from paper_0910_5863_gb300 import problems as P
import oracle

SLICES = 7
BITS = 7
K = 128


def _split(X, e):
    """Digit planes of the rows of X scaled by 2^-e (|x| 2^-e < 1), each digit rounded to
    nearest from the remainder left by the previous ones."""
    R = X * np.exp2(-e)[:, None]
    planes = []
    for p in range(1, SLICES + 1):
        d = np.rint(R * 2.0 ** (BITS * p))
        planes.append(d)
        R = R - d * 2.0 ** (-BITS * p)
    return planes


def _product(A, ea, B, eb):
    """sum over p + q <= SLICES + 1 of 2^-7(p+q) A_p B_q^T, scaled back (float64: the digit
    products and their sums over K columns are integers below 2^53, so exact)."""
    out = np.zeros((A[0].shape[0], B[0].shape[0]))
    for p in range(1, SLICES + 1):
        for q in range(1, SLICES + 2 - p):
            out += (A[p - 1] @ B[q - 1].T) * 2.0 ** (-BITS * (p + q))
    return out * np.exp2(ea)[:, None] * np.exp2(eb)[None, :]


def _row_exponent(X):
    _, e = np.frexp(np.abs(X).max(axis=1))   # max = f 2^e with f in [0.5, 1)
    return e.astype(np.float64)


def _random_block(rng, rows):
    # rows of very different magnitudes, some with a dominant entry
    X = rng.standard_normal((rows, K)) * np.exp2(rng.integers(-30, 30, size=rows))[:, None]
    X[::7, 3] *= 1e6
    return X


def test_digits_are_bf16_exact_and_their_sums_fp32_exact():
    rng = np.random.default_rng(11)
    X = _random_block(rng, 256)
    e = _row_exponent(X)
    assert np.all(np.abs(X) * np.exp2(-e)[:, None] < 1.0)
    planes = _split(X, e)
    assert np.abs(planes[0]).max() <= 128 and all(np.abs(d).max() <= 64 for d in planes[1:])
    # an integer of at most 8 significant bits is exact in bf16 (8-bit significand)
    for d in planes:
        assert np.all(np.abs(d) <= 256) and np.array_equal(d, np.rint(d))
    # |sum_k d_p(i, k) d_q(j, k)| <= 128 * 128 * 128 = 2^21 < 2^24 for every pair of planes
    for p in range(SLICES):
        for q in range(SLICES - p):
            assert (np.abs(planes[p]) @ np.abs(planes[q]).T).max() < 2 ** 24


def test_dropped_products_stay_below_2_to_minus_40():
    rng = np.random.default_rng(12)
    X = _random_block(rng, 192)
    Y = _random_block(rng, 96)
    ex, ey = _row_exponent(X), _row_exponent(Y)
    approx = _product(_split(X, ex), ex, _split(Y, ey), ey)
    exact = X @ Y.T
    err = np.abs(approx - exact) / (np.exp2(ex)[:, None] * np.exp2(ey)[None, :])
    assert err.max() < 2.0 ** -40, err.max()
    # the seventh plane matters: without it on each side the error grows about 2^7-fold
    X6 = _split(X, ex)[:SLICES - 1] + [np.zeros_like(X)]
    Y6 = _split(Y, ey)[:SLICES - 1] + [np.zeros_like(Y)]
    err6 = np.abs(_product(X6, ex, Y6, ey) - exact) / (np.exp2(ex)[:, None] * np.exp2(ey)[None, :])
    assert err6.max() > 16 * err.max()


def _channel_factor():
    """Cholesky factor of S_rr (S_i without its corner dofs, the matrix the local saddle
    factors) of the largest-interior substructure of the 32^3 channel problem whose S_rr is
    definite."""
    prob = P.config_elasticity_channels()
    m = oracle.Model(prob)
    subs = m.subs
    big = [int(k) for k in np.argsort([s.I.size for s in subs])[-6:]]
    m.subs = [subs[k] for k in big]
    m.schur()
    cdofs = set(np.asarray(m.dofs.of_nodes(np.asarray(sorted(m.globs.corners)))).ravel().tolist())
    for sub in sorted(m.subs, key=lambda s: -s.S.shape[0]):
        g = sub.gdof[sub.G]
        r = np.array([k for k in range(len(g)) if int(g[k]) not in cdofs])
        try:
            return np.linalg.cholesky(sub.S[np.ix_(r, r)])
        except np.linalg.LinAlgError:
            continue
    raise AssertionError("no definite S_rr")


def test_row_maximum_exponents_keep_componentwise_accuracy():
    L = _channel_factor()
    Lb = L[:, :K]                              # the first 128-wide block column
    exact = Lb @ Lb.T
    mag = np.abs(Lb) @ np.abs(Lb).T
    a = np.sum(L ** 2, axis=1)                 # the diagonal before this block column
    e_row = _row_exponent(Lb)
    _, e_bound = np.frexp(np.sqrt(a))          # |L_ij| <= sqrt(a_ii)
    e_bound = e_bound.astype(np.float64)
    assert np.all(e_row <= e_bound)
    rel = {}
    for name, e in (("row", e_row), ("bound", e_bound)):
        pl = _split(Lb, e)
        err = np.abs(_product(pl, e, pl, e) - exact)
        rel[name] = (err / np.maximum(mag, 1e-300)).max()
        # both stay at the scale of Cholesky's normwise error bound
        assert (err / np.sqrt(np.outer(a, a))).max() < 1e-12
    assert rel["row"] < 1e-8, rel
    assert rel["bound"] > 100 * rel["row"], rel
