"""The allocation-free Schur-complement entry point (bddc_schur_dense_static).

Some callers cannot allocate device memory (fixed memory budgets, their own
allocator owning the device, no allocation after start-up); for them the
library offers one call whose scratch is a static device array.  These tests
call it through the C ABI:
  * twice in a row on substructure matrices of different sizes and once more on
    the first, each result against the Schur complement the regular setup path
    returns (bddc_get_schur) and against the oracle's Schur complement of that
    substructure, at the tolerance of the other FP64 Schur parity tests;
  * on a dense SPD matrix near the size limit with padded leading dimensions,
    against the plain definition A_GG - A_GI A_II^-1 A_IG;
  * with no interior (S = A) and with an indefinite A_II (BDDC_ENOTSPD, after
    which the next call succeeds);
  * with the device's free memory unchanged across its second and third calls;
  * and the size limit.
This file is collected last on purpose.
"""
import ctypes as C

import numpy as np
import pytest

from paper_0910_5863_gb300 import bddc as B
from paper_0910_5863_gb300 import problems as P
import oracle

pytestmark = pytest.mark.gpu

TOL_S = 1e-11


def _dense_local(sub):
    """A_i ordered [interior; interface] (both ascending in global dof), as the library orders it."""
    perm = np.concatenate([sub.I, sub.G])
    return sub.A.toarray()[np.ix_(perm, perm)]


def _fn():
    lib = B.load()
    f = lib.bddc_schur_dense_static
    f.restype = C.c_int
    f.argtypes = [C.c_int, C.c_int, C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.c_void_p, C.c_char_p, C.c_int]
    return f


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _call(fn, A, ni, lda=None, lds=None):
    """Runs the entry point on the symmetric matrix A (numpy); returns (status, S, message)."""
    import torch

    n = A.shape[0]
    ng = n - ni
    lda = lda or n
    lds = lds or ng
    dA = torch.zeros((n, lda), dtype=torch.float64, device="cuda")   # column c at row c of this array
    dA[:, :n] = torch.from_numpy(np.ascontiguousarray(A.T))
    dS = torch.full((max(ng, 1), lds), float("nan"), dtype=torch.float64, device="cuda")
    msg = C.create_string_buffer(256)
    st = fn(n, ni, dA.data_ptr(), lda, dS.data_ptr(), lds, None, msg, 256)
    S = dS[:ng, :ng].cpu().numpy().T   # column-major result, column j at dS[j]
    return st, S, msg.value


def test_static_scratch_schur_matches_setup_path_and_oracle():
    fn = _fn()
    prob = P.config_small()
    s = B.Solver()
    s.set_mesh_problem(prob)
    s.setup()
    m = oracle.Model(prob)
    m.schur()
    for i in (0, 1, 0):          # different sizes back to back, then the first again
        sub = m.subs[i]
        st, S, msg = _call(fn, _dense_local(sub), sub.I.size)
        assert st == 0, msg
        assert _rel(S, s.schur(i)) < TOL_S, i
        assert _rel(S, sub.S) < TOL_S, i


def test_static_scratch_near_the_limit_with_padding():
    fn = _fn()
    rng = np.random.default_rng(1)
    n, ni = 1000, 640
    Bm = rng.standard_normal((n, n))
    A = Bm @ Bm.T / n + np.eye(n)
    st, S, msg = _call(fn, A, ni, lda=1008, lds=n - ni + 24)
    assert st == 0, msg
    AII, AIG, AGG = A[:ni, :ni], A[:ni, ni:], A[ni:, ni:]
    ref = AGG - AIG.T @ np.linalg.solve(AII, AIG)
    assert _rel(S, ref) < TOL_S


def test_static_scratch_no_interior_and_indefinite():
    fn = _fn()
    rng = np.random.default_rng(2)
    n = 40
    Bm = rng.standard_normal((n, n))
    A = Bm @ Bm.T + n * np.eye(n)
    st, S, msg = _call(fn, A, 0)
    assert st == 0, msg
    assert np.abs(S - A).max() <= 1e-15 * np.abs(A).max()
    bad = A.copy()
    bad[5, :] = 0.0
    bad[:, 5] = 0.0
    bad[5, 5] = -1.0
    st, _, msg = _call(fn, bad, 20)
    assert st == 3, (st, msg)             # BDDC_ENOTSPD
    st, S, msg = _call(fn, A, 20)         # the shared scratch is usable again
    assert st == 0, msg
    ref = A[20:, 20:] - A[:20, 20:].T @ np.linalg.solve(A[:20, :20], A[:20, 20:])
    assert _rel(S, ref) < TOL_S


def test_static_scratch_allocates_nothing():
    import torch

    fn = _fn()
    rng = np.random.default_rng(3)
    n, ni = 300, 200
    Bm = rng.standard_normal((n, n))
    A = Bm @ Bm.T / n + np.eye(n)
    dA = torch.from_numpy(np.ascontiguousarray(A)).cuda()
    dS = torch.zeros((n - ni, n - ni), dtype=torch.float64, device="cuda")
    msg = C.create_string_buffer(256)
    assert fn(n, ni, dA.data_ptr(), n, dS.data_ptr(), n - ni, None, msg, 256) == 0, msg.value  # first call
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(2):
        assert fn(n, ni, dA.data_ptr(), n, dS.data_ptr(), n - ni, None, msg, 256) == 0, msg.value
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_static_scratch_rejects_oversize():
    import torch

    fn = _fn()
    d = torch.zeros(16, dtype=torch.float64, device="cuda")
    msg = C.create_string_buffer(256)
    st = fn(2048, 100, d.data_ptr(), 2048, d.data_ptr(), 1948, None, msg, 256)
    assert st == 1
    assert b"limit" in msg.value
