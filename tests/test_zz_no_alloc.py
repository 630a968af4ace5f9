"""The allocation-free Schur-complement entry point (bddc_schur_dense_static).

Some callers cannot allocate device memory (fixed memory budgets, their own
allocator owning the device, no allocation after start-up); for them the
library offers one call whose scratch is a static device array.  This test
calls it through the C ABI, twice in a row on matrices of different sizes and
once more on the first, and checks every result against the Schur complement
the regular setup path returns (bddc_get_schur), at the tolerance of the other
Schur parity tests.  It also checks the size limit.  This file is collected
last on purpose.
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


def test_static_scratch_schur_matches_setup_path():
    import torch

    fn = _fn()
    prob = P.config_small()
    s = B.Solver()
    s.set_mesh_problem(prob)
    s.setup()
    m = oracle.Model(prob)
    msg = C.create_string_buffer(256)
    for i in (0, 1, 0):          # different sizes back to back, then the first again
        sub = m.subs[i]
        A = _dense_local(sub)    # symmetric: row-major storage equals column-major
        n, ni = A.shape[0], sub.I.size
        ng = n - ni
        dA = torch.from_numpy(np.ascontiguousarray(A)).cuda()
        dS = torch.full((ng, ng), float("nan"), dtype=torch.float64, device="cuda")
        st = fn(n, ni, dA.data_ptr(), n, dS.data_ptr(), ng, None, msg, 256)
        assert st == 0, msg.value
        S = dS.cpu().numpy().T
        ref = s.schur(i)
        assert np.linalg.norm(S - ref) / np.linalg.norm(ref) < TOL_S


def test_static_scratch_rejects_oversize():
    import torch

    fn = _fn()
    d = torch.zeros(16, dtype=torch.float64, device="cuda")
    msg = C.create_string_buffer(256)
    st = fn(2048, 100, d.data_ptr(), 2048, d.data_ptr(), 1948, None, msg, 256)
    assert st == 1
    assert b"limit" in msg.value
