"""Failure detection without a GPU fault: the bounded grid barrier of the PCG
kernel is made to wait for a block that does not exist.  The wait must give up
after its limit, report BDDC_ETIMEOUT through the status word, let every block
return, and leave the CUDA context usable for a normal solve afterwards."""
import time

import numpy as np
import pytest

from paper_0910_5863_gb300 import problems as P
from paper_0910_5863_gb300 import bddc as B

pytestmark = pytest.mark.gpu


def test_barrier_passes_and_times_out():
    import torch
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    s = B.Solver(precision=B.FP64, tol=1e-8)
    assert s.barrier_selftest(0, 1.0) == ("OK", nsm)
    t0 = time.perf_counter()
    status, passed = s.barrier_selftest(1, 0.2)
    dt = time.perf_counter() - t0
    assert status == "ETIMEOUT" and passed == 0
    assert 0.15 < dt < 5.0, dt
    # the context and the handle stay usable
    assert s.barrier_selftest(0, 1.0) == ("OK", nsm)
    prob = P.poisson_cube(8, 2, coef="random_high", seed=5)
    s.set_mesh_problem(prob)
    s.setup()
    u, info = s.solve(B.free_load_vector(prob))
    assert info["converged"] and np.all(np.isfinite(u))
