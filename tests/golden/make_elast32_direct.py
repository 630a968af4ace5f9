"""Writes tests/golden/elast32_direct.txt: how close the oracle's own FP64 solution of the 32^3
elasticity problem (8 channels with E = 1e6, adaptive constraints for lambda > 10, PCG to a
relative residual of 1e-13) comes to the sparse direct solution with one refinement step, the
reference that tests/test_gpu_full_size.py compares the library's solution with.  At this
contrast FP64 solutions stop near that distance whatever the PCG tolerance (the global
residual's floor).  Calls the oracle (and scipy's sparse LU) only:

    python tests/golden/make_elast32_direct.py
"""
import os
import sys

import numpy as np
import scipy.sparse.linalg as spla

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from paper_0910_5863_gb300 import problems as P  # noqa: E402
import oracle  # noqa: E402


def main():
    m = oracle.Model(P.config_elasticity_channels())
    K = m.K.tocsc()
    lu = spla.splu(K)
    u0 = lu.solve(m.F)
    u_ref = u0 + lu.solve(m.F - K @ u0)
    m.schur()
    oracle.adapt(m, 10.0)
    res = m.solve(tol=1e-13)
    err = np.linalg.norm(res.u - u_ref) / np.linalg.norm(u_ref)
    glob = np.linalg.norm(K @ res.u - m.F) / np.linalg.norm(m.F)
    with open(os.path.join(HERE, "elast32_direct.txt"), "w") as f:
        f.write("# Oracle, 32^3 Q1 elasticity, 8 channels E = 1e6 (seed 1), tau = 10, PCG to 1e-13:\n")
        f.write("# relative distance of its solution to the sparse LU solution with one refinement step,\n")
        f.write("# and its global residual |K u - F| / |F| (written by make_elast32_direct.py).\n")
        f.write(f"oracle_u_err {err:.6e}\n")
        f.write(f"oracle_global_residual {glob:.6e}\n")


if __name__ == "__main__":
    main()
