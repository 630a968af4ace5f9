"""Writes tests/golden/elast32_pcg.txt: the oracle's adaptive BDDC on the 32^3 elasticity
problem with 8 stiff channels (64 substructures, corners + adaptive face constraints for
lambda > 10, PCG to 1e-8): the number of added constraints, the PCG iterations and the
Lanczos condition estimate, and the spread of the iteration count when every S_i is
perturbed at the rounding level and when every adaptive row is perturbed at 1e-9
(tests/pcg_spread.py).  Calls the oracle only:

    python tests/golden/make_elast32_pcg.py [--seeds N]
"""
import argparse
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.dirname(HERE))

from paper_0910_5863_gb300 import problems as P  # noqa: E402
import oracle  # noqa: E402
from pcg_spread import perturbed_iteration_range, perturbed_rows_iteration_range  # noqa: E402


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--seeds", type=int, default=8)
    args = ap.parse_args()
    m = oracle.Model(P.config_elasticity_channels())
    m.schur()
    ad = oracle.adapt(m, 10.0)
    res = m.solve(tol=1e-8)
    lmin, lmax = res.condition()
    lo, hi = perturbed_iteration_range(m, tol=1e-8, seeds=args.seeds, delta=1e-12)
    rlo, rhi = perturbed_rows_iteration_range(m, tol=1e-8, seeds=args.seeds, delta=1e-9)
    with open(os.path.join(HERE, "elast32_pcg.txt"), "w") as f:
        f.write("# Oracle, 32^3 Q1 elasticity, 4x4x4 substructures, 8 channels E = 1e6 (seed 1), tau = 10,\n")
        f.write("# PCG to relative residual 1e-8 (written by make_elast32_pcg.py).  iters_lo / iters_hi:\n")
        f.write(f"# the iteration range over {args.seeds} rounding-level perturbations of the S_i (1e-12);\n")
        f.write("# rows_lo / rows_hi: the range when every adaptive row is perturbed by 1e-9 relative.\n")
        f.write(f"n_added {ad.n_added}\n")
        f.write(f"iters {res.iters}\n")
        f.write(f"kappa {lmax / lmin:.10g}\n")
        f.write(f"iters_lo {lo}\n")
        f.write(f"iters_hi {hi}\n")
        f.write(f"rows_lo {rlo}\n")
        f.write(f"rows_hi {rhi}\n")


if __name__ == "__main__":
    main()
