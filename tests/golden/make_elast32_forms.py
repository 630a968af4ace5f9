"""Writes tests/golden/elast32_forms.txt: the oracle's PCG iteration counts (relative residual
1e-8) on the 32^3 elasticity problem with 8 stiff channels (E = 1e6, adaptive constraints for
lambda > 10) with two forms of the same preconditioner: the saddle point of Lemma 2.1 and the
primal form after the generalized change of variables of Section 5 (oracle/change_of_variables.py).
Equal in exact arithmetic; at this conditioning (kappa ~ 7.5e3) their rounding gives different
counts, which measures how far the count of any FP64 implementation can move.  Calls the oracle
only:

    python tests/golden/make_elast32_forms.py
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from paper_0910_5863_gb300 import problems as P  # noqa: E402
import oracle  # noqa: E402
from oracle.bddc import pcg  # noqa: E402
from oracle.change_of_variables import TransformedBDDC  # noqa: E402


def main():
    m = oracle.Model(P.config_elasticity_channels())
    m.schur()
    oracle.adapt(m, 10.0)
    g = m.condensed_rhs()
    lemma = pcg(m.apply_S, m.apply_M, g, 1e-8, 1000)
    cv = TransformedBDDC(m, transform="qr", form="primal")
    primal = pcg(m.apply_S, cv.apply, g, 1e-8, 1000)
    with open(os.path.join(HERE, "elast32_forms.txt"), "w") as f:
        f.write("# Oracle, 32^3 Q1 elasticity, 8 channels E = 1e6 (seed 1), tau = 10, PCG to 1e-8:\n")
        f.write("# iterations with the Lemma 2.1 saddle-point form and with the Section 5 primal form\n")
        f.write("# of the same preconditioner (written by make_elast32_forms.py).\n")
        f.write(f"iters_lemma {lemma.iters}\n")
        f.write(f"iters_primal {primal.iters}\n")


if __name__ == "__main__":
    main()
