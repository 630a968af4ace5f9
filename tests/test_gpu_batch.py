"""The batched workload: independent Poisson problems (2^3 or 3^3 cubic
substructures of 6^3..10^3 elements, lognormal coefficients sigma = 2,
adaptive tau = 10) solved by concurrent library handles on separate streams
(paper_0910_5863_gb300.batch).  Sampled problems are checked against the
oracle; the concurrent run must reproduce a one-worker run bit for bit (the
handles share nothing and every reduction is deterministic)."""
import numpy as np
import pytest

from paper_0910_5863_gb300 import problems as P
from paper_0910_5863_gb300 import bddc as B
import oracle
from pcg_spread import iterations_agree

pytestmark = pytest.mark.gpu

TAU = 10.0


def _sample():
    probs = P.config_batch_poisson()
    dofs = [int((~p.dirichlet).sum()) for p in probs]
    order = np.argsort(dofs, kind="stable")
    pick = [int(order[0]), int(order[len(order) // 2]), int(order[-1])]
    return [probs[i] for i in pick] + probs[:5]


@pytest.fixture(scope="module")
def runs():
    import torch
    from paper_0910_5863_gb300 import batch as BT
    probs = _sample()
    arrays = BT.upload(probs, torch.device("cuda", 0))
    out = {}
    for prec in (B.FP64, B.MIXED):
        _, conc = BT.run(probs, arrays, BT.Pool(prec, workers=4), tau=TAU, keep_solutions=True)
        _, seq = BT.run(probs, arrays, BT.Pool(prec, workers=1), tau=TAU, keep_solutions=True)
        out[prec] = (conc, seq)
    return probs, out


def test_concurrent_equals_sequential(runs):
    probs, out = runs
    for prec, (conc, seq) in out.items():
        for a, b in zip(conc, seq):
            assert a["iters"] == b["iters"] and a["n_added"] == b["n_added"]
            assert np.array_equal(a["u"].cpu().numpy(), b["u"].cpu().numpy()), prec


def test_sampled_against_oracle(runs):
    probs, out = runs
    for k, prob in enumerate(probs[:3]):
        m, ad, ref = oracle.run(prob, tau=TAU, tol=1e-8)
        for prec, (conc, _) in out.items():
            r = conc[k]
            assert r["converged"]
            assert r["n_added"] == ad.n_added, (prob.name, prec, r["n_added"], ad.n_added)
            u = r["u"].cpu().numpy()
            assert np.linalg.norm(m.K @ u - m.F) <= 1e-7 * np.linalg.norm(m.F), (prob.name, prec)
            assert iterations_agree(r["iters"], m, r["kappa"]), (prob.name, prec, r["iters"], ref.iters)
