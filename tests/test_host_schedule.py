"""The host schedule of the PCG local products (csrc/schedule.h, bin_by_cost): the 64-row
blocks of S_i and P~_i are grouped into one bin per SM by longest-processing-time-first
greedy scheduling.  Checked on the CPU (the header is plain C++, compiled here with g++):
a worked example and Graham's tight instance, his (4/3 - 1/(3m)) bound against brute-force
optima on small instances, the output's structure (a permutation, the given order within a
bin), degenerate inputs, and the balance it gives on the 48 x 48 x 24 irregular partition."""
import itertools
import os
import shutil
import subprocess

import numpy as np
import pytest

from paper_0910_5863_gb300 import problems as P
from oracle.globs import Globs

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                    "paper_0910_5863_gb300", "csrc")

DRIVER = r"""
#include <cstdio>
#include "schedule.h"
// stdin: T, then per instance nbins k c_0 .. c_{k-1}; stdout per instance: the bin
// pointers, then the item indices bin by bin.
int main() {
    int T;
    if (scanf("%d", &T) != 1) return 1;
    while (T--) {
        int nbins, k;
        if (scanf("%d %d", &nbins, &k) != 2) return 1;
        std::vector<long long> c(k);
        std::vector<int> items(k);
        for (int i = 0; i < k; ++i) { if (scanf("%lld", &c[i]) != 1) return 1; items[i] = i; }
        std::vector<int> out, ptr;
        bddc::bin_by_cost(items, [&](int i) { return (int64_t)c[i]; }, nbins, out, ptr);
        for (size_t b = 0; b < ptr.size(); ++b) printf("%d ", ptr[b]);
        printf("\n");
        for (int i : out) printf("%d ", i);
        printf("\n");
    }
    return 0;
}
"""


@pytest.fixture(scope="module")
def binner(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("g++ not available")
    d = tmp_path_factory.mktemp("sched")
    src, exe = d / "drv.cpp", d / "drv"
    src.write_text(DRIVER)
    subprocess.run(["g++", "-std=c++17", "-O1", "-I", CSRC, "-o", str(exe), str(src)], check=True)

    def run(instances):
        """instances: list of (nbins, costs) -> list of (binptr, order)."""
        lines = [str(len(instances))]
        for m, c in instances:
            lines.append(f"{m} {len(c)} " + " ".join(str(int(x)) for x in c))
        out = subprocess.run([str(exe)], input="\n".join(lines) + "\n", capture_output=True,
                             text=True, check=True).stdout.split("\n")
        res = []
        for t in range(len(instances)):
            ptr = [int(x) for x in out[2 * t].split()]
            order = [int(x) for x in out[2 * t + 1].split()]
            res.append((ptr, order))
        return res
    return run


def _loads(ptr, order, c):
    return [sum(c[i] for i in order[ptr[b]:ptr[b + 1]]) for b in range(len(ptr) - 1)]


def _check_structure(m, c, ptr, order):
    assert len(ptr) == max(m, 1) + 1 and ptr[0] == 0 and ptr[-1] == len(c)
    assert all(ptr[b] <= ptr[b + 1] for b in range(len(ptr) - 1))
    assert sorted(order) == list(range(len(c)))
    for b in range(len(ptr) - 1):
        seg = order[ptr[b]:ptr[b + 1]]
        assert seg == sorted(seg)          # the items' given order within a bin


def test_worked_example(binner):
    # costs 5 4 3 3 3 on two bins: 5 -> bin 0, 4 -> bin 1, 3 -> bin 1 (4 < 5), 3 -> bin 0
    # (5 < 7), 3 -> bin 1 (7 < 8): loads 8 and 10, where {5, 4} / {3, 3, 3} gives 9
    c = [5, 4, 3, 3, 3]
    (ptr, order), = binner([(2, c)])
    assert ptr == [0, 2, 5] and order == [0, 3, 1, 2, 4]
    assert _loads(ptr, order, c) == [8, 10]


def test_graham_tight_instance(binner):
    # 3 3 2 2 2 on two bins: LPT gives 7 against the optimum 6 = 7/6 of it, Graham's bound
    # 4/3 - 1/(3m) at m = 2 reached exactly
    c = [3, 3, 2, 2, 2]
    (ptr, order), = binner([(2, c)])
    assert max(_loads(ptr, order, c)) == 7


def test_bound_against_brute_force(binner):
    rng = np.random.default_rng(5)
    inst = []
    for _ in range(120):
        m = int(rng.integers(2, 4))
        k = int(rng.integers(1, 8))
        inst.append((m, [int(x) for x in rng.integers(0, 20, size=k)]))
    for (m, c), (ptr, order) in zip(inst, binner(inst)):
        _check_structure(m, c, ptr, order)
        opt = min(max(sum(c[i] for i in range(len(c)) if a[i] == b) for b in range(m))
                  for a in itertools.product(range(m), repeat=len(c)))
        assert max(_loads(ptr, order, c)) * 3 * m <= (4 * m - 1) * opt, (m, c)


def test_degenerate_inputs(binner):
    res = binner([(4, []), (5, [7, 1, 9]), (3, [0, 0, 0, 0]), (0, [2, 3]), (-2, [1])])
    (ptr, order) = res[0]
    assert ptr == [0] * 5 and order == []
    # more bins than items: each item alone, the largest on bin 0, then down
    (ptr, order) = res[1]
    _check_structure(5, [7, 1, 9], ptr, order)
    assert ptr == [0, 1, 2, 3, 3, 3] and order == [2, 0, 1]
    # zero costs: every item goes to bin 0 (its load stays the lowest, ties to the lower bin)
    (ptr, order) = res[2]
    assert ptr == [0, 4, 4, 4] and order == [0, 1, 2, 3]
    # no bins asked for: one bin
    for (m, c), (ptr, order) in zip([(0, [2, 3]), (-2, [1])], res[3:]):
        _check_structure(m, c, ptr, order)
        assert ptr == [0, len(c)]


def test_balance_on_the_irregular_partition(binner):
    """The 48 x 48 x 24 elasticity problem on 64 irregular substructures: 64-row items of
    S_i (cost n_Gamma,i each) on 152 bins.  Handing them out in turn leaves the largest
    block ~9% above the mean; the bins are within 3% of it."""
    prob = P.config_irregular_elasticity()
    g = Globs(prob)
    nG = np.zeros(prob.nsub, dtype=np.int64)
    for n in g.interface_nodes:
        for s in g.sets[n]:
            nG[s] += prob.ncomp
    c = [int(n) for n in nG for _ in range(0, int(n), 64)]
    (ptr, order), = binner([(152, c)])
    _check_structure(152, c, ptr, order)
    mean = sum(c) / 152
    turn = [sum(c[k::152]) for k in range(152)]
    assert max(turn) / mean > 1.05
    assert max(_loads(ptr, order, c)) / mean < 1.03
