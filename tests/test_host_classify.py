"""The library's host mesh analysis (bddc_classify_q1: the classification of
bddc_set_mesh_q1, run without a GPU) against the oracle's glob classification
(Section 2: faces, edges, corners; Assumptions 1 and 2: corner augmentation) on
cubic, irregular and planar partitions."""
import numpy as np
import pytest

from paper_0910_5863_gb300 import bddc as B
from paper_0910_5863_gb300 import problems as P
from oracle.globs import Globs


def _check(prob):
    r = B.classify_mesh(prob)
    g = Globs(prob)
    c = prob.ncomp
    assert (r["n_corners"], r["n_edges"], r["n_faces"]) == g.counts(), prob.name
    assert list(r["corners"]) == list(g.corners), prob.name
    assert r["n_augmented"] == len(g.augmented), prob.name
    assert r["n_free"] == int((~prob.dirichlet.astype(bool)).sum()) * c
    assert r["n_interface"] == len(g.interface_nodes) * c
    return r


@pytest.mark.parametrize("make", [
    lambda: P.config_small(),
    lambda: P.config_adaptive_poisson(),
    lambda: P.poisson_cube(6, 2, coef="lognormal", seed=3),
    lambda: P.poisson_cube(4, 2, s_xyz=(2, 1, 1)),
    lambda: P.elasticity_cube(6, 2),
    lambda: P.elasticity_cube(8, 2, channels=2, seed=3),
])
def test_cubic_partitions(make):
    _check(make())


@pytest.mark.parametrize("seed,grid,nparts", [(1, (12, 12, 8), 8), (2, (10, 8, 8), 6), (3, (16, 12, 6), 12)])
def test_irregular_partitions(seed, grid, nparts):
    """Region-growing partitions: rough interfaces, edge sets with several pieces,
    corners chosen by the neighbour rule."""
    r = _check(P.config_irregular_elasticity(seed=seed, grid=grid, nparts=nparts))
    assert r["n_corners"] > 0 and r["n_faces"] > 0


def test_full_size_configurations():
    """The 32^3 elasticity mesh (4 x 4 x 4 cubes) and the 48 x 48 x 24 mesh in 64
    region-growing substructures (faces and corners of uneven size, augmented corners)."""
    _check(P.config_elasticity_channels())
    r = _check(P.config_irregular_elasticity())
    assert r["n_augmented"] > 0


@pytest.mark.parametrize("k,m", [(2, 2), (2, 4), (3, 4)])
def test_planar_cubes_augmentation(k, m):
    """k x k x 1 cubes fixed on x = 0: face pairs with a floating member get augmented
    corners (Assumption 2); the library promotes the same nodes as the oracle."""
    r = _check(P.planar_cubes(k, m=m))
    assert r["n_augmented"] > 0


def test_errors():
    prob = P.config_small()
    bad = P.config_small()
    bad.elem_sub = bad.elem_sub.copy()
    bad.elem_sub[0] = prob.nsub   # substructure id out of range
    with pytest.raises(B.BddcError) as e:
        B.classify_mesh(bad)
    assert e.value.status == 1
