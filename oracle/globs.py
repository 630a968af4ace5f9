"""Oracle, part 2: interface, globs (faces / edges / corners) and averaging weights.

TEST INFRASTRUCTURE ONLY (see oracle/fe.py).

Section 2 of the paper: the interface is the set of nodes contained in more
than one substructure; a face holds the nodes shared by exactly one pair of
substructures, an edge the nodes shared by one and the same set of more than
two substructures, and a corner is a degenerate, one-node edge.

Reading of the corner definition (the paper's Fig. 3 counts 7 corners in a
2x2x2 cube, which a literal one-node rule does not give): a node of an edge
set is a corner if (i) its set has exactly one node, or (ii) it has at most
one grid neighbour (a node joined to it by an element edge) in its own set
and no grid neighbour whose set is a strict superset of its own.  Globs are
classified on the full mesh; Dirichlet nodes are dropped afterwards.  One face
per pair and one edge per set, even when the set is disconnected.

Weights of the averaging operator E (Section 2, eq. (E); Section 7: weights
proportional to the diagonal of the substructure matrices before the
elimination of interiors): delta_i(x) = a_i(x) / sum_k a_k(x), per dof.
"""
from __future__ import annotations

from collections import defaultdict
import numpy as np

# the 12 element edges in local node numbering a = ax + 2 ay + 4 az
HEX_EDGES = [(a, a ^ (1 << d)) for a in range(8) for d in range(3) if not (a >> d) & 1]


def node_sets(prob):
    """frozenset of substructures containing each node."""
    sets = [set() for _ in range(prob.nn)]
    for e in range(prob.ne):
        s = int(prob.elem_sub[e])
        for n in prob.elems[e]:
            sets[n].add(s)
    return [frozenset(x) for x in sets]


def grid_neighbours(prob):
    nb = [set() for _ in range(prob.nn)]
    for e in range(prob.ne):
        en = prob.elems[e]
        for a, b in HEX_EDGES:
            nb[en[a]].add(int(en[b]))
            nb[en[b]].add(int(en[a]))
    return nb


class Globs:
    """Classification of the interface nodes.

    corners: sorted node ids (Dirichlet nodes removed)
    faces:   dict (i, j) -> sorted node ids (i < j)
    edges:   dict frozenset -> sorted node ids (corners removed)
    sets:    node -> frozenset of substructures
    """

    def __init__(self, prob):
        self.sets = node_sets(prob)
        nb = grid_neighbours(prob)
        by_set = defaultdict(list)
        for n, s in enumerate(self.sets):
            if len(s) >= 2:
                by_set[s].append(n)
        corners = set()
        for s, nodes in by_set.items():
            if len(s) < 3:
                continue
            if len(nodes) == 1:
                corners.add(nodes[0])
                continue
            for n in nodes:
                same = sum(1 for m in nb[n] if self.sets[m] == s)
                sup = any(self.sets[m] > s for m in nb[n])
                if same <= 1 and not sup:
                    corners.add(n)
        dirich = prob.dirichlet
        self.corners = sorted(n for n in corners if not dirich[n])
        self.faces = {}
        self.edges = {}
        for s, nodes in by_set.items():
            keep = sorted(n for n in nodes if not dirich[n] and n not in corners)
            if not keep:
                continue
            if len(s) == 2:
                self.faces[tuple(sorted(s))] = keep
            else:
                self.edges[s] = keep
        self.interface_nodes = sorted(n for n, s in enumerate(self.sets) if len(s) >= 2 and not dirich[n])
        self.corner_set = set(self.corners)
        self.augmented = self._augment(prob)

    def _augment(self, prob):
        """Corner augmentation (reading of Assumptions 1 and 2): for every face pair (i, j),
        in increasing order, one of whose substructures has no Dirichlet node, the
        shared corners must fix the rigid modes -- 1 corner for a scalar problem, 3
        non-collinear corners for elasticity.  While they do not, the face node that
        maximises the smallest squared distance to the current shared corners becomes a
        corner (the lowest node id when there are none yet; ties within 1e-12 relative
        go to the lowest id).  A node promoted for (i, j) lies on that face only, so the
        faces do not interact."""
        need = 1 if prob.ncomp == 1 else 3
        dirich = prob.dirichlet
        anchored = np.zeros(prob.nsub, dtype=bool)
        for e in range(prob.ne):
            if dirich[prob.elems[e]].any():
                anchored[prob.elem_sub[e]] = True
        added = []
        for (i, j) in sorted(self.faces):
            if anchored[i] and anchored[j]:
                continue
            face = list(self.faces[(i, j)])
            pair = {i, j}
            shared = [n for n in self.corners if pair <= self.sets[n]]
            while _corner_rank(prob.xyz, shared, need) < need and face:
                if not shared:
                    pick = face[0]
                else:
                    X = prob.xyz[face][:, None, :] - prob.xyz[shared][None, :, :]
                    dmin = (X ** 2).sum(axis=2).min(axis=1)
                    best = dmin.max()
                    pick = min(n for n, d in zip(face, dmin) if d >= best * (1 - 1e-12))
                face.remove(pick)
                shared.append(pick)
                added.append(pick)
                self.corners.append(pick)
            self.faces[(i, j)] = face
        self.corners = sorted(self.corners)
        self.corner_set = set(self.corners)
        self.faces = {k: v for k, v in self.faces.items() if v}
        return sorted(added)

    def counts(self):
        return len(self.corners), len(self.edges), len(self.faces)


def _corner_rank(xyz, nodes, need):
    """1 if any node (scalar case); for need = 3, 3 if three of the nodes are not collinear."""
    if not nodes:
        return 0
    if need == 1:
        return 1
    P = xyz[nodes]
    D = P[1:] - P[0]
    if D.shape[0] == 0 or np.abs(D).max() == 0:
        return 1
    r = np.linalg.matrix_rank(D, tol=1e-8 * np.abs(D).max())
    return 3 if r >= 2 else 2


def weights(subs, ndof):
    """delta_i per local dof: diag(A_i) normalised over all sharing substructures."""
    total = np.zeros(ndof)
    for s in subs:
        np.add.at(total, s.gdof, s.A.diagonal())
    return [s.A.diagonal() / total[s.gdof] for s in subs]
