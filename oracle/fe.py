"""Oracle, part 1: trilinear (Q1) finite elements and substructure assembly.

TEST INFRASTRUCTURE ONLY.  The oracle is a plain, slow FP64 CPU restatement of
the method, used by the tests, by ``__graft_entry__.smoke`` and by the CPU
baseline leg of ``bench.py``.  The product (the CUDA library and its Python
binding) never imports it.

Follows Section 2 of the paper: each substructure matrix A_i is the
subassembly of the element matrices of the elements in Omega_i (the local
stiffness of eq. (W)/(block-operators)); R maps global to local degrees of
freedom and R^T A R is the global stiffness (eq. (assembled)).  The element
matrices use 2x2x2 Gauss quadrature on the trilinear map.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

GAUSS = np.array([-1.0, 1.0]) / np.sqrt(3.0)
LOCAL = np.array([[a & 1, (a >> 1) & 1, (a >> 2) & 1] for a in range(8)], dtype=np.float64) * 2 - 1


def shape_grads_ref(xi):
    """d N_a / d xi for the 8 trilinear shape functions at reference point xi."""
    g = np.zeros((8, 3))
    for a in range(8):
        s = LOCAL[a]
        f = [(1 + s[d] * xi[d]) for d in range(3)]
        g[a, 0] = s[0] * f[1] * f[2] / 8
        g[a, 1] = f[0] * s[1] * f[2] / 8
        g[a, 2] = f[0] * f[1] * s[2] / 8
    return g


def _quad_points():
    pts = []
    for gz in GAUSS:
        for gy in GAUSS:
            for gx in GAUSS:
                pts.append(np.array([gx, gy, gz]))
    return pts  # all weights are 1


def element_grads(xe):
    """Physical gradients and quadrature weights for one element.

    xe: (8, 3) node coordinates.  Returns list of (grad (8, 3), w*detJ)."""
    out = []
    for xi in _quad_points():
        gr = shape_grads_ref(xi)
        J = xe.T @ gr               # J[d, k] = d x_d / d xi_k
        detJ = np.linalg.det(J)
        gphys = gr @ np.linalg.inv(J)   # dN/dx = dN/dxi * dxi/dx
        out.append((gphys, detJ))
    return out


def poisson_element(xe, k):
    """k * int grad N_a . grad N_b over the element."""
    K = np.zeros((8, 8))
    for g, w in element_grads(xe):
        K += w * (g @ g.T)
    return k * K


def elasticity_D(E, nu):
    lam = E * nu / ((1 + nu) * (1 - 2 * nu))
    mu = E / (2 * (1 + nu))
    D = np.zeros((6, 6))
    D[:3, :3] = lam
    D[np.arange(3), np.arange(3)] += 2 * mu
    D[3, 3] = D[4, 4] = D[5, 5] = mu
    return D


def elasticity_B(g):
    """Strain-displacement matrix (Voigt: xx, yy, zz, xy, yz, xz); dof 3a + c."""
    B = np.zeros((6, 24))
    for a in range(8):
        gx, gy, gz = g[a]
        B[0, 3 * a + 0] = gx
        B[1, 3 * a + 1] = gy
        B[2, 3 * a + 2] = gz
        B[3, 3 * a + 0] = gy
        B[3, 3 * a + 1] = gx
        B[4, 3 * a + 1] = gz
        B[4, 3 * a + 2] = gy
        B[5, 3 * a + 0] = gz
        B[5, 3 * a + 2] = gx
    return B


def elasticity_element(xe, E, nu):
    D = elasticity_D(E, nu)
    K = np.zeros((24, 24))
    for g, w in element_grads(xe):
        B = elasticity_B(g)
        K += w * (B.T @ D @ B)
    return K


def element_matrices(prob):
    """All element matrices.  On a uniform grid every element is the same cube,
    so the unit-coefficient matrix is computed once per distinct shape and
    scaled by the element coefficient (both are linear in k_e / E_e)."""
    ne = prob.ne
    xe0 = prob.xyz[prob.elems[0]]
    edges = prob.xyz[prob.elems[:, 7]] - prob.xyz[prob.elems[:, 0]]
    uniform = np.allclose(edges, edges[0])
    if prob.ncomp == 1:
        unit = poisson_element(xe0, 1.0)
    else:
        unit = elasticity_element(xe0, 1.0, prob.nu)
    if uniform:
        return unit[None, :, :] * prob.coef[:, None, None]
    Ks = []
    for e in range(ne):
        xe = prob.xyz[prob.elems[e]]
        Ks.append(poisson_element(xe, prob.coef[e]) if prob.ncomp == 1
                  else elasticity_element(xe, prob.coef[e], prob.nu))
    return np.array(Ks)


class Dofs:
    """Global free-dof numbering: node-major, component fastest; Dirichlet
    nodes get -1 (eliminated with u = 0)."""

    def __init__(self, prob):
        c = prob.ncomp
        free = ~prob.dirichlet
        self.node_first = -np.ones(prob.nn, dtype=np.int64)
        self.node_first[free] = np.arange(free.sum()) * c
        self.n = int(free.sum()) * c
        self.ncomp = c

    def of_nodes(self, nodes):
        """(len(nodes), ncomp) global dof ids (-1 for Dirichlet)."""
        f = self.node_first[nodes]
        out = f[:, None] + np.arange(self.ncomp)[None, :]
        out[f < 0] = -1
        return out


def assemble_global(prob, Ke=None):
    """K = sum_e over free dofs (scipy CSR) and F (global load vector)."""
    if Ke is None:
        Ke = element_matrices(prob)
    dofs = Dofs(prob)
    c = prob.ncomp
    ed = dofs.of_nodes(prob.elems.ravel()).reshape(prob.ne, 8 * c)
    rows = np.repeat(ed, 8 * c, axis=1).ravel()
    cols = np.tile(ed, (1, 8 * c)).ravel()
    vals = Ke.reshape(prob.ne, -1).ravel()
    keep = (rows >= 0) & (cols >= 0)
    K = sp.coo_matrix((vals[keep], (rows[keep], cols[keep])), shape=(dofs.n, dofs.n)).tocsr()
    F = np.zeros(dofs.n)
    nd = dofs.of_nodes(np.arange(prob.nn))
    m = nd[:, 0] >= 0
    F[nd[m].ravel()] = prob.load[m].ravel()
    return K, F, dofs


class Substructure:
    """Local data of Omega_i: local free dofs (node order, component fastest),
    their global ids, and A_i = sum over the elements of Omega_i."""

    def __init__(self, prob, i, Ke, dofs):
        el = np.nonzero(prob.elem_sub == i)[0]
        self.elements = el
        nodes = np.unique(prob.elems[el].ravel())
        self.nodes = nodes
        gd = dofs.of_nodes(nodes)                    # (nloc_nodes, c)
        keep = gd[:, 0] >= 0
        self.free_nodes = nodes[keep]
        self.gdof = gd[keep].ravel()                 # local dof -> global dof
        nloc = self.gdof.size
        g2l = -np.ones(dofs.n, dtype=np.int64)
        g2l[self.gdof] = np.arange(nloc)
        c = prob.ncomp
        ed = dofs.of_nodes(prob.elems[el].ravel()).reshape(el.size, 8 * c)
        ld = np.where(ed >= 0, g2l[np.maximum(ed, 0)], -1)
        rows = np.repeat(ld, 8 * c, axis=1).ravel()
        cols = np.tile(ld, (1, 8 * c)).ravel()
        vals = Ke[el].reshape(el.size, -1).ravel()
        k = (rows >= 0) & (cols >= 0)
        self.A = sp.coo_matrix((vals[k], (rows[k], cols[k])), shape=(nloc, nloc)).tocsr()
        self.g2l = g2l
