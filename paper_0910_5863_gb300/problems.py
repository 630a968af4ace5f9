"""Seeded synthetic workloads for adaptive BDDC in 3D (mesh, coefficients,
partition, boundary conditions and loads).

This module only *describes* problems: node coordinates, trilinear hexahedral
connectivity, per-element material coefficients, the element -> substructure
map, Dirichlet nodes and nodal loads.  It performs none of the method's
arithmetic (no element matrices, no assembly, no Schur complements); the CPU
oracle and the CUDA library each do that themselves from these arrays.

Random numbers come from splitmix64 (S. Vigna's published 64-bit mixer), one
independent stream per purpose keyed by (seed, purpose id):
    state_0 = seed * 0x9E3779B97F4A7C15 + purpose * 0xD1B54A32D192ED03  (mod 2^64)
    state_k = state_0 + k * 0x9E3779B97F4A7C15, draw_k = mix(state_{k+1})
    uniform = (draw >> 11) * 2^-53
Normal draws use Box-Muller on two consecutive uniforms.

Workloads (the paper's engineering meshes are not public; these stand in for
their shapes, Section 7 of the paper):
  * ``poisson_cube``    -- unit cube, Q1, -div(k grad u) = f, u = 0 on x = 0
  * ``elasticity_cube`` -- unit cube, Q1 linear elasticity, clamped at z = 0,
                           body load (0, 0, -1)
with cubic substructures of m^3 elements, optional stiff element channels,
random high-coefficient elements, lognormal coefficients or z-layers.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import numpy as np

MASK64 = (1 << 64) - 1
GOLDEN = 0x9E3779B97F4A7C15
PURPOSE_MUL = 0xD1B54A32D192ED03

# purpose ids of the independent streams
P_COEF = 1
P_RHS = 2
P_PARTITION = 3
P_PROBLEM = 4
P_CHANNEL = 5


def _mix(z: np.ndarray) -> np.ndarray:
    z = z.astype(np.uint64)
    z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
    z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    return z ^ (z >> np.uint64(31))


def splitmix64_raw(state0: int, n: int) -> np.ndarray:
    """First n outputs of splitmix64 started at 64-bit state ``state0``."""
    k = np.arange(1, n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        states = np.uint64(state0 & MASK64) + k * np.uint64(GOLDEN)
        return _mix(states)


def stream_state(seed: int, purpose: int) -> int:
    return (seed * GOLDEN + purpose * PURPOSE_MUL) & MASK64


class Stream:
    """Sequential draws from one (seed, purpose) splitmix64 stream."""

    def __init__(self, seed: int, purpose: int):
        self.state = stream_state(seed, purpose)

    def raw(self, n: int) -> np.ndarray:
        out = splitmix64_raw(self.state, n)
        self.state = (self.state + n * GOLDEN) & MASK64
        return out

    def uniform(self, n: int) -> np.ndarray:
        return (self.raw(n) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)

    def normal(self, n: int) -> np.ndarray:
        u = self.uniform(2 * n)
        u1 = 1.0 - u[0::2]            # (0, 1]
        u2 = u[1::2]
        return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)

    def below(self, bound: int) -> int:
        return int(self.uniform(1)[0] * bound)


@dataclass
class Problem:
    """A substructured trilinear-hexahedron problem (input arrays only)."""
    name: str
    ncomp: int                    # 1 = Poisson, 3 = elasticity
    grid: tuple                   # (nx, ny, nz) elements
    h: float
    xyz: np.ndarray               # (nn, 3) float64 node coordinates
    elems: np.ndarray             # (ne, 8) int64, local node a = ax + 2 ay + 4 az
    coef: np.ndarray              # (ne,) float64: conductivity k_e or Young modulus E_e
    nu: float                     # Poisson ratio (elasticity only)
    elem_sub: np.ndarray          # (ne,) int32 substructure of each element
    nsub: int
    dirichlet: np.ndarray         # (nn,) bool, all components fixed to 0
    load: np.ndarray              # (nn, ncomp) float64 nodal loads
    meta: dict = field(default_factory=dict)

    @property
    def nn(self) -> int:
        return self.xyz.shape[0]

    @property
    def ne(self) -> int:
        return self.elems.shape[0]


def box_mesh(nx: int, ny: int, nz: int, h: float):
    """Structured box: node id = i + (nx+1)(j + (ny+1) k); element id = ex + nx(ey + ny ez)."""
    i, j, k = np.meshgrid(np.arange(nx + 1), np.arange(ny + 1), np.arange(nz + 1), indexing="ij")
    nid = lambda a, b, c: a + (nx + 1) * (b + (ny + 1) * c)
    xyz = np.zeros(((nx + 1) * (ny + 1) * (nz + 1), 3))
    ids = nid(i, j, k).ravel()
    xyz[ids, 0] = i.ravel() * h
    xyz[ids, 1] = j.ravel() * h
    xyz[ids, 2] = k.ravel() * h
    ex, ey, ez = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    eid = (ex + nx * (ey + ny * ez)).ravel()
    elems = np.zeros((nx * ny * nz, 8), dtype=np.int64)
    for a in range(8):
        ax, ay, az = a & 1, (a >> 1) & 1, (a >> 2) & 1
        elems[eid, a] = nid(ex + ax, ey + ay, ez + az).ravel()
    return xyz, elems


def cubic_partition(nx, ny, nz, sx, sy, sz):
    mx, my, mz = nx // sx, ny // sy, nz // sz
    ex, ey, ez = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    eid = (ex + nx * (ey + ny * ez)).ravel()
    sub = np.zeros(nx * ny * nz, dtype=np.int32)
    sub[eid] = ((ex // mx) + sx * ((ey // my) + sy * (ez // mz))).ravel()
    return sub


def region_growing_partition(nx, ny, nz, nparts, seed):
    """Irregular partition of an nx x ny x nz element grid: nparts distinct seed
    elements drawn uniformly (redrawing repeats), then rounds in which every region,
    in the order 0 .. nparts-1, takes the oldest element of its frontier (the
    unassigned elements face-adjacent to it, in the order first reached; entries
    assigned meanwhile are skipped), i.e. breadth-first growth in round-robin.
    Regions stay face-connected.  Returns elem_sub (int32)."""
    from collections import deque
    ne = nx * ny * nz
    st = Stream(seed, P_PARTITION)
    owner = -np.ones(ne, dtype=np.int64)
    frontier = [deque() for _ in range(nparts)]

    def neighbours(e):
        ex, r = e % nx, e // nx
        ey, ez = r % ny, r // ny
        if ex > 0: yield e - 1
        if ex < nx - 1: yield e + 1
        if ey > 0: yield e - nx
        if ey < ny - 1: yield e + nx
        if ez > 0: yield e - nx * ny
        if ez < nz - 1: yield e + nx * ny

    def take(r, e):
        owner[e] = r
        for q in neighbours(e):
            if owner[q] < 0:
                frontier[r].append(q)

    r = 0
    while r < nparts:
        e = st.below(ne)
        if owner[e] < 0:
            take(r, e)
            r += 1
    left = ne - nparts
    while left > 0:
        for r in range(nparts):
            fr = frontier[r]
            while fr and owner[fr[0]] >= 0:
                fr.popleft()
            if fr:
                take(r, fr.popleft())
                left -= 1
                if left == 0:
                    break
    return owner.astype(np.int32)


def _uniform_loads(nn, seed, dirichlet):
    f = 2.0 * Stream(seed, P_RHS).uniform(nn) - 1.0
    f[dirichlet] = 0.0
    return f.reshape(nn, 1)


def poisson_cube(n: int, s: int, seed: int = 1, coef: str = "one", frac_high: float = 0.2,
                 high: float = 1e4, sigma: float = 2.0, s_xyz=None, name=None) -> Problem:
    """Q1 Poisson on the unit cube with n^3 elements in s^3 cubic substructures.

    coef: "one" (k = 1), "random_high" (exactly round(frac_high*ne) elements get
    k = high, chosen by a seeded partial Fisher-Yates shuffle) or "lognormal"
    (k_e = exp(sigma z), z ~ N(0, 1)).  u = 0 on x = 0; nodal loads f ~ U[-1, 1]
    drawn for every node in node-id order, Dirichlet draws discarded.
    """
    sx, sy, sz = s_xyz if s_xyz is not None else (s, s, s)
    nx = ny = nz = n
    h = 1.0 / n
    xyz, elems = box_mesh(nx, ny, nz, h)
    ne = elems.shape[0]
    k = np.ones(ne)
    if coef == "random_high":
        m = int(round(frac_high * ne))
        st = Stream(seed, P_COEF)
        perm = np.arange(ne)
        u = st.uniform(m)
        for i in range(m):
            j = i + int(u[i] * (ne - i))
            perm[i], perm[j] = perm[j], perm[i]
        k[perm[:m]] = high
    elif coef == "lognormal":
        k = np.exp(sigma * Stream(seed, P_COEF).normal(ne))
    elif coef != "one":
        raise ValueError(coef)
    dirichlet = np.isclose(xyz[:, 0], 0.0)
    load = _uniform_loads(xyz.shape[0], seed, dirichlet)
    return Problem(name or f"poisson{n}_s{sx}{sy}{sz}_{coef}", 1, (nx, ny, nz), h, xyz, elems, k, 0.0,
                   cubic_partition(nx, ny, nz, sx, sy, sz), sx * sy * sz, dirichlet, load,
                   {"seed": seed, "coef": coef})


def _body_load(xyz, elems, h, dirichlet, b=(0.0, 0.0, -1.0)):
    """Nodal loads of a uniform body force on a uniform hexahedral grid: each
    element hands h^3/8 of its force to each of its 8 nodes."""
    nn = xyz.shape[0]
    cnt = np.bincount(elems.ravel(), minlength=nn).astype(np.float64)
    load = np.outer(cnt * h ** 3 / 8.0, np.asarray(b, dtype=np.float64))
    load[dirichlet] = 0.0
    return load


def elasticity_cube(n: int, s: int, seed: int = 1, channels: int = 0, e_channel: float = 1e6,
                    nu: float = 0.3, s_xyz=None, grid=None, layers: int = 0, e_layer: float = 1e3,
                    name=None, partition=None) -> Problem:
    """Q1 linear elasticity on a box of n^3 (or ``grid``) elements with h = 1/n,
    s^3 cubic substructures, clamped at z = 0, body load (0, 0, -1).

    channels: number of straight element channels with E = e_channel; each picks
    an axis in {x, y, z} and a transverse element index pair uniformly and spans
    the whole box, so it crosses substructure faces.
    layers: if > 0, E = e_layer in z-layers floor(ez / layers) odd, 1 otherwise.
    partition: optional (elem_sub, nsub) replacing the cubic substructures.
    """
    nx, ny, nz = grid if grid is not None else (n, n, n)
    sx, sy, sz = s_xyz if s_xyz is not None else (s, s, s)
    h = 1.0 / n
    xyz, elems = box_mesh(nx, ny, nz, h)
    ne = elems.shape[0]
    E = np.ones(ne)
    ex, ey, ez = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    eid = (ex + nx * (ey + ny * ez)).ravel()
    exr, eyr, ezr = ex.ravel(), ey.ravel(), ez.ravel()
    if channels:
        st = Stream(seed, P_CHANNEL)
        for _ in range(channels):
            axis = st.below(3)
            if axis == 0:
                a, b = st.below(ny), st.below(nz)
                sel = (eyr == a) & (ezr == b)
            elif axis == 1:
                a, b = st.below(nx), st.below(nz)
                sel = (exr == a) & (ezr == b)
            else:
                a, b = st.below(nx), st.below(ny)
                sel = (exr == a) & (eyr == b)
            E[eid[sel]] = e_channel
    if layers:
        odd = (ezr // layers) % 2 == 1
        E[eid[odd]] = e_layer
    dirichlet = np.isclose(xyz[:, 2], 0.0)
    load = _body_load(xyz, elems, h, dirichlet)
    esub, nsub = partition if partition is not None else (cubic_partition(nx, ny, nz, sx, sy, sz), sx * sy * sz)
    return Problem(name or f"elast{nx}x{ny}x{nz}_s{sx}{sy}{sz}", 3, (nx, ny, nz), h, xyz, elems, E, nu,
                   esub, nsub, dirichlet, load, {"seed": seed, "channels": channels, "layers": layers})


# --- the named workloads -------------------------------------------------

def config_small(seed: int = 1) -> Problem:
    """12^3 Poisson, 2x2x2 substructures of 6^3, k = 1 (plain BDDC with
    corners + arithmetic edge and face averages; the small parity case)."""
    return poisson_cube(12, 2, seed, "one", name="poisson12_2x2x2")


def config_adaptive_poisson(seed: int = 1) -> Problem:
    """24^3 Poisson, 3x3x3 substructures of 8^3, 20% of elements k = 1e4
    (adaptive BDDC from corners, tau = 10; the timed workload)."""
    return poisson_cube(24, 3, seed, "random_high", name="poisson24_3x3x3_jump1e4")


def config_elasticity_channels(seed: int = 1) -> Problem:
    """32^3 elasticity, 4x4x4 substructures of 8^3, 8 stiff channels E = 1e6."""
    return elasticity_cube(32, 4, seed, channels=8, name="elast32_4x4x4_channels")


def config_irregular_elasticity(seed: int = 1, grid=(48, 48, 24), nparts: int = 64) -> Problem:
    """48 x 48 x 24 elasticity (h = 1/48), nparts irregular substructures by seeded
    region growing, E = 1e3 in the odd z-layers of height 4 elements and 1 elsewhere,
    nu = 0.3, clamped at z = 0, body load (0, 0, -1)."""
    nx, ny, nz = grid
    part = region_growing_partition(nx, ny, nz, nparts, seed)
    return elasticity_cube(nx, 1, seed, grid=grid, layers=4, name=f"elast{nx}x{ny}x{nz}_irregular{nparts}",
                           partition=(part, nparts))


def config_batch_poisson(seed: int = 1, count: int = 256) -> list:
    """count independent Q1 Poisson problems: problem p has s^3 cubic substructures of
    m^3 elements (s in {2, 3}, m in {6, ..., 10}, drawn from the (seed, per-problem)
    stream), k_e = exp(2 z) with z ~ N(0, 1) (lognormal, sigma = 2), u = 0 on x = 0,
    nodal loads U[-1, 1]; problem p uses seed 65536 * seed + p + 1 for its own
    coefficient and load streams."""
    st = Stream(seed, P_PROBLEM)
    out = []
    for p in range(count):
        u = st.uniform(2)
        s = 2 + int(u[0] * 2)
        m = 6 + int(u[1] * 5)
        out.append(poisson_cube(s * m, s, seed=65536 * seed + p + 1, coef="lognormal", sigma=2.0,
                                name=f"batch{p}_poisson{s * m}_s{s}_m{m}"))
    return out


def planar_cubes(k: int, m: int = 8, nu: float = 0.3, name=None) -> Problem:
    """k x k x 1 cubic substructures of m^3 Q1 elasticity elements (h = 1/m per cube,
    the paper's weak-scaling problem, Section 7 and its last table): fixed on the side
    x = 0, loaded on the opposite side x = k by a uniform traction (0, 0, -1)
    distributed to the face nodes by their tributary areas.  E = 1."""
    nx, ny, nz = k * m, k * m, m
    h = 1.0 / m
    xyz, elems = box_mesh(nx, ny, nz, h)
    ne = elems.shape[0]
    dirichlet = np.isclose(xyz[:, 0], 0.0)
    load = np.zeros((xyz.shape[0], 3))
    face = np.isclose(xyz[:, 0], nx * h)
    # tributary area of a node of the loaded face: h^2 / 4 per adjacent face quad
    j = np.rint(xyz[:, 1] / h).astype(int)
    kk = np.rint(xyz[:, 2] / h).astype(int)
    wy = np.where((j == 0) | (j == ny), 0.5, 1.0)
    wz = np.where((kk == 0) | (kk == nz), 0.5, 1.0)
    load[face, 2] = -(h * h) * wy[face] * wz[face]
    return Problem(name or f"planar_cubes_{k}x{k}x1_m{m}", 3, (nx, ny, nz), h, xyz, elems, np.ones(ne), nu,
                   cubic_partition(nx, ny, nz, k, k, 1), k * k, dirichlet, load, {"k": k, "m": m})
