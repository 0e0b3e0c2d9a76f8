"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the CPU oracle.

This module holds no arithmetic of the FEM method itself: it only lays out
structured meshes, draws random numbers and builds boundary masks.  Both sides
(the oracle under ``oracle/`` and the library in ``paper_2111_03541_gb300``)
receive the same arrays from here.

Random numbers come from one counter-based generator, SplitMix64 (Steele, Lea
and Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014):
draw ``i`` of stream ``seed`` is ``mix(seed + (i + 1) * 0x9E3779B97F4A7C15)``.
A uniform double is the top 53 bits times 2^-53; a standard normal comes from
the Box-Muller transform of two uniforms.

Conventions (all indices 0-based, lexicographic x fastest, then y, then z):

* triangle grid ``n x n`` on the unit square: square (i, j) splits along the
  diagonal (i, j)->(i+1, j+1) into triangles (v00, v10, v11) and (v00, v11, v01),
  both counter-clockwise; element id = 2 (j n + i) + t.
* P2 triangles use the (2n+1)^2 grid of vertices and edge midpoints; local
  nodes are the three vertices, then the midpoints of edges (0,1), (1,2), (2,0).
  Edges stay straight: a midpoint sits at the mean of its (jittered) ends.
* Q1 hexahedra on an ``n^3`` box: local node a = i + 2 j + 4 k sits at the
  cube corner (i, j, k).
* jitter moves interior nodes only, each coordinate uniform in [-a h, a h];
  draw ``node * dim + c`` of the jitter stream.
"""
from __future__ import annotations

import math

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# Seeds of the synthetic workloads.
SEED_JITTER = 1001
SEED_COEF = 1002
SEED_ADVECT = 1003
SEED_BATCH = 1004
SEED_GRF = 1005
SEED_CNN = 1006
SEED_FACET = 1007


def splitmix64(seed: int, idx: np.ndarray) -> np.ndarray:
    """SplitMix64 output for counters ``idx`` of stream ``seed`` (uint64 array)."""
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + (idx.astype(np.uint64) + np.uint64(1)) * GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """``n`` doubles in [0, 1) from draws ``offset .. offset+n-1`` of stream ``seed``."""
    z = splitmix64(seed, np.arange(offset, offset + n, dtype=np.uint64))
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def normal(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """``n`` standard normals; normal ``e`` uses draws 2e and 2e+1 (Box-Muller)."""
    u = uniform(seed, 2 * n, 2 * offset)
    u1 = 1.0 - u[0::2]  # (0, 1]
    u2 = u[1::2]
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


def lognormal(seed: int, n: int, sigma: float = 0.5, mu: float = 0.0) -> np.ndarray:
    """Per-element coefficients exp(mu + sigma z), z standard normal."""
    return np.exp(mu + sigma * normal(seed, n))


# ----------------------------------------------------------------------------
# meshes
# ----------------------------------------------------------------------------

def _jitter_grid(coords: np.ndarray, interior: np.ndarray, h: float, alpha: float, seed: int) -> None:
    if alpha == 0.0:
        return
    nn, dim = coords.shape
    u = uniform(seed, nn * dim).reshape(nn, dim)
    coords[interior] += (2.0 * u[interior] - 1.0) * (alpha * h)


def tri_mesh(n: int, order: int = 1, jitter: float = 0.0, seed: int = SEED_JITTER,
             jitter_all: bool = False) -> dict:
    """Triangles on the unit square from an ``n x n`` grid.

    Returns ``coords`` (float64 [nn, 2]), ``conn`` (int32 [2 n^2, 3 or 6]) and,
    for order 2, ``vconn`` (int32 [2 n^2, 3]): the P1 vertex connectivity in the
    (n+1)^2 vertex numbering together with ``vcoords``.
    """
    h = 1.0 / n
    nv = n + 1
    jj, ii = np.meshgrid(np.arange(nv), np.arange(nv), indexing="ij")
    vcoords = np.stack([ii.ravel() * h, jj.ravel() * h], axis=1).astype(np.float64)
    vi, vj = ii.ravel(), jj.ravel()
    interior = (vi > 0) & (vi < n) & (vj > 0) & (vj < n)
    if jitter_all:  # boundary nodes move too (facets off the box's sides)
        interior[:] = True
    _jitter_grid(vcoords, interior, h, jitter, seed)

    j, i = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    i, j = i.ravel(), j.ravel()
    v00 = j * nv + i
    v10 = v00 + 1
    v01 = v00 + nv
    v11 = v01 + 1
    ne = 2 * n * n
    vconn = np.empty((ne, 3), dtype=np.int32)
    vconn[0::2] = np.stack([v00, v10, v11], axis=1)
    vconn[1::2] = np.stack([v00, v11, v01], axis=1)
    if order == 1:
        return {"dim": 2, "elem": "P1", "n": n, "coords": vcoords, "conn": vconn}

    # P2: nodes of the (2n+1)^2 grid; vertex (i, j) is fine node (2i, 2j).
    nf = 2 * n + 1
    fj, fi = np.meshgrid(np.arange(nf), np.arange(nf), indexing="ij")
    fi, fj = fi.ravel(), fj.ravel()
    coords = np.empty((nf * nf, 2), dtype=np.float64)
    vert = (fi % 2 == 0) & (fj % 2 == 0)
    coords[vert] = vcoords[(fj[vert] // 2) * nv + fi[vert] // 2]

    def fine(v):  # vertex index -> fine index
        return (v // nv) * 2 * nf + (v % nv) * 2

    fconn = fine(vconn.astype(np.int64))
    mids = []
    for a, b in ((0, 1), (1, 2), (2, 0)):
        pa, pb = fconn[:, a], fconn[:, b]
        mi = ((pa % nf) + (pb % nf)) // 2
        mj = ((pa // nf) + (pb // nf)) // 2
        m = mj * nf + mi
        # straight edges: midpoint at the mean of the two ends
        coords[m] = 0.5 * (coords[pa] + coords[pb])
        mids.append(m)
    conn = np.concatenate([fconn, np.stack(mids, axis=1)], axis=1).astype(np.int32)
    return {"dim": 2, "elem": "P2", "n": n, "coords": coords, "conn": conn,
            "vcoords": vcoords, "vconn": vconn}


def hex_mesh(n: int, jitter: float = 0.0, seed: int = SEED_JITTER, jitter_all: bool = False) -> dict:
    """Q1 hexahedra on the unit cube from an ``n^3`` grid (``jitter_all``:
    boundary nodes move too, so boundary faces are warped)."""
    h = 1.0 / n
    nv = n + 1
    kk, jj, ii = np.meshgrid(np.arange(nv), np.arange(nv), np.arange(nv), indexing="ij")
    ii, jj, kk = ii.ravel(), jj.ravel(), kk.ravel()
    coords = np.stack([ii * h, jj * h, kk * h], axis=1).astype(np.float64)
    interior = (ii > 0) & (ii < n) & (jj > 0) & (jj < n) & (kk > 0) & (kk < n)
    if jitter_all:
        interior[:] = True
    _jitter_grid(coords, interior, h, jitter, seed)
    k, j, i = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    base = ((k.ravel() * nv) + j.ravel()) * nv + i.ravel()
    conn = np.empty((n ** 3, 8), dtype=np.int32)
    for a in range(8):
        di, dj, dk = a & 1, (a >> 1) & 1, (a >> 2) & 1
        conn[:, a] = base + (dk * nv + dj) * nv + di
    return {"dim": 3, "elem": "Q1", "n": n, "coords": coords, "conn": conn}


def hex_box_mesh(nx: int, ny: int, nz: int, jitter: float = 0.0, seed: int = SEED_JITTER) -> dict:
    """Q1 hexahedra of side h = 1 / nx on the box [0, 1] x [0, ny h] x [0, nz h]
    (nx x ny x nz cells, nodes and elements lexicographic with x fastest):
    ``hex_mesh(n)`` is the case nx = ny = nz = n.  The weak-scaling workload
    of several ranks stacks their cubes along z."""
    h = 1.0 / nx
    kk, jj, ii = np.meshgrid(np.arange(nz + 1), np.arange(ny + 1), np.arange(nx + 1), indexing="ij")
    ii, jj, kk = ii.ravel(), jj.ravel(), kk.ravel()
    coords = np.stack([ii * h, jj * h, kk * h], axis=1).astype(np.float64)
    interior = (ii > 0) & (ii < nx) & (jj > 0) & (jj < ny) & (kk > 0) & (kk < nz)
    _jitter_grid(coords, interior, h, jitter, seed)
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    base = ((k.ravel() * (ny + 1)) + j.ravel()) * (nx + 1) + i.ravel()
    conn = np.empty((nx * ny * nz, 8), dtype=np.int32)
    for a in range(8):
        di, dj, dk = a & 1, (a >> 1) & 1, (a >> 2) & 1
        conn[:, a] = base + (dk * (ny + 1) + dj) * (nx + 1) + di
    return {"dim": 3, "elem": "Q1", "n": nx, "coords": coords, "conn": conn}


def hex20_mesh(n: int, jitter: float = 0.0, seed: int = SEED_JITTER) -> dict:
    """20-node serendipity bricks on the unit cube from an ``n^3`` grid.

    Local nodes: the 8 vertices a = i + 2 j + 4 k at cube corner (i, j, k),
    then the midpoints of the 12 edges: x edges at (y, z) = (j, k) are
    8 + j + 2 k, y edges at (x, z) = (i, k) are 12 + i + 2 k, z edges at
    (x, y) = (i, j) are 16 + i + 2 j.  Global numbering: the (n+1)^3 vertices
    of ``hex_mesh``, then x, y and z edge midpoints (lexicographic, x
    fastest).  Edges stay straight: a midpoint sits at the mean of its
    (jittered) ends.
    """
    v = hex_mesh(n, jitter, seed)
    nv = n + 1
    X = v["coords"]
    r = np.arange
    mids, ids = [], {}
    base = nv ** 3
    for axis in range(3):
        dims = [nv, nv, nv]
        dims[axis] = n  # segments along the axis
        k, j, i = np.meshgrid(r(dims[2]), r(dims[1]), r(dims[0]), indexing="ij")
        i, j, k = i.ravel(), j.ravel(), k.ravel()
        a = (k * nv + j) * nv + i
        step = [1, nv, nv * nv][axis]
        mids.append(0.5 * (X[a] + X[a + step]))
        ids[axis] = (base, dims)
        base += a.shape[0]
    coords = np.concatenate([X] + mids, axis=0)
    ne = n ** 3
    kk, jj, ii = np.meshgrid(r(n), r(n), r(n), indexing="ij")
    ii, jj, kk = ii.ravel(), jj.ravel(), kk.ravel()
    conn = np.empty((ne, 20), dtype=np.int64)
    conn[:, :8] = v["conn"]
    for axis in range(3):
        off, dims = ids[axis]
        for t in range(4):
            b0, b1 = t & 1, t >> 1
            if axis == 0:
                gi, gj, gk = ii, jj + b0, kk + b1
            elif axis == 1:
                gi, gj, gk = ii + b0, jj, kk + b1
            else:
                gi, gj, gk = ii + b0, jj + b1, kk
            conn[:, 8 + 4 * axis + t] = off + (gk * dims[1] + gj) * dims[0] + gi
    return {"dim": 3, "elem": "Q2S", "n": n, "coords": coords, "conn": conn.astype(np.int32)}


def quad8_mesh(n: int, jitter: float = 0.0, seed: int = SEED_JITTER) -> dict:
    """8-node serendipity quadrilaterals on the unit square from an ``n x n``
    grid.  Local nodes: vertices a = i + 2 j at cell corner (i, j), then the
    midpoints of the x edges (at y = j) 4 + j and of the y edges (at x = i)
    6 + i.  Global numbering: the (n+1)^2 vertices (x fastest, interior ones
    jittered as in ``tri_mesh``), then the x-edge midpoints (row by row), then
    the y-edge midpoints.  Edges stay straight.  Element (i, j) is j n + i."""
    h = 1.0 / n
    nv = n + 1
    jj, ii = np.meshgrid(np.arange(nv), np.arange(nv), indexing="ij")
    V = np.stack([ii.ravel() * h, jj.ravel() * h], axis=1).astype(np.float64)
    vi, vj = ii.ravel(), jj.ravel()
    _jitter_grid(V, (vi > 0) & (vi < n) & (vj > 0) & (vj < n), h, jitter, seed)
    xe = lambda i, j: nv * nv + j * n + i            # x edge from (i, j) to (i + 1, j)
    ye = lambda i, j: nv * nv + nv * n + j * nv + i  # y edge from (i, j) to (i, j + 1)
    xi_, xj_ = np.meshgrid(np.arange(n), np.arange(nv), indexing="xy")
    yi_, yj_ = np.meshgrid(np.arange(nv), np.arange(n), indexing="xy")
    xa = (xj_ * nv + xi_).ravel()
    ya = (yj_ * nv + yi_).ravel()
    coords = np.vstack([V, 0.5 * (V[xa] + V[xa + 1]), 0.5 * (V[ya] + V[ya + nv])])
    j, i = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    i, j = i.ravel(), j.ravel()
    v00 = j * nv + i
    conn = np.stack([v00, v00 + 1, v00 + nv, v00 + nv + 1, xe(i, j), xe(i, j + 1), ye(i, j), ye(i + 1, j)],
                    axis=1).astype(np.int32)
    return {"dim": 2, "elem": "Q2Q", "n": n, "coords": coords, "conn": conn}


def thermal_q2q_problem(n: int, jitter: float = 0.2, sigma: float = 0.5,
                        seed_jitter: int = SEED_JITTER, seed_coef: int = SEED_COEF) -> dict:
    """2D thermal conduction on 8-node serendipity quadrilaterals (u = 0 on the boundary, f = 1)."""
    m = quad8_mesh(n, jitter, seed_jitter)
    m["coef"] = lognormal(seed_coef, m["conn"].shape[0], sigma)
    m["bc_mask"], m["bc_val"] = thermal_bc(m)
    m["form"] = "thermal"
    m["source"] = 1.0
    return m


def tet10_mesh(n: int, jitter: float = 0.0, seed: int = SEED_JITTER) -> dict:
    """10-node (quadratic) tetrahedra on the unit cube: each cube of an ``n^3``
    grid split into the 6 tetrahedra around its main diagonal (Kuhn's
    subdivision, conforming across cubes), then one node at the midpoint of
    every edge.  Local nodes: vertices 0..3, then the edges (0,1), (1,2),
    (2,0), (0,3), (1,3), (2,3).  Global numbering: the (n+1)^3 vertices of
    ``hex_mesh`` (jittered the same way), then the edge midpoints in the order
    of their first appearance.  Edges stay straight."""
    from itertools import permutations
    base = hex_mesh(n, jitter, seed)
    X = base["coords"]
    nv = n + 1
    k, j, i = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    c0 = ((k.ravel() * nv) + j.ravel()) * nv + i.ravel()
    step = (1, nv, nv * nv)
    tets = []
    for perm in permutations(range(3)):
        v = [c0]
        for ax in perm:
            v.append(v[-1] + step[ax])
        t = np.stack(v, axis=1)
        # the vertex order's orientation follows the permutation's parity
        odd = sum(1 for a in range(3) for b in range(a + 1, 3) if perm[a] > perm[b]) % 2
        if odd:
            t = t[:, [0, 2, 1, 3]]
        tets.append(t)
    vt = np.stack(tets, axis=1).reshape(-1, 4).astype(np.int64)
    ed = [(0, 1), (1, 2), (2, 0), (0, 3), (1, 3), (2, 3)]
    pairs = np.stack([np.sort(vt[:, [p, q]], axis=1) for p, q in ed], axis=1).reshape(-1, 2)
    key = pairs[:, 0] * X.shape[0] + pairs[:, 1]
    uniq, first, inv = np.unique(key, return_index=True, return_inverse=True)
    order = np.argsort(first)           # number the edges by first appearance
    rank = np.empty_like(order)
    rank[order] = np.arange(order.shape[0])
    eid = rank[inv].reshape(-1, 6)
    ends = pairs[first[order]]
    coords = np.vstack([X, 0.5 * (X[ends[:, 0]] + X[ends[:, 1]])])
    conn = np.concatenate([vt, X.shape[0] + eid], axis=1).astype(np.int32)
    return {"dim": 3, "elem": "P2T", "n": n, "coords": coords, "conn": conn}


def thermal_p2t_problem(n: int, jitter: float = 0.1, sigma: float = 0.5,
                        seed_jitter: int = SEED_JITTER, seed_coef: int = SEED_COEF) -> dict:
    """3D thermal conduction on quadratic tetrahedra (u = 0 on the boundary, f = 1)."""
    m = tet10_mesh(n, jitter, seed_jitter)
    m["coef"] = lognormal(seed_coef, m["conn"].shape[0], sigma)
    m["bc_mask"], m["bc_val"] = thermal_bc(m)
    m["form"] = "thermal"
    m["source"] = 1.0
    return m


def thermal_q2s_problem(n: int, jitter: float = 0.15, sigma: float = 0.5,
                        seed_jitter: int = SEED_JITTER, seed_coef: int = SEED_COEF) -> dict:
    """3D thermal conduction on 20-node serendipity bricks (u = 0 on the boundary, f = 1)."""
    m = hex20_mesh(n, jitter, seed_jitter)
    m["coef"] = lognormal(seed_coef, m["conn"].shape[0], sigma)
    m["bc_mask"], m["bc_val"] = thermal_bc(m)
    m["form"] = "thermal"
    m["source"] = 1.0
    return m


def elastic_q2s_problem(n: int, jitter: float = 0.15, sigma: float = 0.5, nu: float = 0.3,
                        seed_jitter: int = SEED_JITTER, seed_coef: int = SEED_COEF) -> dict:
    """3D linear elasticity on 20-node serendipity bricks (the element of the
    cantilever beams, Sec. 4.2): x = 0 clamped, body force (0, 0, -1)."""
    m = hex20_mesh(n, jitter, seed_jitter)
    m["coef"] = lognormal(seed_coef, m["conn"].shape[0], sigma)  # Young's modulus E
    m["nu"] = nu
    m["body"] = (0.0, 0.0, -1.0)
    m["bc_mask"], m["bc_val"] = elastic_bc(m)
    m["form"] = "elastic"
    return m


# ----------------------------------------------------------------------------
# boundary data
# ----------------------------------------------------------------------------

def boundary_nodes(coords: np.ndarray, tol: float = 1e-14) -> np.ndarray:
    """Boolean mask of nodes on the boundary of the unit square / cube."""
    return np.any((coords <= tol) | (coords >= 1.0 - tol), axis=1)


def thermal_bc(mesh: dict) -> tuple[np.ndarray, np.ndarray]:
    """Dirichlet u = 0 on the whole boundary: (mask u8 [nn], values f64 [nn])."""
    m = boundary_nodes(mesh["coords"]).astype(np.uint8)
    return m, np.zeros(m.shape[0], dtype=np.float64)


def elastic_bc(mesh: dict) -> tuple[np.ndarray, np.ndarray]:
    """Clamp all three displacement components of the nodes on x = 0 (dof 3 node + c)."""
    clamp = mesh["coords"][:, 0] <= 1e-14
    m = np.repeat(clamp, 3).astype(np.uint8)
    return m, np.zeros(m.shape[0], dtype=np.float64)


def oseen_bc(mesh: dict) -> tuple[np.ndarray, np.ndarray]:
    """Lid-driven cavity velocity data plus a pressure pin, dof layout [u1 | u2 | p].

    u = (1, 0) on y = 1 without its two corners, u = 0 on the rest of the
    boundary; the pressure at vertex (0, 0) is pinned to 0.
    """
    c = mesh["coords"]
    n2 = c.shape[0]
    n1 = mesh["vcoords"].shape[0]
    bnd = boundary_nodes(c)
    lid = (c[:, 1] >= 1.0 - 1e-14) & (c[:, 0] > 1e-14) & (c[:, 0] < 1.0 - 1e-14)
    mask = np.zeros(2 * n2 + n1, dtype=np.uint8)
    val = np.zeros(2 * n2 + n1, dtype=np.float64)
    mask[:n2] = bnd
    mask[n2:2 * n2] = bnd
    val[:n2][lid] = 1.0
    mask[2 * n2] = 1  # pressure pin at vertex 0 = (0, 0)
    return mask, val


def advecting_field(coords: np.ndarray, seed: int = SEED_ADVECT, modes: int = 4) -> np.ndarray:
    """Divergence-free nodal field a = (d psi/dy, -d psi/dx), max |a| over nodes = 1.

    psi = sum_{kx,ky in 1..modes} c sin(pi kx x + p1) sin(pi ky y + p2) with
    c ~ N(0, 1) (mode m uses normal m) and phases uniform in [0, 2 pi)
    (draws 2 modes^2 + 2m and 2 modes^2 + 2m + 1).  Returns float64 [2, nn].
    """
    nm = modes * modes
    amp = normal(seed, nm)
    ph = uniform(seed, 2 * nm, offset=2 * nm) * (2.0 * np.pi)
    x, y = coords[:, 0], coords[:, 1]
    a = np.zeros((2, coords.shape[0]), dtype=np.float64)
    for m in range(nm):
        kx, ky = m // modes + 1, m % modes + 1
        p1, p2 = ph[2 * m], ph[2 * m + 1]
        sx, cx = np.sin(np.pi * kx * x + p1), np.cos(np.pi * kx * x + p1)
        sy, cy = np.sin(np.pi * ky * y + p2), np.cos(np.pi * ky * y + p2)
        a[0] += amp[m] * sx * np.pi * ky * cy
        a[1] -= amp[m] * np.pi * kx * cx * sy
    scale = np.sqrt((a * a).sum(axis=0)).max()
    return a / scale


# Boundary facets are faces of mesh elements, named (element, local face):
# triangle face f is the edge from vertex f to vertex (f + 1) % 3 (P2 adds the
# midpoint node 3 + f); hexahedron face 2 d + s is the face where reference
# coordinate d equals 2 s - 1.

SIDES = ("x0", "x1", "y0", "y1", "z0", "z1")


def box_facets(mesh: dict, sides=SIDES) -> tuple[np.ndarray, np.ndarray]:
    """Facets of the structured mesh on the given sides of the box.

    Returns (element int32 [nf], face uint8 [nf]) side by side in the order
    given, ascending element ids within a side (tetrahedra: the faces whose
    vertices lie on the side, face i opposite vertex i).  Triangle grid: square (i, j)
    holds elements 2 (j n + i) (v00, v10, v11) and 2 (j n + i) + 1 (v00, v11,
    v01); hexahedron (i, j, k) is element (k n + j) n + i.
    """
    n = mesh["n"]
    els, faces = [], []
    r = np.arange(n)
    if mesh["elem"] == "Q2Q":
        # element (i, j) = j n + i; edges (0,1|4) y = 0 side, (1,3|7) x = 1,
        # (3,2|5) y = 1, (2,0|6) x = 0
        for side in sides:
            axis, hi = "xyz".index(side[0]), side[1] == "1"
            if axis == 2:
                raise ValueError("a quadrilateral mesh has no z sides")
            k = n - 1 if hi else 0
            e = (r * n + k) if axis == 0 else (k * n + r)
            els.append(e.astype(np.int32))
            faces.append(np.full(n, (1 if hi else 3) if axis == 0 else (2 if hi else 0), np.uint8))
        return np.concatenate(els), np.concatenate(faces)
    if mesh["elem"] == "P2T":
        # tetrahedron face i (opposite vertex i) lies on a side when its three
        # vertices do (boundary nodes are not jittered)
        X, c = mesh["coords"], mesh["conn"][:, :4]
        fv = ((1, 2, 3), (0, 3, 2), (0, 1, 3), (0, 2, 1))
        for side in sides:
            axis, hi = "xyz".index(side[0]), side[1] == "1"
            on = np.abs(X[:, axis] - (1.0 if hi else 0.0)) <= 1e-14
            hit = np.stack([on[c[:, a]] & on[c[:, b]] & on[c[:, d]] for a, b, d in fv], axis=1)
            e, f = np.nonzero(hit)
            els.append(e.astype(np.int32))
            faces.append(f.astype(np.uint8))
        return np.concatenate(els), np.concatenate(faces)
    for side in sides:
        axis, hi = "xyz".index(side[0]), side[1] == "1"
        if mesh["elem"] in ("Q1", "Q2S"):  # bricks: element (k n + j) n + i, face 2 axis + side
            k, j, i = np.meshgrid(r, r, r, indexing="ij")
            idx = (i, j, k)[axis].ravel()
            e = ((k * n + j) * n + i).ravel()[idx == (n - 1 if hi else 0)]
            f = 2 * axis + int(hi)
        else:
            if axis == 2:
                raise ValueError("a triangle mesh has no z sides")
            if axis == 1:  # bottom edge of t = 0 (face 0), top edge of t = 1 (face 1)
                sq = (n - 1 if hi else 0) * n + r
                e, f = (2 * sq + 1, 1) if hi else (2 * sq, 0)
            else:  # right edge of t = 0 (face 1), left edge of t = 1 (face 2)
                sq = r * n + (n - 1 if hi else 0)
                e, f = (2 * sq, 1) if hi else (2 * sq + 1, 2)
        els.append(np.asarray(e, dtype=np.int64))
        faces.append(np.full(len(els[-1]), f, dtype=np.uint8))
    if not els:
        return np.zeros(0, np.int32), np.zeros(0, np.uint8)
    return np.concatenate(els).astype(np.int32), np.concatenate(faces)


def convection_facets(mesh: dict, sides, seed: int = SEED_FACET, h_sigma: float = 0.5) -> dict:
    """Robin (convection) data on the given sides: per facet h lognormal(0,
    h_sigma) (draws 2f, 2f + 1 of the normal stream) and T_env uniform in
    [0.5, 1.5) (draw f of stream seed + 1)."""
    e, f = box_facets(mesh, sides)
    nf = e.shape[0]
    return {"elem": e, "face": f, "h": lognormal(seed, nf, h_sigma), "t_env": 0.5 + uniform(seed + 1, nf)}


def radiation_facets(mesh: dict, sides, es=None, t_env=None, seed: int = SEED_FACET) -> dict:
    """Radiation data on the given sides: per facet es = e_m sigma^b
    (dimensionless; default uniform in [0.5, 1.0), draw f of stream seed + 3)
    and T_env (default uniform in [1.0, 1.5), draw f of stream seed + 4), or
    the constants given."""
    e, f = box_facets(mesh, sides)
    nf = e.shape[0]
    es_ = 0.5 + 0.5 * uniform(seed + 3, nf) if es is None else np.full(nf, float(es))
    te_ = 1.0 + 0.5 * uniform(seed + 4, nf) if t_env is None else np.full(nf, float(t_env))
    return {"elem": e, "face": f, "es": es_, "t_env": te_}


def traction_facets(mesh: dict, sides, stress=None, seed: int = SEED_FACET) -> dict:
    """Loaded-boundary data on the given sides: a 3 x 3 stress sigma^l per
    facet (row-major), the given one on every facet or standard normals
    (draws 9 f .. 9 f + 8 of stream seed + 2)."""
    e, f = box_facets(mesh, sides)
    nf = e.shape[0]
    if stress is None:
        s = normal(seed + 2, 9 * nf).reshape(nf, 3, 3)
    else:
        s = np.broadcast_to(np.asarray(stress, dtype=np.float64).reshape(1, 3, 3), (nf, 3, 3)).copy()
    return {"elem": e, "face": f, "stress": s}


# ----------------------------------------------------------------------------
# the synthetic workloads
# ----------------------------------------------------------------------------

def thermal_p1_problem(n: int = 64, jitter: float = 0.2, sigma: float = 0.5,
                       seed_jitter: int = SEED_JITTER, seed_coef: int = SEED_COEF) -> dict:
    """2D thermal conduction on jittered P1 triangles (64 x 64 grid: 8192 triangles)."""
    m = tri_mesh(n, 1, jitter, seed_jitter)
    m["coef"] = lognormal(seed_coef, m["conn"].shape[0], sigma)
    m["bc_mask"], m["bc_val"] = thermal_bc(m)
    m["form"] = "thermal"
    m["source"] = 1.0
    return m


def thermal_p2_problem(n: int, jitter: float = 0.2, sigma: float = 0.5,
                       seed_jitter: int = SEED_JITTER, seed_coef: int = SEED_COEF) -> dict:
    m = tri_mesh(n, 2, jitter, seed_jitter)
    m["coef"] = lognormal(seed_coef, m["conn"].shape[0], sigma)
    m["bc_mask"], m["bc_val"] = thermal_bc(m)
    m["form"] = "thermal"
    m["source"] = 1.0
    return m


def thermal_q1_problem(n: int, jitter: float = 0.15, sigma: float = 0.5,
                       seed_jitter: int = SEED_JITTER, seed_coef: int = SEED_COEF,
                       coef: np.ndarray | None = None) -> dict:
    m = hex_mesh(n, jitter, seed_jitter)
    m["coef"] = lognormal(seed_coef, m["conn"].shape[0], sigma) if coef is None else coef
    m["bc_mask"], m["bc_val"] = thermal_bc(m)
    m["form"] = "thermal"
    m["source"] = 1.0
    return m


def elastic_problem(n: int = 64, jitter: float = 0.15, sigma: float = 0.5, nu: float = 0.3,
                    seed_jitter: int = SEED_JITTER, seed_coef: int = SEED_COEF) -> dict:
    """3D linear elasticity on jittered Q1 hexahedra (64^3: 262,144 elements)."""
    m = hex_mesh(n, jitter, seed_jitter)
    m["coef"] = lognormal(seed_coef, m["conn"].shape[0], sigma)  # Young's modulus E
    m["nu"] = nu
    m["body"] = (0.0, 0.0, -1.0)
    m["bc_mask"], m["bc_val"] = elastic_bc(m)
    m["form"] = "elastic"
    return m


def elastic_box_problem(nx: int, ny: int, nz: int, jitter: float = 0.15, sigma: float = 0.5, nu: float = 0.3,
                        seed_jitter: int = SEED_JITTER, seed_coef: int = SEED_COEF) -> dict:
    """The elasticity workload of ``elastic_problem`` on an nx x ny x nz box of
    cubes of side 1 / nx (clamped at x = 0, body force (0, 0, -1))."""
    m = hex_box_mesh(nx, ny, nz, jitter, seed_jitter)
    m["coef"] = lognormal(seed_coef, m["conn"].shape[0], sigma)
    m["nu"] = nu
    m["body"] = (0.0, 0.0, -1.0)
    m["bc_mask"], m["bc_val"] = elastic_bc(m)
    m["form"] = "elastic"
    return m


def oseen_problem(n: int = 512, viscosity: float = 0.01, rho: float = 1.0,
                  seed_advect: int = SEED_ADVECT) -> dict:
    """Picard-linearised flow on Taylor-Hood P2-P1 triangles (512^2 grid: 524,288 elements)."""
    m = tri_mesh(n, 2, 0.0)
    m["advect"] = advecting_field(m["coords"], seed_advect)
    m["viscosity"] = viscosity
    m["rho"] = rho
    m["coef"] = np.ones(m["conn"].shape[0], dtype=np.float64)
    m["bc_mask"], m["bc_val"] = oseen_bc(m)
    m["form"] = "oseen"
    return m


def batch_specs(n_problems: int = 512, seed: int = SEED_BATCH,
                lo: float = 1e3, hi: float = 2e5) -> list[dict]:
    """Element type and grid size of each problem of the batched workload.

    Type: uniform draw 2p < 0.5 -> P1, < 0.8 -> P2, else Q1.  Size: element
    count log-uniform in [lo, hi] (draw 2p + 1), rounded to the nearest grid:
    2 n^2 triangles or n^3 hexahedra.
    """
    u = uniform(seed, 2 * n_problems)
    specs = []
    for p in range(n_problems):
        t = "P1" if u[2 * p] < 0.5 else ("P2" if u[2 * p] < 0.8 else "Q1")
        target = math.exp(math.log(lo) + u[2 * p + 1] * (math.log(hi) - math.log(lo)))
        if t == "Q1":
            n = max(2, int(round(target ** (1.0 / 3.0))))
        else:
            n = max(2, int(round(math.sqrt(target / 2.0))))
        specs.append({"type": t, "n": n,
                      "seed_jitter": 1_000_000 + 2 * p, "seed_coef": 1_000_001 + 2 * p})
    return specs


def batch_problem(spec: dict) -> dict:
    if spec["type"] == "P1":
        return thermal_p1_problem(spec["n"], 0.2, 0.5, spec["seed_jitter"], spec["seed_coef"])
    if spec["type"] == "P2":
        return thermal_p2_problem(spec["n"], 0.2, 0.5, spec["seed_jitter"], spec["seed_coef"])
    return thermal_q1_problem(spec["n"], 0.15, 0.5, spec["seed_jitter"], spec["seed_coef"])


def grf_cells(n: int = 128, corr_len: float = 0.1, sigma: float = 1.0,
              seed: int = SEED_GRF) -> np.ndarray:
    """Gaussian random field on the n^3 cells of the unit cube (x fastest).

    Squared-exponential covariance exp(-r^2 / (2 l^2)), sampled by filtering
    white noise in Fourier space on the periodic n^3 grid.  The filter's
    point variance sum_k filt(k)^2 / n^3 (Parseval) scales the field to
    standard deviation ``sigma`` in expectation, so the mean stays a proper
    zero-mean random component.  Returns float64 [n^3].
    """
    w = normal(seed, n ** 3).reshape(n, n, n)
    k = 2.0 * np.pi * np.fft.fftfreq(n, d=1.0 / n)
    kz, ky, kx = np.meshgrid(k, k, k, indexing="ij")
    filt = np.exp(-0.25 * corr_len ** 2 * (kx ** 2 + ky ** 2 + kz ** 2))
    g = np.fft.ifftn(np.fft.fftn(w) * filt).real
    g *= sigma / np.sqrt(np.sum(filt ** 2) / n ** 3)
    return g.ravel()


def grf_thermal_problem(n: int = 128, system: int = 0) -> dict:
    """3D thermal conduction on an unjittered Q1 grid with k = exp(GRF), f = 1, u = 0 on the boundary."""
    k = np.exp(grf_cells(n, seed=SEED_GRF + system))
    return thermal_q1_problem(n, 0.0, 0.0, coef=k)
