"""Structure of the synthetic quadratic meshes (host logic, no method
arithmetic): conformity, orientation, counts and boundary sets of the
10-node tetrahedra (Kuhn's split), the 8-node quadrilaterals and the 20-node
bricks."""
from collections import Counter

import numpy as np

import gen


def test_kuhn_tetrahedra_conform_and_cover_the_cube():
    n = 4
    m = gen.tet10_mesh(n, 0.1)
    X, c = m["coords"], m["conn"]
    assert c.shape == (6 * n ** 3, 10)
    V = X[c[:, :4]]
    det = np.einsum("ij,ij->i", V[:, 1] - V[:, 0], np.cross(V[:, 2] - V[:, 0], V[:, 3] - V[:, 0]))
    assert (det > 0).all() and abs(det.sum() / 6 - 1.0) < 1e-13
    # every triangle is shared by two tetrahedra, except the 12 n^2 on the boundary
    faces = Counter(tuple(sorted(t[list(f)])) for t in c[:, :4] for f in ((1, 2, 3), (0, 3, 2), (0, 1, 3), (0, 2, 1)))
    assert set(faces.values()) <= {1, 2}
    bnd = [f for f, k in faces.items() if k == 1]
    assert len(bnd) == 12 * n ** 2
    on = np.any((X <= 1e-14) | (X >= 1 - 1e-14), axis=1)
    assert all(on[list(f)].all() for f in bnd)
    # one node per edge, shared by every tetrahedron around the edge
    ed = {}
    for t in c:
        for k, (p, q) in enumerate(((0, 1), (1, 2), (2, 0), (0, 3), (1, 3), (2, 3))):
            key = (min(t[p], t[q]), max(t[p], t[q]))
            assert ed.setdefault(key, t[4 + k]) == t[4 + k]
    assert len(ed) == X.shape[0] - (n + 1) ** 3
    # the box facets are exactly the boundary triangles
    e, f = gen.box_facets(m, gen.SIDES)
    fv = ((1, 2, 3), (0, 3, 2), (0, 1, 3), (0, 2, 1))
    got = sorted(tuple(sorted(c[el, list(fv[fa])])) for el, fa in zip(e, f))
    assert got == sorted(bnd)


def test_quad8_mesh_conforms():
    n = 5
    m = gen.quad8_mesh(n, 0.2)
    X, c = m["coords"], m["conn"]
    assert X.shape[0] == (n + 1) ** 2 + 2 * n * (n + 1) and c.shape == (n * n, 8)
    # counter-clockwise cells: positive signed area of the ring 0, 1, 3, 2
    ring = X[c[:, [0, 1, 3, 2]]]
    area = 0.5 * np.sum(ring[:, :, 0] * np.roll(ring[:, :, 1], -1, axis=1)
                        - np.roll(ring[:, :, 0], -1, axis=1) * ring[:, :, 1], axis=1)
    assert (area > 0).all() and abs(area.sum() - 1.0) < 1e-13
    # each midpoint node belongs to one edge (the same two vertices everywhere)
    ends = {}
    for t in c:
        for mid, (p, q) in zip(t[4:], ((0, 1), (2, 3), (0, 2), (1, 3))):
            key = (min(t[p], t[q]), max(t[p], t[q]))
            assert ends.setdefault(mid, key) == key
    assert Counter(Counter(c[:, 4:].ravel()).values()) == Counter({2: 2 * n * (n - 1), 1: 4 * n})
    e, f = gen.box_facets(m, ("x0", "x1", "y0", "y1"))
    assert e.shape[0] == 4 * n


def test_hex20_mesh_conforms():
    n = 3
    m = gen.hex20_mesh(n, 0.15)
    X, c = m["coords"], m["conn"]
    assert X.shape[0] == (n + 1) ** 3 + 3 * n * (n + 1) ** 2 and c.shape == (n ** 3, 20)
    pairs = [(0, 1), (2, 3), (4, 5), (6, 7), (0, 2), (1, 3), (4, 6), (5, 7), (0, 4), (1, 5), (2, 6), (3, 7)]
    for t in c:
        for k, (p, q) in enumerate(pairs):
            assert np.abs(X[t[8 + k]] - 0.5 * (X[t[p]] + X[t[q]])).max() < 1e-15
    # an interior edge node is shared by 4 bricks, a face edge by 2, a box edge by 1
    share = Counter(Counter(c[:, 8:].ravel()).values())
    assert share == Counter({4: 3 * n * (n - 1) ** 2, 2: 3 * n * 4 * (n - 1), 1: 12 * n})
