"""Pins of the oracle's 10-node (quadratic) tetrahedron, the quadratic simplex
of the paper's 3D experiments (Sec. 4.1, Sec. 4.3): basis, the collapsed
64-point rule, element matrices and assembled systems.

Expected values come from the basis's defining properties (nodal
interpolation, reproduction of all quadratics), the exact simplex moments
a! b! c! / (a + b + c + 3)!, the closed-form load moments of quadratic
simplices (-V/20 at a vertex, V/5 at an edge), invariants of the assembled
Laplacian (zero row sums, symmetry, one zero eigenvalue per element, linear
and harmonic quadratic fields in the kernel: straight-edged tetrahedra are
affine even when jittered), a brute-force pattern and the O(h^3) rate on a
manufactured solution.
"""
import itertools
from math import factorial

import numpy as np
import scipy.sparse as sp

import gen

REF = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], float)
EDGES = [(0, 1), (1, 2), (2, 0), (0, 3), (1, 3), (2, 3)]


def _ref_nodes():
    return np.vstack([REF] + [0.5 * (REF[p] + REF[q]) for p, q in EDGES])


def _tet(seed=3):
    rng = np.random.default_rng(seed)
    V = REF * 0.8 + rng.uniform(-0.1, 0.1, (4, 3)) + 0.3
    return V, np.vstack([V] + [0.5 * (V[p] + V[q]) for p, q in EDGES])


def test_basis_interpolates_and_reproduces_quadratics(orc):
    R = _ref_nodes()
    Nn = np.array([orc.shape(orc.P2T, r)[0] for r in R])
    assert np.abs(Nn - np.eye(10)).max() < 1e-15
    rng = np.random.default_rng(4)
    for x in rng.dirichlet(np.ones(4), 8)[:, 1:]:
        N, dN = orc.shape(orc.P2T, x)
        for i, j, k in itertools.product(range(3), repeat=3):
            if i + j + k > 2:
                continue
            f = R[:, 0] ** i * R[:, 1] ** j * R[:, 2] ** k
            assert abs(N @ f - x[0] ** i * x[1] ** j * x[2] ** k) < 1e-15
            g = np.array([i * x[0] ** max(i - 1, 0) * x[1] ** j * x[2] ** k,
                          j * x[0] ** i * x[1] ** max(j - 1, 0) * x[2] ** k,
                          k * x[0] ** i * x[1] ** j * x[2] ** max(k - 1, 0)])
            assert np.abs(dN.T @ f - g).max() < 1e-14
    x = np.array([0.2, 0.3, 0.1])
    N, _ = orc.shape(orc.P2T, x)
    assert abs(N @ (R[:, 0] * R[:, 1] * R[:, 2]) - 0.2 * 0.3 * 0.1) > 1e-3  # a cubic is not


def test_collapsed_rule_exact_to_degree_5(orc):
    pts, w = orc.quad(orc.QTET64)
    assert pts.shape == (64, 3) and (w > 0).all() and (pts.sum(axis=1) < 1).all() and (pts > 0).all()
    for a, b, c in itertools.product(range(6), repeat=3):
        if a + b + c > 5:
            continue
        exact = factorial(a) * factorial(b) * factorial(c) / factorial(a + b + c + 3)
        assert abs(np.sum(w * pts[:, 0] ** a * pts[:, 1] ** b * pts[:, 2] ** c) - exact) < 1e-16
    assert abs(np.sum(w * pts[:, 0] ** 6) - factorial(6) / factorial(9)) > 1e-9


def test_element_volume_load_and_stiffness(orc):
    V, X = _tet()
    vol = abs(np.linalg.det(V[1:] - V[0])) / 6
    assert abs(orc.elem_measure(orc.P2T, orc.QTET64, X) - vol) < 1e-16
    Ke, de, det = orc.elem_thermal(orc.P2T, orc.QTET64, X, k=1.7, f=2.0)
    assert abs(det - 6 * vol) < 1e-15
    assert np.abs(de[:4] + 2.0 * vol / 20).max() < 1e-16
    assert np.abs(de[4:] - 2.0 * vol / 5).max() < 1e-16
    assert np.abs(Ke - Ke.T).max() < 1e-14
    assert np.abs(Ke.sum(axis=1)).max() < 1e-14
    ev = np.linalg.eigvalsh(Ke)
    assert abs(ev[0]) < 1e-13 and ev[1] > 1e-3 * ev[-1]


def _csr(s):
    n = s["row_ptr"].shape[0] - 1
    return sp.csr_matrix((s["val"], s["col"], s["row_ptr"]), shape=(n, n))


def test_laplacian_invariants_and_harmonic_quadratics(orc):
    prob = gen.thermal_p2t_problem(3)
    s = orc.assemble(prob, dirichlet=False)
    K = _csr(s)
    scale = np.abs(s["val"]).max()
    assert np.abs(K @ np.ones(K.shape[0])).max() < 1e-13 * scale
    assert abs(K - K.T).max() < 1e-14 * scale
    assert abs(s["d"].sum() - 1.0) < 1e-13
    prob["coef"] = np.full(prob["conn"].shape[0], 1.3)
    s = orc.assemble(prob, dirichlet=False)
    x = prob["coords"]
    inner = ~gen.boundary_nodes(x)
    for u in (0.3 + 1.1 * x[:, 0] - 0.7 * x[:, 1] + 0.4 * x[:, 2],
              x[:, 0] ** 2 + x[:, 1] ** 2 - 2.0 * x[:, 2] ** 2 + 0.5 * x[:, 0] * x[:, 1] - 0.3 * x[:, 1] * x[:, 2]):
        assert np.abs((_csr(s) @ u)[inner]).max() < 1e-12 * np.abs(s["val"]).max()


def test_pattern_matches_brute_force(orc):
    prob = gen.thermal_p2t_problem(2)
    s = orc.assemble(prob, dirichlet=False)
    n = prob["coords"].shape[0]
    pairs = sorted({(int(a), int(b)) for el in prob["conn"] for a in el for b in el} | {(g, g) for g in range(n)})
    rows = np.repeat(np.arange(n), np.diff(s["row_ptr"]))
    assert list(zip(rows.tolist(), s["col"].tolist())) == pairs
    assert np.diff(s["row_ptr"]).max() == 65


def test_mms_third_order(orc):
    errs = []
    for n in (2, 4, 8):
        prob = gen.thermal_p2t_problem(n, jitter=0.1)
        prob["coef"] = np.ones(prob["conn"].shape[0])
        c = prob["coords"]
        u = np.prod(np.sin(np.pi * c), axis=1)
        s = orc.assemble(prob, fnodal=3 * np.pi ** 2 * u)
        x, _, rr = orc.pcg(s, tol=1e-13)
        assert rr <= 1e-12
        errs.append(np.sqrt(np.mean((x - u) ** 2)))
    rates = np.log(np.array(errs[:-1]) / np.array(errs[1:])) / np.log(2.0)
    assert rates.min() >= 2.7, (errs, rates)


# ---------------------------------------------------------------------------
# convection on the 6-node faces (Sec. 4.1, h(T, T_env - T) on the surface of
# the 3D thermal case)
# ---------------------------------------------------------------------------

# P2 triangle mass matrix times 180 / area (vertices, then the midpoints of
# edges (0,1), (1,2), (2,0)): the closed form of int N_a N_b
P2_MASS = np.array([[6, -1, -1, 0, -4, 0], [-1, 6, -1, 0, 0, -4], [-1, -1, 6, -4, 0, 0],
                    [0, 0, -4, 32, 16, 16], [-4, 0, 0, 16, 32, 16], [0, -4, 0, 16, 16, 32]], float)


def test_face_tables_orientation_and_midpoints(orc):
    V, X = _tet(seed=7)
    for face in range(4):
        loc = orc.facet_nodes(orc.P2T, face)
        assert len(loc) == 6 and face not in loc[:3]
        Xf = X[loc]
        n = np.cross(Xf[1] - Xf[0], Xf[2] - Xf[0])
        assert n @ (Xf[0] - V[face]) > 0  # outward: away from the opposite vertex
        for m, (p, q) in enumerate(((0, 1), (1, 2), (2, 0))):
            assert np.abs(Xf[3 + m] - 0.5 * (Xf[p] + Xf[q])).max() < 1e-15


def test_face_convection_closed_form(orc):
    _, X = _tet(seed=8)
    loc = orc.facet_nodes(orc.P2T, 2)
    Xf = X[loc]
    area = 0.5 * np.linalg.norm(np.cross(Xf[1] - Xf[0], Xf[2] - Xf[0]))
    Kf, df, meas = orc.facet_thermal(orc.P2T, Xf, h=1.7, t_env=0.6)
    assert abs(meas - area) < 1e-16
    assert np.abs(Kf - 1.7 * area / 180.0 * P2_MASS).max() < 1e-15
    assert np.abs(df - 1.7 * 0.6 * area * np.array([0, 0, 0, 1, 1, 1]) / 3.0).max() < 1e-15
    # radiation at a uniform temperature: load es (T_env^4 - T^4) int N_m,
    # tangent 4 es T^3 times the mass matrix
    Kr, rr = orc.facet_radiation(orc.P2T, Xf, 0.8, 1.3, np.full(6, 1.1))
    assert np.abs(rr - 0.8 * (1.3 ** 4 - 1.1 ** 4) * area * np.array([0, 0, 0, 1, 1, 1]) / 3.0).max() < 1e-14
    assert np.abs(Kr - 4 * 0.8 * 1.1 ** 3 * area / 180.0 * P2_MASS).max() < 1e-14


def test_assembled_convection_on_the_surface(orc):
    prob = gen.thermal_p2t_problem(3)
    base = orc.assemble(prob, dirichlet=False)
    fac = gen.convection_facets(prob, gen.SIDES)
    fac["h"] = np.full(fac["elem"].shape[0], 2.5)
    fac["t_env"] = np.full(fac["elem"].shape[0], 0.7)
    prob["facets"] = fac
    s = orc.assemble(prob, dirichlet=False)
    Kc = _csr(s) - _csr(base)
    one = np.ones(Kc.shape[0])
    assert abs(one @ Kc @ one - 2.5 * 6.0) < 1e-12          # h times the cube's surface
    assert abs((s["d"] - base["d"]).sum() - 2.5 * 0.7 * 6.0) < 1e-12
    x = prob["coords"]
    assert abs(x[:, 0] @ Kc @ one - 2.5 * 3.0) < 1e-12       # int x over the surface = 3
    assert abs(Kc - Kc.T).max() < 1e-15


def test_capacity_matrix_closed_form(orc):
    """Consistent mass matrix of the affine 10-node tetrahedron: V / 420 times
    [6 I - J on the vertices (off-diagonal 1), -4 between a vertex and an edge
    touching it, -6 between a vertex and the opposite edge, 32 on the edge
    diagonal, 16 between edges sharing a vertex, 8 between opposite edges]."""
    V, X = _tet(seed=12)
    vol = abs(np.linalg.det(V[1:] - V[0])) / 6
    Me, det = orc.elem_capacity(orc.P2T, X, 1.0)
    M = np.zeros((10, 10))
    for a in range(4):
        for b in range(4):
            M[a, b] = 6.0 if a == b else 1.0
    for k, (p, q) in enumerate(EDGES):
        for a in range(4):
            M[a, 4 + k] = M[4 + k, a] = -4.0 if a in (p, q) else -6.0
        for l, (r, t) in enumerate(EDGES):
            M[4 + k, 4 + l] = 32.0 if k == l else (16.0 if len({p, q} & {r, t}) == 1 else 8.0)
    assert np.abs(Me - vol / 420.0 * M).max() < 1e-15
    assert abs(Me.sum() - vol) < 1e-15
    assert np.abs(Me.sum(axis=1) - vol * np.array([-1 / 20] * 4 + [1 / 5] * 6)).max() < 1e-15


def test_radiation_tangent_is_the_derivative_on_a_face(orc):
    """Radiation on a 6-node face with a varying temperature: the tangent is
    minus the derivative of the load (central differences)."""
    rng = np.random.default_rng(12)
    V = np.array([[0.1, 0.0, 0.2], [1.1, 0.2, 0.0], [0.3, 0.9, 0.4]])
    Xf = np.vstack([V, 0.5 * (V[0] + V[1]), 0.5 * (V[1] + V[2]), 0.5 * (V[2] + V[0])])
    T = 0.7 + 0.5 * rng.random(6)
    Kf, _ = orc.facet_radiation(orc.P2T, Xf, 0.8, 1.3, T)
    h = 1e-6
    for b in range(6):
        e = np.zeros(6)
        e[b] = h
        _, rp = orc.facet_radiation(orc.P2T, Xf, 0.8, 1.3, T + e)
        _, rm = orc.facet_radiation(orc.P2T, Xf, 0.8, 1.3, T - e)
        assert np.abs(-(rp - rm) / (2 * h) - Kf[:, b]).max() < 1e-8 * np.abs(Kf).max()
