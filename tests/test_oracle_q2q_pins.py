"""Pins of the oracle's 8-node serendipity quadrilateral (the quadratic
serendipity rectangles of the 2D thermal case, Sec. 4.1) and of the
convection on its edges.

Expected values come from the basis's defining properties (nodal
interpolation, reproduction of the 8 serendipity monomials), exact Gauss
moments, the shoelace area of the straight-edged element, the closed-form
loads of a parallelogram (-A/12 at a vertex, A/3 at a midpoint), invariants
of the assembled Laplacian (zero row sums, symmetry, linear fields in the
kernel of jittered meshes, harmonic quadratics on affine ones), a
brute-force pattern, O(h^3) on affine cells and about O(h^2) on jittered ones
(the serendipity loss on non-affine cells) for a manufactured solution, and the
closed-form mass matrix of a straight 3-node edge.
"""
import itertools

import numpy as np
import scipy.sparse as sp

import gen

REF = np.array([[-1, -1], [1, -1], [-1, 1], [1, 1], [0, -1], [0, 1], [-1, 0], [1, 0]], float)
MONO = [(0, 0), (1, 0), (0, 1), (2, 0), (1, 1), (0, 2), (2, 1), (1, 2)]


def _quad(seed=3, amp=0.12):
    rng = np.random.default_rng(seed)
    V = np.array([[0, 0], [1, 0], [0, 1], [1, 1]], float) + rng.uniform(-amp, amp, (4, 2))
    return V, np.vstack([V, 0.5 * (V[0] + V[1]), 0.5 * (V[2] + V[3]), 0.5 * (V[0] + V[2]), 0.5 * (V[1] + V[3])])


def test_basis_interpolates_and_reproduces_the_space(orc):
    Nn = np.array([orc.shape(orc.Q2Q, r)[0] for r in REF])
    assert np.abs(Nn - np.eye(8)).max() == 0.0
    rng = np.random.default_rng(5)
    for x in rng.uniform(-1, 1, (8, 2)):
        N, dN = orc.shape(orc.Q2Q, x)
        for i, j in MONO:
            f = REF[:, 0] ** i * REF[:, 1] ** j
            assert abs(N @ f - x[0] ** i * x[1] ** j) < 1e-15
            g = np.array([i * x[0] ** max(i - 1, 0) * x[1] ** j, j * x[0] ** i * x[1] ** max(j - 1, 0)])
            assert np.abs(dN.T @ f - g).max() < 1e-14
    N, _ = orc.shape(orc.Q2Q, np.array([0.3, -0.4]))
    assert abs(N @ (REF[:, 0] ** 2 * REF[:, 1] ** 2) - (0.3 * 0.4) ** 2) > 1e-3


def test_gauss9_exact_to_degree5_per_variable(orc):
    pts, w = orc.quad(orc.QQUAD9)
    assert pts.shape == (9, 2)
    for a, b in itertools.product(range(6), repeat=2):
        exact = np.prod([0.0 if k % 2 else 2.0 / (k + 1) for k in (a, b)])
        assert abs(np.sum(w * pts[:, 0] ** a * pts[:, 1] ** b) - exact) < 1e-15
    assert abs(np.sum(w * pts[:, 0] ** 6) - 2.0 * 2.0 / 7.0) > 1e-3


def test_area_and_parallelogram_loads(orc):
    V, X = _quad()
    ring = V[[0, 1, 3, 2]]
    area = 0.5 * abs(np.sum(ring[:, 0] * np.roll(ring[:, 1], -1) - np.roll(ring[:, 0], -1) * ring[:, 1]))
    assert abs(orc.elem_measure(orc.Q2Q, orc.QQUAD9, X) - area) < 1e-15
    # a parallelogram: consistent loads -A/12 (vertices), A/3 (midpoints)
    P = np.array([[0.1, 0.2], [1.3, 0.5], [0.4, 1.1], [1.6, 1.4]])
    XP = np.vstack([P, 0.5 * (P[0] + P[1]), 0.5 * (P[2] + P[3]), 0.5 * (P[0] + P[2]), 0.5 * (P[1] + P[3])])
    e1, e2 = P[1] - P[0], P[2] - P[0]
    A = abs(e1[0] * e2[1] - e1[1] * e2[0])
    Ke, de, det = orc.elem_thermal(orc.Q2Q, orc.QQUAD9, XP, k=1.0, f=3.0)
    assert np.abs(de[:4] + 3.0 * A / 12).max() < 1e-14 and np.abs(de[4:] - 3.0 * A / 3).max() < 1e-14
    assert np.abs(Ke - Ke.T).max() < 1e-14 and np.abs(Ke.sum(axis=1)).max() < 1e-14
    ev = np.linalg.eigvalsh(Ke)
    assert abs(ev[0]) < 1e-13 and ev[1] > 1e-3 * ev[-1]


def _csr(s):
    n = s["row_ptr"].shape[0] - 1
    return sp.csr_matrix((s["val"], s["col"], s["row_ptr"]), shape=(n, n))


def test_laplacian_invariants(orc):
    prob = gen.thermal_q2q_problem(4)
    s = orc.assemble(prob, dirichlet=False)
    K = _csr(s)
    scale = np.abs(s["val"]).max()
    assert np.abs(K @ np.ones(K.shape[0])).max() < 1e-13 * scale
    assert abs(K - K.T).max() < 1e-14 * scale
    assert abs(s["d"].sum() - 1.0) < 1e-13
    prob["coef"] = np.full(prob["conn"].shape[0], 1.3)
    x = prob["coords"]
    inner = ~gen.boundary_nodes(x)
    s = orc.assemble(prob, dirichlet=False)
    u = 0.3 + 1.1 * x[:, 0] - 0.7 * x[:, 1]
    assert np.abs((_csr(s) @ u)[inner]).max() < 1e-13 * np.abs(s["val"]).max()
    prob = gen.thermal_q2q_problem(4, jitter=0.0)
    prob["coef"] = np.ones(prob["conn"].shape[0])
    x = prob["coords"]
    s = orc.assemble(prob, dirichlet=False)
    for u in (x[:, 0] ** 2 - x[:, 1] ** 2, x[:, 0] * x[:, 1] + 0.5 * x[:, 0]):
        assert np.abs((_csr(s) @ u)[inner]).max() < 1e-13 * np.abs(s["val"]).max()


def test_pattern_matches_brute_force(orc):
    prob = gen.thermal_q2q_problem(3)
    s = orc.assemble(prob, dirichlet=False)
    n = prob["coords"].shape[0]
    pairs = sorted({(int(a), int(b)) for el in prob["conn"] for a in el for b in el} | {(g, g) for g in range(n)})
    rows = np.repeat(np.arange(n), np.diff(s["row_ptr"]))
    assert list(zip(rows.tolist(), s["col"].tolist())) == pairs
    assert np.diff(s["row_ptr"]).max() == 21


def _mms_rates(orc, jitter):
    errs = []
    for n in (4, 8, 16):
        prob = gen.thermal_q2q_problem(n, jitter=jitter)
        prob["coef"] = np.ones(prob["conn"].shape[0])
        c = prob["coords"]
        u = np.sin(np.pi * c[:, 0]) * np.sin(np.pi * c[:, 1])
        s = orc.assemble(prob, fnodal=2 * np.pi ** 2 * u)
        x, _, rr = orc.pcg(s, tol=1e-13)
        assert rr <= 1e-12
        errs.append(np.sqrt(np.mean((x - u) ** 2)))
    return np.log(np.array(errs[:-1]) / np.array(errs[1:])) / np.log(2.0)


def test_mms_rates(orc):
    # affine (parallelogram) cells: the serendipity space holds all
    # quadratics, O(h^3) (observed 3.8, 3.9)
    assert _mms_rates(orc, 0.0).min() >= 2.7
    # jittered cells are not affine: serendipity elements then lose the
    # quadratics in physical coordinates (Arnold, Boffi and Falk, 2002) and
    # the rate falls to about 2 (observed 3.3, 2.1)
    assert _mms_rates(orc, 0.15).min() >= 1.8


def test_edges_tables_and_convection(orc):
    V, X = _quad(seed=6)
    centre = V.mean(axis=0)
    for face in range(4):
        loc = orc.facet_nodes(orc.Q2Q, face)
        Xf = X[loc]
        assert np.abs(Xf[2] - 0.5 * (Xf[0] + Xf[1])).max() < 1e-15  # the midpoint third
        t = Xf[1] - Xf[0]
        assert np.array([t[1], -t[0]]) @ (Xf[0] - centre) > 0       # counter-clockwise: outward on the right
        L = np.linalg.norm(t)
        Kf, df, meas = orc.facet_thermal(orc.Q2Q, Xf, h=1.5, t_env=0.8)
        assert abs(meas - L) < 1e-15
        M = L / 30.0 * np.array([[4, -1, 2], [-1, 4, 2], [2, 2, 16]])
        assert np.abs(Kf - 1.5 * M).max() < 1e-15
        assert np.abs(df - 1.5 * 0.8 * L * np.array([1, 1, 4]) / 6.0).max() < 1e-15
    # the four sides of the unit square: perimeter 4
    prob = gen.thermal_q2q_problem(5)
    e, f = gen.box_facets(prob, ("x0", "x1", "y0", "y1"))
    tot = sum(orc.facet_thermal(orc.Q2Q, prob["coords"][prob["conn"][el][orc.facet_nodes(orc.Q2Q, int(fa))]],
                                1.0, 1.0)[2] for el, fa in zip(e, f))
    assert abs(tot - 4.0) < 1e-13


def test_capacity_on_a_parallelogram(orc):
    """Mass matrix of the 8-node element on a parallelogram: total mass the
    area, row sums the consistent loads (-A/12, A/3), symmetric positive
    definite."""
    P = np.array([[0.1, 0.2], [1.3, 0.5], [0.4, 1.1], [1.6, 1.4]])
    XP = np.vstack([P, 0.5 * (P[0] + P[1]), 0.5 * (P[2] + P[3]), 0.5 * (P[0] + P[2]), 0.5 * (P[1] + P[3])])
    e1, e2 = P[1] - P[0], P[2] - P[0]
    A = abs(e1[0] * e2[1] - e1[1] * e2[0])
    Me, det = orc.elem_capacity(orc.Q2Q, XP, 2.0)
    assert abs(Me.sum() - 2.0 * A) < 1e-14
    assert np.abs(Me.sum(axis=1) - 2.0 * A * np.array([-1 / 12] * 4 + [1 / 3] * 4)).max() < 1e-14
    assert np.abs(Me - Me.T).max() < 1e-15 and np.linalg.eigvalsh(Me)[0] > 0
