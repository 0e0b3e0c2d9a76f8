"""Pins of the oracle's 20-node serendipity brick (the quadratic serendipity
elements of the paper's experiments, Sec. 4.2): basis, 3 x 3 x 3 Gauss rule,
geometry and assembled systems.

Expected values come from the basis's defining properties (nodal
interpolation, reproduction of the serendipity polynomial space), exact
polynomial moments, the trilinear element's volume, invariants of the
assembled Laplacian (zero row sums, symmetry, harmonic quadratics in the
kernel on affine meshes, linear fields on jittered ones), a brute-force
pattern, and the O(h^3) convergence rate on a manufactured solution.
"""
import itertools

import numpy as np
import pytest
import scipy.sparse as sp

import gen


def _ref_nodes():
    pts = [[2 * (a & 1) - 1, 2 * ((a >> 1) & 1) - 1, 2 * ((a >> 2) & 1) - 1] for a in range(8)]
    for axis in range(3):
        d1, d2 = (1, 2) if axis == 0 else ((0, 2) if axis == 1 else (0, 1))
        for t in range(4):
            p = [0, 0, 0]
            p[d1] = 2 * (t & 1) - 1
            p[d2] = 2 * ((t >> 1) & 1) - 1
            pts.append(p)
    return np.array(pts, float)


# monomials x^i y^j z^k of the 20-dimensional serendipity space
SERENDIPITY = [(0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 1, 0), (0, 1, 1), (1, 0, 1), (1, 1, 1),
               (2, 0, 0), (0, 2, 0), (0, 0, 2), (2, 1, 0), (2, 0, 1), (1, 2, 0), (0, 2, 1), (1, 0, 2), (0, 1, 2),
               (2, 1, 1), (1, 2, 1), (1, 1, 2)]


def test_basis_interpolates_and_reproduces_the_space(orc):
    R = _ref_nodes()
    Nn = np.array([orc.shape(orc.Q2S, r)[0] for r in R])
    assert np.abs(Nn - np.eye(20)).max() == 0.0
    rng = np.random.default_rng(3)
    for x in rng.uniform(-1, 1, (8, 3)):
        N, dN = orc.shape(orc.Q2S, x)
        for (i, j, k) in SERENDIPITY:
            f = R[:, 0] ** i * R[:, 1] ** j * R[:, 2] ** k
            assert abs(N @ f - x[0] ** i * x[1] ** j * x[2] ** k) < 1e-14
            # gradient of the interpolant = gradient of the monomial
            g = np.array([i * x[0] ** max(i - 1, 0) * x[1] ** j * x[2] ** k,
                          j * x[0] ** i * x[1] ** max(j - 1, 0) * x[2] ** k,
                          k * x[0] ** i * x[1] ** j * x[2] ** max(k - 1, 0)])
            assert np.abs(dN.T @ f - g).max() < 1e-13
    # a monomial outside the space (x^2 y^2) is not reproduced
    x = np.array([0.3, -0.4, 0.2])
    N, _ = orc.shape(orc.Q2S, x)
    assert abs(N @ (R[:, 0] ** 2 * R[:, 1] ** 2) - (0.3 * 0.4) ** 2) > 1e-3


def test_gauss27_exact_to_degree5_per_variable(orc):
    pts, w = orc.quad(orc.QHEX27)
    assert pts.shape == (27, 3)
    for a, b, c in itertools.product(range(6), repeat=3):
        exact = np.prod([0.0 if k % 2 else 2.0 / (k + 1) for k in (a, b, c)])
        assert abs(np.sum(w * pts[:, 0] ** a * pts[:, 1] ** b * pts[:, 2] ** c) - exact) < 1e-14
    assert abs(np.sum(w * pts[:, 0] ** 6) - 8.0 / 7.0) > 1e-3


def test_volume_matches_the_trilinear_element(orc):
    rng = np.random.default_rng(5)
    V = np.array([[a & 1, (a >> 1) & 1, (a >> 2) & 1] for a in range(8)], float) + rng.uniform(-0.15, 0.15, (8, 3))
    X = np.vstack([V] + [0.5 * (V[a0] + V[a1]) for a0, a1 in
                         [(0, 1), (2, 3), (4, 5), (6, 7), (0, 2), (1, 3), (4, 6), (5, 7), (0, 4), (1, 5), (2, 6),
                          (3, 7)]])
    vol27 = orc.elem_measure(orc.Q2S, orc.QHEX27, X)
    vol8 = orc.elem_measure(orc.Q1, orc.QHEX8, V)  # detJ of a trilinear map: exact with 2 points
    assert abs(vol27 - vol8) < 1e-15


def _csr(s):
    n = s["row_ptr"].shape[0] - 1
    return sp.csr_matrix((s["val"], s["col"], s["row_ptr"]), shape=(n, n))


def test_laplacian_invariants(orc):
    prob = gen.thermal_q2s_problem(3)
    s = orc.assemble(prob, dirichlet=False)
    K = _csr(s)
    scale = np.abs(s["val"]).max()
    assert np.abs(K @ np.ones(K.shape[0])).max() < 1e-13 * scale
    assert abs(K - K.T).max() < 1e-14 * scale
    assert abs(s["d"].sum() - 1.0) < 1e-13
    # patch test on the jittered mesh: linear fields, constant k
    prob["coef"] = np.full(prob["conn"].shape[0], 1.3)
    s = orc.assemble(prob, dirichlet=False)
    K = _csr(s)
    x = prob["coords"]
    u = 0.3 + 1.1 * x[:, 0] - 0.7 * x[:, 1] + 0.4 * x[:, 2]
    inner = ~gen.boundary_nodes(x)
    assert np.abs((K @ u)[inner]).max() < 1e-13 * np.abs(s["val"]).max()


def test_harmonic_quadratic_in_the_kernel_on_affine_meshes(orc):
    prob = gen.thermal_q2s_problem(3, jitter=0.0)
    prob["coef"] = np.ones(prob["conn"].shape[0])
    s = orc.assemble(prob, dirichlet=False)
    x = prob["coords"]
    u = x[:, 0] ** 2 + x[:, 1] ** 2 - 2.0 * x[:, 2] ** 2 + 0.5 * x[:, 0] * x[:, 1] - 0.3 * x[:, 1] * x[:, 2]
    inner = ~gen.boundary_nodes(x)
    assert np.abs((_csr(s) @ u)[inner]).max() < 1e-13 * np.abs(s["val"]).max()


def test_pattern_matches_brute_force(orc):
    prob = gen.thermal_q2s_problem(2)
    s = orc.assemble(prob, dirichlet=False)
    n = prob["coords"].shape[0]
    pairs = sorted({(int(a), int(b)) for el in prob["conn"] for a in el for b in el} | {(g, g) for g in range(n)})
    rows = np.repeat(np.arange(n), np.diff(s["row_ptr"]))
    assert list(zip(rows.tolist(), s["col"].tolist())) == pairs
    assert np.diff(s["row_ptr"]).max() == 81  # a vertex of the 2 x 2 x 2 block


def test_mms_third_order(orc):
    errs = []
    ns = (2, 4, 8)
    for n in ns:
        prob = gen.thermal_q2s_problem(n, jitter=0.1)
        prob["coef"] = np.ones(prob["conn"].shape[0])
        c = prob["coords"]
        u = np.prod(np.sin(np.pi * c), axis=1)
        s = orc.assemble(prob, fnodal=3 * np.pi ** 2 * u)
        x, _, rr = orc.pcg(s, tol=1e-13)
        assert rr <= 1e-12
        errs.append(np.sqrt(np.mean((x - u) ** 2)))
    rates = np.log(np.array(errs[:-1]) / np.array(errs[1:])) / np.log(2.0)
    assert rates.min() >= 2.8, (errs, rates)
