"""Pins of the CPU oracle against what FEM and the mathematics fix.

Each test reaches the expected value by a route other than the oracle's own
quadrature loops: closed forms, exact rational integration over triangles,
Kronecker products of 1D integrals, invariants (symmetry, zero row sums,
rigid-body modes, the patch test, load sums), dense direct solves and observed
convergence rates on manufactured solutions.
"""
from fractions import Fraction
from math import factorial

import numpy as np
import pytest
import scipy.sparse as sp

import gen


# ---------------------------------------------------------------------------
# quadrature
# ---------------------------------------------------------------------------

def _tri_moment(i, j):
    # int over reference triangle of xi^i eta^j = i! j! / (i+j+2)!
    return factorial(i) * factorial(j) / factorial(i + j + 2)


@pytest.mark.parametrize("kind,deg", [(0, 2), (1, 4)])
def test_triangle_rules_exact_to_degree(orc, kind, deg):
    pts, w = orc.quad(kind)
    for i in range(deg + 1):
        for j in range(deg + 1 - i):
            got = np.sum(w * pts[:, 0] ** i * pts[:, 1] ** j)
            assert abs(got - _tri_moment(i, j)) < 5e-16, (i, j)
    # one degree higher is not integrated exactly by either rule
    errs = [abs(np.sum(w * pts[:, 0] ** i * pts[:, 1] ** (deg + 1 - i)) - _tri_moment(i, deg + 1 - i))
            for i in range(deg + 2)]
    assert max(errs) > 1e-6


def test_hex_gauss_exact_to_degree3_per_variable(orc):
    pts, w = orc.quad(2)
    for a in range(4):
        for b in range(4):
            for c in range(4):
                exact = np.prod([0.0 if k % 2 else 2.0 / (k + 1) for k in (a, b, c)])
                got = np.sum(w * pts[:, 0] ** a * pts[:, 1] ** b * pts[:, 2] ** c)
                assert abs(got - exact) < 1e-15
    got4 = np.sum(w * pts[:, 0] ** 4)
    assert abs(got4 - 8 * 2.0 / 5) > 0.1


# ---------------------------------------------------------------------------
# shape functions
# ---------------------------------------------------------------------------

NODES = {
    0: np.array([[0, 0], [1, 0], [0, 1]], float),
    1: np.array([[0, 0], [1, 0], [0, 1], [0.5, 0], [0.5, 0.5], [0, 0.5]], float),
    2: np.array([[2 * (a & 1) - 1, 2 * ((a >> 1) & 1) - 1, 2 * ((a >> 2) & 1) - 1] for a in range(8)], float),
}


@pytest.mark.parametrize("elem", [0, 1, 2])
def test_basis_partition_kronecker_reproduction(orc, elem):
    rng = np.random.default_rng(0)
    dim = 3 if elem == 2 else 2
    nodes = NODES[elem]
    for a, xa in enumerate(nodes):
        N, _ = orc.shape(elem, xa)
        e = np.zeros(len(nodes))
        e[a] = 1.0
        assert np.allclose(N, e, atol=1e-15)
    for _ in range(20):
        xi = rng.uniform(-1, 1, dim) if elem == 2 else rng.dirichlet(np.ones(3))[1:]
        N, dN = orc.shape(elem, xi)
        assert abs(N.sum() - 1.0) < 1e-14
        assert np.abs(dN.sum(axis=0)).max() < 1e-14
        # linear fields are reproduced, with their gradients
        c = rng.normal(size=dim)
        assert abs(N @ (nodes @ c) - xi @ c) < 1e-14
        assert np.allclose(dN.T @ (nodes @ c), c, atol=1e-14)
        if elem == 1:  # quadratic fields too
            f = lambda x: 1 + x[..., 0] * x[..., 1] - 2 * x[..., 0] ** 2 + 3 * x[..., 1] ** 2
            assert abs(N @ f(nodes) - f(xi)) < 1e-13


# ---------------------------------------------------------------------------
# geometry
# ---------------------------------------------------------------------------

def test_triangle_measure_is_shoelace(orc):
    m = gen.tri_mesh(6, 1, 0.2)
    for e in range(m["conn"].shape[0]):
        X = m["coords"][m["conn"][e]]
        area = 0.5 * ((X[1, 0] - X[0, 0]) * (X[2, 1] - X[0, 1]) - (X[2, 0] - X[0, 0]) * (X[1, 1] - X[0, 1]))
        assert abs(orc.elem_measure(0, 0, X) - area) < 1e-16


@pytest.mark.parametrize("mesh", ["p1", "p2", "q1"])
def test_total_measure_is_one(orc, mesh):
    if mesh == "q1":
        m = gen.hex_mesh(5, 0.15)
        tot = sum(orc.elem_measure(2, 2, m["coords"][c]) for c in m["conn"])
    else:
        m = gen.tri_mesh(7, 1 if mesh == "p1" else 2, 0.2)
        elem, q = (0, 0) if mesh == "p1" else (1, 1)
        tot = sum(orc.elem_measure(elem, q, m["coords"][c]) for c in m["conn"])
    assert abs(tot - 1.0) < 1e-13


# ---------------------------------------------------------------------------
# element matrices against closed forms / exact integration
# ---------------------------------------------------------------------------

def test_p1_reference_triangle_closed_form(orc):
    X = np.array([[0, 0], [1, 0], [0, 1]], float)
    Ke, de, _ = orc.elem_thermal(0, 0, X, 2.0, 1.0)
    ref = 2.0 / 2 * np.array([[2, -1, -1], [-1, 1, 0], [-1, 0, 1]], float)
    assert np.allclose(Ke, ref, atol=1e-15)
    assert np.allclose(de, np.full(3, 1.0 / 6), atol=1e-16)


def test_p1_jittered_matches_gradient_formula(orc):
    m = gen.tri_mesh(5, 1, 0.2)
    for e in range(m["conn"].shape[0]):
        X = m["coords"][m["conn"][e]]
        Minv = np.linalg.inv(np.column_stack([np.ones(3), X]))  # rows: (1, x, y) -> lambda
        G = Minv[1:, :].T  # G[a] = grad lambda_a
        area = 0.5 * abs(np.linalg.det(np.column_stack([np.ones(3), X])))
        Ke, de, _ = orc.elem_thermal(0, 0, X, 1.7, 1.0)
        assert np.allclose(Ke, 1.7 * area * G @ G.T, rtol=1e-13, atol=1e-13)
        assert np.allclose(de, area / 3, rtol=1e-14)


# exact integration of barycentric polynomials {(i, j, k): coefficient}

def _pmul(p, q):
    r = {}
    for (a, ca) in p.items():
        for (b, cb) in q.items():
            k = (a[0] + b[0], a[1] + b[1], a[2] + b[2])
            r[k] = r.get(k, 0) + ca * cb
    return r


def _padd(p, q, s=1):
    r = dict(p)
    for k, c in q.items():
        r[k] = r.get(k, 0) + s * c
    return r


def _pint(p, area):
    tot = Fraction(0)
    for (i, j, k), c in p.items():
        tot += c * Fraction(2 * factorial(i) * factorial(j) * factorial(k), factorial(i + j + k + 2))
    return tot * area


def _lam(k):
    e = [0, 0, 0]
    e[k] = 1
    return {tuple(e): Fraction(1)}


ONE = {(0, 0, 0): Fraction(1)}


def _p2_basis_and_grads(X):
    """P2 basis as barycentric polynomials and its gradient components, exactly."""
    x = [Fraction(float(v)) for v in X[:3, 0]]
    y = [Fraction(float(v)) for v in X[:3, 1]]
    a2 = (x[1] - x[0]) * (y[2] - y[0]) - (x[2] - x[0]) * (y[1] - y[0])
    gl = [((y[1] - y[2]) / a2, (x[2] - x[1]) / a2),
          ((y[2] - y[0]) / a2, (x[0] - x[2]) / a2),
          ((y[0] - y[1]) / a2, (x[1] - x[0]) / a2)]
    N, G = [], []
    for i in range(3):
        N.append(_padd(_pmul(_lam(i), {k: 2 * v for k, v in _lam(i).items()}), _lam(i), -1))
        d4 = _padd({k: 4 * v for k, v in _lam(i).items()}, ONE, -1)
        G.append([{k: v * gl[i][c] for k, v in d4.items()} for c in range(2)])
    for p, q in ((0, 1), (1, 2), (2, 0)):
        N.append({k: 4 * v for k, v in _pmul(_lam(p), _lam(q)).items()})
        G.append([_padd({k: 4 * v * gl[p][c] for k, v in _lam(q).items()},
                        {k: 4 * v * gl[q][c] for k, v in _lam(p).items()}) for c in range(2)])
    return N, G, a2 / 2


def test_p2_jittered_matches_exact_rational_integrals(orc):
    m = gen.tri_mesh(3, 2, 0.2)
    for e in range(0, m["conn"].shape[0], 3):
        X = m["coords"][m["conn"][e]]
        N, G, area = _p2_basis_and_grads(X)
        Ke, de, _ = orc.elem_thermal(1, 0, X, 1.0, 1.0)  # 3-point rule is exact here
        Ke6, de6, _ = orc.elem_thermal(1, 1, X, 1.0, 1.0)
        for a in range(6):
            exact_d = float(_pint(N[a], area))
            assert abs(de[a] - exact_d) < 1e-16 and abs(de6[a] - exact_d) < 1e-16
            for b in range(6):
                ex = float(_pint(_padd(_pmul(G[a][0], G[b][0]), _pmul(G[a][1], G[b][1])), area))
                assert abs(Ke[a, b] - ex) < 1e-13 * max(1.0, abs(ex))
                assert abs(Ke6[a, b] - ex) < 1e-13 * max(1.0, abs(ex))


def _kron3(az, ay, ax):
    return np.kron(az, np.kron(ay, ax))


def _cube_1d(h):
    S = np.array([[1, -1], [-1, 1]], float) / h   # int phi_i' phi_j'
    M = h * np.array([[2, 1], [1, 2]], float) / 6  # int phi_i phi_j
    Cm = np.array([[-0.5, -0.5], [0.5, 0.5]])      # Cm[i, j] = int phi_i' phi_j
    return S, M, Cm


def _cube_D(h):
    """D[c][cp][a, b] = int d_c N_a d_cp N_b over a cube of side h (a = i + 2j + 4k)."""
    S, M, Cm = _cube_1d(h)
    D = [[None] * 3 for _ in range(3)]
    for c in range(3):
        for cp in range(3):
            f = []
            for axis in range(3):  # x, y, z
                if axis == c and axis == cp:
                    f.append(S)
                elif axis == c:
                    f.append(Cm)          # derivative on the test function
                elif axis == cp:
                    f.append(Cm.T)        # derivative on the trial function
                else:
                    f.append(M)
            D[c][cp] = _kron3(f[2], f[1], f[0])
    return D


def test_q1_thermal_cube_kronecker(orc):
    h = 0.37
    X = NODES[2] * 0.5 * h + 0.5 * h + np.array([0.1, -0.2, 0.3])
    Ke, de, _ = orc.elem_thermal(2, 2, X, 2.5, 1.0)
    S, M, _ = _cube_1d(h)
    ref = 2.5 * (_kron3(M, M, S) + _kron3(M, S, M) + _kron3(S, M, M))
    assert np.allclose(Ke, ref, rtol=1e-14, atol=1e-15)
    # per unit k: diagonal h/3, edge neighbour 0, face and body diagonal -h/12
    assert abs(ref[0, 0] / 2.5 - h / 3) < 1e-15 and abs(ref[0, 1]) < 1e-15
    assert abs(ref[0, 3] / 2.5 + h / 12) < 1e-15 and abs(ref[0, 7] / 2.5 + h / 12) < 1e-15
    assert np.allclose(de, h ** 3 / 8, rtol=1e-14)


def test_q1_elastic_cube_kronecker(orc):
    h = 0.5
    X = NODES[2] * 0.5 * h
    E, nu = 3.0, 0.3
    lam = E * nu / ((1 + nu) * (1 - 2 * nu))
    mu = E / (2 * (1 + nu))
    Ke, de, _ = orc.elem_elastic(X, E, nu, (0.0, 0.0, -1.0))
    D = _cube_D(h)
    lap = D[0][0] + D[1][1] + D[2][2]
    ref = np.zeros((24, 24))
    for c in range(3):
        for cp in range(3):
            # lambda d_c N_a d_cp N_b + mu d_cp N_a d_c N_b (+ mu grad.grad on the diagonal)
            blk = lam * D[c][cp] + mu * D[cp][c]
            if c == cp:
                blk = blk + mu * lap
            ref[c::3, cp::3] = blk
    assert np.allclose(Ke, ref, rtol=1e-13, atol=1e-14)
    assert np.allclose(de[2::3], -h ** 3 / 8, rtol=1e-14) and np.allclose(de[0::3], 0.0)


def _affine_hex(J0, shift):
    return NODES[2] @ J0.T + shift


def test_q1_sheared_parallelepiped_exact(orc):
    """Affine (non-symmetric Jacobian) hexahedron: 2-point Gauss is exact, and
    the exact integrals follow from reference 1D integrals and the constant J."""
    J0 = np.array([[0.30, 0.05, -0.02], [0.04, 0.25, 0.06], [-0.03, 0.07, 0.35]])
    X = _affine_hex(J0, np.array([0.2, 0.1, 0.4]))
    # reference cube [-1,1]^3 integrals of dN/dxi: 1D matrices on [-1, 1]
    S, M, Cm = _cube_1d(2.0)
    Dref = _cube_D(2.0)  # int_ref dxi_i N_a dxi_j N_b
    Jinv = np.linalg.inv(J0)
    det = np.linalg.det(J0)
    Dphys = [[sum(Jinv[i, c] * Jinv[j, cp] * Dref[i][j] for i in range(3) for j in range(3)) * det
              for cp in range(3)] for c in range(3)]
    Ke, _, _ = orc.elem_thermal(2, 2, X, 1.0, 1.0)
    assert np.allclose(Ke, Dphys[0][0] + Dphys[1][1] + Dphys[2][2], rtol=1e-12, atol=1e-14)
    E, nu = 2.0, 0.25
    lam = E * nu / ((1 + nu) * (1 - 2 * nu))
    mu = E / (2 * (1 + nu))
    Kel, _, _ = orc.elem_elastic(X, E, nu)
    lap = Dphys[0][0] + Dphys[1][1] + Dphys[2][2]
    for c in range(3):
        for cp in range(3):
            blk = lam * Dphys[c][cp] + mu * Dphys[cp][c] + (mu * lap if c == cp else 0)
            assert np.allclose(Kel[c::3, cp::3], blk, rtol=1e-12, atol=1e-14)


# ---------------------------------------------------------------------------
# flow element
# ---------------------------------------------------------------------------

def test_oseen_element_exact_for_constant_advection(orc):
    m = gen.tri_mesh(3, 2, 0.2)
    a = (0.6, -0.3)
    mu, rho = 0.01, 1.3
    for e in range(0, m["conn"].shape[0], 4):
        X = m["coords"][m["conn"][e]]
        aN = np.tile(a, (6, 1))
        A, BT, B, Mp, _ = orc.elem_oseen(X, aN, mu, rho)
        N, G, area = _p2_basis_and_grads(X)
        Mlin = [_lam(0), _lam(1), _lam(2)]
        fa = [Fraction(v) for v in a]
        for ia in range(6):
            adv = _padd({k: v * fa[0] for k, v in G[ia][0].items()},
                        {k: v * fa[1] for k, v in G[ia][1].items()})
            for ib in range(6):
                visc = _padd(_pmul(G[ia][0], G[ib][0]), _pmul(G[ia][1], G[ib][1]))
                ex = float(Fraction(mu) * _pint(visc, area) - Fraction(rho) * _pint(_pmul(adv, N[ib]), area))
                assert abs(A[ia, ib] - ex) < 1e-14 * max(1.0, abs(ex)) + 1e-16
        for i in range(2):
            for pa in range(3):
                for vb in range(6):
                    ex = float(_pint(_pmul(Mlin[pa], G[vb][i]), area))
                    assert abs(B[i, pa, vb] - ex) < 1e-15
                    assert abs(BT[i, vb, pa] + ex) < 1e-15
        for pa in range(3):
            assert abs(Mp[pa] - float(_pint(_pmul(Mlin[pa], Mlin[pa]), area))) < 1e-16


# ---------------------------------------------------------------------------
# assembled systems: invariants
# ---------------------------------------------------------------------------

def _csr(s):
    n = s["row_ptr"].shape[0] - 1
    return sp.csr_matrix((s["val"], s["col"], s["row_ptr"]), shape=(n, n))


@pytest.mark.parametrize("kind", ["p1", "p2", "q1"])
def test_neumann_laplacian_rows_sum_to_zero_and_symmetric(orc, kind):
    prob = {"p1": lambda: gen.thermal_p1_problem(8), "p2": lambda: gen.thermal_p2_problem(5),
            "q1": lambda: gen.thermal_q1_problem(4)}[kind]()
    s = orc.assemble(prob, dirichlet=False)
    K = _csr(s)
    scale = np.abs(s["val"]).max()
    assert np.abs(K @ np.ones(K.shape[0])).max() < 1e-13 * scale
    assert abs(K - K.T).max() < 1e-14 * scale
    assert abs(s["d"].sum() - 1.0) < 1e-13  # f = 1 on the unit square / cube


@pytest.mark.parametrize("kind", ["p1", "q1"])
def test_patch_test_linear_field(orc, kind):
    prob = gen.thermal_p1_problem(8) if kind == "p1" else gen.thermal_q1_problem(4)
    prob["coef"] = np.full(prob["conn"].shape[0], 1.3)  # the patch test needs constant k
    s = orc.assemble(prob, dirichlet=False)
    K = _csr(s)
    c = prob["coords"]
    u = 0.3 + 1.1 * c[:, 0] - 0.7 * c[:, 1] + (0.4 * c[:, 2] if c.shape[1] == 3 else 0)
    inner = ~gen.boundary_nodes(c)
    assert np.abs((K @ u)[inner]).max() < 1e-13 * np.abs(s["val"]).max()


def test_elastic_rigid_modes_symmetry_load(orc):
    prob = gen.elastic_problem(4)
    s = orc.assemble(prob, dirichlet=False)
    K = _csr(s)
    x = prob["coords"]
    scale = np.abs(s["val"]).max()
    modes = []
    for c in range(3):
        t = np.zeros_like(x)
        t[:, c] = 1
        modes.append(t.ravel())
    for w in np.eye(3):
        modes.append(np.cross(w, x).ravel())
    for u in modes:
        assert np.abs(K @ u).max() < 1e-13 * scale
    assert abs(K - K.T).max() < 1e-14 * scale
    assert abs(s["d"][2::3].sum() + 1.0) < 1e-13 and np.abs(s["d"][0::3]).max() == 0
    # patch test (constant E): a linear displacement field has zero interior residual
    prob["coef"] = np.full(prob["conn"].shape[0], 2.1)
    s = orc.assemble(prob, dirichlet=False)
    K = _csr(s)
    scale = np.abs(s["val"]).max()
    A = np.array([[0.1, 0.2, -0.1], [0.05, -0.3, 0.2], [0.3, 0.1, 0.15]])
    u = (x @ A.T).ravel()
    inner = np.repeat(~gen.boundary_nodes(x), 3)
    assert np.abs((K @ u)[inner]).max() < 1e-13 * scale


def test_oseen_assembled_invariants(orc):
    prob = gen.oseen_problem(6)
    n2 = prob["coords"].shape[0]
    s = orc.assemble(prob, dirichlet=False)
    K = _csr(s).toarray()
    A1 = K[:n2, :n2]
    B1 = K[2 * n2:, :n2]
    BT1 = K[:n2, 2 * n2:]
    assert np.abs(K[:n2, n2:2 * n2]).max() == 0  # no u1-u2 coupling
    assert np.allclose(A1, K[n2:2 * n2, n2:2 * n2], atol=0)
    assert np.abs(B1 @ np.ones(n2)).max() < 1e-14  # B annihilates constant velocity
    assert np.allclose(BT1, -B1.T, atol=1e-16)
    # viscous part has zero row sums: rebuild with rho = 0
    p0 = dict(prob)
    p0["rho"] = 0.0
    K0 = _csr(orc.assemble(p0, dirichlet=False)).toarray()
    assert np.abs(K0[:n2, :n2] @ np.ones(n2)).max() < 1e-15
    # constant advection: convection block is skew on interior dofs
    pc = dict(prob)
    pc["advect"] = np.tile(np.array([[0.7], [-0.4]]), (1, n2))
    pc["viscosity"] = 0.0
    Kc = _csr(orc.assemble(pc, dirichlet=False)).toarray()[:n2, :n2]
    inner = ~gen.boundary_nodes(prob["coords"])
    S = (Kc + Kc.T)[np.ix_(inner, inner)]
    assert np.abs(S).max() < 1e-14
    # diagonal of the consistent P1 mass: each triangle gives 3 x area / 6
    assert abs(s["pmass"].sum() - 0.5) < 1e-14


# ---------------------------------------------------------------------------
# pattern: brute force set of dof pairs and closed-form counts
# ---------------------------------------------------------------------------

def _brute_pattern(prob):
    pairs = set()
    conn = prob["conn"]
    if prob["form"] == "thermal":
        n = prob["coords"].shape[0]
        for el in conn:
            pairs.update((int(a), int(b)) for a in el for b in el)
    elif prob["form"] == "elastic":
        n = 3 * prob["coords"].shape[0]
        for el in conn:
            pairs.update((3 * int(a) + c, 3 * int(b) + d) for a in el for b in el
                         for c in range(3) for d in range(3))
    else:
        n2 = prob["coords"].shape[0]
        n = 2 * n2 + prob["vcoords"].shape[0]
        for el, pe in zip(conn, prob["vconn"]):
            for i in range(2):
                pairs.update((i * n2 + int(a), i * n2 + int(b)) for a in el for b in el)
                pairs.update((i * n2 + int(a), 2 * n2 + int(b)) for a in el for b in pe)
                pairs.update((2 * n2 + int(b), i * n2 + int(a)) for a in el for b in pe)
    pairs.update((g, g) for g in range(n))
    return n, sorted(pairs)


@pytest.mark.parametrize("kind", ["p1", "p2", "q1", "el", "os"])
def test_pattern_matches_brute_force(orc, kind):
    prob = {"p1": lambda: gen.thermal_p1_problem(5), "p2": lambda: gen.thermal_p2_problem(4),
            "q1": lambda: gen.thermal_q1_problem(3), "el": lambda: gen.elastic_problem(3),
            "os": lambda: gen.oseen_problem(3)}[kind]()
    s = orc.assemble(prob, dirichlet=False)
    n, pairs = _brute_pattern(prob)
    rows = np.repeat(np.arange(n), np.diff(s["row_ptr"]))
    got = list(zip(rows.tolist(), s["col"].tolist()))
    assert got == pairs


def test_pattern_closed_form_counts(orc):
    for n in (3, 8, 64):
        s = orc.assemble(gen.thermal_p1_problem(n, jitter=0.0), dirichlet=False)
        assert s["col"].shape[0] == (n + 1) ** 2 + 2 * (3 * n * n + 2 * n)
    for n in (2, 5):
        s = orc.assemble(gen.elastic_problem(n, jitter=0.0), dirichlet=False)
        assert s["col"].shape[0] == 9 * (4 + 3 * (n - 1)) ** 3


# ---------------------------------------------------------------------------
# Dirichlet elimination and solvers against dense direct solves
# ---------------------------------------------------------------------------

def test_dirichlet_elimination_equals_partitioned_solve(orc):
    prob = gen.thermal_p1_problem(6)
    rng = np.random.default_rng(3)
    prob["bc_val"] = np.where(prob["bc_mask"] > 0, rng.normal(size=prob["bc_mask"].shape), 0.0)
    full = orc.assemble(prob, dirichlet=False)
    K = _csr(full).toarray()
    b = prob["bc_mask"].astype(bool)
    i = ~b
    xi = np.linalg.solve(K[np.ix_(i, i)], full["d"][i] - K[np.ix_(i, b)] @ prob["bc_val"][b])
    s = orc.assemble(prob)
    x = np.linalg.solve(_csr(s).toarray(), s["d"])
    assert np.allclose(x[b], prob["bc_val"][b], atol=1e-15)
    assert np.allclose(x[i], xi, rtol=1e-11, atol=1e-14)
    Kd = _csr(s).toarray()
    assert np.abs(Kd[np.ix_(i, b)]).max() == 0 and np.abs(Kd[np.ix_(b, i)]).max() == 0
    assert np.allclose(np.diag(Kd)[b], 1.0)


@pytest.mark.parametrize("kind", ["p1", "el"])
def test_pcg_matches_dense_solve(orc, kind):
    prob = gen.thermal_p1_problem(12) if kind == "p1" else gen.elastic_problem(4)
    s = orc.assemble(prob)
    x, it, rr = orc.pcg(s, tol=1e-12)
    assert it > 0 and rr <= 1e-12
    xd = np.linalg.solve(_csr(s).toarray(), s["d"])
    assert np.linalg.norm(x - xd) <= 1e-9 * np.linalg.norm(xd)


def test_gmres_matches_dense_solve(orc):
    prob = gen.oseen_problem(4)
    s = orc.assemble(prob)
    pd = orc.oseen_precond(s, prob)
    x, it, rr = orc.gmres(s, pd, m=50, tol=1e-11)
    assert it > 0 and rr <= 1e-11
    xd = np.linalg.solve(_csr(s).toarray(), s["d"])
    assert np.linalg.norm(x - xd) <= 1e-7 * np.linalg.norm(xd)
    x5, it5, rr5 = orc.gmres(s, np.ones_like(pd), m=5, tol=1e-10, maxit=200000)
    assert rr5 <= 1e-10 and np.linalg.norm(x5 - xd) <= 1e-6 * np.linalg.norm(xd)


# ---------------------------------------------------------------------------
# convergence on manufactured solutions
# ---------------------------------------------------------------------------

def _mms_error(orc, prob):
    c = prob["coords"]
    dim = c.shape[1]
    u = np.prod(np.sin(np.pi * c), axis=1)
    prob["coef"] = np.ones(prob["conn"].shape[0])
    s = orc.assemble(prob, fnodal=dim * np.pi ** 2 * u)
    x, _, rr = orc.pcg(s, tol=1e-13)  # PCG itself is pinned against dense solves below
    assert rr <= 1e-12
    return np.sqrt(np.mean((x - u) ** 2))


@pytest.mark.parametrize("kind,ns,rate", [("p1", (16, 32, 64), 1.9), ("p2", (4, 8, 16), 2.9),
                                          ("q1", (8, 16, 32), 1.8)])
def test_mms_convergence_rate(orc, kind, ns, rate):
    errs = []
    for n in ns:
        if kind == "p1":
            prob = gen.thermal_p1_problem(n, jitter=0.2)
        elif kind == "p2":
            prob = gen.thermal_p2_problem(n, jitter=0.2)
        else:
            prob = gen.thermal_q1_problem(n, jitter=0.15)
        errs.append(_mms_error(orc, prob))
    rates = np.log(np.array(errs[:-1]) / np.array(errs[1:])) / np.log(np.array(ns[1:]) / np.array(ns[:-1]))
    assert rates.min() >= rate, (errs, rates)


# ---------------------------------------------------------------------------
# convolution layers of the learned preconditioner
# ---------------------------------------------------------------------------

def test_conv3d_fwd_matches_independent_correlation(orc):
    from scipy.ndimage import correlate
    rng = np.random.default_rng(21)
    x = rng.normal(size=(5, 6, 7, 3))
    w = rng.normal(size=(4, 3, 27))
    b = rng.normal(size=4)
    out = orc.conv3d_fwd(x, w, b)
    ref = np.zeros_like(out)
    for co in range(4):
        acc = np.full(x.shape[:3], b[co])
        for ci in range(3):
            acc += correlate(x[..., ci], w[co, ci].reshape(3, 3, 3), mode="constant", cval=0.0)
        ref[..., co] = acc
    assert np.abs(out - ref).max() < 1e-12
    r = orc.conv3d_fwd(x, w, b, relu=True)
    assert np.abs(r - np.maximum(ref, 0.0)).max() < 1e-12


def test_conv3d_gradients_central_differences(orc):
    rng = np.random.default_rng(22)
    x = rng.normal(size=(4, 5, 3, 2))
    w = rng.normal(size=(3, 2, 27))
    b = rng.normal(size=3)
    g = rng.normal(size=(4, 5, 3, 3))  # loss = sum(g * conv(x))

    def loss(xx, ww, bb):
        return float(np.sum(g * orc.conv3d_fwd(xx, ww, bb)))

    gin = orc.conv3d_bwd_data(g, w, 2)
    gw, gb = orc.conv3d_bwd_weight(x, g)
    h = 1e-6
    for idx in [(0, 0, 0, 0), (3, 4, 2, 1), (2, 2, 1, 0)]:
        xp, xm = x.copy(), x.copy()
        xp[idx] += h
        xm[idx] -= h
        fd = (loss(xp, w, b) - loss(xm, w, b)) / (2 * h)
        assert abs(fd - gin[idx]) <= 1e-6 * max(1.0, abs(fd))
    for idx in [(0, 0, 0), (2, 1, 13), (1, 0, 26)]:
        wp, wm = w.copy(), w.copy()
        wp[idx] += h
        wm[idx] -= h
        fd = (loss(x, wp, b) - loss(x, wm, b)) / (2 * h)
        assert abs(fd - gw[idx]) <= 1e-6 * max(1.0, abs(fd))
    for c in range(3):
        bp, bm = b.copy(), b.copy()
        bp[c] += h
        bm[c] -= h
        fd = (loss(x, w, bp) - loss(x, w, bm)) / (2 * h)
        assert abs(fd - gb[c]) <= 1e-6 * max(1.0, abs(fd))


@pytest.mark.parametrize("make", [lambda: gen.elastic_problem(6), lambda: gen.thermal_q1_problem(5),
                                  lambda: gen.thermal_p1_problem(9), lambda: gen.thermal_p2_problem(7),
                                  lambda: gen.elastic_q2s_problem(3), lambda: gen.thermal_p2t_problem(3)],
                         ids=["elastic_q1", "thermal_q1", "thermal_p1", "thermal_p2", "elastic_q2s", "thermal_p2t"])
def test_threaded_oracle_is_bit_identical(orc, make):
    """The all-core build of the oracle (OpenMP, used as the CPU baseline)
    gives the serial oracle's K and d bit for bit."""
    import os
    prob = make()
    a = orc.assemble(prob)
    try:
        b = orc.assemble_threads(prob, max(2, os.cpu_count() or 2))
    except RuntimeError:
        pytest.skip("no OpenMP build of the oracle on this host")
    for k in ("row_ptr", "col", "val", "d"):
        assert np.array_equal(a[k], b[k]), k
