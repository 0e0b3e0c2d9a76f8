"""Pins of the oracle's transient pieces: the capacity matrix C int N_a N_b
(the rate term -C(T, T_t) of Sec. 4.1), generalised-alpha time stepping
(Sec. 2.1 Eq. time_constraints and time_effective, Blocks C and D) and the
nonlinear radiation term e_m sigma^b (T, T_env^4 - T^4) of Sec. 4.1 inside its
Newton sub-steps.

Expected values come from exact barycentric integration, Kronecker products of
1D integrals, the total volume, the double root -rho_inf of the first-order
generalised-alpha amplification matrix at infinite stiffness (Jansen,
Whiting and Hulbert 2000), exact solutions of scalar ODEs, the matrix
exponential of the semi-discrete system, the steady state, closed-form facet
integrals at constant temperature, central differences of the radiation
load, and the exact solution of a radiating slab.
"""
from fractions import Fraction
from math import factorial

import numpy as np
import pytest
import scipy.linalg
import scipy.sparse as sp

import gen


def _csr(s):
    n = s["row_ptr"].shape[0] - 1
    return sp.csr_matrix((s["val"], s["col"], s["row_ptr"]), shape=(n, n))


def _scalar(v):
    return {"row_ptr": np.array([0, 1], np.int64), "col": np.array([0], np.int32), "val": np.array([float(v)]),
            "d": np.zeros(1)}


# ---------------------------------------------------------------------------
# capacity matrices
# ---------------------------------------------------------------------------

def _bary_integral(powers):
    # int over a triangle of area A of l0^i l1^j l2^k = 2A i! j! k! / (i + j + k + 2)!, per unit 2A
    i, j, k = powers
    return Fraction(factorial(i) * factorial(j) * factorial(k), factorial(i + j + k + 2))


def _p2_basis_poly(a):
    # P2 basis in barycentric monomials {(i, j, k): coefficient}
    if a < 3:
        e = [0, 0, 0]
        e2 = [0, 0, 0]
        e[a] = 2
        e2[a] = 1
        return {tuple(e): 2, tuple(e2): -1}  # l (2 l - 1)
    p, q = [(0, 1), (1, 2), (2, 0)][a - 3]
    e = [0, 0, 0]
    e[p] += 1
    e[q] += 1
    return {tuple(e): 4}


def _p2_mass_exact():
    M = np.zeros((6, 6), dtype=object)
    for a in range(6):
        for b in range(6):
            s = Fraction(0)
            for ea, ca in _p2_basis_poly(a).items():
                for eb, cb in _p2_basis_poly(b).items():
                    s += ca * cb * _bary_integral(tuple(x + y for x, y in zip(ea, eb)))
            M[a, b] = s
    return M  # times 2A


def test_p1_capacity_closed_form(orc):
    X = np.array([[0.1, 0.2], [0.9, 0.3], [0.4, 1.0]])
    A = 0.5 * ((X[1, 0] - X[0, 0]) * (X[2, 1] - X[0, 1]) - (X[2, 0] - X[0, 0]) * (X[1, 1] - X[0, 1]))
    M, det = orc.elem_capacity(orc.P1, X, 2.0)
    assert np.abs(M - 2.0 * A / 12.0 * (np.ones((3, 3)) + np.eye(3))).max() < 1e-16


def test_p2_capacity_exact_barycentric(orc):
    X = np.array([[0.1, 0.2], [0.9, 0.3], [0.4, 1.0]])
    X6 = np.vstack([X, 0.5 * (X[0] + X[1]), 0.5 * (X[1] + X[2]), 0.5 * (X[2] + X[0])])
    A = 0.5 * ((X[1, 0] - X[0, 0]) * (X[2, 1] - X[0, 1]) - (X[2, 0] - X[0, 0]) * (X[1, 1] - X[0, 1]))
    M, det = orc.elem_capacity(orc.P2, X6, 1.5)
    ref = 1.5 * 2.0 * A * _p2_mass_exact().astype(float)
    assert np.abs(M - ref).max() < 1e-15
    # the classical table: A / 180 [6 -1 -1 0 -4 0; ...; 32 16 16 ...]
    assert _p2_mass_exact()[0, 0] * 360 == 6 and _p2_mass_exact()[3, 3] * 360 == 32
    assert _p2_mass_exact()[0, 4] * 360 == -4 and _p2_mass_exact()[0, 3] == 0


def test_q1_capacity_box_kronecker(orc):
    a, b, c = 0.3, 0.5, 0.7
    X = np.array([[a * (k & 1), b * ((k >> 1) & 1), c * ((k >> 2) & 1)] for k in range(8)], float)
    M, det = orc.elem_capacity(orc.Q1, X, 1.3)
    m1 = lambda L: L / 6.0 * np.array([[2.0, 1.0], [1.0, 2.0]])
    ref = 1.3 * np.kron(m1(c), np.kron(m1(b), m1(a)))  # node a = i + 2j + 4k: x fastest
    assert np.abs(M - ref).max() < 1e-16


@pytest.mark.parametrize("kind", ["p1", "p2", "q1"])
def test_capacity_assembly_invariants(orc, kind):
    prob = {"p1": lambda: gen.thermal_p1_problem(7), "p2": lambda: gen.thermal_p2_problem(5),
            "q1": lambda: gen.thermal_q1_problem(4)}[kind]()
    Cel = gen.lognormal(77, prob["conn"].shape[0], 0.3)
    M = orc.capacity(prob, Cel)
    K = orc.assemble(prob, dirichlet=False)
    assert np.array_equal(M["row_ptr"], K["row_ptr"]) and np.array_equal(M["col"], K["col"])
    Md = _csr(M).toarray()
    assert np.abs(Md - Md.T).max() < 1e-17
    # total capacity = sum_e C_e |e|: constant C on the unit square / cube gives 1
    ones = orc.capacity(prob, np.ones_like(Cel))
    assert abs(ones["val"].sum() - 1.0) < 1e-13
    assert np.linalg.eigvalsh(Md).min() > 0


# ---------------------------------------------------------------------------
# generalised-alpha
# ---------------------------------------------------------------------------

def _decay_sequence(orc, rho, steps=8, stiff=1e8):
    prm = orc.genalpha_params(rho)
    phi, u, a = np.array([1.0]), np.array([-stiff]), np.zeros(1)
    out = []
    for _ in range(steps):
        phi, u, a, its = orc.genalpha(_scalar(stiff), _scalar(1.0), np.zeros(1), np.zeros(1, np.uint8),
                                      np.zeros(1), phi, u, a, prm, 1.0, 1)
        out.append(phi[0])
    return np.array(out)


@pytest.mark.parametrize("rho", [0.0, 0.25, 0.5, 0.8, 1.0])
def test_high_frequency_double_root(orc, rho):
    # at infinite stiffness both roots of the amplification matrix are -rho_inf:
    # phi_{n+2} - 2 lam phi_{n+1} + lam^2 phi_n = 0 with lam = -rho_inf
    s = _decay_sequence(orc, rho)
    lam = -rho
    res = s[2:] - 2 * lam * s[1:-1] + lam ** 2 * s[:-2]
    assert np.abs(res).max() <= 1e-6 * np.abs(s).max()
    if rho == 1.0:
        assert np.allclose(np.abs(s), 1.0, atol=1e-6)
    if rho == 0.0:
        assert np.abs(s[3:]).max() < 1e-6


@pytest.mark.parametrize("rho", [0.0, 0.5, 1.0])
def test_second_order_scalar(orc, rho):
    # m phi' + k phi = f, phi(0) = 0: phi(T) = f / k (1 - exp(-k T / m))
    m, k, f, T = 1.0, 2.0, 1.0, 1.0
    prm = orc.genalpha_params(rho)
    errs = []
    for steps in (10, 20, 40):
        phi, u, a, its = orc.genalpha(_scalar(k), _scalar(m), np.array([f]), np.zeros(1, np.uint8), np.zeros(1),
                                      np.zeros(1), np.array([f / m]), np.zeros(1), prm, T / steps, steps)
        errs.append(abs(phi[0] - f / k * (1.0 - np.exp(-k * T / m))))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert rates.min() > 1.9, (errs, rates)


def _heat_system(orc, kind="p1"):
    """Conduction with k = 1, f = 1, u = 0 on the boundary, unassembled
    Dirichlet rows: P1 triangles, 8-node quadrilaterals or 10-node
    tetrahedra (the elements of the paper's 2D and 3D thermal cases)."""
    prob = {"p1": lambda: gen.thermal_p1_problem(6), "q2q": lambda: gen.thermal_q2q_problem(4),
            "p2t": lambda: gen.thermal_p2t_problem(2)}[kind]()
    prob["coef"] = np.full(prob["conn"].shape[0], 1.0)
    K = orc.assemble(prob, dirichlet=False)
    M = orc.capacity(prob, np.full(prob["conn"].shape[0], 1.0))
    F = K["d"].copy()
    return prob, K, M, F


@pytest.mark.parametrize("kind", ["p1", "q2q", "p2t"])
def test_fe_heat_matches_matrix_exponential(orc, kind):
    prob, K, M, F = _heat_system(orc, kind)
    mask = prob["bc_mask"]
    free = mask == 0
    x = prob["coords"]
    phi0 = np.where(free, np.prod(np.sin(np.pi * x), axis=1), 0.0)
    Kd, Md = _csr(K).toarray()[np.ix_(free, free)], _csr(M).toarray()[np.ix_(free, free)]
    T = 0.05
    # exact semi-discrete solution: phi' = M^-1 (F - K phi)
    A = -np.linalg.solve(Md, Kd)
    g = np.linalg.solve(Md, F[free])
    ps = np.linalg.solve(Kd, F[free])  # steady state
    exact = ps + scipy.linalg.expm(A * T) @ (phi0[free] - ps)
    prm = orc.genalpha_params(0.5)
    u0 = orc.initial_rate(K, M, F, mask, phi0)
    assert np.abs(u0[free] - (g + A @ phi0[free])).max() < 1e-10 * np.abs(u0).max()
    errs = []
    for steps in (8, 16, 32):
        phi, u, a, its = orc.genalpha(K, M, F, mask, np.zeros_like(F), phi0, u0, np.zeros_like(F), prm,
                                      T / steps, steps)
        assert (its == 1).all()  # a linear form converges in one Newton solve
        errs.append(np.abs(phi[free] - exact).max())
        assert np.abs(phi[~free]).max() == 0
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert rates.min() > 1.9 and errs[-1] < 1e-4, (errs, rates)


@pytest.mark.parametrize("kind", ["p1", "q2q", "p2t"])
def test_steady_state_reached(orc, kind):
    prob, K, M, F = _heat_system(orc, kind)
    mask = prob["bc_mask"]
    free = mask == 0
    prm = orc.genalpha_params(0.0)
    phi0 = np.zeros_like(F)
    u0 = orc.initial_rate(K, M, F, mask, phi0)
    phi, u, a, its = orc.genalpha(K, M, F, mask, np.zeros_like(F), phi0, u0, np.zeros_like(F), prm, 10.0, 12)
    Kd = _csr(K).toarray()[np.ix_(free, free)]
    ps = np.linalg.solve(Kd, F[free])
    assert np.abs(phi[free] - ps).max() < 1e-10 * np.abs(ps).max()
    assert np.abs(u).max() < 1e-8 * np.abs(ps).max()


# ---------------------------------------------------------------------------
# radiation e_m sigma^b (T, T_env^4 - T^4) (Sec. 4.1) inside the Newton steps
# ---------------------------------------------------------------------------

def test_radiation_facet_constant_temperature(orc):
    es, te, T = 0.7, 1.3, 0.9
    # P1 edge of length 1, P2 edge of length 1.3, Q1 unit square face
    cases = [(orc.P1, np.array([[0.1, 0.2], [0.7, 1.0]]), 1.0, np.array([0.5, 0.5]),
              np.array([[1 / 3, 1 / 6], [1 / 6, 1 / 3]])),
             (orc.P2, np.array([[0.3, -0.2], [-0.9, 0.3], [-0.3, 0.05]]), 1.3, np.array([1 / 6, 1 / 6, 2 / 3]),
              np.array([[4, -1, 2], [-1, 4, 2], [2, 2, 16]]) / 30.0),
             (orc.Q1, np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [1, 1, 0]], float), 1.0, np.full(4, 0.25),
              np.kron(np.array([[2, 1], [1, 2]]) / 6.0, np.array([[2, 1], [1, 2]]) / 6.0))]
    for elem, X, L, intN, mass in cases:
        Kf, rf = orc.facet_radiation(elem, X, es, te, np.full(X.shape[0], T))
        assert np.abs(rf - es * (te ** 4 - T ** 4) * L * intN).max() < 1e-15
        assert np.abs(Kf - 4 * es * T ** 3 * L * mass).max() < 1e-15


def test_radiation_tangent_is_the_derivative(orc):
    rng = np.random.default_rng(4)
    X = np.array([[a & 1, (a >> 1) & 1, 0.0] for a in range(4)], float) + rng.uniform(-0.2, 0.2, (4, 3))
    T = 0.8 + 0.4 * rng.random(4)
    Kf, rf = orc.facet_radiation(orc.Q1, X, 0.6, 1.2, T)
    h = 1e-6
    for b in range(4):
        e = np.zeros(4)
        e[b] = h
        _, rp = orc.facet_radiation(orc.Q1, X, 0.6, 1.2, T + e)
        _, rm = orc.facet_radiation(orc.Q1, X, 0.6, 1.2, T - e)
        assert np.abs(-(rp - rm) / (2 * h) - Kf[:, b]).max() < 1e-8 * np.abs(Kf).max()


@pytest.mark.parametrize("kind", ["p1", "p2", "q1", "q2q", "p2t"])
def test_radiation_slab_steady_state(orc, kind):
    # T = T0 on x = 0, k dT/dn = es (T_env^4 - T^4) on x = 1, insulated
    # elsewhere, no source: T = T0 + b x with k b = es (T_env^4 - (T0 + b)^4)
    import scipy.optimize
    prob = {"p1": lambda: gen.thermal_p1_problem(6), "p2": lambda: gen.thermal_p2_problem(4),
            "q1": lambda: gen.thermal_q1_problem(3), "q2q": lambda: gen.thermal_q2q_problem(3),
            "p2t": lambda: gen.thermal_p2t_problem(2)}[kind]()
    k, es, T0, Te = 1.7, 0.8, 0.4, 1.5
    prob["coef"] = np.full(prob["conn"].shape[0], k)
    prob["source"] = 0.0
    x = prob["coords"]
    left = x[:, 0] <= 1e-14
    prob["bc_mask"] = left.astype(np.uint8)
    prob["bc_val"] = np.where(left, T0, 0.0)
    K = orc.assemble(prob, dirichlet=False)
    M = orc.capacity(prob, np.ones(prob["conn"].shape[0]))
    rad = gen.radiation_facets(prob, ("x1",), es=es, t_env=Te)
    phi0 = np.where(left, T0, T0)
    u0 = np.zeros_like(phi0)
    phi, u, a, its = orc.genalpha(K, M, K["d"], prob["bc_mask"], prob["bc_val"], phi0, u0, np.zeros_like(phi0),
                                  orc.genalpha_params(0.0), 50.0, 8, prob=prob, radiation=rad)
    # the physical root: T(1) = T0 + b > 0
    b = scipy.optimize.brentq(lambda b: k * b - es * (Te ** 4 - (T0 + b) ** 4), -T0, 5.0, xtol=1e-15)
    assert np.abs(phi - (T0 + b * x[:, 0])).max() < 1e-10
    assert its.max() <= 8 and its[0] >= 3  # nonlinear: several Newton solves, converging fast


def test_radiation_newton_uses_the_exact_tangent(orc):
    # with the tangent c1 (K + K_rad) + c2 / (b1 dt) M Newton converges
    # quadratically: a few solves per step (a tangent with the wrong scale on
    # the radiation part needs 11 or more here)
    prob = gen.thermal_q1_problem(3)
    k, T0, Te = 1.7, 0.4, 1.5
    prob["coef"] = np.full(prob["conn"].shape[0], k)
    prob["source"] = 0.0
    x = prob["coords"]
    left = x[:, 0] <= 1e-14
    prob["bc_mask"] = left.astype(np.uint8)
    prob["bc_val"] = np.where(left, T0, 0.0)
    K = orc.assemble(prob, dirichlet=False)
    M = orc.capacity(prob, np.ones(prob["conn"].shape[0]))
    rad = gen.radiation_facets(prob, ("x1", "y1", "z1"), es=0.8, t_env=Te)
    phi0 = np.full(x.shape[0], T0)
    u0 = orc.initial_rate(K, M, K["d"], prob["bc_mask"], phi0)
    phi, u, a, its = orc.genalpha(K, M, K["d"], prob["bc_mask"], prob["bc_val"], phi0, u0, np.zeros_like(phi0),
                                  orc.genalpha_params(0.5), 0.02, 6, newton_tol=1e-10, max_newton=30, prob=prob,
                                  radiation=rad)
    assert its.max() <= 7, its
