"""Pins of the oracle's steady Navier-Stokes form with SUPG (Sec. 4.3) on
Taylor-Hood P2-P1 triangles and of its Newton tangent.

Expected values come from outside the routine: central finite differences of
its residual (the complex-step tangent), the pinned Picard (Oseen) element on
linear velocity fields (the SUPG-free residual equals the Oseen operator with
the advecting field set to the velocity), an exact steady flow (Poiseuille:
every interior velocity row and every pressure row vanishes, with the SUPG
terms switched on), and the quadratic convergence of Newton's method on the
lid-driven cavity.
"""
import numpy as np

import gen

MU, RHO, TM, TC = 0.05, 1.3, 0.02, 0.03


def _tri(seed=4):
    rng = np.random.default_rng(seed)
    V = np.array([[0.0, 0.0], [1.0, 0.1], [0.2, 0.9]]) + rng.uniform(-0.1, 0.1, (3, 2))
    X = np.vstack([V, 0.5 * (V[0] + V[1]), 0.5 * (V[1] + V[2]), 0.5 * (V[2] + V[0])])
    return V, X


def test_complex_step_tangent_matches_finite_differences(orc):
    V, X = _tri()
    rng = np.random.default_rng(6)
    U, P = rng.normal(size=(6, 2)), rng.normal(size=3)
    r, Ke, det = orc.elem_ns(V, U, P, MU, RHO, TM, TC)
    assert det > 0
    h = 1e-6
    fd = np.zeros((15, 15))
    for c in range(15):
        Up, Um, Pp, Pm = U.copy(), U.copy(), P.copy(), P.copy()
        if c < 12:
            Up.flat[c] += h
            Um.flat[c] -= h
        else:
            Pp[c - 12] += h
            Pm[c - 12] -= h
        fd[:, c] = (orc.elem_ns(V, Up, Pp, MU, RHO, TM, TC)[0] - orc.elem_ns(V, Um, Pm, MU, RHO, TM, TC)[0]) / (2 * h)
    assert np.abs(Ke - fd).max() < 1e-7 * np.abs(Ke).max()
    # the SUPG terms couple every block: u1-u2 and pressure-pressure entries exist
    assert np.abs(Ke[0:12:2, 1:12:2]).max() > 1e-3 and np.abs(Ke[12:, 12:]).max() > 1e-6


def test_without_supg_equals_the_oseen_operator_on_linear_fields(orc):
    V, X = _tri(seed=5)
    A_lin = np.array([[0.7, -0.4], [0.3, -0.7]])  # divergence-free is not needed here
    U = X @ A_lin.T + np.array([0.2, -0.1])        # linear: exact under both rules
    P = np.array([0.3, -1.2, 0.8])
    r, _, _ = orc.elem_ns(V, U, P, MU, RHO, 0.0, 0.0)
    A, BT, B, _, _ = orc.elem_oseen(X, U, MU, RHO)
    ru = np.stack([A @ U[:, i] + BT[i] @ P for i in range(2)], axis=1)   # [6][2]
    rp = B[0] @ U[:, 0] + B[1] @ U[:, 1]
    scale = np.abs(r).max()
    assert np.abs(r[:12].reshape(6, 2) - ru).max() < 1e-14 * scale * 10
    assert np.abs(r[12:] - rp).max() < 1e-14 * scale * 10


def test_poiseuille_is_an_exact_discrete_solution(orc):
    prob = gen.oseen_problem(5, viscosity=MU, rho=RHO)
    x = prob["coords"]
    n2, n1 = x.shape[0], prob["vcoords"].shape[0]
    state = np.concatenate([x[:, 1] * (1.0 - x[:, 1]), np.zeros(n2), -2.0 * MU * prob["vcoords"][:, 0] + 0.4])
    R, _ = orc.ns_system(prob, state, TM, TC)
    inner = ~gen.boundary_nodes(x)
    scale = np.abs(orc.ns_system(prob, np.ones(2 * n2 + n1), TM, TC)[0]).max()
    assert np.abs(R[:n2][inner]).max() < 1e-13 * scale
    assert np.abs(R[n2:2 * n2][inner]).max() < 1e-13 * scale
    assert np.abs(R[2 * n2:]).max() < 1e-13 * scale
    # a wrong pressure gradient leaves a residual
    bad = state.copy()
    bad[2 * n2:] *= 1.5
    assert np.abs(orc.ns_system(prob, bad, TM, TC)[0][:n2][inner]).max() > 1e-6


def test_newton_converges_quadratically_on_the_cavity(orc):
    prob = gen.oseen_problem(4, viscosity=0.02, rho=1.0)
    x, hist = orc.ns_newton(prob, 0.01, 0.01, tol=1e-13)
    assert hist[-1] <= 1e-13 * hist[0] and len(hist) <= 8
    # quadratic: once small, each residual is about the square of the previous
    small = [(a, b) for a, b in zip(hist[:-1], hist[1:]) if a < 1e-2 and b > 1e-15]
    assert small and all(b < 50.0 * a * a for a, b in small)
