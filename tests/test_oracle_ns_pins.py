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


# ---------------------------------------------------------------------------
# the same form on Taylor-Hood tetrahedra (the 3D flow case)
# ---------------------------------------------------------------------------

def test_tetrahedron_tangent_matches_finite_differences(orc):
    rng = np.random.default_rng(8)
    V = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], float) * 0.9 + rng.uniform(-0.1, 0.1, (4, 3))
    U, P = rng.normal(size=(10, 3)), rng.normal(size=4)
    r, Ke, det = orc.elem_ns3(V, U, P, MU, RHO, TM, TC)
    assert det > 0
    h = 1e-6
    for c in (0, 7, 17, 29, 31):
        Up, Um, Pp, Pm = U.copy(), U.copy(), P.copy(), P.copy()
        if c < 30:
            Up.flat[c] += h
            Um.flat[c] -= h
        else:
            Pp[c - 30] += h
            Pm[c - 30] -= h
        fd = (orc.elem_ns3(V, Up, Pp, MU, RHO, TM, TC)[0] - orc.elem_ns3(V, Um, Pm, MU, RHO, TM, TC)[0]) / (2 * h)
        assert np.abs(Ke[:, c] - fd).max() < 1e-7 * np.abs(Ke).max()


def test_tetrahedra_poiseuille_is_an_exact_discrete_solution(orc):
    m = gen.tet10_mesh(2, 0.1)
    X, c = m["coords"], m["conn"]
    nv = 27  # the (n + 1)^3 vertices come first: the P1 pressure nodes
    n2 = X.shape[0]
    u = np.zeros((n2, 3))
    u[:, 0] = X[:, 1] * (1.0 - X[:, 1])
    p = -2.0 * MU * X[:nv, 0] + 0.3
    R = np.zeros(3 * n2 + nv)
    scale = 0.0
    for el in c:
        r, _, _ = orc.elem_ns3(X[el[:4]], u[el], p[el[:4]], MU, RHO, TM, TC)
        for a in range(10):
            for i in range(3):
                R[i * n2 + el[a]] += r[3 * a + i]
        for b in range(4):
            R[3 * n2 + el[b]] += r[30 + b]
        scale = max(scale, np.abs(orc.elem_ns3(X[el[:4]], np.ones((10, 3)), np.ones(4), MU, RHO, TM, TC)[0]).max())
    inner = ~gen.boundary_nodes(X)
    for i in range(3):
        assert np.abs(R[i * n2:(i + 1) * n2][inner]).max() < 1e-13 * scale
    assert np.abs(R[3 * n2:]).max() < 1e-13 * scale


def test_rotation_covariance(orc):
    """Rotating the element and the nodal velocities rotates the velocity
    residual and leaves the pressure residual unchanged (the form is built
    from vectors and scalars only): catches a dropped or misplaced component."""
    rng = np.random.default_rng(10)
    # 2D
    V, X = _tri(seed=9)
    U, P = rng.normal(size=(6, 2)), rng.normal(size=3)
    t = 0.7
    Q = np.array([[np.cos(t), -np.sin(t)], [np.sin(t), np.cos(t)]])
    r, _, _ = orc.elem_ns(V, U, P, MU, RHO, TM, TC)
    rq, _, _ = orc.elem_ns(V @ Q.T, U @ Q.T, P, MU, RHO, TM, TC)
    s = np.abs(r).max()
    assert np.abs(rq[:12].reshape(6, 2) - r[:12].reshape(6, 2) @ Q.T).max() < 1e-13 * s
    assert np.abs(rq[12:] - r[12:]).max() < 1e-13 * s
    # 3D
    V3 = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], float) * 0.9 + rng.uniform(-0.1, 0.1, (4, 3))
    U3, P3 = rng.normal(size=(10, 3)), rng.normal(size=4)
    Q3, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    if np.linalg.det(Q3) < 0:
        Q3[:, 0] *= -1.0  # a rotation keeps the vertex order positive
    r, _, _ = orc.elem_ns3(V3, U3, P3, MU, RHO, TM, TC)
    rq, _, _ = orc.elem_ns3(V3 @ Q3.T, U3 @ Q3.T, P3, MU, RHO, TM, TC)
    s = np.abs(r).max()
    assert np.abs(rq[:30].reshape(10, 3) - r[:30].reshape(10, 3) @ Q3.T).max() < 1e-12 * s
    assert np.abs(rq[30:] - r[30:]).max() < 1e-12 * s
