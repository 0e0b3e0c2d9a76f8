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


# ---------------------------------------------------------------------------
# the SUPG terms themselves (Sec. 4.3: tau^m rho (v_i,j u_j, R^m_i),
# tau^m (q_,i, R^m_i), tau^c (v_i,i, R^c)), on fields where the strong
# residuals have closed forms: u = A x + b (so grad u = A, Laplacian 0) and
# p = g . x + p0 give R^m = rho A (A x + b) + g and R^c = tr A.  The
# difference r(tau_m, tau_c) - r(0, 0) is compared with an independent
# evaluation of those three integrals on a collapsed (Duffy) Gauss-Legendre
# rule, a different exact rule from the oracle's; the form must also be
# affine in tau_m and tau_c separately.
# ---------------------------------------------------------------------------

def _collapsed_rule(dim, n=6):
    """Points (barycentric coordinates l_1..l_dim of the reference simplex)
    and weights of the collapsed Gauss-Legendre product rule, exact for
    polynomials of degree <= 2 n - 2 - dim on the unit simplex of volume
    1 / dim!."""
    xg, wg = np.polynomial.legendre.leggauss(n)
    xg, wg = 0.5 * (xg + 1.0), 0.5 * wg
    pts, wts = [], []
    if dim == 2:
        for s, ws in zip(xg, wg):
            for t, wt in zip(xg, wg):
                pts.append((s, t * (1.0 - s)))
                wts.append(ws * wt * (1.0 - s))
    else:
        for s, ws in zip(xg, wg):
            for t, wt in zip(xg, wg):
                for v, wv in zip(xg, wg):
                    pts.append((s, t * (1.0 - s), v * (1.0 - s) * (1.0 - t)))
                    wts.append(ws * wt * wv * (1.0 - s) ** 2 * (1.0 - t))
    return np.array(pts), np.array(wts)


def _supg_terms(V, A, b, g, rho, tm, tc):
    """The SUPG part of the residual on the affine Taylor-Hood simplex with
    vertices V (dim + 1 rows), evaluated independently: velocity rows
    (node-major, dof (a, i) at dim a + i) then pressure vertex rows."""
    dim = V.shape[1]
    E = V[1:] - V[0]                     # columns of the affine map
    Jm = E.T
    det = np.linalg.det(Jm)
    Ginv = np.linalg.inv(Jm)             # rows: gradients of l_1..l_dim
    gl = np.vstack([-Ginv.sum(axis=0), Ginv])  # gradients of the barycentrics
    edges = [(0, 1), (1, 2), (2, 0)] if dim == 2 else [(0, 1), (1, 2), (2, 0), (0, 3), (1, 3), (2, 3)]
    nv = dim + 1
    nn = nv + len(edges)
    pts, wts = _collapsed_rule(dim)
    rv = np.zeros((nn, dim))
    rp = np.zeros(nv)
    Rc = np.trace(A)
    for lam, w in zip(pts, wts):
        l = np.concatenate([[1.0 - lam.sum()], lam])
        x = V[0] + Jm @ lam
        u = A @ x + b
        Rm = rho * (A @ u) + g
        grads = [(4.0 * l[v] - 1.0) * gl[v] for v in range(nv)]
        grads += [4.0 * (l[q] * gl[p] + l[p] * gl[q]) for p, q in edges]
        wd = w * abs(det)
        for a, gN in enumerate(grads):
            adv = gN @ u
            rv[a] += wd * (tm * rho * adv * Rm + tc * gN * Rc)
        for v in range(nv):
            rp[v] += wd * tm * (gl[v] @ Rm)
    return np.concatenate([rv.ravel(), rp])


def _linear_state(V, A, b, g, p0):
    dim = V.shape[1]
    edges = [(0, 1), (1, 2), (2, 0)] if dim == 2 else [(0, 1), (1, 2), (2, 0), (0, 3), (1, 3), (2, 3)]
    X = np.vstack([V] + [0.5 * (V[p] + V[q]) for p, q in edges])
    return X @ A.T + b, V @ g + p0


def test_supg_terms_against_an_independent_evaluation(orc):
    rng = np.random.default_rng(21)
    for dim, elem in ((2, orc.elem_ns), (3, orc.elem_ns3)):
        V = np.vstack([np.zeros(dim), np.eye(dim)]) * 0.8 + rng.uniform(-0.1, 0.1, (dim + 1, dim))
        A = rng.normal(size=(dim, dim))  # tr A != 0: the continuity residual is on
        b, g, p0 = rng.normal(size=dim), rng.normal(size=dim), 0.7
        U, P = _linear_state(V, A, b, g, p0)
        tm, tc = 0.037, 0.021
        r00 = elem(V, U, P, MU, RHO, 0.0, 0.0)[0]
        rtt = elem(V, U, P, MU, RHO, tm, tc)[0]
        ref = _supg_terms(V, A, b, g, RHO, tm, tc)
        scale = np.abs(ref).max()
        assert scale > 1e-3 and np.abs(ref[:-(dim + 1)]).max() > 1e-3 and np.abs(ref[-(dim + 1):]).max() > 1e-4
        assert np.abs((rtt - r00) - ref).max() <= 1e-12 * scale
        # each term on its own (a flipped sign or a dropped rho in one of them fails here)
        assert np.abs((elem(V, U, P, MU, RHO, tm, 0.0)[0] - r00) - _supg_terms(V, A, b, g, RHO, tm, 0.0)).max() \
            <= 1e-12 * scale
        assert np.abs((elem(V, U, P, MU, RHO, 0.0, tc)[0] - r00) - _supg_terms(V, A, b, g, RHO, 0.0, tc)).max() \
            <= 1e-12 * scale


def test_supg_residual_is_affine_in_each_stabilisation_parameter(orc):
    rng = np.random.default_rng(22)
    for dim, elem, nu, npr in ((2, orc.elem_ns, 6, 3), (3, orc.elem_ns3, 10, 4)):
        V = np.vstack([np.zeros(dim), np.eye(dim)]) * 0.9 + rng.uniform(-0.1, 0.1, (dim + 1, dim))
        U, P = rng.normal(size=(nu, dim)), rng.normal(size=npr)  # a general (quadratic) state
        r = lambda tm, tc: elem(V, U, P, MU, RHO, tm, tc)[0]
        r00 = r(0.0, 0.0)
        dm, dc = r(0.05, 0.0) - r00, r(0.0, 0.04) - r00
        scale = np.abs(r00).max() + np.abs(dm).max() + np.abs(dc).max()
        assert np.abs(r(0.1, 0.0) - r00 - 2.0 * dm).max() <= 1e-13 * scale
        assert np.abs(r(0.0, 0.12) - r00 - 3.0 * dc).max() <= 1e-13 * scale
        assert np.abs(r(0.05, 0.04) - r00 - dm - dc).max() <= 1e-13 * scale
        assert np.abs(dm).max() > 1e-6 and np.abs(dc).max() > 1e-6
