"""Pins of the oracle's terms on the 8-node faces of the 20-node brick
(convection, Sec. 4.1; the loaded boundary (d_i, sigma^l_ij n_j) of the
cantilever beams, Sec. 4.2): face tables, closed forms on flat faces and
the balance of a uniform stress over the closed surface."""
import numpy as np

import gen


def _brick(seed=3, amp=0.12):
    rng = np.random.default_rng(seed)
    V = np.array([[a & 1, (a >> 1) & 1, (a >> 2) & 1] for a in range(8)], float) + rng.uniform(-amp, amp, (8, 3))
    pairs = [(0, 1), (2, 3), (4, 5), (6, 7), (0, 2), (1, 3), (4, 6), (5, 7), (0, 4), (1, 5), (2, 6), (3, 7)]
    return V, np.vstack([V] + [0.5 * (V[p] + V[q]) for p, q in pairs])


def test_face_tables_match_the_quadrilateral_convention(orc):
    V, X = _brick()
    centre = V.mean(axis=0)
    for face in range(6):
        loc = orc.facet_nodes(orc.Q2S, face)
        assert len(loc) == 8
        assert loc[:4] == orc.facet_nodes(orc.Q1, face)  # the vertices as on the Q1 brick
        Xf = X[loc]
        for j in range(2):  # 4 + j: between face vertices 2j and 2j + 1
            assert np.abs(Xf[4 + j] - 0.5 * (Xf[2 * j] + Xf[2 * j + 1])).max() < 1e-15
        for i in range(2):  # 6 + i: between face vertices i and i + 2
            assert np.abs(Xf[6 + i] - 0.5 * (Xf[i] + Xf[i + 2])).max() < 1e-15
        # outward: the traction of sigma = I is the outward area vector
        df = orc.facet_traction(face, Xf, np.eye(3), elem=orc.Q2S)
        assert df.sum(axis=0) @ (Xf[:4].mean(axis=0) - centre) > 0


def test_flat_face_closed_forms(orc):
    # a flat parallelogram face of area A: int N_m = -A/12 (vertices), A/3 (midpoints)
    V = np.array([[a & 1, (a >> 1) & 1, (a >> 2) & 1] for a in range(8)], float) @ np.array(
        [[1.2, 0.1, 0.0], [0.2, 0.9, 0.1], [0.0, 0.1, 1.1]]).T
    pairs = [(0, 1), (2, 3), (4, 5), (6, 7), (0, 2), (1, 3), (4, 6), (5, 7), (0, 4), (1, 5), (2, 6), (3, 7)]
    X = np.vstack([V] + [0.5 * (V[p] + V[q]) for p, q in pairs])
    for face in range(6):
        Xf = X[orc.facet_nodes(orc.Q2S, face)]
        An = np.cross(Xf[1] - Xf[0], Xf[2] - Xf[0])
        A = np.linalg.norm(An)
        mom = A * np.array([-1 / 12] * 4 + [1 / 3] * 4)
        Kf, df, meas = orc.facet_thermal(orc.Q2S, Xf, 1.7, 0.4)
        assert abs(meas - A) < 1e-14
        assert np.abs(Kf.sum(axis=1) - 1.7 * mom).max() < 1e-14 and np.abs(df - 1.7 * 0.4 * mom).max() < 1e-14
        sigma = np.array([[0.3, -0.2, 0.5], [0.1, 0.7, -0.4], [0.2, 0.0, 0.9]])
        dt = orc.facet_traction(face, Xf, sigma, elem=orc.Q2S)
        n = An / A * np.sign(An @ (Xf[:4].mean(axis=0) - V.mean(axis=0)))
        assert np.abs(dt - np.outer(mom, sigma @ n)).max() < 1e-14


def test_uniform_stress_balances_over_the_closed_surface(orc):
    prob = gen.elastic_q2s_problem(3)
    prob["body"] = (0.0, 0.0, 0.0)
    base = orc.assemble(prob, dirichlet=False)
    fac = gen.traction_facets(prob, gen.SIDES, stress=np.array([[0.3, -0.2, 0.5], [0.1, 0.7, -0.4], [0.2, 0.0, 0.9]]))
    prob["facets"] = fac
    s = orc.assemble(prob, dirichlet=False)
    load = (s["d"] - base["d"]).reshape(-1, 3)
    assert np.abs(load.sum(axis=0)).max() < 1e-13        # sigma n integrates to zero over a closed surface
    x = prob["coords"]
    # first moment: sum_a x_a (x) f_a = V sigma^T for a uniform stress (divergence theorem)
    M = x.T @ load
    assert np.abs(M - np.array([[0.3, -0.2, 0.5], [0.1, 0.7, -0.4], [0.2, 0.0, 0.9]]).T).max() < 1e-12


def test_flat_face_mass_matrix_by_independent_quadrature(orc):
    """The whole face matrix (not only its row sums): on a flat parallelogram
    face the map is affine with Jacobian A / 4, so Kf = h A / 4 int N_a N_b
    over [-1, 1]^2, here by 5 x 5 Gauss-Legendre (numpy) of the pinned
    8-node basis."""
    V = np.array([[a & 1, (a >> 1) & 1, (a >> 2) & 1] for a in range(8)], float) @ np.array(
        [[1.2, 0.1, 0.0], [0.2, 0.9, 0.1], [0.0, 0.1, 1.1]]).T
    pairs = [(0, 1), (2, 3), (4, 5), (6, 7), (0, 2), (1, 3), (4, 6), (5, 7), (0, 4), (1, 5), (2, 6), (3, 7)]
    X = np.vstack([V] + [0.5 * (V[p] + V[q]) for p, q in pairs])
    g, w = np.polynomial.legendre.leggauss(5)
    ref = np.zeros((8, 8))
    for u, wu in zip(g, w):
        for v, wv in zip(g, w):
            N, _ = orc.shape(orc.Q2Q, np.array([u, v]))
            ref += wu * wv * np.outer(N, N)
    for face in (0, 3, 5):
        Xf = X[orc.facet_nodes(orc.Q2S, face)]
        A = np.linalg.norm(np.cross(Xf[1] - Xf[0], Xf[2] - Xf[0]))
        Kf, _, _ = orc.facet_thermal(orc.Q2S, Xf, 1.7, 0.4)
        assert np.abs(Kf - 1.7 * A / 4.0 * ref).max() < 1e-14


def test_radiation_on_flat_faces_closed_forms(orc):
    """Radiation e_m sigma^b (T, T_env^4 - T^4) (Sec. 4.1) on a flat 8-node
    face at a uniform temperature: load es (T_env^4 - T^4) int N_m (-A/12 at
    the vertices, A/3 at the midpoints), tangent 4 es T^3 times the face mass
    matrix, i.e. 4 es T^3 / h times the convection matrix of the same face."""
    V = np.array([[a & 1, (a >> 1) & 1, (a >> 2) & 1] for a in range(8)], float) @ np.array(
        [[1.2, 0.1, 0.0], [0.2, 0.9, 0.1], [0.0, 0.1, 1.1]]).T
    pairs = [(0, 1), (2, 3), (4, 5), (6, 7), (0, 2), (1, 3), (4, 6), (5, 7), (0, 4), (1, 5), (2, 6), (3, 7)]
    X = np.vstack([V] + [0.5 * (V[p] + V[q]) for p, q in pairs])
    es, te, T, h = 0.7, 1.3, 0.9, 1.7
    for face in range(6):
        Xf = X[orc.facet_nodes(orc.Q2S, face)]
        A = np.linalg.norm(np.cross(Xf[1] - Xf[0], Xf[2] - Xf[0]))
        mom = A * np.array([-1 / 12] * 4 + [1 / 3] * 4)
        Kr, rr = orc.facet_radiation(orc.Q2S, Xf, es, te, np.full(8, T))
        Kc, _, _ = orc.facet_thermal(orc.Q2S, Xf, h, 0.0)
        assert np.abs(rr - es * (te ** 4 - T ** 4) * mom).max() < 1e-14
        assert np.abs(Kr - 4 * es * T ** 3 / h * Kc).max() < 1e-14 * np.abs(Kr).max()
        assert np.abs(Kr - Kr.T).max() <= 1e-15 * np.abs(Kr).max()  # symmetric up to product order


def test_radiation_tangent_is_the_derivative_on_warped_faces(orc):
    """On the warped faces of a jittered brick, with a varying temperature,
    the tangent is minus the derivative of the load (central differences)."""
    _, X = _brick(seed=9, amp=0.15)
    rng = np.random.default_rng(10)
    for face in range(6):
        Xf = X[orc.facet_nodes(orc.Q2S, face)]
        T = 0.7 + 0.5 * rng.random(8)
        Kf, _ = orc.facet_radiation(orc.Q2S, Xf, 0.6, 1.2, T)
        hstep = 1e-6
        for b in range(8):
            e = np.zeros(8)
            e[b] = hstep
            _, rp = orc.facet_radiation(orc.Q2S, Xf, 0.6, 1.2, T + e)
            _, rm = orc.facet_radiation(orc.Q2S, Xf, 0.6, 1.2, T - e)
            assert np.abs(-(rp - rm) / (2 * hstep) - Kf[:, b]).max() < 1e-8 * np.abs(Kf).max()
