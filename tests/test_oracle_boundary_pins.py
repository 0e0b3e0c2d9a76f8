"""Pins of the oracle's boundary (facet) terms: convection h(T, T_env - T) of
Sec. 4.1 and the loaded boundary (d_i, sigma^l_ij n_j) of Sec. 4.2.

Expected values come from closed-form 1D and tensor-product mass matrices,
the vector area of a quadrilateral from its diagonals, the divergence theorem
on a closed element surface, and patch tests whose exact solutions are linear
fields (reproduced exactly by P1, P2 and Q1 elements).
"""
import numpy as np
import pytest
import scipy.sparse as sp

import gen

M1D = np.array([[2.0, 1.0], [1.0, 2.0]]) / 3.0  # int_{-1}^{1} N_a N_b du, N = (1 -+ u) / 2


def _csr(s):
    n = s["row_ptr"].shape[0] - 1
    return sp.csr_matrix((s["val"], s["col"], s["row_ptr"]), shape=(n, n))


def _vector_area(Xf):
    # facet node m = b_u + 2 b_v: cyclic order 0, 1, 3, 2; vector area of a
    # (possibly warped) quadrilateral = half the cross product of its diagonals
    return 0.5 * np.cross(Xf[3] - Xf[0], Xf[2] - Xf[1])


def _orientation(face):
    d, s = divmod(face, 2)
    return (1.0 if s else -1.0) * (-1.0 if d == 1 else 1.0)


# ---------------------------------------------------------------------------
# single facets: closed forms
# ---------------------------------------------------------------------------

def test_p1_edge_closed_form(orc):
    X = np.array([[0.1, 0.2], [0.7, 1.0]])
    L = 1.0
    K, d, meas = orc.facet_thermal(orc.P1, X, 2.0, 3.0)
    assert abs(meas - L) < 1e-15
    assert np.abs(K - 2.0 * L / 6.0 * np.array([[2, 1], [1, 2]])).max() < 1e-15
    assert np.abs(d - 2.0 * 3.0 * L / 2.0).max() < 1e-15


def test_p2_edge_closed_form(orc):
    # straight quadratic edge: L/30 [[4, -1, 2], [-1, 4, 2], [2, 2, 16]], load L [1/6, 1/6, 2/3]
    X = np.array([[0.3, -0.2], [-0.9, 0.3], [-0.3, 0.05]])
    L = 1.3
    K, d, meas = orc.facet_thermal(orc.P2, X, 0.7, -1.5)
    assert abs(meas - L) < 1e-15
    assert np.abs(K - 0.7 * L / 30.0 * np.array([[4, -1, 2], [-1, 4, 2], [2, 2, 16]])).max() < 1e-15
    assert np.abs(d - 0.7 * -1.5 * L * np.array([1 / 6, 1 / 6, 2 / 3])).max() < 1e-15


def test_q1_face_parallelogram_kronecker(orc):
    # affine face x = c0 + c1 u + c2 v in general position: |x_u x x_v| = |c1 x c2|
    c0 = np.array([0.2, -0.1, 0.4])
    c1 = np.array([0.3, 0.1, -0.2])
    c2 = np.array([-0.05, 0.25, 0.15])
    Xf = np.array([c0 + (2 * (m & 1) - 1) * c1 + (2 * (m >> 1) - 1) * c2 for m in range(4)])
    J = np.linalg.norm(np.cross(c1, c2))
    K, d, meas = orc.facet_thermal(orc.Q1, Xf, 1.7, 0.9)
    assert abs(meas - 4.0 * J) < 1e-15
    assert np.abs(K - 1.7 * J * np.kron(M1D, M1D)).max() < 1e-15
    assert np.abs(d - 1.7 * 0.9 * J).max() < 1e-15  # int N_m du dv = 1


def test_facet_node_tables(orc):
    assert orc.facet_nodes(orc.P1, 2) == [2, 0]
    assert orc.facet_nodes(orc.P2, 1) == [1, 2, 4]
    want = {0: [0, 2, 4, 6], 1: [1, 3, 5, 7], 2: [0, 1, 4, 5], 3: [2, 3, 6, 7], 4: [0, 1, 2, 3], 5: [4, 5, 6, 7]}
    for f, loc in want.items():
        assert orc.facet_nodes(orc.Q1, f) == loc
    with pytest.raises(ValueError):
        orc.facet_nodes(orc.Q1, 6)


def _jittered_hex(seed=5, amp=0.2):
    rng = np.random.default_rng(seed)
    X = np.array([[a & 1, (a >> 1) & 1, (a >> 2) & 1] for a in range(8)], float)
    return X + rng.uniform(-amp, amp, size=X.shape)


def test_traction_face_total_is_sigma_times_vector_area(orc):
    X = _jittered_hex()
    sigma = np.array([[1.0, 0.3, -0.2], [0.5, -0.7, 0.1], [0.2, 0.4, 0.9]])
    for face in range(6):
        Xf = X[orc.facet_nodes(orc.Q1, face)]
        df = orc.facet_traction(face, Xf, sigma)
        want = sigma @ (_orientation(face) * _vector_area(Xf))
        assert np.abs(df.sum(axis=0) - want).max() < 1e-15


def test_traction_outward_on_unit_cube(orc):
    X = np.array([[a & 1, (a >> 1) & 1, (a >> 2) & 1] for a in range(8)], float)
    for face in range(6):
        d, s = divmod(face, 2)
        n = np.zeros(3)
        n[d] = 1.0 if s else -1.0
        df = orc.facet_traction(face, X[orc.facet_nodes(orc.Q1, face)], np.eye(3))
        assert np.abs(df - 0.25 * n).max() < 1e-16  # sigma = I: load n |face| / 4 per node


def test_traction_closed_surface_sums_to_zero(orc):
    # divergence theorem: the outward vector areas of a closed surface cancel
    X = _jittered_hex(seed=11, amp=0.3)
    rng = np.random.default_rng(2)
    sigma = rng.normal(size=(3, 3))
    tot = np.zeros(3)
    for face in range(6):
        tot += orc.facet_traction(face, X[orc.facet_nodes(orc.Q1, face)], sigma).sum(axis=0)
    assert np.abs(tot).max() < 1e-15


def test_convection_rigid_motion_invariance(orc):
    X = _jittered_hex(seed=7)
    Xf = X[orc.facet_nodes(orc.Q1, 3)]
    th = 0.7
    R = np.array([[np.cos(th), -np.sin(th), 0], [np.sin(th), np.cos(th), 0], [0, 0, 1]])
    R = R @ np.array([[1, 0, 0], [0, np.cos(0.4), -np.sin(0.4)], [0, np.sin(0.4), np.cos(0.4)]])
    K0, d0, m0 = orc.facet_thermal(orc.Q1, Xf, 1.1, 0.3)
    K1, d1, m1 = orc.facet_thermal(orc.Q1, Xf @ R.T + np.array([3.0, -1.0, 2.0]), 1.1, 0.3)
    assert np.abs(K1 - K0).max() < 1e-15 and abs(m1 - m0) < 1e-15
    assert np.allclose(K0, K0.T, atol=0) and np.all(np.linalg.eigvalsh(K0) > 0)


# ---------------------------------------------------------------------------
# assembled systems: patch tests with exact linear solutions
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("kind", ["p1", "p2", "q1"])
def test_robin_patch_test(orc, kind):
    # T = T0 on x = 0, k dT/dn = h (T_env - T) on x = 1, insulated elsewhere,
    # no source: T = T0 + b x with b = h (T_env - T0) / (k + h)
    prob = {"p1": lambda: gen.thermal_p1_problem(6), "p2": lambda: gen.thermal_p2_problem(4),
            "q1": lambda: gen.thermal_q1_problem(3)}[kind]()
    k, h, T0, Tenv = 1.7, 2.3, 0.4, 1.9
    prob["coef"] = np.full(prob["conn"].shape[0], k)
    prob["source"] = 0.0
    x = prob["coords"]
    left = x[:, 0] <= 1e-14
    prob["bc_mask"] = left.astype(np.uint8)
    prob["bc_val"] = np.where(left, T0, 0.0)
    fac = gen.convection_facets(prob, ("x1",))
    fac["h"][:] = h
    fac["t_env"][:] = Tenv
    prob["facets"] = fac
    s = orc.assemble(prob)
    T = np.linalg.solve(_csr(s).toarray(), s["d"])
    exact = T0 + h * (Tenv - T0) / (k + h) * x[:, 0]
    assert np.abs(T - exact).max() < 1e-13


def test_robin_makes_neumann_laplacian_definite(orc):
    prob = gen.thermal_q1_problem(3)
    prob["facets"] = gen.convection_facets(prob, gen.SIDES)
    s = orc.assemble(prob, dirichlet=False)
    K = _csr(s).toarray()
    assert np.abs(K - K.T).max() < 1e-15 * np.abs(K).max()
    assert np.linalg.eigvalsh(K).min() > 1e-6
    # total load: source over the unit cube plus sum_f h_f T_env,f |f| (flat faces)
    area = 1.0 / 9.0
    want = 1.0 + np.sum(prob["facets"]["h"] * prob["facets"]["t_env"]) * area
    assert abs(s["d"].sum() - want) < 1e-13


def test_traction_patch_test_general_stress(orc):
    # uniform stress sigma: u = eps x with eps = ((1 + nu) sigma - nu tr(sigma) I) / E,
    # u prescribed on z = 0, traction sigma n on the other five sides
    prob = gen.elastic_problem(3)
    E, nu = 2.1, 0.3
    prob["coef"] = np.full(prob["conn"].shape[0], E)
    prob["nu"] = nu
    prob["body"] = (0.0, 0.0, 0.0)
    sigma = np.array([[0.8, 0.3, -0.2], [0.3, -0.5, 0.4], [-0.2, 0.4, 0.6]])
    eps = ((1 + nu) * sigma - nu * np.trace(sigma) * np.eye(3)) / E
    x = prob["coords"]
    u = x @ eps.T
    bottom = np.repeat(x[:, 2] <= 1e-14, 3)
    prob["bc_mask"] = bottom.astype(np.uint8)
    prob["bc_val"] = np.where(bottom, u.ravel(), 0.0)
    prob["facets"] = gen.traction_facets(prob, ("x0", "x1", "y0", "y1", "z1"), stress=sigma)
    s = orc.assemble(prob)
    got = np.linalg.solve(_csr(s).toarray(), s["d"])
    assert np.abs(got - u.ravel()).max() < 1e-13


def test_traction_total_load_on_warped_boundary(orc):
    # every boundary node moved: the boundary is a closed warped surface, and
    # the loads of a uniform stress on all of it cancel (divergence theorem)
    m = gen.hex_mesh(3, jitter=0.2, jitter_all=True)
    prob = dict(m, form="elastic", coef=np.ones(27), nu=0.25, body=(0.0, 0.0, 0.0),
                bc_mask=np.zeros(3 * m["coords"].shape[0], np.uint8),
                bc_val=np.zeros(3 * m["coords"].shape[0]))
    prob["facets"] = gen.traction_facets(prob, gen.SIDES, stress=np.arange(9.0).reshape(3, 3) - 4.0)
    s = orc.assemble(prob, dirichlet=False)
    assert np.abs(s["d"].reshape(-1, 3).sum(axis=0)).max() < 1e-13


def test_bad_facet_rejected(orc):
    prob = gen.thermal_p1_problem(3)
    fac = gen.convection_facets(prob, ("x0",))
    fac["face"][1] = 3
    prob["facets"] = fac
    with pytest.raises(orc.AssemblyError):
        orc.assemble(prob)
