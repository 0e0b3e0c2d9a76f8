"""Pins of the oracle's linear elasticity on 20-node serendipity bricks (the
element of the 3D cantilever beams, Sec. 4.2; stress-strain law of Sec. 4.2).

Expected values come from mechanics and exact integration, not from the
oracle: rigid-body modes in the kernel (exactly six zero eigenvalues of an
element), the strain energy of a linear field against the element volume from
the divergence theorem, the block-trace identity tr K_ab = (lambda + 4 mu)
K^th_ab with the pinned scalar Laplacian, interior rows that vanish for linear
fields on jittered meshes, exact reproduction of a quadratic displacement
with its constant body force on affine meshes (rows and a full solve), and a
brute-force 3 x 3-block pattern.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import gen

E0, NU = 2.3, 0.3


def lame(E, nu):
    return E * nu / ((1 + nu) * (1 - 2 * nu)), E / (2 * (1 + nu))


def _brick(seed=5, amp=0.15):
    rng = np.random.default_rng(seed)
    V = np.array([[a & 1, (a >> 1) & 1, (a >> 2) & 1] for a in range(8)], float) + rng.uniform(-amp, amp, (8, 3))
    edges = [(0, 1), (2, 3), (4, 5), (6, 7), (0, 2), (1, 3), (4, 6), (5, 7), (0, 4), (1, 5), (2, 6), (3, 7)]
    return V, np.vstack([V] + [0.5 * (V[a0] + V[a1]) for a0, a1 in edges])


def _volume_divergence(V):
    """Volume of the trilinear brick as (1/3) of the flux of x through its six
    bilinear faces (divergence theorem), each face integrated exactly by 3 x 3
    Gauss (the integrand x . (x_u x x_v) is quadratic in u and in v)."""
    faces = [(0, 4, 6, 2), (1, 3, 7, 5), (0, 1, 5, 4), (2, 6, 7, 3), (0, 2, 3, 1), (4, 5, 7, 6)]
    g, w = np.polynomial.legendre.leggauss(3)
    g, w = 0.5 * (g + 1), 0.5 * w
    vol = 0.0
    for f in faces:
        P = V[list(f)]  # u along P0->P1, v along P0->P3: x_u x x_v points outward
        for u, wu in zip(g, w):
            for v, wv in zip(g, w):
                x = (1 - u) * (1 - v) * P[0] + u * (1 - v) * P[1] + u * v * P[2] + (1 - u) * v * P[3]
                xu = (1 - v) * (P[1] - P[0]) + v * (P[2] - P[3])
                xv = (1 - u) * (P[3] - P[0]) + u * (P[2] - P[1])
                vol += wu * wv * x @ np.cross(xu, xv) / 3.0
    return vol


def _rigid_modes(X):
    """Three translations and three infinitesimal rotations, dof 3 a + c."""
    modes = []
    for c in range(3):
        u = np.zeros_like(X)
        u[:, c] = 1.0
        modes.append(u.ravel())
    for axis in range(3):
        w = np.zeros(3)
        w[axis] = 1.0
        modes.append(np.cross(w, X).ravel())
    return np.array(modes)


def test_element_rigid_modes_and_rank(orc):
    _, X = _brick()
    Ke, de, det = orc.elem_elastic(X, E0, NU, elem=orc.Q2S)
    assert det > 0
    scale = np.abs(Ke).max()
    assert np.abs(Ke - Ke.T).max() < 1e-14 * scale
    assert np.abs(Ke @ _rigid_modes(X).T).max() < 1e-13 * scale
    ev = np.linalg.eigvalsh(Ke)
    assert np.abs(ev[:6]).max() < 1e-12 * ev[-1]
    assert ev[6] > 1e-4 * ev[-1]  # full integration: no spurious zero-energy modes


def test_element_energy_of_a_linear_field(orc):
    V, X = _brick(seed=9)
    A = np.array([[0.3, -0.7, 0.2], [0.5, 0.1, -0.4], [-0.2, 0.6, 0.8]])  # not symmetric
    u = (X @ A.T + np.array([0.1, -0.2, 0.3])).ravel()
    Ke, _, _ = orc.elem_elastic(X, E0, NU, elem=orc.Q2S)
    eps = 0.5 * (A + A.T)
    lam, mu = lame(E0, NU)
    exact = _volume_divergence(V) * (lam * np.trace(eps) ** 2 + 2 * mu * np.sum(eps * eps))
    assert abs(u @ Ke @ u - exact) < 1e-13 * exact
    # the antisymmetric part of A (a rotation) stores no energy
    W = 0.5 * (A - A.T)
    r = (X @ W.T).ravel()
    assert abs(r @ Ke @ r) < 1e-13 * exact


def test_block_trace_is_the_scalar_laplacian(orc):
    _, X = _brick(seed=11)
    Ke, _, _ = orc.elem_elastic(X, E0, NU, elem=orc.Q2S)
    Kth, _, _ = orc.elem_thermal(orc.Q2S, orc.QHEX27, X, k=1.0, f=0.0)
    lam, mu = lame(E0, NU)
    tr = np.einsum("acbc->ab", Ke.reshape(20, 3, 20, 3))
    assert np.abs(tr - (lam + 4 * mu) * Kth).max() < 1e-13 * np.abs(tr).max()
    # with nu = 0 (lambda = 0) the blocks are mu (M_ab^T + tr M_ab I): the
    # off-diagonal entries of a block are the transposed ones of the thermal
    # direction tensor, so block (a, a) is symmetric
    K0, _, _ = orc.elem_elastic(X, E0, 0.0, elem=orc.Q2S)
    B = K0.reshape(20, 3, 20, 3)
    for a in range(20):
        assert np.abs(B[a, :, a, :] - B[a, :, a, :].T).max() < 1e-14 * np.abs(K0).max()


def test_element_load(orc):
    V, X = _brick(seed=13)
    b = np.array([0.4, -1.1, 2.0])
    _, de, _ = orc.elem_elastic(X, E0, NU, body=b, elem=orc.Q2S)
    de = de.reshape(20, 3)
    # the 20 shape functions sum to one: the loads add up to b times the volume
    assert np.abs(de.sum(axis=0) - b * _volume_divergence(V)).max() < 1e-14
    # component c of every node's load is b_c times the same scalar moment
    assert np.abs(de[:, 0] / b[0] - de[:, 1] / b[1]).max() < 1e-15


def _csr(s):
    n = s["row_ptr"].shape[0] - 1
    return sp.csr_matrix((s["val"], s["col"], s["row_ptr"]), shape=(n, n))


def test_assembled_kernel_and_patch(orc):
    prob = gen.elastic_q2s_problem(3)
    s = orc.assemble(prob, dirichlet=False)
    K = _csr(s)
    scale = np.abs(s["val"]).max()
    assert abs(K - K.T).max() < 1e-14 * scale
    x = prob["coords"]
    for m in _rigid_modes(x):
        assert np.abs(K @ m).max() < 1e-12 * scale
    # body force (0, 0, -1) over the unit cube
    assert np.abs(s["d"].reshape(-1, 3).sum(axis=0) - np.array([0.0, 0.0, -1.0])).max() < 1e-13
    # patch test on the jittered mesh: linear field, uniform material, no body force
    prob["coef"] = np.full(prob["conn"].shape[0], E0)
    prob["body"] = (0.0, 0.0, 0.0)
    s = orc.assemble(prob, dirichlet=False)
    A = np.array([[0.3, -0.7, 0.2], [0.5, 0.1, -0.4], [-0.2, 0.6, 0.8]])
    u = (x @ A.T).ravel()
    inner = np.repeat(~gen.boundary_nodes(x), 3)
    assert np.abs((_csr(s) @ u)[inner]).max() < 1e-12 * np.abs(s["val"]).max()


def _quadratic_field(x):
    """u_i = x^T H_i x / 2 with symmetric H_i, and its body force b = -div sigma
    for uniform lambda, mu: (div sigma)_i = lambda sum_k (H_k)_ki
    + mu (tr H_i + sum_j (H_j)_ij)."""
    H = np.array([[[1.0, 0.3, -0.2], [0.3, -0.5, 0.4], [-0.2, 0.4, 0.7]],
                  [[0.2, -0.6, 0.1], [-0.6, 0.9, 0.3], [0.1, 0.3, -0.4]],
                  [[-0.3, 0.2, 0.5], [0.2, 0.1, -0.7], [0.5, -0.7, 0.6]]])
    u = 0.5 * np.einsum("nj,ijk,nk->ni", x, H, x)
    lam, mu = lame(E0, NU)
    div = np.array([lam * sum(H[k][k, i] for k in range(3))
                    + mu * (np.trace(H[i]) + sum(H[j][i, j] for j in range(3))) for i in range(3)])
    return u, -div


def test_quadratic_field_reproduced_on_affine_meshes(orc):
    prob = gen.elastic_q2s_problem(3, jitter=0.0)
    prob["coef"] = np.full(prob["conn"].shape[0], E0)
    x = prob["coords"]
    u, b = _quadratic_field(x)
    prob["body"] = tuple(b)
    s = orc.assemble(prob, dirichlet=False)
    inner = np.repeat(~gen.boundary_nodes(x), 3)
    r = _csr(s) @ u.ravel() - s["d"]
    assert np.abs(r[inner]).max() < 1e-12 * np.abs(s["val"]).max()
    # the full solve with u on the whole boundary returns u at every node
    bnd = np.repeat(gen.boundary_nodes(x), 3)
    prob["bc_mask"] = bnd.astype(np.uint8)
    prob["bc_val"] = np.where(bnd, u.ravel(), 0.0)
    s = orc.assemble(prob)
    xs, _, rr = orc.pcg(s, tol=1e-14)
    assert np.abs(xs - u.ravel()).max() < 1e-11 * np.abs(u).max()


def test_pattern_matches_brute_force(orc):
    prob = gen.elastic_q2s_problem(2)
    s = orc.assemble(prob, dirichlet=False)
    n = prob["coords"].shape[0]
    pairs = sorted({(int(a), int(b)) for el in prob["conn"] for a in el for b in el} | {(g, g) for g in range(n)})
    ent = sorted((3 * a + c, 3 * b + cp) for a, b in pairs for c in range(3) for cp in range(3))
    rows = np.repeat(np.arange(3 * n), np.diff(s["row_ptr"]))
    assert list(zip(rows.tolist(), s["col"].tolist())) == ent
    assert np.diff(s["row_ptr"]).max() == 243


def test_two_dimensional_elements_rejected(orc):
    prob = gen.thermal_p1_problem(3)
    prob["form"] = "elastic"
    prob["nu"] = NU
    prob["body"] = (0.0, 0.0, -1.0)
    with pytest.raises(orc.AssemblyError):
        orc.assemble(prob)
