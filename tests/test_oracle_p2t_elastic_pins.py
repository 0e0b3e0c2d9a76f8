"""Pins of the oracle's linear elasticity (Sec. 4.2 form, -(d_i,j, sigma_ij))
on 10-node quadratic tetrahedra: symmetry and the rigid-body null space, the
energy of a uniform strain, the body load's closed form, the trace of the
3x3 blocks against the conduction element, and the patch test on an
assembled mesh."""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import gen

V0 = np.array([[0.1, 0.0, 0.05], [1.2, 0.1, -0.1], [0.2, 0.9, 0.1], [0.15, 0.2, 1.1]])


def _tet10(V):
    """Vertices, then the edges (0,1), (1,2), (2,0), (0,3), (1,3), (2,3)."""
    edges = [(0, 1), (1, 2), (2, 0), (0, 3), (1, 3), (2, 3)]
    return np.vstack([V] + [0.5 * (V[p] + V[q]) for p, q in edges])


def _volume(V):
    return abs(np.linalg.det(np.array([V[1] - V[0], V[2] - V[0], V[3] - V[0]]))) / 6.0


def _lame(E, nu):
    return E * nu / ((1 + nu) * (1 - 2 * nu)), E / (2 * (1 + nu))


def test_symmetric_with_the_rigid_body_null_space(orc):
    X = _tet10(V0)
    Ke, _, det = orc.elem_elastic(X, 2.3, 0.3, elem=orc.P2T)
    assert det > 0
    s = np.abs(Ke).max()
    assert np.abs(Ke - Ke.T).max() <= 1e-14 * s
    modes = [np.tile(np.eye(3)[c], 10) for c in range(3)] + [np.cross(ax, X).ravel() for ax in np.eye(3)]
    for r in modes:
        assert np.abs(Ke @ r).max() <= 1e-13 * s * np.abs(r).max()
    ev = np.linalg.eigvalsh(0.5 * (Ke + Ke.T))
    assert ev.min() > -1e-12 * ev.max()
    assert np.sum(ev < 1e-10 * ev.max()) == 6  # exactly the six rigid-body modes


def test_uniform_strain_energy(orc):
    """u = eps x with a symmetric eps: u^T K u = V (lambda (tr eps)^2 + 2 mu eps:eps)."""
    X = _tet10(V0)
    E, nu = 2.3, 0.3
    lam, mu = _lame(E, nu)
    A = np.random.default_rng(3).normal(size=(3, 3))
    eps = 0.5 * (A + A.T)
    u = (X @ eps.T).ravel()
    Ke, _, _ = orc.elem_elastic(X, E, nu, elem=orc.P2T)
    energy = _volume(V0) * (lam * np.trace(eps) ** 2 + 2 * mu * np.sum(eps * eps))
    assert abs(u @ Ke @ u - energy) <= 1e-12 * energy


def test_body_load_closed_form(orc):
    """de[3a + c] = b_c int N_a: -V/20 at the vertices, V/5 at the edge nodes."""
    X = _tet10(V0)
    b = np.array([0.3, -0.7, 1.1])
    _, de, _ = orc.elem_elastic(X, 1.0, 0.25, body=b, elem=orc.P2T)
    intN = _volume(V0) * np.array([-1 / 20] * 4 + [1 / 5] * 6)
    assert np.abs(de.reshape(10, 3) - np.outer(intN, b)).max() <= 1e-15


def test_trace_of_the_blocks_is_the_conduction_element(orc):
    """With nu = 0 (lambda = 0) the block (a, b) is mu (g_b g_a^T + (g_a . g_b) I)
    integrated, so its trace is 4 mu int grad N_a . grad N_b: 4 mu times the
    conduction element with k = 1."""
    X = _tet10(V0)
    E = 1.7
    Ke, _, _ = orc.elem_elastic(X, E, 0.0, elem=orc.P2T)
    Kt, _, _ = orc.elem_thermal(orc.P2T, orc.QTET64, X, 1.0, 0.0)
    tr = sum(Ke[c::3, c::3] for c in range(3))
    mu = E / 2
    assert np.abs(tr - 4 * mu * Kt).max() <= 1e-13 * 4 * mu * np.abs(Kt).max()


def test_patch_test_on_an_assembled_mesh(orc):
    """A linear displacement imposed on the boundary of a jittered mesh of
    quadratic tetrahedra (homogeneous material, no body force) is reproduced
    at every node by the assembled system."""
    m = gen.tet10_mesh(3, 0.1)
    X = m["coords"]
    A = np.array([[0.01, 0.02, -0.01], [0.03, -0.02, 0.01], [0.0, 0.015, 0.02]])
    u = X @ A.T + np.array([0.1, -0.2, 0.05])
    bnd = np.any((X < 1e-12) | (X > 1 - 1e-12), axis=1)
    prob = dict(m, form="elastic", coef=np.full(m["conn"].shape[0], 2.0), nu=0.3, body=(0.0, 0.0, 0.0))
    prob["bc_mask"] = np.repeat(bnd, 3).astype(np.uint8)
    prob["bc_val"] = np.where(prob["bc_mask"] != 0, u.ravel(), 0.0)
    s = orc.assemble(prob)
    n = s["d"].shape[0]
    K = sp.csr_matrix((s["val"], s["col"], s["row_ptr"]), shape=(n, n))
    x = spla.spsolve(K.tocsc(), s["d"])
    assert np.abs(x - u.ravel()).max() <= 1e-12 * np.abs(u).max()
