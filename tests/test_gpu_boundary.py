"""Parity of the boundary (facet) terms with the CPU FP64 oracle, through the
C ABI: convection h(T, T_env - T) (Sec. 4.1) on P1/P2 edges and Q1 faces, and
the loaded boundary (d_i, sigma^l_ij n_j) (Sec. 4.2) on Q1 faces.

Meshes with every node jittered (``jitter_all``) give warped, tilted facets;
Dirichlet sides there are picked by grid index.  Tolerances: as the domain
parity (row-scaled 1e-12 for K, 1e-12 of max |d| for d); the mixed path's
d (exact fixed-point load plus the FP64 boundary load) also within 1e-12.
"""
import numpy as np
import pytest

import gen

pytestmark = pytest.mark.gpu

TOL = 1e-12


@pytest.fixture(scope="module")
def mf():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2111_03541_gb300 as mf
    mf.lib()
    return mf


def _grid_index(prob, axis):
    """Grid index of every node along axis (x fastest, then y, then z)."""
    nn = prob["coords"].shape[0]
    per = prob["n"] + 1 if prob["elem"] != "P2" else 2 * prob["n"] + 1
    return (np.arange(nn) // per ** axis) % per


def _thermal(kind, n, sides, dirichlet="x0", jitter_all=False, bval_seed=None):
    if kind == "Q1":
        m = gen.hex_mesh(n, 0.15, jitter_all=jitter_all)
    else:
        m = gen.tri_mesh(n, 1 if kind == "P1" else 2, 0.2, jitter_all=jitter_all)
    prob = dict(m, form="thermal", source=1.0, coef=gen.lognormal(gen.SEED_COEF, m["conn"].shape[0], 0.5))
    nn = m["coords"].shape[0]
    mask = np.zeros(nn, np.uint8)
    if dirichlet:
        mask[_grid_index(prob, "xyz".index(dirichlet[0])) == 0] = 1
    prob["bc_mask"] = mask
    prob["bc_val"] = np.zeros(nn)
    if bval_seed is not None:
        prob["bc_val"] = np.where(mask > 0, gen.normal(bval_seed, nn), 0.0)
    prob["facets"] = gen.convection_facets(prob, sides)
    return prob


def _elastic(n, sides, jitter_all=False, stress=None):
    m = gen.hex_mesh(n, 0.15, jitter_all=jitter_all)
    prob = dict(m, form="elastic", nu=0.3, body=(0.0, 0.0, -1.0),
                coef=gen.lognormal(gen.SEED_COEF, m["conn"].shape[0], 0.5))
    clamp = _grid_index(prob, 0) == 0
    prob["bc_mask"] = np.repeat(clamp, 3).astype(np.uint8)
    prob["bc_val"] = np.zeros(3 * m["coords"].shape[0])
    prob["facets"] = gen.traction_facets(prob, sides, stress=stress)
    return prob


def row_scaled_error(rp, val, ref):
    n = rp.shape[0] - 1
    rows = np.repeat(np.arange(n), np.diff(rp))
    rmax = np.zeros(n)
    np.maximum.at(rmax, rows, np.abs(ref))
    emax = np.zeros(n)
    np.maximum.at(emax, rows, np.abs(val - ref))
    ok = rmax > 0
    assert (emax[~ok] == 0).all()
    return (emax[ok] / rmax[ok]).max()


def _gpu(mf, prob, prec=0, bc=True):
    P = mf.Problem(prob)
    coeffs = P.make_coeffs(bc=bc)
    if not bc:
        P.facet_coeffs.bc_mask = None
        P.facet_coeffs.bc_val = None
    vals, d = P.assemble(prec=prec, coeffs=coeffs)
    rp, ci = P.csr_arrays()
    return P, rp.cpu().numpy(), ci.cpu().numpy(), vals.cpu().numpy(), d.cpu().numpy()


THERMAL = {
    "p1_20": lambda: _thermal("P1", 20, ("x1", "y0", "y1")),
    "p1_all_jitter_17": lambda: _thermal("P1", 17, ("x0", "x1", "y0", "y1"), jitter_all=True, bval_seed=5),
    "p2_9": lambda: _thermal("P2", 9, ("x1", "y1")),
    "p2_all_jitter_11": lambda: _thermal("P2", 11, ("x0", "x1", "y0", "y1"), jitter_all=True, bval_seed=6),
    "q1_8": lambda: _thermal("Q1", 8, ("x1", "y0", "z1")),
    "q1_all_jitter_9": lambda: _thermal("Q1", 9, gen.SIDES, jitter_all=True, bval_seed=7),
}


@pytest.mark.parametrize("case", list(THERMAL))
def test_convection_parity(mf, orc, case):
    prob = THERMAL[case]()
    P, rp, ci, val, d = _gpu(mf, prob)
    ref = orc.assemble(prob)
    assert np.array_equal(rp, ref["row_ptr"]) and np.array_equal(ci, ref["col"])
    assert row_scaled_error(rp, val, ref["val"]) <= TOL
    assert np.abs(d - ref["d"]).max() <= TOL * np.abs(ref["d"]).max()


@pytest.mark.parametrize("case", ["p1_20", "q1_all_jitter_9"])
def test_convection_parity_without_dirichlet(mf, orc, case):
    prob = THERMAL[case]()
    P, rp, ci, val, d = _gpu(mf, prob, bc=False)
    ref = orc.assemble(prob, dirichlet=False)
    assert row_scaled_error(rp, val, ref["val"]) <= TOL
    assert np.abs(d - ref["d"]).max() <= TOL * np.abs(ref["d"]).max()


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("jitter_all", [False, True])
def test_traction_parity(mf, orc, prec, jitter_all):
    prob = _elastic(9, ("x1", "y0", "y1", "z0", "z1"), jitter_all=jitter_all)
    P, rp, ci, val, d = _gpu(mf, prob, prec=prec)
    ref = orc.assemble(prob)
    assert np.array_equal(rp, ref["row_ptr"]) and np.array_equal(ci, ref["col"])
    assert row_scaled_error(rp, val, ref["val"]) <= (TOL if prec == 0 else 1e-11)
    assert np.abs(d - ref["d"]).max() <= TOL * np.abs(ref["d"]).max()


@pytest.mark.parametrize("case", ["p2_all_jitter_11", "q1_all_jitter_9", "elastic"])
def test_boundary_bit_reproducible(mf, case):
    import torch
    prob = _elastic(8, gen.SIDES[1:], jitter_all=True) if case == "elastic" else THERMAL[case]()
    P = mf.Problem(prob)
    v1, d1 = [t.clone() for t in P.assemble()]
    P.values.fill_(float("nan"))
    P.d.fill_(float("nan"))
    v2, d2 = P.assemble()
    assert torch.equal(v1, v2) and torch.equal(d1, d2)


def test_zero_facets_is_a_no_op(mf):
    import torch
    prob = _thermal("Q1", 5, ())
    assert prob["facets"]["elem"].shape[0] == 0
    P = mf.Problem(prob)
    v1, d1 = [t.clone() for t in P.assemble()]
    plain = dict(prob)
    del plain["facets"]
    Q = mf.Problem(plain)
    v2, d2 = Q.assemble()
    assert torch.equal(v1, v2) and torch.equal(d1, d2)


def test_bad_facets_rejected(mf):
    for bad in ("face", "elem"):
        prob = _thermal("Q1", 3, ("x1",))
        if bad == "face":
            prob["facets"]["face"][2] = 6
        else:
            prob["facets"]["elem"][1] = 27
        with pytest.raises(mf.MFError) as ei:
            mf.Problem(prob)
        assert ei.value.status == mf.MF_ERR_BAD_MESH
    prob = _thermal("P1", 3, ("x1",))
    prob["facets"]["face"][0] = 3
    with pytest.raises(mf.MFError) as ei:
        mf.Problem(prob)
    assert ei.value.status == mf.MF_ERR_BAD_MESH
    mf.mf_sync_status()  # nothing left latched


def test_boundary_invalid_arguments(mf):
    import torch
    P = mf.Problem(gen.oseen_problem(3))
    e = torch.zeros(1, dtype=torch.int32, device="cuda")
    f = torch.zeros(1, dtype=torch.uint8, device="cuda")
    with pytest.raises(mf.MFError) as ei:
        mf.mf_facets_create(P.mesh, P.pattern, e, f)
    assert ei.value.status == mf.MF_ERR_INVALID_ARG
    Q = mf.Problem(_thermal("P1", 4, ("x1",)))
    with pytest.raises(mf.MFError) as ei:
        mf.mf_assemble_boundary(Q.facets, mf.FacetCoeffs(), Q.csr, Q.d)
    assert ei.value.status == mf.MF_ERR_INVALID_ARG
    with pytest.raises(mf.MFError) as ei:
        mf.mf_assemble_boundary(Q.facets, Q.facet_coeffs, P.csr, Q.d)
    assert ei.value.status == mf.MF_ERR_INVALID_ARG


def test_nonfinite_facet_coefficient_latched(mf):
    P = mf.Problem(_thermal("P2", 4, ("y1",)))
    P.f_h[1] = float("inf")
    P.assemble()
    with pytest.raises(mf.MFError) as ei:
        mf.mf_sync_status()
    assert ei.value.status == mf.MF_ERR_NONFINITE
    P.f_h[1] = 1.0
    P.assemble()
    mf.mf_sync_status()


# ---------------------------------------------------------------------------
# solutions: patch tests with exact linear fields, solved on the GPU
# ---------------------------------------------------------------------------

def test_robin_patch_solution(mf):
    prob = _thermal("Q1", 6, ("x1",))
    k, h, T0, Tenv = 1.7, 2.3, 0.4, 1.9
    prob["coef"][:] = k
    prob["source"] = 0.0
    prob["bc_val"] = np.where(prob["bc_mask"] > 0, T0, 0.0)
    prob["facets"]["h"][:] = h
    prob["facets"]["t_env"][:] = Tenv
    P = mf.Problem(prob)
    P.assemble()
    x, st, info = P.solve(tol=1e-13)
    assert st == mf.MF_OK
    exact = T0 + h * (Tenv - T0) / (k + h) * prob["coords"][:, 0]
    assert np.abs(x.cpu().numpy() - exact).max() < 1e-10


@pytest.mark.parametrize("prec", [0, 1])
def test_traction_patch_solution(mf, prec):
    prob = _elastic(4, ("x0", "x1", "y0", "y1", "z1"))
    E, nu = 2.1, 0.25  # lambda / mu = 2 nu / (1 - 2 nu) = 1
    prob["coef"][:] = E
    prob["nu"] = nu
    prob["body"] = (0.0, 0.0, 0.0)
    sigma = np.array([[0.8, 0.3, -0.2], [0.3, -0.5, 0.4], [-0.2, 0.4, 0.6]])
    eps = ((1 + nu) * sigma - nu * np.trace(sigma) * np.eye(3)) / E
    u = prob["coords"] @ eps.T
    bottom = np.repeat(prob["coords"][:, 2] <= 1e-14, 3)
    prob["bc_mask"] = bottom.astype(np.uint8)
    prob["bc_val"] = np.where(bottom, u.ravel(), 0.0)
    prob["facets"] = gen.traction_facets(prob, ("x0", "x1", "y0", "y1", "z1"), stress=sigma)
    P = mf.Problem(prob)
    P.assemble(prec=prec)
    x, st, info = P.solve(tol=1e-13)
    assert st == mf.MF_OK
    assert np.abs(x.cpu().numpy() - u.ravel()).max() < (1e-10 if prec == 0 else 1e-8) * np.abs(u).max()


# ---------------------------------------------------------------------------
# full sizes: sampled boundary rows
# ---------------------------------------------------------------------------

def _sampled(mf, orc, prob, nodes, dofs_per_node, prec=0, tol=TOL):
    P = mf.Problem(prob)
    vals, d = P.assemble(prec=prec)
    rp, ci = P.csr_arrays()
    rp, ci, vals, d = rp.cpu().numpy(), ci.cpu().numpy(), vals.cpu().numpy(), d.cpu().numpy()
    keep = np.zeros(prob["coords"].shape[0], np.uint8)
    keep[nodes] = 1
    ref = orc.assemble(prob, keep_nodes=keep)
    rows = [dofs_per_node * int(n) + c for n in nodes for c in range(dofs_per_node)]
    dscale = max(np.abs(ref["d"][rows]).max(), 1e-300)
    for r, (cols, v) in zip(rows, orc.rows_of(ref, rows)):
        s = slice(rp[r], rp[r + 1])
        assert np.array_equal(ci[s], cols)
        assert np.abs(vals[s] - v).max() <= tol * np.abs(v).max()
        assert abs(d[r] - ref["d"][r]) <= TOL * dscale
    return P


def _box_nodes(n, rng, count):
    nv = n + 1
    corners = [0, n, n * nv, n * nv + n, n * nv * nv, n * nv * nv + n, nv ** 3 - nv, nv ** 3 - 1]
    edges = [n // 2, n * nv + n // 2, (n // 2) * nv + n, (n // 2) * nv * nv]
    faces = []
    for _ in range(count):
        i, j = rng.integers(1, n, 2)
        side = rng.integers(0, 6)
        axis, hi = divmod(side, 2)
        ijk = [i, j]
        ijk.insert(axis, n if hi else 0)
        faces.append((ijk[2] * nv + ijk[1]) * nv + ijk[0])
    return np.unique(np.array(corners + edges + faces))


def test_grf_thermal_convection_full_size_sampled_rows(mf, orc):
    """128^3 Q1 thermal, k = exp(GRF), convection on five sides, T = 0 on x = 0."""
    base = gen.grf_thermal_problem(128)
    prob = dict(base)
    x = base["coords"]
    left = x[:, 0] <= 1e-14
    prob["bc_mask"] = left.astype(np.uint8)
    prob["bc_val"] = np.zeros(x.shape[0])
    prob["facets"] = gen.convection_facets(prob, ("x1", "y0", "y1", "z0", "z1"))
    nodes = _box_nodes(128, np.random.default_rng(23), 40)
    P = _sampled(mf, orc, prob, nodes, 1)
    assert P.nnz == (4 + 3 * 127) ** 3


@pytest.mark.parametrize("prec", [0, 1])
def test_elastic_traction_full_size_sampled_rows(mf, orc, prec):
    """64^3 Q1 elasticity clamped at x = 0 with a random stress load on the other five sides."""
    prob = gen.elastic_problem(64)
    prob["facets"] = gen.traction_facets(prob, ("x1", "y0", "y1", "z0", "z1"))
    nodes = _box_nodes(64, np.random.default_rng(29), 40)
    _sampled(mf, orc, prob, nodes, 3, prec=prec, tol=TOL if prec == 0 else 1e-11)


def test_single_element_all_faces(mf, orc):
    # one hexahedron, convection on all six faces, no Dirichlet: every node
    # sits on three facets
    prob = _thermal("Q1", 1, gen.SIDES, dirichlet=None, jitter_all=True)
    P, rp, ci, val, d = _gpu(mf, prob, bc=False)
    ref = orc.assemble(prob, dirichlet=False)
    assert row_scaled_error(rp, val, ref["val"]) <= TOL
    assert np.abs(d - ref["d"]).max() <= TOL * np.abs(ref["d"]).max()


def test_facets_on_fully_constrained_rows(mf, orc):
    # convection on the Dirichlet side itself: rows stay identities, d = bc_val
    prob = _thermal("P2", 5, ("x0", "x1"), bval_seed=11)
    P, rp, ci, val, d = _gpu(mf, prob)
    ref = orc.assemble(prob)
    assert row_scaled_error(rp, val, ref["val"]) <= TOL
    assert np.abs(d - ref["d"]).max() <= TOL * np.abs(ref["d"]).max()
    m = prob["bc_mask"] > 0
    assert np.array_equal(d[m], prob["bc_val"][m])


# ---------------------------------------------------------------------------
# 8-node faces of the 20-node brick (the cantilever beams' loads, Sec. 4.2;
# convection, Sec. 4.1): 3 x 3 Gauss on the vertices' bilinear map
# ---------------------------------------------------------------------------
_Q2S_EDGES = [(0, 1), (2, 3), (4, 5), (6, 7), (0, 2), (1, 3), (4, 6), (5, 7), (0, 4), (1, 5), (2, 6), (3, 7)]


def _warp_hex20(m, amp=0.08, seed=11):
    """Every vertex jittered (boundary ones too: warped, tilted faces), the
    edge midpoints moved to the means of their ends (straight edges)."""
    X = m["coords"].copy()
    c = m["conn"]
    verts = np.unique(c[:, :8])
    h = 1.0 / m["n"]
    X[verts] += np.random.default_rng(seed).uniform(-amp * h, amp * h, (verts.shape[0], 3))
    for k, (a, b) in enumerate(_Q2S_EDGES):
        X[c[:, 8 + k]] = 0.5 * (X[c[:, a]] + X[c[:, b]])
    return dict(m, coords=X)


def _q2s_thermal(n, sides, warp=False):
    m = gen.hex20_mesh(n, 0.15)
    if warp:
        m = _warp_hex20(m)
    prob = dict(m, form="thermal", source=1.0, coef=gen.lognormal(gen.SEED_COEF, m["conn"].shape[0], 0.5))
    nn = m["coords"].shape[0]
    mask = np.zeros(nn, np.uint8)
    # x = 0 side by the vertices of the x = 0 faces (also when warped)
    e0, f0 = gen.box_facets(m, ("x0",))
    for e in e0:
        mask[m["conn"][e, [0, 2, 4, 6, 12, 14, 16, 18]]] = 1
    prob["bc_mask"] = mask
    prob["bc_val"] = np.where(mask > 0, gen.normal(9, nn), 0.0)
    prob["facets"] = gen.convection_facets(prob, sides)
    return prob


def _q2s_elastic(n, sides, warp=False):
    prob = gen.elastic_q2s_problem(n)
    if warp:
        prob = dict(prob, coords=_warp_hex20(prob)["coords"])
    prob["facets"] = gen.traction_facets(prob, sides)
    return prob


@pytest.mark.parametrize("warp", [False, True])
def test_q2s_face_convection_parity(mf, orc, warp):
    prob = _q2s_thermal(5, ("x1", "y0", "y1", "z0", "z1"), warp=warp)
    P, rp, ci, val, d = _gpu(mf, prob)
    ref = orc.assemble(prob)
    assert np.array_equal(rp, ref["row_ptr"]) and np.array_equal(ci, ref["col"])
    assert row_scaled_error(rp, val, ref["val"]) <= TOL
    assert np.abs(d - ref["d"]).max() <= TOL * np.abs(ref["d"]).max()


@pytest.mark.parametrize("warp", [False, True])
def test_q2s_face_traction_parity(mf, orc, warp):
    prob = _q2s_elastic(4, ("x1", "y0", "y1", "z0", "z1"), warp=warp)
    P, rp, ci, val, d = _gpu(mf, prob)
    ref = orc.assemble(prob)
    assert np.array_equal(rp, ref["row_ptr"]) and np.array_equal(ci, ref["col"])
    assert row_scaled_error(rp, val, ref["val"]) <= TOL
    assert np.abs(d - ref["d"]).max() <= TOL * np.abs(ref["d"]).max()


def test_q2s_uniform_stress_balances_over_the_closed_surface(mf):
    """A uniform stress on all six sides with no body force and no clamp:
    the loads sum to zero (int sigma n over a closed surface), per component."""
    prob = gen.elastic_q2s_problem(3)
    prob["body"] = (0.0, 0.0, 0.0)
    prob["bc_mask"] = np.zeros_like(prob["bc_mask"])
    prob["facets"] = gen.traction_facets(prob, gen.SIDES, stress=np.arange(9.0).reshape(3, 3) - 4.0)
    P, rp, ci, val, d = _gpu(mf, prob, bc=False)
    tot = d.reshape(-1, 3).sum(axis=0)
    assert np.abs(tot).max() <= 1e-12 * np.abs(d).max()
