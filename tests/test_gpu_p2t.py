"""Parity of the 10-node quadratic tetrahedron (thermal form, FP64) with the
CPU FP64 oracle, through the C ABI: pattern bit-exact (rows of up to 65
entries), values row-scaled within 1e-12, sampled rows of the 48^3 Kuhn mesh
(663,552 elements), a PCG solve, reproducibility, degenerate cases and the
combinations the element does not provide.
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


def _gpu(mf, prob, bc=True):
    P = mf.Problem(prob)
    vals, d = P.assemble(coeffs=P.make_coeffs(bc=bc))
    rp, ci = P.csr_arrays()
    return P, rp.cpu().numpy(), ci.cpu().numpy(), vals.cpu().numpy(), d.cpu().numpy()


CASES = {
    "p2t_2": lambda: gen.thermal_p2t_problem(2),
    "p2t_5": lambda: gen.thermal_p2t_problem(5),
    "p2t_affine_3": lambda: gen.thermal_p2t_problem(3, jitter=0.0),
}


@pytest.mark.parametrize("case", list(CASES))
def test_pattern_and_values(mf, orc, case):
    prob = CASES[case]()
    P, rp, ci, val, d = _gpu(mf, prob)
    ref = orc.assemble(prob)
    assert np.array_equal(rp, ref["row_ptr"]) and np.array_equal(ci, ref["col"])
    assert np.diff(rp).max() == 65
    assert row_scaled_error(rp, val, ref["val"]) <= TOL
    assert np.abs(d - ref["d"]).max() <= TOL * np.abs(ref["d"]).max()


def test_values_without_dirichlet_and_lifted(mf, orc):
    prob = gen.thermal_p2t_problem(4)
    P, rp, ci, val, d = _gpu(mf, prob, bc=False)
    ref = orc.assemble(prob, dirichlet=False)
    assert row_scaled_error(rp, val, ref["val"]) <= TOL
    assert np.abs(d - ref["d"]).max() <= TOL * np.abs(ref["d"]).max()
    prob["bc_val"] = np.where(prob["bc_mask"] > 0, gen.normal(12, prob["bc_mask"].shape[0]), 0.0)
    P, rp, ci, val, d = _gpu(mf, prob)
    ref = orc.assemble(prob)
    assert row_scaled_error(rp, val, ref["val"]) <= TOL
    assert np.abs(d - ref["d"]).max() <= TOL * np.abs(ref["d"]).max()


def test_bit_reproducible(mf):
    import torch
    P = mf.Problem(gen.thermal_p2t_problem(6))
    v1, d1 = [t.clone() for t in P.assemble()]
    P.values.fill_(float("nan"))
    v2, d2 = P.assemble()
    assert torch.equal(v1, v2) and torch.equal(d1, d2)


def test_pcg_matches_oracle(mf, orc):
    prob = gen.thermal_p2t_problem(6)
    P = mf.Problem(prob)
    P.assemble()
    x, st, info = P.solve(tol=1e-12)
    assert st == mf.MF_OK
    ref = orc.assemble(prob)
    xo, _, _ = orc.pcg(ref, tol=1e-14)
    assert np.abs(x.cpu().numpy() - xo).max() <= 1e-9 * np.abs(xo).max()


def test_harmonic_quadratic_solved_exactly(mf):
    """A harmonic quadratic prescribed on the boundary of a jittered mesh (no
    source, uniform conductivity) is in the P2 space of the affine
    tetrahedra: the GPU solve returns it at every node."""
    prob = gen.thermal_p2t_problem(5)
    prob["source"] = 0.0
    prob["coef"] = np.full(prob["conn"].shape[0], 1.3)
    x = prob["coords"]
    u = x[:, 0] ** 2 + x[:, 1] ** 2 - 2.0 * x[:, 2] ** 2 + 0.5 * x[:, 0] * x[:, 1] - 0.3 * x[:, 1] * x[:, 2]
    prob["bc_val"] = np.where(prob["bc_mask"] > 0, u, 0.0)
    P = mf.Problem(prob)
    P.assemble()
    xs, st, info = P.solve(tol=1e-13)
    assert st == mf.MF_OK
    assert np.abs(xs.cpu().numpy() - u).max() < 1e-10


def test_full_size_sampled_rows(mf, orc):
    """The 48^3 Kuhn mesh (663,552 elements, 912,673 nodes): sampled rows."""
    prob = gen.thermal_p2t_problem(48)
    P = mf.Problem(prob)
    vals, d = P.assemble()
    rp, ci = P.csr_arrays()
    rp, ci, vals, d = rp.cpu().numpy(), ci.cpu().numpy(), vals.cpu().numpy(), d.cpu().numpy()
    nn = prob["coords"].shape[0]
    assert nn == 912673
    rng = np.random.default_rng(41)
    nodes = np.unique(np.concatenate([rng.integers(0, nn, 40), [0, 50, 49 ** 3 // 2, 49 ** 3, nn - 1]]))
    keep = np.zeros(nn, np.uint8)
    keep[nodes] = 1
    ref = orc.assemble(prob, keep_nodes=keep)
    dscale = np.abs(ref["d"][nodes]).max()
    for r, (cols, v) in zip(nodes, orc.rows_of(ref, nodes)):
        s = slice(rp[r], rp[r + 1])
        assert np.array_equal(ci[s], cols)
        assert np.abs(vals[s] - v).max() <= TOL * np.abs(v).max()
        assert abs(d[r] - ref["d"][r]) <= TOL * dscale


def test_single_tetrahedron(mf, orc):
    prob = gen.thermal_p2t_problem(1, jitter=0.0)
    prob["conn"] = prob["conn"][:1]
    prob["coef"] = prob["coef"][:1]
    used = np.unique(prob["conn"])
    remap = -np.ones(prob["coords"].shape[0], np.int64)
    remap[used] = np.arange(used.shape[0])
    prob["conn"] = remap[prob["conn"]].astype(np.int32)
    prob["coords"] = prob["coords"][used]
    prob["bc_mask"] = prob["bc_mask"][used]
    prob["bc_val"] = prob["bc_val"][used]
    P, rp, ci, val, d = _gpu(mf, prob, bc=False)
    ref = orc.assemble(prob, dirichlet=False)
    assert np.array_equal(rp, ref["row_ptr"]) and np.diff(rp).min() == 10
    assert row_scaled_error(rp, val, ref["val"]) <= TOL
    assert np.abs(d - ref["d"]).max() <= TOL * np.abs(ref["d"]).max()


def test_all_constrained(mf, orc):
    prob = gen.thermal_p2t_problem(2)
    prob["bc_mask"][:] = 1
    prob["bc_val"] = np.linspace(-1.0, 1.0, prob["bc_mask"].shape[0])
    P, rp, ci, val, d = _gpu(mf, prob)
    ref = orc.assemble(prob)
    assert np.array_equal(val, ref["val"]) and np.array_equal(d, prob["bc_val"])


def test_nan_conductivity_latched(mf):
    P = mf.Problem(gen.thermal_p2t_problem(2))
    P.coef[7] = float("nan")
    P.assemble()
    with pytest.raises(mf.MFError) as ei:
        mf.mf_sync_status()
    assert ei.value.status == mf.MF_ERR_NONFINITE
    P.coef[7] = 1.0
    P.assemble()
    mf.mf_sync_status()


def test_inverted_tetrahedron_rejected(mf):
    prob = gen.thermal_p2t_problem(2)
    c = prob["conn"][5].copy()
    # swap vertices 1 and 2 (and the edges (0,1) <-> (2,0), (1,3) <-> (2,3))
    prob["conn"][5] = c[[0, 2, 1, 3, 6, 5, 4, 7, 9, 8]]
    with pytest.raises(mf.MFError) as ei:
        mf.Problem(prob)
    assert ei.value.status == mf.MF_ERR_BAD_MESH


def test_unsupported_combinations(mf):
    import torch
    prob = gen.thermal_p2t_problem(2)
    P = mf.Problem(prob)
    C = torch.ones(P.conn.shape[0], dtype=torch.float64, device="cuda")
    with pytest.raises(mf.MFError) as ei:  # the capacity form is FP64 only
        mf.mf_assemble(mf.MF_FORM_CAPACITY, P.mesh, P.pattern, P.make_coeffs(coef=C), mf.MF_PREC_MIXED, P.csr, P.d)
    assert ei.value.status == mf.MF_ERR_UNSUPPORTED
    with pytest.raises(mf.MFError) as ei:
        mf.mf_pattern_build(P.mesh, mf.MF_FORM_ELASTIC)
    assert ei.value.status == mf.MF_ERR_UNSUPPORTED
    e = torch.zeros(1, dtype=torch.int32, device="cuda")
    f = torch.full((1,), 4, dtype=torch.uint8, device="cuda")  # a tetrahedron has faces 0..3
    with pytest.raises(mf.MFError) as ei:
        mf.mf_facets_create(P.mesh, P.pattern, e, f)
    assert ei.value.status == mf.MF_ERR_BAD_MESH
    with pytest.raises(mf.MFError) as ei:
        mf.mf_batch_create([P])
    assert ei.value.status == mf.MF_ERR_UNSUPPORTED


def _p2t_convection(n, sides, dirichlet_x0=True, bval_seed=None):
    prob = gen.thermal_p2t_problem(n)
    x = prob["coords"]
    mask = (np.abs(x[:, 0]) <= 1e-14).astype(np.uint8) if dirichlet_x0 else np.zeros(x.shape[0], np.uint8)
    prob["bc_mask"] = mask
    prob["bc_val"] = np.zeros(x.shape[0])
    if bval_seed is not None:
        prob["bc_val"] = np.where(mask > 0, gen.normal(bval_seed, x.shape[0]), 0.0)
    prob["facets"] = gen.convection_facets(prob, sides)
    return prob


@pytest.mark.parametrize("case", ["five_sides_4", "all_sides_lifted_5"])
def test_convection_on_faces_parity(mf, orc, case):
    """Convection h(T, T_env - T) on the 6-node faces (the surface terms of the
    3D thermal case) added to the assembled system, against the oracle."""
    prob = (_p2t_convection(4, ("x1", "y0", "y1", "z0", "z1")) if case == "five_sides_4"
            else _p2t_convection(5, gen.SIDES, bval_seed=9))
    P, rp, ci, val, d = _gpu(mf, prob)
    ref = orc.assemble(prob)
    assert np.array_equal(rp, ref["row_ptr"]) and np.array_equal(ci, ref["col"])
    assert row_scaled_error(rp, val, ref["val"]) <= TOL
    assert np.abs(d - ref["d"]).max() <= TOL * np.abs(ref["d"]).max()


def test_convection_on_faces_without_dirichlet_and_reproducible(mf, orc):
    import torch
    prob = _p2t_convection(4, gen.SIDES, dirichlet_x0=False)
    P = mf.Problem(prob)
    coeffs = P.make_coeffs(bc=False)
    P.facet_coeffs.bc_mask = None
    P.facet_coeffs.bc_val = None
    v1, d1 = [t.clone() for t in P.assemble(coeffs=coeffs)]
    v2, d2 = P.assemble(coeffs=coeffs)
    assert torch.equal(v1, v2) and torch.equal(d1, d2)
    rp, ci = P.csr_arrays()
    ref = orc.assemble(prob, dirichlet=False)
    assert row_scaled_error(rp.cpu().numpy(), v1.cpu().numpy(), ref["val"]) <= TOL
    assert np.abs(d1.cpu().numpy() - ref["d"]).max() <= TOL * np.abs(ref["d"]).max()
    # the surface terms alone: the sum of all added entries is sum_f h_f A_f
    # (the domain rows sum to zero), whose areas add up to the cube's 6
    fac = prob["facets"]
    e, f = fac["elem"], fac["face"]
    X = prob["coords"]
    fv = ((1, 2, 3), (0, 3, 2), (0, 1, 3), (0, 2, 1))
    area = np.array([0.5 * np.linalg.norm(np.cross(X[prob["conn"][el][fv[fa][1]]] - X[prob["conn"][el][fv[fa][0]]],
                                                     X[prob["conn"][el][fv[fa][2]]] - X[prob["conn"][el][fv[fa][0]]]))
                     for el, fa in zip(e, f)])
    assert abs(area.sum() - 6.0) < 1e-12
    assert abs(v1.cpu().numpy().sum() - (fac["h"] * area).sum()) < 1e-11 * (fac["h"] * area).sum()


def test_capacity_parity(mf, orc):
    """The capacity form C int N_a N_b (the rate term of Sec. 4.1) against the oracle."""
    import torch
    prob = gen.thermal_p2t_problem(4)
    P = mf.Problem(prob)
    C = gen.lognormal(77, prob["conn"].shape[0], 0.3)
    vals = torch.empty(P.nnz, dtype=torch.float64, device="cuda")
    d = torch.empty(P.n, dtype=torch.float64, device="cuda")
    csr = mf.CSR(P.csr.n_rows, P.csr.nnz, P.csr.row_ptr, P.csr.col_idx, vals.data_ptr())
    Ct = torch.from_numpy(np.ascontiguousarray(C)).cuda()
    mf.mf_assemble(mf.MF_FORM_CAPACITY, P.mesh, P.pattern, P.make_coeffs(coef=Ct, bc=False), mf.MF_PREC_FP64, csr, d)
    rp, ci = P.csr_arrays()
    ref = orc.capacity(prob, C)
    assert np.array_equal(rp.cpu().numpy(), ref["row_ptr"]) and np.array_equal(ci.cpu().numpy(), ref["col"])
    assert row_scaled_error(ref["row_ptr"], vals.cpu().numpy(), ref["val"]) <= TOL
    assert (d.cpu().numpy() == 0).all()
