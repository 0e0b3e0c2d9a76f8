"""Parity of the 8-node serendipity quadrilateral (thermal form, FP64) and of
the convection on its edges with the CPU FP64 oracle, through the C ABI:
pattern bit-exact, values row-scaled within 1e-12, sampled rows of a 256^2
mesh, a PCG solve, reproducibility, the 2D thermal case's set-up (sides
fixed, convection on the top edge), degenerate cases and the combinations
the element does not provide.
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
    coeffs = P.make_coeffs(bc=bc)
    if not bc and P.facets:
        P.facet_coeffs.bc_mask = None
        P.facet_coeffs.bc_val = None
    vals, d = P.assemble(coeffs=coeffs)
    rp, ci = P.csr_arrays()
    return P, rp.cpu().numpy(), ci.cpu().numpy(), vals.cpu().numpy(), d.cpu().numpy()


CASES = {
    "q2q_3": lambda: gen.thermal_q2q_problem(3),
    "q2q_7": lambda: gen.thermal_q2q_problem(7),
    "q2q_affine_4": lambda: gen.thermal_q2q_problem(4, jitter=0.0),
}


@pytest.mark.parametrize("case", list(CASES))
def test_pattern_and_values(mf, orc, case):
    prob = CASES[case]()
    P, rp, ci, val, d = _gpu(mf, prob)
    ref = orc.assemble(prob)
    assert np.array_equal(rp, ref["row_ptr"]) and np.array_equal(ci, ref["col"])
    assert row_scaled_error(rp, val, ref["val"]) <= TOL
    assert np.abs(d - ref["d"]).max() <= TOL * np.abs(ref["d"]).max()


def test_values_without_dirichlet_and_lifted(mf, orc):
    prob = gen.thermal_q2q_problem(5)
    P, rp, ci, val, d = _gpu(mf, prob, bc=False)
    ref = orc.assemble(prob, dirichlet=False)
    assert row_scaled_error(rp, val, ref["val"]) <= TOL
    assert np.abs(d - ref["d"]).max() <= TOL * np.abs(ref["d"]).max()
    prob["bc_val"] = np.where(prob["bc_mask"] > 0, gen.normal(12, prob["bc_mask"].shape[0]), 0.0)
    P, rp, ci, val, d = _gpu(mf, prob)
    ref = orc.assemble(prob)
    assert row_scaled_error(rp, val, ref["val"]) <= TOL
    assert np.abs(d - ref["d"]).max() <= TOL * np.abs(ref["d"]).max()


def test_bit_reproducible_and_pcg(mf, orc):
    import torch
    prob = gen.thermal_q2q_problem(12)
    P = mf.Problem(prob)
    v1, d1 = [t.clone() for t in P.assemble()]
    P.values.fill_(float("nan"))
    v2, d2 = P.assemble()
    assert torch.equal(v1, v2) and torch.equal(d1, d2)
    x, st, info = P.solve(tol=1e-12)
    assert st == mf.MF_OK
    xo, _, _ = orc.pcg(orc.assemble(prob), tol=1e-14)
    assert np.abs(x.cpu().numpy() - xo).max() <= 1e-9 * np.abs(xo).max()


def test_full_size_sampled_rows(mf, orc):
    """256^2 quadrilaterals (65,536 elements, 197,633 nodes): sampled rows."""
    prob = gen.thermal_q2q_problem(256)
    P = mf.Problem(prob)
    vals, d = P.assemble()
    rp, ci = P.csr_arrays()
    rp, ci, vals, d = rp.cpu().numpy(), ci.cpu().numpy(), vals.cpu().numpy(), d.cpu().numpy()
    nn = prob["coords"].shape[0]
    assert nn == 197633
    rng = np.random.default_rng(43)
    nodes = np.unique(np.concatenate([rng.integers(0, nn, 40), [0, 258, 257 ** 2 // 2, 257 ** 2, nn - 1]]))
    keep = np.zeros(nn, np.uint8)
    keep[nodes] = 1
    ref = orc.assemble(prob, keep_nodes=keep)
    dscale = np.abs(ref["d"][nodes]).max()
    for r, (cols, v) in zip(nodes, orc.rows_of(ref, nodes)):
        s = slice(rp[r], rp[r + 1])
        assert np.array_equal(ci[s], cols)
        assert np.abs(vals[s] - v).max() <= TOL * np.abs(v).max()
        assert abs(d[r] - ref["d"][r]) <= TOL * dscale


def _case_2d_thermal(n):
    """Left and right sides fixed (T = 1.2), convection on the top edge (the
    2D thermal case's set-up, with synthetic coefficients), insulated bottom."""
    prob = gen.thermal_q2q_problem(n)
    x = prob["coords"]
    side = (np.abs(x[:, 0]) <= 1e-14) | (np.abs(x[:, 0] - 1.0) <= 1e-14)
    prob["bc_mask"] = side.astype(np.uint8)
    prob["bc_val"] = np.where(side, 1.2, 0.0)
    prob["facets"] = gen.convection_facets(prob, ("y1",))
    return prob


def test_top_edge_convection_parity(mf, orc):
    prob = _case_2d_thermal(9)
    P, rp, ci, val, d = _gpu(mf, prob)
    ref = orc.assemble(prob)
    assert np.array_equal(rp, ref["row_ptr"]) and np.array_equal(ci, ref["col"])
    assert row_scaled_error(rp, val, ref["val"]) <= TOL
    assert np.abs(d - ref["d"]).max() <= TOL * np.abs(ref["d"]).max()
    x, st, info = P.solve(tol=1e-12)
    assert st == mf.MF_OK
    xo, _, _ = orc.pcg(ref, tol=1e-14)
    assert np.abs(x.cpu().numpy() - xo).max() <= 1e-9 * np.abs(xo).max()


def test_all_edges_convection_without_dirichlet(mf, orc):
    prob = gen.thermal_q2q_problem(6)
    prob["facets"] = gen.convection_facets(prob, ("x0", "x1", "y0", "y1"))
    P, rp, ci, val, d = _gpu(mf, prob, bc=False)
    ref = orc.assemble(prob, dirichlet=False)
    assert row_scaled_error(rp, val, ref["val"]) <= TOL
    assert np.abs(d - ref["d"]).max() <= TOL * np.abs(ref["d"]).max()


def test_single_element_and_all_constrained(mf, orc):
    prob = gen.thermal_q2q_problem(1, jitter=0.0)
    P, rp, ci, val, d = _gpu(mf, prob, bc=False)
    ref = orc.assemble(prob, dirichlet=False)
    assert np.array_equal(rp, ref["row_ptr"]) and np.diff(rp).min() == 8
    assert row_scaled_error(rp, val, ref["val"]) <= TOL
    prob = gen.thermal_q2q_problem(2)
    prob["bc_mask"][:] = 1
    prob["bc_val"] = np.linspace(-1.0, 1.0, prob["bc_mask"].shape[0])
    P, rp, ci, val, d = _gpu(mf, prob)
    ref = orc.assemble(prob)
    assert np.array_equal(val, ref["val"]) and np.array_equal(d, prob["bc_val"])


def test_nan_conductivity_latched(mf):
    P = mf.Problem(gen.thermal_q2q_problem(2))
    P.coef[1] = float("nan")
    P.assemble()
    with pytest.raises(mf.MFError) as ei:
        mf.mf_sync_status()
    assert ei.value.status == mf.MF_ERR_NONFINITE
    P.coef[1] = 1.0
    P.assemble()
    mf.mf_sync_status()


def test_mirrored_element_rejected(mf):
    prob = gen.thermal_q2q_problem(2)
    c = prob["conn"][1].copy()
    prob["conn"][1] = c[[1, 0, 3, 2, 4, 5, 7, 6]]  # mirror in x: clockwise
    with pytest.raises(mf.MFError) as ei:
        mf.Problem(prob)
    assert ei.value.status == mf.MF_ERR_BAD_MESH


def test_unsupported_combinations(mf):
    import torch
    P = mf.Problem(gen.thermal_q2q_problem(2))
    C = torch.ones(P.conn.shape[0], dtype=torch.float64, device="cuda")
    with pytest.raises(mf.MFError) as ei:  # the capacity form is FP64 only
        mf.mf_assemble(mf.MF_FORM_CAPACITY, P.mesh, P.pattern, P.make_coeffs(coef=C), mf.MF_PREC_MIXED, P.csr, P.d)
    assert ei.value.status == mf.MF_ERR_UNSUPPORTED
    with pytest.raises(mf.MFError) as ei:
        mf.mf_pattern_build(P.mesh, mf.MF_FORM_ELASTIC)
    assert ei.value.status == mf.MF_ERR_UNSUPPORTED
    with pytest.raises(mf.MFError) as ei:
        mf.mf_batch_create([P])
    assert ei.value.status == mf.MF_ERR_UNSUPPORTED


def test_capacity_parity(mf, orc):
    """The capacity form C int N_a N_b (the rate term of Sec. 4.1) against the oracle."""
    import torch
    prob = gen.thermal_q2q_problem(7)
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
