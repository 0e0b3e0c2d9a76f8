"""Parity of the 20-node serendipity brick (thermal form, FP64) with the CPU
FP64 oracle, through the C ABI: pattern bit-exact (rows of up to 81
entries), values row-scaled within 1e-12, sampled rows at 32^3, a PCG solve,
reproducibility and the combinations the element does not provide.
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
    "q2s_3": lambda: gen.thermal_q2s_problem(3),
    "q2s_5": lambda: gen.thermal_q2s_problem(5),
    "q2s_affine_4": lambda: gen.thermal_q2s_problem(4, jitter=0.0),
}


@pytest.mark.parametrize("case", list(CASES))
def test_pattern_and_values(mf, orc, case):
    prob = CASES[case]()
    P, rp, ci, val, d = _gpu(mf, prob)
    ref = orc.assemble(prob)
    assert np.array_equal(rp, ref["row_ptr"]) and np.array_equal(ci, ref["col"])
    assert np.diff(rp).max() == 81
    assert row_scaled_error(rp, val, ref["val"]) <= TOL
    assert np.abs(d - ref["d"]).max() <= TOL * np.abs(ref["d"]).max()


def test_values_without_dirichlet_and_lifted(mf, orc):
    prob = gen.thermal_q2s_problem(4)
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
    P = mf.Problem(gen.thermal_q2s_problem(6))
    v1, d1 = [t.clone() for t in P.assemble()]
    P.values.fill_(float("nan"))
    v2, d2 = P.assemble()
    assert torch.equal(v1, v2) and torch.equal(d1, d2)


def test_pcg_matches_oracle(mf, orc):
    prob = gen.thermal_q2s_problem(6)
    P = mf.Problem(prob)
    P.assemble()
    x, st, info = P.solve(tol=1e-12)
    assert st == mf.MF_OK
    ref = orc.assemble(prob)
    xo, _, _ = orc.pcg(ref, tol=1e-14)
    assert np.abs(x.cpu().numpy() - xo).max() <= 1e-9 * np.abs(xo).max()


def test_full_size_sampled_rows(mf, orc):
    """32^3 serendipity bricks (32,768 elements, 140,481 nodes): sampled rows."""
    prob = gen.thermal_q2s_problem(32)
    P = mf.Problem(prob)
    vals, d = P.assemble()
    rp, ci = P.csr_arrays()
    rp, ci, vals, d = rp.cpu().numpy(), ci.cpu().numpy(), vals.cpu().numpy(), d.cpu().numpy()
    nn = prob["coords"].shape[0]
    assert nn == 33 ** 3 + 3 * 32 * 33 * 33
    rng = np.random.default_rng(31)
    nodes = np.unique(np.concatenate([rng.integers(0, nn, 40), [0, 34, 33 ** 3 // 2, 33 ** 3, nn - 1]]))
    keep = np.zeros(nn, np.uint8)
    keep[nodes] = 1
    ref = orc.assemble(prob, keep_nodes=keep)
    dscale = np.abs(ref["d"][nodes]).max()
    for r, (cols, v) in zip(nodes, orc.rows_of(ref, nodes)):
        s = slice(rp[r], rp[r + 1])
        assert np.array_equal(ci[s], cols)
        assert np.abs(vals[s] - v).max() <= TOL * np.abs(v).max()
        assert abs(d[r] - ref["d"][r]) <= TOL * dscale


def test_unsupported_combinations(mf):
    import torch
    prob = gen.thermal_q2s_problem(2)
    P = mf.Problem(prob)
    C = torch.ones(P.conn.shape[0], dtype=torch.float64, device="cuda")
    with pytest.raises(mf.MFError) as ei:
        mf.mf_assemble(mf.MF_FORM_CAPACITY, P.mesh, P.pattern, P.make_coeffs(coef=C), mf.MF_PREC_FP64, P.csr, P.d)
    assert ei.value.status == mf.MF_ERR_UNSUPPORTED
    with pytest.raises(mf.MFError) as ei:
        mf.mf_pattern_build(P.mesh, mf.MF_FORM_OSEEN)
    assert ei.value.status == mf.MF_ERR_UNSUPPORTED
    e = torch.zeros(1, dtype=torch.int32, device="cuda")
    f = torch.zeros(1, dtype=torch.uint8, device="cuda")
    fs = mf.mf_facets_create(P.mesh, P.pattern, e, f)  # 8-node faces carry facet terms
    mf.mf_facets_destroy(fs)
    with pytest.raises(mf.MFError) as ei:
        mf.mf_batch_create([P])
    assert ei.value.status == mf.MF_ERR_UNSUPPORTED


def test_inverted_brick_rejected(mf):
    prob = gen.thermal_q2s_problem(2)
    c = prob["conn"][3].copy()
    # mirror the element in x: swap vertices i = 0 <-> 1 (and the y/z edges at x = 0 <-> 1)
    perm = [1, 0, 3, 2, 5, 4, 7, 6, 8, 9, 10, 11, 13, 12, 15, 14, 17, 16, 19, 18]
    prob["conn"][3] = c[perm]
    with pytest.raises(mf.MFError) as ei:
        mf.Problem(prob)
    assert ei.value.status == mf.MF_ERR_BAD_MESH


def test_single_brick(mf, orc):
    prob = gen.thermal_q2s_problem(1, jitter=0.0)
    P, rp, ci, val, d = _gpu(mf, prob, bc=False)
    ref = orc.assemble(prob, dirichlet=False)
    assert np.array_equal(rp, ref["row_ptr"]) and np.array_equal(ci, ref["col"])
    assert np.diff(rp).min() == 20  # every node couples with all 20
    assert row_scaled_error(rp, val, ref["val"]) <= TOL
    assert np.abs(d - ref["d"]).max() <= TOL * np.abs(ref["d"]).max()


def test_all_constrained(mf, orc):
    prob = gen.thermal_q2s_problem(2)
    prob["bc_mask"][:] = 1
    prob["bc_val"] = np.linspace(-1.0, 1.0, prob["bc_mask"].shape[0])
    P, rp, ci, val, d = _gpu(mf, prob)
    ref = orc.assemble(prob)
    assert np.array_equal(val, ref["val"]) and np.array_equal(d, prob["bc_val"])


def test_nan_conductivity_latched(mf):
    P = mf.Problem(gen.thermal_q2s_problem(2))
    P.coef[3] = float("nan")
    P.assemble()
    with pytest.raises(mf.MFError) as ei:
        mf.mf_sync_status()
    assert ei.value.status == mf.MF_ERR_NONFINITE
    P.coef[3] = 1.0
    P.assemble()
    mf.mf_sync_status()
