"""Parity of linear elasticity on 20-node serendipity bricks (FP64) with the
CPU FP64 oracle, through the C ABI: pattern bit-exact (rows of up to 243
entries), values row-scaled within 1e-12, sampled rows at 32^3, a PCG solve,
reproducibility, degenerate cases and the combinations the element does not
provide.
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
    "el_q2s_3": lambda: gen.elastic_q2s_problem(3),
    "el_q2s_5": lambda: gen.elastic_q2s_problem(5),
    "el_q2s_affine_4": lambda: gen.elastic_q2s_problem(4, jitter=0.0),
    "el_q2s_nu_049": lambda: gen.elastic_q2s_problem(3, nu=0.49),
}


@pytest.mark.parametrize("case", list(CASES))
def test_pattern_and_values(mf, orc, case):
    prob = CASES[case]()
    P, rp, ci, val, d = _gpu(mf, prob)
    ref = orc.assemble(prob)
    assert np.array_equal(rp, ref["row_ptr"]) and np.array_equal(ci, ref["col"])
    assert np.diff(rp).max() == 243
    assert row_scaled_error(rp, val, ref["val"]) <= TOL
    assert np.abs(d - ref["d"]).max() <= TOL * np.abs(ref["d"]).max()


def test_values_without_dirichlet_and_lifted(mf, orc):
    prob = gen.elastic_q2s_problem(4)
    prob["body"] = (0.3, -0.8, 1.1)
    P, rp, ci, val, d = _gpu(mf, prob, bc=False)
    ref = orc.assemble(prob, dirichlet=False)
    assert row_scaled_error(rp, val, ref["val"]) <= TOL
    assert np.abs(d - ref["d"]).max() <= TOL * np.abs(ref["d"]).max()
    # nonzero prescribed displacements on the clamped face and on single
    # components elsewhere (rows next to them carry the lifting)
    m = prob["bc_mask"].copy()
    m[3 * np.arange(0, m.shape[0] // 3, 7) + 1] = 1
    prob["bc_mask"] = m
    prob["bc_val"] = np.where(m > 0, gen.normal(12, m.shape[0]), 0.0)
    P, rp, ci, val, d = _gpu(mf, prob)
    ref = orc.assemble(prob)
    assert row_scaled_error(rp, val, ref["val"]) <= TOL
    assert np.abs(d - ref["d"]).max() <= TOL * np.abs(ref["d"]).max()


def test_bit_reproducible(mf):
    import torch
    P = mf.Problem(gen.elastic_q2s_problem(6))
    v1, d1 = [t.clone() for t in P.assemble()]
    P.values.fill_(float("nan"))
    P.d.fill_(float("nan"))
    v2, d2 = P.assemble()
    assert torch.equal(v1, v2) and torch.equal(d1, d2)


def test_pcg_matches_oracle(mf, orc):
    prob = gen.elastic_q2s_problem(5)
    P = mf.Problem(prob)
    P.assemble()
    x, st, info = P.solve(tol=1e-12)
    assert st == mf.MF_OK
    ref = orc.assemble(prob)
    xo, _, _ = orc.pcg(ref, tol=1e-14)
    assert np.abs(x.cpu().numpy() - xo).max() <= 1e-9 * np.abs(xo).max()


def test_quadratic_field_solved_exactly(mf):
    """A quadratic displacement with its constant body force (uniform E, nu,
    affine bricks, the field prescribed on the whole boundary) is in the
    serendipity space: the GPU solve returns it at every node."""
    import torch
    prob = gen.elastic_q2s_problem(4, jitter=0.0)
    E, nu = 2.3, 0.3
    prob["coef"] = np.full(prob["conn"].shape[0], E)
    lam, mu = E * nu / ((1 + nu) * (1 - 2 * nu)), E / (2 * (1 + nu))
    H = np.array([[[1.0, 0.3, -0.2], [0.3, -0.5, 0.4], [-0.2, 0.4, 0.7]],
                  [[0.2, -0.6, 0.1], [-0.6, 0.9, 0.3], [0.1, 0.3, -0.4]],
                  [[-0.3, 0.2, 0.5], [0.2, 0.1, -0.7], [0.5, -0.7, 0.6]]])
    x = prob["coords"]
    u = 0.5 * np.einsum("nj,ijk,nk->ni", x, H, x).ravel()
    div = [lam * sum(H[k][k, i] for k in range(3)) + mu * (np.trace(H[i]) + sum(H[j][i, j] for j in range(3)))
           for i in range(3)]
    prob["body"] = tuple(-np.array(div))
    bnd = np.repeat(gen.boundary_nodes(x), 3)
    prob["bc_mask"] = bnd.astype(np.uint8)
    prob["bc_val"] = np.where(bnd, u, 0.0)
    P = mf.Problem(prob)
    P.assemble()
    xs, st, info = P.solve(tol=1e-13)
    assert st == mf.MF_OK
    assert np.abs(xs.cpu().numpy() - u).max() < 1e-10 * np.abs(u).max()


def test_full_size_sampled_rows(mf, orc):
    """32^3 serendipity bricks (32,768 elements, 421,443 dofs): sampled rows."""
    prob = gen.elastic_q2s_problem(32)
    P = mf.Problem(prob)
    vals, d = P.assemble()
    rp, ci = P.csr_arrays()
    rp, ci, vals, d = rp.cpu().numpy(), ci.cpu().numpy(), vals.cpu().numpy(), d.cpu().numpy()
    nn = prob["coords"].shape[0]
    assert rp.shape[0] - 1 == 3 * nn == 421443
    rng = np.random.default_rng(37)
    nodes = np.unique(np.concatenate([rng.integers(0, nn, 30), [0, 34, 33 ** 3 // 2, 33 ** 3, nn - 1]]))
    keep = np.zeros(nn, np.uint8)
    keep[nodes] = 1
    ref = orc.assemble(prob, keep_nodes=keep)
    rows = np.concatenate([3 * nodes + c for c in range(3)])
    dscale = np.abs(ref["d"][rows]).max()
    for r, (cols, v) in zip(rows, orc.rows_of(ref, rows)):
        s = slice(rp[r], rp[r + 1])
        assert np.array_equal(ci[s], cols)
        assert np.abs(vals[s] - v).max() <= TOL * np.abs(v).max()
        assert abs(d[r] - ref["d"][r]) <= TOL * dscale


def test_single_brick(mf, orc):
    prob = gen.elastic_q2s_problem(1, jitter=0.0)
    P, rp, ci, val, d = _gpu(mf, prob, bc=False)
    ref = orc.assemble(prob, dirichlet=False)
    assert np.array_equal(rp, ref["row_ptr"]) and np.array_equal(ci, ref["col"])
    assert np.diff(rp).min() == 60  # every dof couples with all 60
    assert row_scaled_error(rp, val, ref["val"]) <= TOL
    assert np.abs(d - ref["d"]).max() <= TOL * np.abs(ref["d"]).max()


def test_all_constrained(mf, orc):
    prob = gen.elastic_q2s_problem(2)
    prob["bc_mask"][:] = 1
    prob["bc_val"] = np.linspace(-1.0, 1.0, prob["bc_mask"].shape[0])
    P, rp, ci, val, d = _gpu(mf, prob)
    ref = orc.assemble(prob)
    assert np.array_equal(val, ref["val"]) and np.array_equal(d, prob["bc_val"])


def test_nan_modulus_latched(mf):
    P = mf.Problem(gen.elastic_q2s_problem(2))
    P.coef[5] = float("nan")
    P.assemble()
    with pytest.raises(mf.MFError) as ei:
        mf.mf_sync_status()
    assert ei.value.status == mf.MF_ERR_NONFINITE
    P.coef[5] = 1.0
    P.assemble()
    mf.mf_sync_status()


def test_unsupported_combinations(mf):
    import torch
    prob = gen.elastic_q2s_problem(2)
    P = mf.Problem(prob)
    with pytest.raises(mf.MFError) as ei:
        mf.mf_assemble(mf.MF_FORM_ELASTIC, P.mesh, P.pattern, P.make_coeffs(), mf.MF_PREC_MIXED, P.csr, P.d)
    assert ei.value.status == mf.MF_ERR_UNSUPPORTED
    e = torch.zeros(1, dtype=torch.int32, device="cuda")
    f = torch.zeros(1, dtype=torch.uint8, device="cuda")
    fs = mf.mf_facets_create(P.mesh, P.pattern, e, f)  # 8-node faces carry facet terms
    mf.mf_facets_destroy(fs)
    with pytest.raises(mf.MFError) as ei:  # batching takes thermal problems
        mf.mf_batch_create([P])
    assert ei.value.status == mf.MF_ERR_INVALID_ARG
    with pytest.raises(mf.MFError) as ei:
        mf.mf_pattern_build(P.mesh, mf.MF_FORM_OSEEN)
    assert ei.value.status == mf.MF_ERR_UNSUPPORTED
