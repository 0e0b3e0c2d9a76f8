"""Mixed-precision (tensor-core) assembly of Q1 elasticity against the oracle.

Contract: the CSR pattern is the same bit for bit; K within 1e-11 row-scaled
of the FP64 oracle (the slices keep about 40 bits of the scaled gradients);
the solution of the mixed system within 1e-8 relative of the oracle's
tightly solved x*; two assemblies bit-identical.  Any Poisson ratio in
(-1, 0.5) is accepted (lambda / mu enters once per CSR block as an exact
53-bit multiplier), and the fixed-point scale follows the coordinates and
coefficients of each assembly.
"""
import numpy as np
import pytest

import gen

pytestmark = pytest.mark.gpu

TOL_K = 1e-11


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
    emax = np.zeros(n)
    rmax = np.zeros(n)
    np.maximum.at(emax, rows, np.abs(val - ref))
    np.maximum.at(rmax, rows, np.abs(ref))
    ok = rmax > 0
    assert (emax[~ok] == 0).all()
    return (emax[ok] / rmax[ok]).max()


@pytest.mark.parametrize("n,nu", [(1, 0.3), (5, 0.3), (9, 0.3), (13, 0.3), (6, 0.25), (6, 0.45), (6, 0.0),
                                  (6, 0.49), (6, -0.3), (5, 0.3141592653589793), (4, 1e-12)])
def test_mixed_values_against_oracle(mf, orc, n, nu):
    prob = gen.elastic_problem(n, nu=nu)
    P = mf.Problem(prob)
    vals, d = P.assemble(mf.MF_PREC_MIXED)
    mf.mf_sync_status()
    rp, ci = P.csr_arrays()
    rp = rp.cpu().numpy()
    ref = orc.assemble(prob)
    assert np.array_equal(rp, ref["row_ptr"]) and np.array_equal(ci.cpu().numpy(), ref["col"])
    err = row_scaled_error(rp, vals.cpu().numpy(), ref["val"])
    assert err <= TOL_K, err
    assert np.abs(d.cpu().numpy() - ref["d"]).max() <= 1e-12 * np.abs(ref["d"]).max()


def test_mixed_without_dirichlet_keeps_rigid_modes(mf, orc):
    import torch
    prob = gen.elastic_problem(6)
    P = mf.Problem(prob)
    vals, d = P.assemble(mf.MF_PREC_MIXED, coeffs=P.make_coeffs(bc=False))
    x = prob["coords"]
    scale = vals.abs().max().item()
    for w in np.eye(3):
        u = torch.from_numpy(np.cross(w, x).ravel()).cuda()
        y = torch.empty_like(u)
        mf.mf_spmv(P.csr, u, y)
        assert y.abs().max().item() <= 1e-11 * scale


def test_mixed_solution_within_1e8(mf, orc):
    import torch
    prob = gen.elastic_problem(12)
    P = mf.Problem(prob)
    P.assemble(mf.MF_PREC_MIXED)
    x, st, info = P.solve(tol=1e-12, max_iter=100000)
    assert st == mf.MF_OK
    ref = orc.assemble(prob)
    xo, _, rr = orc.pcg(ref, tol=1e-14, maxit=100000)
    err = np.linalg.norm(x.cpu().numpy() - xo) / np.linalg.norm(xo)
    assert err <= 1e-8, err


def test_mixed_bit_reproducible(mf):
    import torch
    P = mf.Problem(gen.elastic_problem(11))
    v1, d1 = [t.clone() for t in P.assemble(mf.MF_PREC_MIXED)]
    P.values.zero_()
    v2, d2 = P.assemble(mf.MF_PREC_MIXED)
    assert torch.equal(v1, v2) and torch.equal(d1, d2)


def test_mixed_alternating_coefficients_on_one_pattern(mf):
    """Re-assembly on one pattern keeps no state from the call before: five
    calls with two coefficient sets (different Poisson ratio, coefficients,
    lifting and Dirichlet data; an FP64 call in between) give, bit for bit,
    what a fresh pattern gives for the same coefficients."""
    import torch
    prob = gen.elastic_problem(9)
    rng = np.random.default_rng(21)
    prob["bc_val"] = np.where(prob["bc_mask"] != 0, rng.standard_normal(prob["bc_val"].shape[0]), 0.0)
    P = mf.Problem(prob)
    coef_b = P.coef * 3.0
    cA = P.make_coeffs()
    cB = P.make_coeffs(coef=coef_b, bc=False)
    cB.nu = 0.45

    def run(Q, c):
        v, d = Q.assemble(mf.MF_PREC_MIXED, coeffs=c)
        mf.mf_sync_status()
        return v.clone(), d.clone()

    seq = [run(P, cA), run(P, cB)]
    P.assemble(mf.MF_PREC_FP64)
    seq += [run(P, cA), run(P, cB), run(P, cA)]
    Q = mf.Problem(prob)
    fresh_b = run(Q, cB)  # cB names no buffer of P's pattern
    for k, (v, d) in enumerate(seq):
        ref = seq[0] if k % 2 == 0 else fresh_b
        assert torch.equal(v, ref[0]) and torch.equal(d, ref[1]), k
    assert not torch.equal(seq[0][0], seq[1][0])


def test_mixed_nan_coordinate_latched(mf):
    """A NaN coordinate (one node: its 8 elements, mixed with finite ones in
    their warps) is reported as MF_ERR_NONFINITE by the fixed-point bound
    pass, and the next assembly with the coordinate restored is clean."""
    import torch
    P = mf.Problem(gen.elastic_problem(6))
    v0, d0 = [t.clone() for t in P.assemble(mf.MF_PREC_MIXED)]
    mf.mf_sync_status()
    node = 3 * 49 + 2 * 7 + 3  # an interior node of the 7 x 7 x 7 node lattice
    keep = P.coords[node, 1].item()
    P.coords[node, 1] = float("nan")
    P.assemble(mf.MF_PREC_MIXED)
    with pytest.raises(mf.MFError) as ei:
        mf.mf_sync_status()
    assert ei.value.status == mf.MF_ERR_NONFINITE
    P.coords[node, 1] = keep
    v1, d1 = P.assemble(mf.MF_PREC_MIXED)
    mf.mf_sync_status()
    assert torch.equal(v0, v1) and torch.equal(d0, d1)


def test_mixed_full_size_sampled_rows(mf, orc):
    prob = gen.elastic_problem(64)
    P = mf.Problem(prob)
    vals, d = P.assemble(mf.MF_PREC_MIXED)
    rp, ci = P.csr_arrays()
    rp, ci, vals = rp.cpu().numpy(), ci.cpu().numpy(), vals.cpu().numpy()
    nn = prob["coords"].shape[0]
    nodes = np.unique(np.concatenate([np.random.default_rng(13).integers(0, nn, 30), [1, 66, nn - 2]]))
    keep = np.zeros(nn, np.uint8)
    keep[nodes] = 1
    ref = orc.assemble(prob, keep_nodes=keep)
    rows = [3 * n + c for n in nodes for c in range(3)]
    for r, (cols, v) in zip(rows, orc.rows_of(ref, rows)):
        s = slice(rp[r], rp[r + 1])
        assert np.array_equal(ci[s], cols)
        assert np.abs(vals[s] - v).max() <= TOL_K * np.abs(v).max()


def test_mixed_full_32cube(mf, orc):
    """32^3 = 32,768 elements, every row compared."""
    prob = gen.elastic_problem(32)
    P = mf.Problem(prob)
    vals, d = P.assemble(mf.MF_PREC_MIXED)
    mf.mf_sync_status()
    rp, ci = P.csr_arrays()
    rp = rp.cpu().numpy()
    ref = orc.assemble(prob)
    assert np.array_equal(rp, ref["row_ptr"]) and np.array_equal(ci.cpu().numpy(), ref["col"])
    assert row_scaled_error(rp, vals.cpu().numpy(), ref["val"]) <= TOL_K
    assert np.abs(d.cpu().numpy() - ref["d"]).max() <= 1e-12 * np.abs(ref["d"]).max()


def test_mixed_lifting_nonzero_dirichlet(mf, orc):
    """Nonzero prescribed displacements: lifted right-hand side against the oracle."""
    prob = gen.elastic_problem(7)
    rng = np.random.default_rng(5)
    prob["bc_val"] = np.where(prob["bc_mask"] != 0, rng.standard_normal(prob["bc_val"].shape[0]), 0.0)
    P = mf.Problem(prob)
    vals, d = P.assemble(mf.MF_PREC_MIXED)
    mf.mf_sync_status()
    rp, _ = P.csr_arrays()
    ref = orc.assemble(prob)
    assert row_scaled_error(rp.cpu().numpy(), vals.cpu().numpy(), ref["val"]) <= TOL_K
    assert np.abs(d.cpu().numpy() - ref["d"]).max() <= 1e-10 * np.abs(ref["d"]).max()


def test_mixed_scale_follows_moved_coordinates(mf, orc):
    """The fixed-point scale is taken per assembly: moving the nodes (here a
    uniform stretch by 3, which scales K by 3) after the pattern was built
    still gives the oracle's K of the moved mesh."""
    import torch
    prob = gen.elastic_problem(6)
    P = mf.Problem(prob)
    P.assemble(mf.MF_PREC_MIXED)
    moved = dict(prob)
    moved["coords"] = prob["coords"] * 3.0
    P.coords.copy_(torch.from_numpy(moved["coords"]).to(P.coords.device))
    vals, d = P.assemble(mf.MF_PREC_MIXED)
    mf.mf_sync_status()
    rp, _ = P.csr_arrays()
    ref = orc.assemble(moved)
    assert row_scaled_error(rp.cpu().numpy(), vals.cpu().numpy(), ref["val"]) <= TOL_K
    assert np.abs(d.cpu().numpy() - ref["d"]).max() <= 1e-12 * np.abs(ref["d"]).max()
