"""Steady Navier-Stokes with SUPG (Sec. 4.3) on the GPU against the oracle.
The GPU forms the element residual and tangent in double-float (FP32 pairs,
about 47 bits) and sums them into the CSR rows in FP64.

The oracle's or_ns_system gives the residual R and the tangent K = dR/dx by
complex-step differentiation of its residual (its own 16-point rule); the
GPU path forms the tangent by hand-derived derivatives on a collapsed 4 x 4
Gauss rule, so the two agree only if both the form and its derivative are
right.  Contract: the CSR pattern equals the oracle's element couplings (every
block present); K within 1e-12 row-scaled and d = -R within 1e-12 of the
residual scale; Newton from the Dirichlet values takes the oracle's number of
steps and reaches its solution.
"""
import numpy as np
import pytest

import gen

pytestmark = pytest.mark.gpu
MU, RHO, TM, TC = 0.05, 1.3, 0.02, 0.03


@pytest.fixture(scope="module")
def mf():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2111_03541_gb300 as mf
    mf.lib()
    return mf


def ns_problem(n, jitter=0.0, mu=MU, rho=RHO, tm=TM, tc=TC, seed=3):
    prob = gen.oseen_problem(n, viscosity=mu, rho=rho)
    if jitter > 0.0:
        m = gen.tri_mesh(n, 2, jitter)
        for k in ("coords", "conn", "vconn", "vcoords"):
            prob[k] = m[k]
    prob["form"] = "ns"
    prob["tau_m"], prob["tau_c"] = tm, tc
    n2, n1 = prob["coords"].shape[0], prob["vcoords"].shape[0]
    prob["state"] = np.random.default_rng(seed).standard_normal(2 * n2 + n1)
    return prob


def oracle_rows(orc, prob):
    R, K = orc.ns_system(prob, prob["state"], prob["tau_m"], prob["tau_c"])
    K = K.tocsr()
    K.sort_indices()
    return R, K


def row_scaled_error(rp, val, ref):
    n = rp.shape[0] - 1
    rows = np.repeat(np.arange(n), np.diff(rp))
    emax = np.zeros(n)
    rmax = np.zeros(n)
    np.maximum.at(emax, rows, np.abs(val - ref))
    np.maximum.at(rmax, rows, np.abs(ref))
    ok = rmax > 0
    assert (emax[~ok] <= 1e-300).all()
    return (emax[ok] / rmax[ok]).max()


@pytest.mark.parametrize("n,jitter", [(1, 0.0), (2, 0.0), (5, 0.0), (8, 0.2), (13, 0.2)])
def test_ns_tangent_and_residual_against_oracle(mf, orc, n, jitter):
    prob = ns_problem(n, jitter)
    P = mf.Problem(prob)
    vals, d = P.assemble(coeffs=P.make_coeffs(bc=False))
    mf.mf_sync_status()
    rp, ci = P.csr_arrays()
    rp, ci = rp.cpu().numpy(), ci.cpu().numpy()
    R, K = oracle_rows(orc, prob)
    assert np.array_equal(rp, K.indptr) and np.array_equal(ci, K.indices)
    assert row_scaled_error(rp, vals.cpu().numpy(), K.data) <= 1e-12
    assert np.abs(d.cpu().numpy() + R).max() <= 1e-12 * np.abs(R).max()


def test_ns_every_block_present(mf, orc):
    prob = ns_problem(4)
    P = mf.Problem(prob)
    rp, ci = P.csr_arrays()
    rp, ci = rp.cpu().numpy(), ci.cpu().numpy()
    n2 = prob["coords"].shape[0]
    row_u1, row_p = 5, 2 * n2 + 3
    cols_u1 = ci[rp[row_u1]:rp[row_u1 + 1]]
    cols_p = ci[rp[row_p]:rp[row_p + 1]]
    assert (cols_u1 >= n2).any() and (cols_u1 < n2).any() and (cols_u1 >= 2 * n2).any()  # u1-u2 and u-p
    assert ((cols_p >= 2 * n2) & (cols_p != row_p)).any()  # p-p beyond the diagonal


def test_ns_dirichlet_elimination(mf, orc):
    """State on the Dirichlet data: free rows keep the oracle's tangent on free
    columns (constrained columns zeroed, nothing lifted), constrained rows are
    identity rows with d = 0, and d = -R on the free rows."""
    prob = ns_problem(6)
    mask = prob["bc_mask"] > 0
    prob["state"] = np.where(mask, prob["bc_val"], prob["state"])
    P = mf.Problem(prob)
    vals, d = P.assemble()
    mf.mf_sync_status()
    rp, ci = P.csr_arrays()
    rp, ci, vals, d = rp.cpu().numpy(), ci.cpu().numpy(), vals.cpu().numpy(), d.cpu().numpy()
    R, K = oracle_rows(orc, prob)
    rows = np.repeat(np.arange(rp.shape[0] - 1), np.diff(rp))
    ref = np.where(mask[rows] | mask[ci], 0.0, K.data)
    ref = np.where(mask[rows] & (rows == ci), 1.0, ref)
    assert row_scaled_error(rp, vals, ref) <= 1e-12
    assert (d[mask] == 0.0).all()
    assert np.abs(d[~mask] + R[~mask]).max() <= 1e-12 * np.abs(R).max()


def test_ns_bit_reproducible(mf):
    import torch
    P = mf.Problem(ns_problem(9, 0.2))
    v1, d1 = [t.clone() for t in P.assemble()]
    P.values.zero_()
    v2, d2 = P.assemble()
    assert torch.equal(v1, v2) and torch.equal(d1, d2)


@pytest.mark.parametrize("n", [4, 8])
def test_ns_newton_matches_oracle(mf, orc, n):
    """Lid-driven cavity (Re 50), Newton from the Dirichlet values: the GPU
    takes the oracle's number of steps (quadratic convergence) and reaches
    its solution."""
    prob = ns_problem(n, mu=0.02, rho=1.0, tm=0.01, tc=0.01)
    xo, hist_o = orc.ns_newton(prob, 0.01, 0.01, tol=1e-12)
    import torch
    P = mf.Problem(prob)
    P.advect.zero_()
    st, hist, steps = P.newton(tol=1e-12, max_newton=30, lin_tol=1e-12)
    assert st == mf.MF_OK
    assert steps == len(hist_o) - 1
    assert hist[0] == pytest.approx(hist_o[0], rel=1e-12)
    x = P.advect.cpu().numpy()
    assert np.linalg.norm(x - xo) <= 1e-9 * np.linalg.norm(xo)
    # quadratic: once small, each norm is about the square of the previous;
    # norms below 1e-13 are at the floor of the double-float residual (about
    # 2^-47 of its terms) and say nothing about the rate
    small = [(a, b) for a, b in zip(hist[:-1], hist[1:]) if a < 1e-2 and b > 1e-13]
    assert small and all(b < 50.0 * a * a for a, b in small)
