"""FP64 iterative refinement around an FP32 inner Jacobi-PCG (the mixed
path's solve, MF_SOLVER_PCG_REFINED), against the oracle.

Contract (reading 12): the refined solution of the mixed-assembled system
lies within 1e-8 relative of the oracle's tight solution x*; x* is
meaningful because the oracle's own kappa_est * relres is below 1e-9.  At
64^3 x* is the committed golden file written by
tests/golden/make_elastic_64cube_solution.py (oracle only), compared on its
1,024 sampled dofs.
"""
import os

import numpy as np
import pytest

import gen

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "elastic_q1_64cube_solution.txt")


@pytest.fixture(scope="module")
def mf():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2111_03541_gb300 as mf
    mf.lib()
    return mf


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_refined_solve_against_oracle_12cube(mf, orc, prec):
    prob = gen.elastic_problem(12)
    P = mf.Problem(prob)
    P.assemble(mf.MF_PREC_MIXED if prec == "mixed" else mf.MF_PREC_FP64)
    x, st, info = P.solve(solver=mf.MF_SOLVER_PCG_REFINED, tol=1e-12, max_iter=100000, inner_tol=1e-4)
    assert st == mf.MF_OK and info.converged and info.rel_residual <= 1e-12
    assert info.refinements >= 2  # the FP32 inner solves alone cannot reach 1e-12
    ref = orc.assemble(prob)
    xo, _, rr = orc.pcg(ref, tol=1e-14, maxit=100000)
    err = np.linalg.norm(x.cpu().numpy() - xo) / np.linalg.norm(xo)
    assert err <= 1e-8, err


def test_refined_matches_fp64_pcg_on_p1(mf):
    """A scalar system (2D thermal, P1): refined and plain FP64 PCG agree."""
    import torch
    P = mf.Problem(gen.thermal_p1_problem(64))
    P.assemble()
    x64, st, _ = P.solve(tol=1e-12)
    xr, st2, info = P.solve(solver=mf.MF_SOLVER_PCG_REFINED, tol=1e-12, inner_tol=1e-3)
    assert st == mf.MF_OK and st2 == mf.MF_OK and info.refinements >= 1
    assert (torch.linalg.norm(xr - x64) / torch.linalg.norm(x64)).item() <= 1e-9


def test_refined_mixed_64cube_against_golden(mf):
    head, idx, val = {}, [], []
    with open(GOLDEN) as f:
        for line in f:
            if line.startswith("#"):
                continue
            a, b = line.split()
            if a.isdigit():
                idx.append(int(a))
                val.append(float(b))
            else:
                head[a] = float(b)
    assert head["kappa_est"] * head["relres"] <= 1e-9  # x* is tight enough to judge 1e-8
    prob = gen.elastic_problem(64)
    P = mf.Problem(prob)
    P.assemble(mf.MF_PREC_MIXED)
    # the FP64 residual of this system has a rounding floor near 2e-12: 1e-11 is reachable
    x, st, info = P.solve(solver=mf.MF_SOLVER_PCG_REFINED, tol=1e-11, max_iter=200000, inner_tol=1e-4)
    assert st == mf.MF_OK and info.converged and info.refinements <= 20
    xs = x.cpu().numpy()[np.array(idx)]
    ref = np.array(val)
    err = np.linalg.norm(xs - ref) / np.linalg.norm(ref)
    assert err <= 1e-8, err


def test_refinement_stops_at_the_rounding_floor(mf):
    """A tolerance below the FP64 residual's rounding floor ends in a
    'stagnated' error after a few refinements, not at the iteration cap."""
    P = mf.Problem(gen.elastic_problem(16))
    P.assemble(mf.MF_PREC_MIXED)
    x, st, info = P.solve(solver=mf.MF_SOLVER_PCG_REFINED, tol=1e-30, max_iter=10 ** 7, inner_tol=1e-4)
    assert st == mf.MF_ERR_NOT_CONVERGED and not info.converged
    assert info.refinements <= 40 and info.iterations < 10 ** 6
    assert info.rel_residual <= 1e-12
