"""The flow system (Sec. 4.3 Picard form, Taylor-Hood P2-P1, lid-driven
cavity data) solved by GMRES(50) with the block upper-triangular
preconditioner (pressure mass over the viscosity for the Schur complement,
one geometric multigrid V-cycle for the velocity block): the solution
matches a direct solve of the oracle's system, and the iteration count stays
bounded as the grid is refined (16^2 .. 64^2)."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import gen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mf():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2111_03541_gb300 as mf
    mf.lib()
    return mf


def hierarchy(mf, n, coarsest=4):
    probs, m = [], n
    while m >= coarsest:
        probs.append(gen.oseen_problem(m))
        m //= 2
    Ps = [mf.Problem(p) for p in probs]
    for P in Ps:
        P.assemble()
    pm = Ps[0].pressure_mass_diag()
    mg = mf.mf_flow_mg_create([P.csr for P in Ps], [p["n"] for p in probs], [P.bc_mask for P in Ps], pm,
                              probs[0]["viscosity"])
    return probs, Ps, mg


def solve(mf, n, tol=1e-10):
    probs, Ps, mg = hierarchy(mf, n)
    try:
        x, st, info = Ps[0].solve(solver=mf.MF_SOLVER_GMRES_FLOW_MG, restart=50, tol=tol, max_iter=2000,
                                  flow_mg=mg, check_every=1)
    finally:
        mf.mf_flow_mg_destroy(mg)
    return probs[0], x, st, info


@pytest.mark.parametrize("n", [16, 32])
def test_flow_mg_solves_the_oracle_system(mf, orc, n):
    """Backward error: the GPU solution leaves a residual below 5e-11 in the
    oracle's own system; forward error: within 10 kappa_1 relres of the direct
    solve of that system (kappa_1 from a 1-norm condition estimate)."""
    prob, x, st, info = solve(mf, n, tol=1e-11)
    assert st == mf.MF_OK and info.converged and info.rel_residual <= 1e-11
    assert info.iterations <= 200, info.iterations
    ref = orc.assemble(prob)
    nr = ref["row_ptr"].shape[0] - 1
    K = sp.csr_matrix((ref["val"], ref["col"], ref["row_ptr"]), shape=(nr, nr)).tocsc()
    xg = x.cpu().numpy()
    assert np.linalg.norm(ref["d"] - K @ xg) <= 5e-11 * np.linalg.norm(ref["d"])
    lu = spla.splu(K)
    kinv = spla.LinearOperator(K.shape, matvec=lu.solve, rmatvec=lambda v: lu.solve(v, trans="T"))
    kappa = spla.norm(K, 1) * spla.onenormest(kinv)
    xr = lu.solve(ref["d"])
    err = np.linalg.norm(xg - xr) / np.linalg.norm(xr)
    assert err <= 10 * kappa * 1e-11, (err, kappa)


def test_flow_mg_iterations_do_not_grow_with_the_grid(mf):
    its = {}
    for n in (16, 32, 64):
        _, _, st, info = solve(mf, n, tol=1e-8)
        assert st == mf.MF_OK and info.converged
        its[n] = info.iterations
    assert its[16] <= 120 and its[64] <= 1.5 * its[16] + 10, its
