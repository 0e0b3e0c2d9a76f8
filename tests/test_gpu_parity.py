"""Parity of the CUDA path (through the C ABI) with the CPU FP64 oracle.

Pattern: bit-exact.  Values: row-scaled max error <= 1e-12, i.e.
max_i max_j |K_ij - K^ora_ij| / max_j |K^ora_ij|, and max_i |d_i - d^ora_i| <=
1e-12 max |d^ora|.  Sizes span several thread blocks and ragged tails; the
full-size elasticity case is checked on sampled rows the oracle assembles one
by one.
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


def _partly_jittered_q1(n):
    """Unjittered Q1 box whose interior nodes with x < 0.4 are moved: elements
    away from them stay exact translates of element 0, the others are not."""
    prob = gen.thermal_q1_problem(n, jitter=0.0)
    X = prob["coords"].copy()
    h = 1.0 / n
    inner = (X[:, 0] > 1e-12) & (X[:, 0] < 0.4) & (np.abs(X[:, 1] - 0.5) < 0.5 - 1e-12) & \
        (np.abs(X[:, 2] - 0.5) < 0.5 - 1e-12)
    idx = np.nonzero(inner)[0]
    X[idx] += 0.15 * h * (2.0 * gen.uniform(4321, 3 * idx.size).reshape(-1, 3) - 1.0)
    prob["coords"] = X
    return prob


def _box_q1(n, scale=(1.0, 1.0, 1.0), shear=0.0):
    """Unjittered Q1 box of side h = 1/n, n a power of two so that every
    element is an exact translate of element 0; ``scale`` stretches the axes
    by powers of two (a rectangular cell, still exact), ``shear`` adds shear *
    y to x (a sheared cell: translates, but not class-constant reference
    entries)."""
    prob = gen.thermal_q1_problem(n, jitter=0.0)
    X = prob["coords"].copy()
    X[:, 0] += shear * X[:, 1]
    X *= np.asarray(scale)
    prob["coords"] = X
    return prob


CASES = {
    "p1_64": lambda: gen.thermal_p1_problem(64),
    "p1_13": lambda: gen.thermal_p1_problem(13),
    "p2_11": lambda: gen.thermal_p2_problem(11),
    "q1_9": lambda: gen.thermal_q1_problem(9),
    "q1_affine_11": lambda: gen.thermal_q1_problem(11, jitter=0.0),
    "q1_partly_translate_10": lambda: _partly_jittered_q1(10),
    "q1_box_16": lambda: _box_q1(16),
    "q1_box_rect_8": lambda: _box_q1(8, scale=(1.0, 0.5, 2.0)),
    "q1_box_sheared_8": lambda: _box_q1(8, shear=0.25),
    "el_7": lambda: gen.elastic_problem(7),
    "el_12": lambda: gen.elastic_problem(12),
    "os_9": lambda: gen.oseen_problem(9),
    "os_20": lambda: gen.oseen_problem(20),
}


def row_scaled_error(rp, col, val, ref):
    err = 0.0
    n = rp.shape[0] - 1
    a = np.abs(val - ref)
    scale = np.abs(ref)
    rows = np.repeat(np.arange(n), np.diff(rp))
    rmax = np.zeros(n)
    np.maximum.at(rmax, rows, scale)
    emax = np.zeros(n)
    np.maximum.at(emax, rows, a)
    ok = rmax > 0
    err = (emax[ok] / rmax[ok]).max() if ok.any() else 0.0
    assert (emax[~ok] == 0).all()
    return err


def _gpu(mf, prob, bc=True):
    P = mf.Problem(prob)
    coeffs = P.make_coeffs(bc=bc)
    vals, d = P.assemble(coeffs=coeffs)
    rp, ci = P.csr_arrays()
    return P, rp.cpu().numpy(), ci.cpu().numpy(), vals.cpu().numpy(), d.cpu().numpy()


@pytest.mark.parametrize("case", list(CASES))
def test_pattern_and_values(mf, orc, case):
    prob = CASES[case]()
    P, rp, ci, val, d = _gpu(mf, prob)
    ref = orc.assemble(prob)
    assert np.array_equal(rp, ref["row_ptr"]) and np.array_equal(ci, ref["col"])
    assert row_scaled_error(rp, ci, val, ref["val"]) <= TOL
    assert np.abs(d - ref["d"]).max() <= TOL * np.abs(ref["d"]).max()


@pytest.mark.parametrize("case", ["p1_13", "q1_9", "q1_box_16", "el_7", "os_9"])
def test_values_without_dirichlet(mf, orc, case):
    prob = CASES[case]()
    P, rp, ci, val, d = _gpu(mf, prob, bc=False)
    ref = orc.assemble(prob, dirichlet=False)
    assert row_scaled_error(rp, ci, val, ref["val"]) <= TOL
    assert np.abs(d - ref["d"]).max() <= TOL * max(np.abs(ref["d"]).max(), 1e-300)


@pytest.mark.parametrize("case", ["p1_64", "el_12", "os_20"])
def test_assembly_bit_reproducible(mf, case):
    import torch
    P = mf.Problem(CASES[case]())
    v1, d1 = [t.clone() for t in P.assemble()]
    P.values.fill_(float("nan"))
    v2, d2 = P.assemble()
    assert torch.equal(v1, v2) and torch.equal(d1, d2)


@pytest.mark.parametrize("case", ["q1_6", "q1_box_8"])
def test_nonzero_dirichlet_values_lifted(mf, orc, case):
    prob = gen.thermal_q1_problem(6) if case == "q1_6" else _box_q1(8)
    rng = np.random.default_rng(7)
    prob["bc_val"] = np.where(prob["bc_mask"] > 0, rng.normal(size=prob["bc_mask"].shape), 0.0)
    P, rp, ci, val, d = _gpu(mf, prob)
    ref = orc.assemble(prob)
    assert row_scaled_error(rp, ci, val, ref["val"]) <= TOL
    assert np.abs(d - ref["d"]).max() <= TOL * np.abs(ref["d"]).max()


def test_pressure_mass_diag(mf, orc):
    prob = gen.oseen_problem(10)
    P = mf.Problem(prob)
    pm = P.pressure_mass_diag().cpu().numpy()
    ref = orc.assemble(prob)["pmass"]
    assert np.abs(pm - ref).max() <= TOL * np.abs(ref).max()


def test_elastic_full_size_sampled_rows(mf, orc):
    """64^3 Q1 elasticity (262,144 elements): closed-form nnz and sampled rows."""
    prob = gen.elastic_problem(64)
    P = mf.Problem(prob)
    assert P.nnz == 9 * (4 + 3 * 63) ** 3 == 64_701_513
    vals, d = P.assemble()
    rp, ci = P.csr_arrays()
    rp, ci = rp.cpu().numpy(), ci.cpu().numpy()
    vals, d = vals.cpu().numpy(), d.cpu().numpy()
    nn = prob["coords"].shape[0]
    rng = np.random.default_rng(11)
    nodes = np.unique(np.concatenate([rng.integers(0, nn, 40), [0, 1, 65, nn - 1, nn // 2, 65 * 65 + 66]]))
    keep = np.zeros(nn, np.uint8)
    keep[nodes] = 1
    ref = orc.assemble(prob, keep_nodes=keep)
    rows = [3 * n + c for n in nodes for c in range(3)]
    for r, (cols, v) in zip(rows, orc.rows_of(ref, rows)):
        s = slice(rp[r], rp[r + 1])
        assert np.array_equal(ci[s], cols)
        scale = np.abs(v).max()
        assert np.abs(vals[s] - v).max() <= TOL * scale
        assert abs(d[r] - ref["d"][r]) <= TOL * max(abs(ref["d"][r]), 1e-300) or abs(d[r] - ref["d"][r]) < 1e-20


def test_pcg_matches_oracle_solution(mf, orc):
    import torch
    prob = gen.thermal_p1_problem(64)
    P = mf.Problem(prob)
    P.assemble()
    x, st, info = P.solve(tol=1e-10)
    assert st == mf.MF_OK and info.converged and info.rel_residual <= 1e-10
    ref = orc.assemble(prob)
    xo, it, rr = orc.pcg(ref, tol=1e-13)
    xg = x.cpu().numpy()
    assert np.linalg.norm(xg - xo) <= 1e-7 * np.linalg.norm(xo)
    # same iteration count as the oracle's PCG at the same tolerance, up to rounding
    _, it_o, _ = orc.pcg(ref, tol=1e-10)
    assert abs(info.iterations - it_o) <= 2
    # warm start from the solution converges at once
    x2, st2, info2 = P.solve(x=x.clone(), tol=1e-10)
    assert info2.iterations <= 1


def test_pcg_elastic_small(mf, orc):
    prob = gen.elastic_problem(6)
    P = mf.Problem(prob)
    P.assemble()
    x, st, info = P.solve(tol=1e-11)
    assert st == mf.MF_OK and info.rel_residual <= 1e-11
    ref = orc.assemble(prob)
    xo, _, _ = orc.pcg(ref, tol=1e-14)
    assert np.linalg.norm(x.cpu().numpy() - xo) <= 1e-8 * np.linalg.norm(xo)


def test_gmres_flow_matches_oracle(mf, orc):
    prob = gen.oseen_problem(8)
    P = mf.Problem(prob)
    P.assemble()
    pd = P.flow_precond(1.0)
    ref = orc.assemble(prob)
    pref = orc.oseen_precond(ref, prob)
    pref[2 * prob["coords"].shape[0]:] *= prob["viscosity"]  # p_scale = 1: diag(M_p)
    pref[prob["bc_mask"] > 0] = 1.0
    assert np.abs(pd.cpu().numpy() - pref).max() <= TOL * np.abs(pref).max()
    x, st, info = P.solve(solver=mf.MF_SOLVER_GMRES, tol=1e-10, restart=50, precond=pd, max_iter=20000,
                          check_every=10)
    assert st == mf.MF_OK and info.rel_residual <= 1e-10
    xo = np.linalg.solve(_dense(ref), ref["d"])
    assert np.linalg.norm(x.cpu().numpy() - xo) <= 1e-7 * np.linalg.norm(xo)


def _dense(s):
    n = s["row_ptr"].shape[0] - 1
    A = np.zeros((n, n))
    rows = np.repeat(np.arange(n), np.diff(s["row_ptr"]))
    A[rows, s["col"]] = s["val"]
    return A


def test_spmv_matches_oracle(mf, orc):
    import torch
    prob = gen.elastic_problem(9)
    P = mf.Problem(prob)
    P.assemble()
    xh = np.random.default_rng(5).normal(size=P.n)
    x = torch.from_numpy(xh).cuda()
    y = torch.empty_like(x)
    mf.mf_spmv(P.csr, x, y)
    ref = orc.assemble(prob)
    yo = orc.spmv(ref, xh)
    assert np.abs(y.cpu().numpy() - yo).max() <= 1e-12 * np.abs(yo).max()


# ---------------------------------------------------------------------------
# error paths (host-side faults only: bad inputs, iteration caps)
# ---------------------------------------------------------------------------

def test_inverted_element_rejected(mf):
    prob = gen.thermal_p1_problem(4)
    prob["conn"][3] = prob["conn"][3][[0, 2, 1]]  # clockwise: detJ < 0
    with pytest.raises(mf.MFError) as ei:
        mf.Problem(prob)
    assert ei.value.status == mf.MF_ERR_BAD_MESH


def test_index_out_of_range_rejected(mf):
    prob = gen.elastic_problem(3)
    prob["conn"][5, 2] = prob["coords"].shape[0] + 7
    with pytest.raises(mf.MFError) as ei:
        mf.Problem(prob)
    assert ei.value.status == mf.MF_ERR_BAD_MESH


def test_nan_coefficient_latched(mf):
    import torch
    prob = gen.thermal_q1_problem(4)
    P = mf.Problem(prob)
    P.coef[7] = float("nan")
    P.assemble()
    with pytest.raises(mf.MFError) as ei:
        mf.mf_sync_status()
    assert ei.value.status == mf.MF_ERR_NONFINITE
    P.coef[7] = 1.0
    P.assemble()
    mf.mf_sync_status()  # the status word was cleared; the context is usable


def test_iteration_cap_reports_not_converged(mf):
    P = mf.Problem(gen.thermal_p1_problem(32))
    P.assemble()
    x, st, info = P.solve(tol=1e-12, max_iter=5, check_every=3)
    assert st == mf.MF_ERR_NOT_CONVERGED and info.iterations == 5 and not info.converged
    assert info.rel_residual > 1e-12


def test_invalid_arguments(mf):
    import ctypes as C
    P = mf.Problem(gen.thermal_p1_problem(4))
    bad = mf.CSR()
    with pytest.raises(mf.MFError) as ei:
        mf.mf_assemble(mf.MF_FORM_ELASTIC, P.mesh, P.pattern, P.coeffs, mf.MF_PREC_FP64, P.csr, P.d)
    assert ei.value.status == mf.MF_ERR_INVALID_ARG
    with pytest.raises(mf.MFError) as ei:
        mf.mf_assemble(mf.MF_FORM_THERMAL, P.mesh, P.pattern, P.coeffs, mf.MF_PREC_FP64, bad, P.d)
    assert ei.value.status == mf.MF_ERR_INVALID_ARG
    with pytest.raises(mf.MFError) as ei:
        mf.mf_pattern_build(P.mesh, mf.MF_FORM_ELASTIC)
    assert ei.value.status == mf.MF_ERR_UNSUPPORTED


# ---------------------------------------------------------------------------
# degenerate and maximum-size cases
# ---------------------------------------------------------------------------

def test_empty_mesh_rejected(mf):
    import torch
    X = torch.zeros((4, 2), dtype=torch.float64, device="cuda")
    C = torch.zeros((0, 3), dtype=torch.int32, device="cuda")
    desc = mf.MeshDesc(dim=2, elem=mf.MF_P1_TRI, n_nodes=4, n_elems=0, coords=X.data_ptr(), conn=C.data_ptr(),
                       n_pnodes=0, pconn=None)
    with pytest.raises(mf.MFError) as ei:
        mf.mf_mesh_create(desc)
    assert ei.value.status == mf.MF_ERR_INVALID_ARG


@pytest.mark.parametrize("kind", ["p1", "q1", "el"])
def test_single_cell_all_constrained(mf, orc, kind):
    prob = {"p1": lambda: gen.thermal_p1_problem(1), "q1": lambda: gen.thermal_q1_problem(1),
            "el": lambda: gen.elastic_problem(1)}[kind]()
    prob["bc_mask"][:] = 1
    prob["bc_val"] = np.linspace(-1.0, 1.0, prob["bc_mask"].shape[0])
    P, rp, ci, val, d = _gpu(mf, prob)
    ref = orc.assemble(prob)
    assert np.array_equal(val, ref["val"]) and np.array_equal(d, ref["d"])
    K = _dense({"row_ptr": rp, "col": ci, "val": val})
    assert np.array_equal(K, np.eye(K.shape[0])) and np.array_equal(d, prob["bc_val"])


def _sampled_rows(mf, orc, prob, rows_of_node, nodes, pnodes=None, tol=TOL):
    P = mf.Problem(prob)
    vals, d = P.assemble()
    rp, ci = P.csr_arrays()
    rp, ci, vals, d = rp.cpu().numpy(), ci.cpu().numpy(), vals.cpu().numpy(), d.cpu().numpy()
    keep = np.zeros(prob["coords"].shape[0], np.uint8)
    keep[nodes] = 1
    kp = None
    if pnodes is not None:
        kp = np.zeros(prob["vcoords"].shape[0], np.uint8)
        kp[pnodes] = 1
    ref = orc.assemble(prob, keep_nodes=keep, keep_pnodes=kp)
    for r, (cols, v) in zip(rows_of_node, orc.rows_of(ref, rows_of_node)):
        s = slice(rp[r], rp[r + 1])
        assert np.array_equal(ci[s], cols)
        assert np.abs(vals[s] - v).max() <= tol * max(np.abs(v).max(), 1e-300)
        assert abs(d[r] - ref["d"][r]) <= tol * max(np.abs(ref["d"]).max(), 1e-300)
    return P


def test_flow_full_size_sampled_rows(mf, orc):
    """512^2 Taylor-Hood (524,288 elements, 2,364,419 dofs): sampled u1, u2 and p rows."""
    prob = gen.oseen_problem(512)
    n2 = prob["coords"].shape[0]
    n1 = prob["vcoords"].shape[0]
    rng = np.random.default_rng(17)
    nodes = np.unique(np.concatenate([rng.integers(0, n2, 25), [0, 1, 1025, n2 - 1, n2 // 2]]))
    pnodes = np.unique(np.concatenate([rng.integers(0, n1, 25), [0, 1, n1 - 1]]))
    rows = [int(n) for n in nodes] + [int(n2 + n) for n in nodes] + [int(2 * n2 + p) for p in pnodes]
    # a pressure row needs the elements at its vertex: keep the P2 node of that vertex too
    vert = pnodes // 513 * 2 * 1025 + (pnodes % 513) * 2
    P = _sampled_rows(mf, orc, prob, rows, np.unique(np.concatenate([nodes, vert])), pnodes)
    assert P.n == 2 * n2 + n1 == 2_364_419


def test_grf_thermal_full_size_sampled_rows(mf, orc):
    """128^3 Q1 thermal with k = exp(GRF) (2,097,152 elements): sampled rows."""
    prob = gen.grf_thermal_problem(128)
    nn = prob["coords"].shape[0]
    rng = np.random.default_rng(19)
    nodes = np.unique(np.concatenate([rng.integers(0, nn, 40), [0, 130, nn - 1, nn // 2]]))
    P = _sampled_rows(mf, orc, prob, [int(n) for n in nodes], nodes)
    assert P.nnz == (4 + 3 * 127) ** 3
