"""Parity of the transient pieces with the CPU FP64 oracle, through the C ABI:
the capacity matrix C int N_a N_b (MF_FORM_CAPACITY), generalised-alpha time
stepping (mf_genalpha_run, mf_genalpha_initial_rate) and the nonlinear
radiation term e_m sigma^b (T, T_env^4 - T^4) in its Newton sub-steps.

Capacity: pattern bit-exact, values row-scaled within 1e-12.  Time stepping:
both sides solve every Newton step by Jacobi-PCG to a relative residual of
1e-13, so the states agree to the solves' accuracy: within 1e-10 of the
state's maximum after the steps run here.
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
    prob = gen.thermal_q1_problem(n, jitter=0.0)
    X = prob["coords"].copy()
    h = 1.0 / n
    inner = (X[:, 0] > 1e-12) & (X[:, 0] < 0.4) & (np.abs(X[:, 1] - 0.5) < 0.5 - 1e-12) & \
        (np.abs(X[:, 2] - 0.5) < 0.5 - 1e-12)
    idx = np.nonzero(inner)[0]
    X[idx] += 0.15 * h * (2.0 * gen.uniform(4321, 3 * idx.size).reshape(-1, 3) - 1.0)
    prob["coords"] = X
    return prob


CAP = {
    "p1_20": lambda: gen.thermal_p1_problem(20),
    "p2_9": lambda: gen.thermal_p2_problem(9),
    "q1_8": lambda: gen.thermal_q1_problem(8),
    "q1_affine_11": lambda: gen.thermal_q1_problem(11, jitter=0.0),
    "q1_partly_translate_10": lambda: _partly_jittered_q1(10),
    "q1_box_16": lambda: gen.thermal_q1_problem(16, jitter=0.0),  # exact translates of a cube: box rows
}


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


def _capacity_gpu(mf, P, C, bc=False):
    import torch
    vals = torch.empty(P.nnz, dtype=torch.float64, device="cuda")
    d = torch.empty(P.n, dtype=torch.float64, device="cuda")
    csr = mf.CSR(P.csr.n_rows, P.csr.nnz, P.csr.row_ptr, P.csr.col_idx, vals.data_ptr())
    Ct = torch.from_numpy(np.ascontiguousarray(C)).cuda()
    coeffs = P.make_coeffs(coef=Ct, bc=bc)
    mf.mf_assemble(mf.MF_FORM_CAPACITY, P.mesh, P.pattern, coeffs, mf.MF_PREC_FP64, csr, d)
    return vals, d, csr


@pytest.mark.parametrize("case", list(CAP))
def test_capacity_parity(mf, orc, case):
    prob = CAP[case]()
    C = gen.lognormal(77, prob["conn"].shape[0], 0.3)
    P = mf.Problem(prob)
    vals, d, _ = _capacity_gpu(mf, P, C)
    rp, ci = P.csr_arrays()
    rp, ci = rp.cpu().numpy(), ci.cpu().numpy()
    ref = orc.capacity(prob, C)
    assert np.array_equal(rp, ref["row_ptr"]) and np.array_equal(ci, ref["col"])
    assert row_scaled_error(rp, vals.cpu().numpy(), ref["val"]) <= TOL
    assert np.abs(d.cpu().numpy()).max() == 0.0


@pytest.mark.parametrize("n,jitter", [(6, 0.15), (8, 0.0)])
def test_capacity_with_dirichlet(mf, orc, n, jitter):
    prob = gen.thermal_q1_problem(n, jitter=jitter)
    prob["bc_val"] = np.where(prob["bc_mask"] > 0, gen.normal(9, prob["bc_mask"].shape[0]), 0.0)
    C = gen.lognormal(78, prob["conn"].shape[0], 0.3)
    P = mf.Problem(prob)
    vals, d, _ = _capacity_gpu(mf, P, C, bc=True)
    ref = orc.capacity(prob, C)
    ref["d"] = np.zeros(prob["coords"].shape[0])
    orc.apply_dirichlet(ref, prob["bc_mask"], prob["bc_val"])
    rp, _ = P.csr_arrays()
    assert row_scaled_error(rp.cpu().numpy(), vals.cpu().numpy(), ref["val"]) <= TOL
    assert np.abs(d.cpu().numpy() - ref["d"]).max() <= TOL * np.abs(ref["d"]).max()


def test_capacity_rejected_in_mixed_precision(mf):
    import torch
    P = mf.Problem(gen.thermal_p1_problem(4))
    C = torch.ones(P.conn.shape[0], dtype=torch.float64, device="cuda")
    with pytest.raises(mf.MFError) as ei:
        mf.mf_assemble(mf.MF_FORM_CAPACITY, P.mesh, P.pattern, P.make_coeffs(coef=C), mf.MF_PREC_MIXED, P.csr, P.d)
    assert ei.value.status == mf.MF_ERR_UNSUPPORTED


# ---------------------------------------------------------------------------
# generalised-alpha
# ---------------------------------------------------------------------------

def _transient_setup(mf, orc, prob, C):
    """GPU K (domain + boundary terms, no elimination), M, F and the oracle's."""
    import torch
    P = mf.Problem(prob)
    coeffs = P.make_coeffs(bc=False)
    mf.mf_assemble(P.form, P.mesh, P.pattern, coeffs, mf.MF_PREC_FP64, P.csr, P.d)
    if P.facets:
        fc = mf.FacetCoeffs(h=P.facet_coeffs.h, t_env=P.facet_coeffs.t_env)
        mf.mf_assemble_boundary(P.facets, fc, P.csr, P.d)
    Mv, _, _ = _capacity_gpu(mf, P, C)
    K = orc.assemble(prob, dirichlet=False)
    M = orc.capacity(prob, C)
    return P, Mv, K, M


def _run_both(mf, orc, prob, C, rho, dt, steps, phi0):
    import torch
    P, Mv, K, M = _transient_setup(mf, orc, prob, C)
    F = K["d"]
    mask, bval = prob["bc_mask"], prob["bc_val"]
    # oracle
    u0o = orc.initial_rate(K, M, F, mask, np.where(mask > 0, bval, phi0))
    po, uo, ao, itso = orc.genalpha(K, M, F, mask, bval, phi0, u0o, np.zeros_like(F), orc.genalpha_params(rho), dt,
                                    steps)
    # GPU
    phi = torch.from_numpy(np.where(mask > 0, bval, phi0)).cuda()
    u = torch.empty_like(phi)
    a = torch.zeros_like(phi)
    mf.mf_genalpha_initial_rate(P.csr, Mv, P.d, P.bc_mask, phi, u)
    assert np.abs(u.cpu().numpy() - u0o).max() <= 1e-10 * max(np.abs(u0o).max(), 1e-300)
    prm = mf.mf_genalpha_params_from_rho(rho)
    st, nits, pits = mf.mf_genalpha_run(P.csr, Mv, P.d, P.bc_mask, P.bc_val, phi, u, a, prm, dt, steps,
                                        pcg_tol=1e-13)
    return P, Mv, (phi.cpu().numpy(), u.cpu().numpy(), nits, pits), (po, uo, itso)


@pytest.mark.parametrize("kind,rho", [("p1", 0.5), ("p2", 0.0), ("q1", 0.8)])
def test_genalpha_parity(mf, orc, kind, rho):
    prob = {"p1": lambda: gen.thermal_p1_problem(16), "p2": lambda: gen.thermal_p2_problem(7),
            "q1": lambda: gen.thermal_q1_problem(6)}[kind]()
    left = prob["coords"][:, 0] <= 1e-14
    prob["bc_mask"] = left.astype(np.uint8)
    prob["bc_val"] = np.where(left, 0.3, 0.0)
    sides = ("x1", "y0", "y1") if kind != "q1" else ("x1", "y0", "z1")
    prob["facets"] = gen.convection_facets(prob, sides)
    C = gen.lognormal(79, prob["conn"].shape[0], 0.3)
    x = prob["coords"]
    phi0 = np.sin(np.pi * x[:, 0]) * np.cos(0.5 * np.pi * x[:, 1])
    P, Mv, (pg, ug, nits, pits), (po, uo, itso) = _run_both(mf, orc, prob, C, rho, 2e-3, 6, phi0)
    assert np.array_equal(nits, itso) and (nits == 1).all()
    assert np.abs(pg - po).max() <= 1e-10 * np.abs(po).max()
    assert np.abs(ug - uo).max() <= 1e-9 * np.abs(uo).max()


def test_genalpha_bit_reproducible(mf, orc):
    import torch
    prob = gen.thermal_q1_problem(6)
    C = np.ones(prob["conn"].shape[0])
    P, Mv, K, M = _transient_setup(mf, orc, prob, C)
    prm = mf.mf_genalpha_params_from_rho(0.5)
    out = []
    for _ in range(2):
        phi = torch.zeros(P.n, dtype=torch.float64, device="cuda")
        u = torch.zeros_like(phi)
        a = torch.zeros_like(phi)
        mf.mf_genalpha_run(P.csr, Mv, P.d, P.bc_mask, P.bc_val, phi, u, a, prm, 1e-2, 4)
        out.append((phi.clone(), u.clone()))
    assert torch.equal(out[0][0], out[1][0]) and torch.equal(out[0][1], out[1][1])


@pytest.mark.parametrize("rho", [0.0, 0.5, 1.0])
def test_genalpha_high_frequency_double_root(mf, rho):
    # one dof, stiffness 1e8, unit capacity: phi_{n+2} - 2 lam phi_{n+1} + lam^2 phi_n = 0, lam = -rho_inf
    import torch
    rp = torch.tensor([0, 1], dtype=torch.int64, device="cuda")
    ci = torch.tensor([0], dtype=torch.int32, device="cuda")
    kv = torch.tensor([1e8], dtype=torch.float64, device="cuda")
    mv = torch.tensor([1.0], dtype=torch.float64, device="cuda")
    F = torch.zeros(1, dtype=torch.float64, device="cuda")
    K = mf.CSR(1, 1, rp.data_ptr(), ci.data_ptr(), kv.data_ptr())
    phi = torch.ones(1, dtype=torch.float64, device="cuda")
    u = torch.full((1,), -1e8, dtype=torch.float64, device="cuda")
    a = torch.zeros(1, dtype=torch.float64, device="cuda")
    prm = mf.mf_genalpha_params_from_rho(rho)
    seq = []
    for _ in range(8):
        mf.mf_genalpha_run(K, mv, F, None, None, phi, u, a, prm, 1.0, 1, pcg_tol=1e-14)
        seq.append(phi.item())
    s = np.array(seq)
    lam = -rho
    assert np.abs(s[2:] - 2 * lam * s[1:-1] + lam ** 2 * s[:-2]).max() <= 1e-6 * np.abs(s).max()


def test_genalpha_steady_state(mf, orc):
    import torch
    prob = gen.thermal_p1_problem(12)
    C = np.ones(prob["conn"].shape[0])
    P, Mv, K, M = _transient_setup(mf, orc, prob, C)
    phi = torch.zeros(P.n, dtype=torch.float64, device="cuda")
    u = torch.empty_like(phi)
    a = torch.zeros_like(phi)
    mf.mf_genalpha_initial_rate(P.csr, Mv, P.d, P.bc_mask, phi, u)
    prm = mf.mf_genalpha_params_from_rho(0.0)
    mf.mf_genalpha_run(P.csr, Mv, P.d, P.bc_mask, P.bc_val, phi, u, a, prm, 10.0, 12, pcg_tol=1e-13)
    ref = orc.assemble(prob)
    xs, _, _ = orc.pcg(ref, tol=1e-14)
    assert np.abs(phi.cpu().numpy() - xs).max() <= 1e-10 * np.abs(xs).max()


def test_genalpha_invalid_arguments(mf):
    import torch
    P = mf.Problem(gen.thermal_p1_problem(4))
    P.assemble()
    x = torch.zeros(P.n, dtype=torch.float64, device="cuda")
    prm = mf.mf_genalpha_params_from_rho(0.5)
    with pytest.raises(mf.MFError) as ei:
        mf.mf_genalpha_run(P.csr, P.values, P.d, None, None, x, x, x, prm, 0.0, 1)
    assert ei.value.status == mf.MF_ERR_INVALID_ARG
    with pytest.raises(mf.MFError) as ei:
        mf.mf_genalpha_params_from_rho(1.5)
    assert ei.value.status == mf.MF_ERR_INVALID_ARG
    with pytest.raises(mf.MFError) as ei:
        mf.mf_genalpha_run(P.csr, P.values, P.d, P.bc_mask, None, x, x, x, prm, 0.1, 1)
    assert ei.value.status == mf.MF_ERR_INVALID_ARG


# ---------------------------------------------------------------------------
# radiation inside the Newton sub-steps
# ---------------------------------------------------------------------------

def _oracle_radiation_load(orc, prob, rad, T):
    elem = {"P1": orc.P1, "P2": orc.P2, "Q1": orc.Q1}[prob["elem"]]
    R = np.zeros(prob["coords"].shape[0])
    for e, f, es, te in zip(rad["elem"], rad["face"], rad["es"], rad["t_env"]):
        nodes = prob["conn"][e][orc.facet_nodes(elem, int(f))]
        _, rf = orc.facet_radiation(elem, prob["coords"][nodes], es, te, T[nodes])
        R[nodes] += rf
    return R


def _radiation_case(kind):
    prob = {"p1": lambda: gen.thermal_p1_problem(10), "p2": lambda: gen.thermal_p2_problem(6),
            "q1": lambda: gen.thermal_q1_problem(5)}[kind]()
    prob["source"] = 0.0
    x = prob["coords"]
    left = x[:, 0] <= 1e-14
    prob["bc_mask"] = left.astype(np.uint8)
    prob["bc_val"] = np.where(left, 1.0, 0.0)
    sides = ("x1", "y1") if kind != "q1" else ("x1", "y1", "z1")
    rad = gen.radiation_facets(prob, sides)
    return prob, rad


def _gpu_radiation(mf, P, rad):
    import torch
    e = torch.from_numpy(rad["elem"]).cuda()
    f = torch.from_numpy(rad["face"]).cuda()
    F = mf.mf_facets_create(P.mesh, P.pattern, e, f)
    es = torch.from_numpy(rad["es"]).cuda()
    te = torch.from_numpy(rad["t_env"]).cuda()
    return F, es, te, (e, f)


@pytest.mark.parametrize("kind", ["p1", "p2", "q1"])
def test_genalpha_radiation_parity(mf, orc, kind):
    import torch
    prob, rad = _radiation_case(kind)
    C = gen.lognormal(80, prob["conn"].shape[0], 0.3)
    P, Mv, K, M = _transient_setup(mf, orc, prob, C)
    mask, bval = prob["bc_mask"], prob["bc_val"]
    # an undamped Newton on T^4 needs a predictor close enough: start at the
    # Dirichlet value and take steps of 0.01
    phi0 = np.full(prob["coords"].shape[0], 1.0)
    prm = orc.genalpha_params(0.5)
    Fo = K["d"] + _oracle_radiation_load(orc, prob, rad, phi0)
    u0o = orc.initial_rate(K, M, Fo, mask, phi0)
    po, uo, ao, itso = orc.genalpha(K, M, K["d"], mask, bval, phi0, u0o, np.zeros_like(phi0), prm, 0.01, 4,
                                    newton_tol=1e-10, max_newton=30, prob=prob, radiation=rad)
    Fh, es, te, keep = _gpu_radiation(mf, P, rad)
    phi = torch.from_numpy(phi0.copy()).cuda()
    u = torch.empty_like(phi)
    a = torch.zeros_like(phi)
    mf.mf_genalpha_initial_rate(P.csr, Mv, P.d, P.bc_mask, phi, u, rad=Fh, rad_es=es, rad_tenv=te)
    assert np.abs(u.cpu().numpy() - u0o).max() <= 1e-10 * np.abs(u0o).max()
    st, nits, pits = mf.mf_genalpha_run(P.csr, Mv, P.d, P.bc_mask, P.bc_val, phi, u, a,
                                        mf.mf_genalpha_params_from_rho(0.5), 0.01, 4, newton_tol=1e-10, max_newton=30,
                                        pcg_tol=1e-13, rad=Fh, rad_es=es, rad_tenv=te)
    mf.mf_facets_destroy(Fh)
    assert np.array_equal(nits, itso) and nits.max() > 1  # nonlinear: several solves per step
    assert np.abs(phi.cpu().numpy() - po).max() <= 1e-10 * np.abs(po).max()
    assert np.abs(u.cpu().numpy() - uo).max() <= 1e-8 * np.abs(uo).max()


@pytest.mark.parametrize("kind", ["p1", "q1"])
def test_radiation_slab_steady_state_gpu(mf, orc, kind):
    # T = T0 + b x, k b = es (T_env^4 - (T0 + b)^4)
    import scipy.optimize
    import torch
    prob = gen.thermal_p1_problem(8) if kind == "p1" else gen.thermal_q1_problem(4)
    k, es, T0, Te = 1.7, 0.8, 0.4, 1.5
    prob["coef"] = np.full(prob["conn"].shape[0], k)
    prob["source"] = 0.0
    x = prob["coords"]
    left = x[:, 0] <= 1e-14
    prob["bc_mask"] = left.astype(np.uint8)
    prob["bc_val"] = np.where(left, T0, 0.0)
    rad = gen.radiation_facets(prob, ("x1",), es=es, t_env=Te)
    P, Mv, K, M = _transient_setup(mf, orc, prob, np.ones(prob["conn"].shape[0]))
    Fh, es_t, te_t, keep = _gpu_radiation(mf, P, rad)
    phi = torch.full((P.n,), T0, dtype=torch.float64, device="cuda")
    u = torch.zeros_like(phi)
    a = torch.zeros_like(phi)
    mf.mf_genalpha_run(P.csr, Mv, P.d, P.bc_mask, P.bc_val, phi, u, a, mf.mf_genalpha_params_from_rho(0.0), 50.0, 8,
                       max_newton=30, pcg_tol=1e-13, rad=Fh, rad_es=es_t, rad_tenv=te_t)
    mf.mf_facets_destroy(Fh)
    b = scipy.optimize.brentq(lambda b: k * b - es * (Te ** 4 - (T0 + b) ** 4), -T0, 5.0, xtol=1e-15)
    assert np.abs(phi.cpu().numpy() - (T0 + b * x[:, 0])).max() < 1e-10


# ---------------------------------------------------------------------------
# degenerate cases
# ---------------------------------------------------------------------------

def test_genalpha_zero_steps_keeps_the_state(mf, orc):
    import torch
    prob = gen.thermal_p1_problem(6)
    P, Mv, K, M = _transient_setup(mf, orc, prob, np.ones(prob["conn"].shape[0]))
    phi = torch.linspace(0.0, 1.0, P.n, dtype=torch.float64, device="cuda")
    u = torch.full_like(phi, 0.25)
    a = torch.full_like(phi, -0.5)
    mask = P.bc_mask.bool()
    p0, u0, a0 = phi.clone(), u.clone(), a.clone()
    st, nits, pits = mf.mf_genalpha_run(P.csr, Mv, P.d, P.bc_mask, P.bc_val, phi, u, a,
                                        mf.mf_genalpha_params_from_rho(0.5), 0.1, 0)
    # only the Dirichlet dofs are set (value bc_val, zero rates)
    assert torch.equal(phi[~mask], p0[~mask]) and torch.equal(u[~mask], u0[~mask]) and torch.equal(a[~mask], a0[~mask])
    assert torch.equal(phi[mask], P.bc_val[mask]) and (u[mask] == 0).all() and (a[mask] == 0).all()


def test_genalpha_without_dirichlet_conserves_heat(mf, orc):
    # pure Neumann, F = 0: the total heat 1^T M phi is constant in time
    import torch
    prob = gen.thermal_q1_problem(5)
    prob["source"] = 0.0
    P, Mv, K, M = _transient_setup(mf, orc, prob, gen.lognormal(81, prob["conn"].shape[0], 0.3))
    x = torch.from_numpy(prob["coords"][:, 0].copy()).cuda()
    phi = torch.cos(np.pi * x)
    u = torch.empty_like(phi)
    a = torch.zeros_like(phi)
    mf.mf_genalpha_initial_rate(P.csr, Mv, P.d, None, phi, u)
    Md = _csr_t(P, Mv)
    h0 = float((Md @ phi.cpu().numpy()).sum())
    mf.mf_genalpha_run(P.csr, Mv, P.d, None, None, phi, u, a, mf.mf_genalpha_params_from_rho(0.5), 0.05, 5,
                       pcg_tol=1e-13)
    h1 = float((Md @ phi.cpu().numpy()).sum())
    assert abs(h1 - h0) <= 1e-10 * np.abs(Md @ phi.cpu().numpy()).sum()


def _csr_t(P, vals):
    import scipy.sparse as sp
    rp, ci = P.csr_arrays()
    return sp.csr_matrix((vals.cpu().numpy(), ci.cpu().numpy(), rp.cpu().numpy()), shape=(P.n, P.n))


def test_radiation_with_no_facets_is_linear(mf, orc):
    # an empty radiation set changes nothing: bit-identical to the run without it
    import torch
    prob = gen.thermal_p1_problem(8)
    P, Mv, K, M = _transient_setup(mf, orc, prob, np.ones(prob["conn"].shape[0]))
    e = torch.zeros(0, dtype=torch.int32, device="cuda")
    f = torch.zeros(0, dtype=torch.uint8, device="cuda")
    R = mf.mf_facets_create(P.mesh, P.pattern, e, f)
    es = torch.zeros(0, dtype=torch.float64, device="cuda")
    out = []
    for rk in ({}, {"rad": R, "rad_es": es, "rad_tenv": es}):
        phi = torch.zeros(P.n, dtype=torch.float64, device="cuda")
        u = torch.zeros_like(phi)
        a = torch.zeros_like(phi)
        mf.mf_genalpha_run(P.csr, Mv, P.d, P.bc_mask, P.bc_val, phi, u, a, mf.mf_genalpha_params_from_rho(0.5), 0.01,
                           3, **rk)
        out.append(phi.clone())
    mf.mf_facets_destroy(R)
    assert torch.equal(out[0], out[1])


def test_radiation_facets_on_another_pattern_rejected(mf, orc):
    import torch
    p1 = gen.thermal_p1_problem(4)
    P, Mv, K, M = _transient_setup(mf, orc, p1, np.ones(p1["conn"].shape[0]))
    Q = mf.Problem(gen.thermal_p1_problem(4))
    rad = gen.radiation_facets(p1, ("x1",))
    Fh, es, te, keep = _gpu_radiation(mf, Q, rad)
    x = torch.zeros(P.n, dtype=torch.float64, device="cuda")
    with pytest.raises(mf.MFError) as ei:
        mf.mf_genalpha_run(P.csr, Mv, P.d, None, None, x, x.clone(), x.clone(), mf.mf_genalpha_params_from_rho(0.5),
                           0.01, 1, rad=Fh, rad_es=es, rad_tenv=te)
    assert ei.value.status == mf.MF_ERR_INVALID_ARG
    mf.mf_facets_destroy(Fh)
