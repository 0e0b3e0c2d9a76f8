"""Margins of the double-float element kernels (20-node bricks, thermal and
elastic; 10-node tetrahedra; 8-node quadrilaterals) on strongly distorted
meshes with a high coefficient contrast, and on larger meshes compared in
full: the FP32-pair arithmetic (about 47 bits) must keep every CSR row within
the FP64 bound of 1e-12 row-scaled of the FP64 oracle, also where the
element maps are far from affine (jitter up to 0.4 h) and the lognormal
coefficients spread over several orders of magnitude (sigma 2)."""
import numpy as np
import pytest

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


CASES = {
    "q2s_thermal_jitter40_contrast": lambda: gen.thermal_q2s_problem(4, jitter=0.4, sigma=2.0),
    "q2s_thermal_12cube": lambda: gen.thermal_q2s_problem(12, jitter=0.3, sigma=2.0),
    "q2s_elastic_jitter30_contrast": lambda: gen.elastic_q2s_problem(4, jitter=0.3, sigma=2.0),
    "q2s_elastic_nu049_jitter30": lambda: gen.elastic_q2s_problem(3, jitter=0.3, sigma=2.0, nu=0.49),
    "p2t_jitter25_contrast": lambda: gen.thermal_p2t_problem(4, jitter=0.25, sigma=2.0),
    "p2t_12cube": lambda: gen.thermal_p2t_problem(12, jitter=0.2, sigma=2.0),
    "q2q_jitter30_contrast": lambda: gen.thermal_q2q_problem(16, jitter=0.3, sigma=2.0),
}


@pytest.mark.parametrize("case", list(CASES))
def test_double_float_kernels_within_fp64_bound(mf, orc, case):
    prob = CASES[case]()
    P = mf.Problem(prob)
    vals, d = P.assemble()
    mf.mf_sync_status()
    rp, ci = P.csr_arrays()
    rp = rp.cpu().numpy()
    ref = orc.assemble(prob)
    assert np.array_equal(rp, ref["row_ptr"]) and np.array_equal(ci.cpu().numpy(), ref["col"])
    err = row_scaled_error(rp, vals.cpu().numpy(), ref["val"])
    derr = np.abs(d.cpu().numpy() - ref["d"]).max() / np.abs(ref["d"]).max()
    print(f"{case}: K row-scaled {err:.2e}, d {derr:.2e}")
    assert err <= 1e-12, err
    assert derr <= 1e-12, derr
