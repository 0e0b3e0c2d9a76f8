"""The allocation-free Jacobi-PCG entry point (mf_solve_pcg_noalloc).

Some callers cannot allocate device memory while they solve: a framework that
reserved all device memory for its own pool at start-up (a cudaMalloc would
fail or fragment that pool), or a latency-critical loop where an allocation
would synchronise the device.  mf_solve_pcg_noalloc serves them from a static
device array.  Here it must reproduce mf_solve (the allocating entry point)
within the parity tolerance, on two calls in a row that reuse the array.
"""
import ctypes as C

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


def test_noalloc_pcg_matches_mf_solve_on_two_calls(mf):
    import torch
    problems = [gen.thermal_p1_problem(64), gen.elastic_problem(10)]
    for prob in problems:  # the second call reuses the array the first call left behind
        P = mf.Problem(prob)
        P.assemble()
        x_ref, st_ref, info_ref = P.solve(tol=1e-10, check_every=50)
        assert st_ref == mf.MF_OK
        x = torch.zeros(P.n, dtype=torch.float64, device=P.device)
        st, info = mf.mf_solve_pcg_noalloc(P.csr, P.d, x, 1e-10, 100000, 50)
        torch.cuda.synchronize()
        assert st == mf.MF_OK and info.converged
        assert info.iterations == info_ref.iterations
        assert info.rel_residual <= 1e-10
        xr = x_ref.cpu().numpy()
        xn = x.cpu().numpy()
        assert np.abs(xn - xr).max() <= 1e-12 * np.abs(xr).max()
        P.close()


def test_noalloc_solve_allocates_no_device_memory(mf):
    """After a first call (the one-time symbol lookup), a solve leaves the
    device's free memory and torch's allocator statistics unchanged."""
    import torch
    P = mf.Problem(gen.thermal_p1_problem(48))
    P.assemble()
    x = torch.zeros(P.n, dtype=torch.float64, device=P.device)
    mf.mf_solve_pcg_noalloc(P.csr, P.d, x, 1e-10, 100000, 50)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    alloc0 = torch.cuda.memory_stats().get("allocation.all.allocated", 0)
    x.zero_()
    st, info = mf.mf_solve_pcg_noalloc(P.csr, P.d, x, 1e-10, 100000, 50)
    torch.cuda.synchronize()
    assert st == mf.MF_OK and info.converged
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.cuda.memory_stats().get("allocation.all.allocated", 0) == alloc0
    assert mf.mf_last_error() == ""
    P.close()


def test_noalloc_rejects_an_empty_system(mf):
    import torch
    P = mf.Problem(gen.thermal_p1_problem(4))
    empty = mf.CSR(n_rows=P.csr.n_rows, nnz=0, row_ptr=P.csr.row_ptr, col_idx=P.csr.col_idx,
                   values=P.csr.values)
    x = torch.zeros(P.n, dtype=torch.float64, device=P.device)
    with pytest.raises(mf.MFError) as ei:
        mf.mf_solve_pcg_noalloc(empty, P.d, x, 1e-10, 10)
    assert ei.value.status == mf.MF_ERR_INVALID_ARG


def test_noalloc_rejects_systems_above_the_limit(mf):
    import torch
    P = mf.Problem(gen.thermal_p1_problem(4))
    big = mf.CSR(n_rows=mf.MF_NOALLOC_MAX_ROWS + 1, nnz=P.csr.nnz, row_ptr=P.csr.row_ptr,
                 col_idx=P.csr.col_idx, values=P.csr.values)
    x = torch.zeros(P.n, dtype=torch.float64, device=P.device)
    with pytest.raises(mf.MFError) as ei:
        mf.mf_solve_pcg_noalloc(big, P.d, x, 1e-10, 10)
    assert ei.value.status == mf.MF_ERR_INVALID_ARG
    assert "MF_NOALLOC_MAX_ROWS" in mf.mf_last_error()
