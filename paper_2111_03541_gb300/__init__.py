"""Python binding of libmf (GB300 FEM assembly + Krylov hot path of MetaFEM, arXiv 2111.03541).

Argument marshalling only: every step of assembly and solve runs in the CUDA
kernels of ``libmf.so`` (built in-tree by ``paper_2111_03541_gb300.build``).
PyTorch provides device memory and streams.  There is no CPU fallback: if the
library is missing, importing the binding's entry points raises.

The ``mf_*`` functions mirror the C ABI of ``include/mf.h`` one to one.  The
``Problem`` class is a convenience that moves a problem made by ``gen`` to
the GPU and keeps its handles.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB = os.path.join(HERE, "libmf.so")

MF_OK, MF_ERR_INVALID_ARG, MF_ERR_BAD_MESH, MF_ERR_NONFINITE, MF_ERR_OOM, MF_ERR_CUDA, \
    MF_ERR_NOT_CONVERGED, MF_ERR_TIMEOUT, MF_ERR_UNSUPPORTED = range(9)
MF_P1_TRI, MF_P2_TRI, MF_Q1_HEX, MF_Q2S_HEX, MF_P2_TET, MF_Q2S_QUAD = 0, 1, 2, 3, 4, 5
MF_FORM_THERMAL, MF_FORM_ELASTIC, MF_FORM_OSEEN, MF_FORM_CAPACITY, MF_FORM_NS = 0, 1, 2, 3, 4
MF_PREC_FP64, MF_PREC_MIXED = 0, 1
MF_SOLVER_PCG, MF_SOLVER_GMRES, MF_SOLVER_PCG_REFINED, MF_SOLVER_GMRES_FLOW_MG = 0, 1, 2, 3

ELEM = {"P1": MF_P1_TRI, "P2": MF_P2_TRI, "Q1": MF_Q1_HEX, "Q2S": MF_Q2S_HEX, "P2T": MF_P2_TET, "Q2Q": MF_Q2S_QUAD}
FORM = {"thermal": MF_FORM_THERMAL, "elastic": MF_FORM_ELASTIC, "oseen": MF_FORM_OSEEN, "ns": MF_FORM_NS}


class MFError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"mf status {status}: {msg}")
        self.status = status


class MeshDesc(C.Structure):
    _fields_ = [("dim", C.c_int32), ("elem", C.c_int32), ("n_nodes", C.c_int64), ("n_elems", C.c_int64),
                ("coords", C.c_void_p), ("conn", C.c_void_p), ("n_pnodes", C.c_int64), ("pconn", C.c_void_p)]


class Coeffs(C.Structure):
    _fields_ = [("elem_coef", C.c_void_p), ("nu", C.c_double), ("visc", C.c_double), ("rho", C.c_double),
                ("source", C.c_double * 3), ("advect", C.c_void_p), ("bc_mask", C.c_void_p),
                ("bc_val", C.c_void_p), ("tau_m", C.c_double), ("tau_c", C.c_double)]


class CSR(C.Structure):
    _fields_ = [("n_rows", C.c_int64), ("nnz", C.c_int64), ("row_ptr", C.c_void_p), ("col_idx", C.c_void_p),
                ("values", C.c_void_p)]


class SolverOpts(C.Structure):
    _fields_ = [("solver", C.c_int32), ("restart", C.c_int32), ("tol", C.c_double), ("max_iter", C.c_int64),
                ("precond_diag", C.c_void_p), ("check_every", C.c_int32), ("inner_tol", C.c_double),
                ("flow_mg", C.c_void_p)]


class BatchTiling(C.Structure):
    _fields_ = [("elem_tile", C.c_int32), ("elem_block", C.c_int32), ("node_tile", C.c_int32),
                ("grid_per_sm", C.c_int32)]


class FacetCoeffs(C.Structure):
    _fields_ = [("h", C.c_void_p), ("t_env", C.c_void_p), ("stress", C.c_void_p),
                ("bc_mask", C.c_void_p), ("bc_val", C.c_void_p)]


class GenAlphaParams(C.Structure):
    _fields_ = [("b1", C.c_double), ("b2", C.c_double), ("c1", C.c_double), ("c2", C.c_double),
                ("c3", C.c_double)]


class SolveInfo(C.Structure):
    _fields_ = [("iterations", C.c_int64), ("rel_residual", C.c_double), ("converged", C.c_int32),
                ("refinements", C.c_int64)]


_lib = None

# name -> argtypes (all return mf_status as int, except mf_last_error)
_SIGS = {
    "mf_mesh_create": [C.POINTER(MeshDesc), C.c_void_p, C.POINTER(C.c_void_p)],
    "mf_mesh_destroy": [C.c_void_p],
    "mf_pattern_build": [C.c_void_p, C.c_int32, C.c_void_p, C.POINTER(C.c_void_p)],
    "mf_pattern_csr": [C.c_void_p, C.POINTER(CSR)],
    "mf_pattern_copy_csr": [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p],
    "mf_pattern_destroy": [C.c_void_p],
    "mf_assemble": [C.c_int32, C.c_void_p, C.c_void_p, C.POINTER(Coeffs), C.c_int32, C.POINTER(CSR), C.c_void_p,
                    C.c_void_p],
    "mf_ns_newton": [C.c_void_p, C.c_void_p, C.POINTER(Coeffs), C.c_void_p, C.c_double, C.c_int32,
                     C.POINTER(SolverOpts), C.c_void_p, C.POINTER(C.c_int32), C.c_void_p],
    "mf_facets_create": [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p,
                         C.POINTER(C.c_void_p)],
    "mf_facets_destroy": [C.c_void_p],
    "mf_assemble_boundary": [C.c_void_p, C.POINTER(FacetCoeffs), C.POINTER(CSR), C.c_void_p, C.c_void_p],
    "mf_genalpha_params_from_rho": [C.c_double, C.POINTER(GenAlphaParams)],
    "mf_genalpha_run": [C.POINTER(CSR), C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                        C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(GenAlphaParams), C.c_double,
                        C.c_int64, C.c_double, C.c_int32, C.c_double, C.c_int64, C.c_void_p, C.c_void_p,
                        C.c_void_p],
    "mf_genalpha_initial_rate": [C.POINTER(CSR), C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                 C.c_void_p, C.c_void_p, C.c_void_p, C.c_double, C.c_int64, C.c_void_p],
    "mf_pressure_mass_diag": [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p],
    "mf_flow_mg_create": [C.c_int32, C.POINTER(C.POINTER(CSR)), C.c_void_p, C.POINTER(C.c_void_p), C.c_void_p,
                          C.c_double, C.c_void_p, C.POINTER(C.c_void_p)],
    "mf_flow_mg_destroy": [C.c_void_p],
    "mf_flow_precond": [C.c_void_p, C.c_void_p, C.POINTER(CSR), C.c_void_p, C.c_double, C.c_void_p, C.c_void_p],
    "mf_solve": [C.POINTER(CSR), C.c_void_p, C.c_void_p, C.POINTER(SolverOpts), C.POINTER(SolveInfo), C.c_void_p],
    "mf_solve_pcg_noalloc": [C.POINTER(CSR), C.c_void_p, C.c_void_p, C.c_double, C.c_int64, C.c_int32,
                             C.POINTER(SolveInfo), C.c_void_p],
    "mf_spmv": [C.POINTER(CSR), C.c_void_p, C.c_void_p, C.c_void_p],
    "mf_sync_status": [C.c_void_p],
    "mf_batch_create": [C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                        C.POINTER(C.c_void_p)],
    "mf_batch_set_tiling": [C.c_void_p, C.POINTER(BatchTiling)],
    "mf_batch_get_tiling": [C.c_void_p, C.POINTER(BatchTiling)],
    "mf_batch_autotune": [C.c_void_p, C.c_char_p, C.c_void_p, C.POINTER(BatchTiling)],
    "mf_batch_assemble": [C.c_void_p, C.c_void_p],
    "mf_batch_destroy": [C.c_void_p],
    "mf_cnn_create": [C.c_void_p, C.POINTER(C.c_void_p)],
    "mf_cnn_destroy": [C.c_void_p],
    "mf_cnn_get_params": [C.c_void_p, C.c_void_p, C.c_int64],
    "mf_cnn_get_grads": [C.c_void_p, C.c_void_p, C.c_int64],
    "mf_cnn_forward": [C.c_void_p, C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p],
    "mf_cnn_backward": [C.c_void_p, C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p],
    "mf_cnn_train_step": [C.c_void_p, C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.POINTER(CSR), C.c_void_p,
                          C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_float, C.c_float,
                          C.POINTER(C.c_double), C.c_void_p],
    "mf_cnn_node_logk": [C.c_int32, C.c_int32, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p],
    "mf_cnn_input": [C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p],
    "mf_axpby": [C.c_int64, C.c_double, C.c_void_p, C.c_double, C.c_void_p, C.c_void_p],
    "mf_solve_fcg_cnn": [C.POINTER(CSR), C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_int32, C.c_int32,
                         C.c_void_p, C.c_void_p, C.c_double, C.c_int64, C.c_int32, C.POINTER(SolveInfo),
                         C.POINTER(C.c_int64), C.c_void_p],
    "mf_set_kernel_timing": [C.c_int32],
    "mf_kernel_times": [C.c_char_p, C.c_size_t],
}


def lib() -> C.CDLL:
    """Loads libmf.so; raises if it has not been built (no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB):
            raise RuntimeError(f"{LIB} is missing: build it with python -m paper_2111_03541_gb300.build")
        L = C.CDLL(LIB)
        for name, argt in _SIGS.items():
            f = getattr(L, name)
            f.argtypes = argt
            f.restype = C.c_int
        L.mf_cnn_num_params.argtypes = []
        L.mf_cnn_num_params.restype = C.c_int64
        L.mf_last_error.argtypes = []
        L.mf_last_error.restype = C.c_char_p
        _lib = L
    return _lib


def exported_symbols() -> list[str]:
    return list(_SIGS) + ["mf_last_error", "mf_cnn_num_params"]


def _check(status: int, allow=()) -> int:
    if status != MF_OK and status not in allow:
        raise MFError(status, lib().mf_last_error().decode())
    return status


def _ptr(t) -> int | None:
    return None if t is None else t.data_ptr()


def _stream(stream) -> int | None:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return getattr(stream, "cuda_stream", stream)


# ---------------------------------------------------------------------------
# the C ABI, one to one
# ---------------------------------------------------------------------------

def mf_mesh_create(desc: MeshDesc, stream=None) -> C.c_void_p:
    h = C.c_void_p()
    _check(lib().mf_mesh_create(C.byref(desc), _stream(stream), C.byref(h)))
    return h


def mf_mesh_destroy(h) -> None:
    _check(lib().mf_mesh_destroy(h))


def mf_pattern_build(mesh, form: int, stream=None) -> C.c_void_p:
    h = C.c_void_p()
    _check(lib().mf_pattern_build(mesh, form, _stream(stream), C.byref(h)))
    return h


def mf_pattern_csr(pattern) -> CSR:
    c = CSR()
    _check(lib().mf_pattern_csr(pattern, C.byref(c)))
    return c


def mf_pattern_copy_csr(pattern, row_ptr, col_idx, stream=None) -> None:
    _check(lib().mf_pattern_copy_csr(pattern, _ptr(row_ptr), _ptr(col_idx), _stream(stream)))


def mf_pattern_destroy(h) -> None:
    _check(lib().mf_pattern_destroy(h))


def mf_assemble(form: int, mesh, pattern, coeffs: Coeffs, prec: int, K: CSR, d, stream=None) -> None:
    _check(lib().mf_assemble(form, mesh, pattern, C.byref(coeffs), prec, C.byref(K), _ptr(d), _stream(stream)))


def mf_ns_newton(mesh, pattern, coeffs: Coeffs, x, newton_tol: float, max_newton: int, lin: SolverOpts,
                 stream=None) -> tuple[int, list[float], int]:
    """Newton on the Navier-Stokes form: (status, residual norms before each
    step, steps taken); MF_ERR_NOT_CONVERGED is returned, not raised."""
    hist = (C.c_double * (max_newton + 1))()
    steps = C.c_int32(0)
    st = lib().mf_ns_newton(mesh, pattern, C.byref(coeffs), _ptr(x), newton_tol, max_newton, C.byref(lin),
                            C.cast(hist, C.c_void_p), C.byref(steps), _stream(stream))
    if st not in (MF_OK, MF_ERR_NOT_CONVERGED):
        _check(st)
    n = min(steps.value + 1, max_newton + 1)  # one norm per evaluated state
    return st, [hist[i] for i in range(n)], steps.value


def mf_facets_create(mesh, pattern, elem, face, stream=None) -> C.c_void_p:
    """elem: int32 device tensor of parent elements, face: uint8 device tensor of local faces."""
    h = C.c_void_p()
    n = 0 if elem is None else elem.numel()
    _check(lib().mf_facets_create(mesh, pattern, n, _ptr(elem), _ptr(face), _stream(stream), C.byref(h)))
    return h


def mf_facets_destroy(h) -> None:
    _check(lib().mf_facets_destroy(h))


def mf_assemble_boundary(facets, coeffs: FacetCoeffs, K: CSR, d, stream=None) -> None:
    _check(lib().mf_assemble_boundary(facets, C.byref(coeffs), C.byref(K), _ptr(d), _stream(stream)))


def mf_genalpha_params_from_rho(rho_inf: float) -> GenAlphaParams:
    p = GenAlphaParams()
    _check(lib().mf_genalpha_params_from_rho(rho_inf, C.byref(p)))
    return p


def mf_genalpha_run(K: CSR, M_values, F, bc_mask, bc_val, phi, u, a, prm: GenAlphaParams, dt: float, steps: int,
                    newton_tol: float = 1e-8, max_newton: int = 10, pcg_tol: float = 1e-12,
                    pcg_max_iter: int = 100000, stream=None, allow=(), rad=None, rad_es=None, rad_tenv=None):
    """Returns (status, newton solves per step, PCG iterations per step) as numpy arrays.
    rad: a facet set handle (radiation), rad_es / rad_tenv: per-facet device tensors."""
    import numpy as np
    nits = np.zeros(max(steps, 1), dtype=np.int64)
    pits = np.zeros(max(steps, 1), dtype=np.int64)
    st = _check(lib().mf_genalpha_run(C.byref(K), _ptr(M_values), _ptr(F), _ptr(bc_mask), _ptr(bc_val), rad,
                                      _ptr(rad_es), _ptr(rad_tenv), _ptr(phi), _ptr(u), _ptr(a), C.byref(prm), dt,
                                      steps, newton_tol, max_newton, pcg_tol, pcg_max_iter, nits.ctypes.data,
                                      pits.ctypes.data, _stream(stream)), allow)
    return st, nits[:steps], pits[:steps]


def mf_genalpha_initial_rate(K: CSR, M_values, F, bc_mask, phi, u, pcg_tol: float = 1e-13,
                             pcg_max_iter: int = 100000, stream=None, rad=None, rad_es=None, rad_tenv=None) -> None:
    _check(lib().mf_genalpha_initial_rate(C.byref(K), _ptr(M_values), _ptr(F), _ptr(bc_mask), rad, _ptr(rad_es),
                                          _ptr(rad_tenv), _ptr(phi), _ptr(u), pcg_tol, pcg_max_iter,
                                          _stream(stream)))


def mf_pressure_mass_diag(mesh, pattern, out, stream=None) -> None:
    _check(lib().mf_pressure_mass_diag(mesh, pattern, _ptr(out), _stream(stream)))


def mf_flow_mg_create(systems, cells, bc_masks, pmass, visc: float, stream=None):
    """systems: CSR structures of the flow systems, finest first; cells: grid
    cells per side of each; bc_masks: their device masks; pmass: the finest
    pressure-mass diagonal (device).  Returns the opaque hierarchy handle."""
    import numpy as np
    n = len(systems)
    arr = (C.POINTER(CSR) * n)(*[C.pointer(k) for k in systems])
    cl = np.ascontiguousarray(cells, dtype=np.int64)
    masks = (C.c_void_p * n)(*[_ptr(m) for m in bc_masks])
    out = C.c_void_p()
    _check(lib().mf_flow_mg_create(n, arr, cl.ctypes.data_as(C.c_void_p), masks, _ptr(pmass), visc,
                                   _stream(stream), C.byref(out)))
    return out


def mf_flow_mg_destroy(mg) -> None:
    _check(lib().mf_flow_mg_destroy(mg))


def mf_flow_precond(mesh, pattern, K: CSR, bc_mask, p_scale: float, out, stream=None) -> None:
    _check(lib().mf_flow_precond(mesh, pattern, C.byref(K), _ptr(bc_mask), p_scale, _ptr(out), _stream(stream)))


def mf_solve(K: CSR, d, x, opts: SolverOpts, stream=None, allow=(MF_ERR_NOT_CONVERGED,)) -> tuple[int, SolveInfo]:
    info = SolveInfo()
    st = _check(lib().mf_solve(C.byref(K), _ptr(d), _ptr(x), C.byref(opts), C.byref(info), _stream(stream)), allow)
    return st, info


MF_NOALLOC_MAX_ROWS = 1 << 20


def mf_solve_pcg_noalloc(K: CSR, d, x, tol: float, max_iter: int, check_every: int = 50, stream=None,
                         allow=(MF_ERR_NOT_CONVERGED,)) -> tuple[int, SolveInfo]:
    """Jacobi-PCG that makes no device allocation (work vectors in a static device array)."""
    info = SolveInfo()
    st = _check(lib().mf_solve_pcg_noalloc(C.byref(K), _ptr(d), _ptr(x), tol, max_iter, check_every,
                                           C.byref(info), _stream(stream)), allow)
    return st, info


def mf_spmv(K: CSR, x, y, stream=None) -> None:
    _check(lib().mf_spmv(C.byref(K), _ptr(x), _ptr(y), _stream(stream)))


def mf_sync_status(stream=None) -> None:
    _check(lib().mf_sync_status(_stream(stream)))


def mf_batch_create(problems: list, stream=None) -> C.c_void_p:
    """Batch of thermal ``Problem`` objects (their mesh, pattern, coefficients and buffers)."""
    n = len(problems)
    meshes = (C.c_void_p * n)(*[p.mesh.value for p in problems])
    pats = (C.c_void_p * n)(*[p.pattern.value for p in problems])
    coeffs = (Coeffs * n)(*[p.coeffs for p in problems])
    vals = (C.c_void_p * n)(*[_ptr(p.values) for p in problems])
    ds = (C.c_void_p * n)(*[_ptr(p.d) for p in problems])
    h = C.c_void_p()
    _check(lib().mf_batch_create(n, meshes, pats, coeffs, vals, ds, C.byref(h)))
    return h


def mf_batch_set_tiling(batch, tiling: BatchTiling) -> None:
    _check(lib().mf_batch_set_tiling(batch, C.byref(tiling)))


def mf_batch_get_tiling(batch) -> BatchTiling:
    t = BatchTiling()
    _check(lib().mf_batch_get_tiling(batch, C.byref(t)))
    return t


def mf_batch_autotune(batch, cache_path: str | None = None, stream=None) -> BatchTiling:
    t = BatchTiling()
    _check(lib().mf_batch_autotune(batch, None if cache_path is None else cache_path.encode(), _stream(stream),
                                   C.byref(t)))
    return t


def mf_batch_assemble(batch, stream=None) -> None:
    _check(lib().mf_batch_assemble(batch, _stream(stream)))


def mf_batch_destroy(batch) -> None:
    _check(lib().mf_batch_destroy(batch))


def mf_cnn_num_params() -> int:
    return int(lib().mf_cnn_num_params())


def mf_cnn_create(init) -> C.c_void_p:
    """init: float32 numpy array of mf_cnn_num_params() initial parameters."""
    import numpy as np
    init = np.ascontiguousarray(init, dtype=np.float32)
    h = C.c_void_p()
    _check(lib().mf_cnn_create(init.ctypes.data, C.byref(h)))
    return h


def mf_cnn_destroy(h) -> None:
    _check(lib().mf_cnn_destroy(h))


def mf_cnn_get_params(h):
    import numpy as np
    out = np.empty(mf_cnn_num_params(), dtype=np.float32)
    _check(lib().mf_cnn_get_params(h, out.ctypes.data, out.size))
    return out


def mf_cnn_get_grads(h):
    import numpy as np
    out = np.empty(mf_cnn_num_params(), dtype=np.float32)
    _check(lib().mf_cnn_get_grads(h, out.ctypes.data, out.size))
    return out


def mf_cnn_forward(h, B, nz, ny, nx, x, y, stream=None) -> None:
    _check(lib().mf_cnn_forward(h, B, nz, ny, nx, _ptr(x), _ptr(y), _stream(stream)))


def mf_cnn_backward(h, B, nz, ny, nx, x, gy, stream=None) -> None:
    _check(lib().mf_cnn_backward(h, B, nz, ny, nx, _ptr(x), _ptr(gy), _stream(stream)))


def mf_cnn_train_step(h, nz, ny, nx, K: CSR, kvals, r, x, mask, lr, weight_decay, err=None, stream=None) -> float:
    B = len(kvals)
    arr = lambda ts: (C.c_void_p * B)(*[_ptr(t) for t in ts])
    loss = C.c_double()
    _check(lib().mf_cnn_train_step(h, B, nz, ny, nx, C.byref(K), arr(kvals), arr(r),
                                   None if err is None else arr(err), arr(x), _ptr(mask),
                                   lr, weight_decay, C.byref(loss), _stream(stream)))
    return loss.value


def mf_cnn_node_logk(nz, ny, nx, kcell, out, stream=None) -> None:
    _check(lib().mf_cnn_node_logk(nz, ny, nx, _ptr(kcell), _ptr(out), _stream(stream)))


def mf_cnn_input(n, r, logk, x, stream=None) -> None:
    _check(lib().mf_cnn_input(n, _ptr(r), _ptr(logk), _ptr(x), _stream(stream)))


def mf_axpby(n, a, x, b, y, stream=None) -> None:
    _check(lib().mf_axpby(n, a, _ptr(x), b, _ptr(y), _stream(stream)))


def mf_solve_fcg_cnn(K: CSR, d, x, cnn, nz, ny, nx, logk, mask, tol, max_iter, m_dirs=1, stream=None,
                     allow=(MF_ERR_NOT_CONVERGED,)):
    info = SolveInfo()
    fb = C.c_int64()
    st = _check(lib().mf_solve_fcg_cnn(C.byref(K), _ptr(d), _ptr(x), cnn, nz, ny, nx, _ptr(logk), _ptr(mask), tol,
                                       max_iter, m_dirs, C.byref(info), C.byref(fb), _stream(stream)), allow)
    return st, info, fb.value


def mf_set_kernel_timing(enable: bool) -> None:
    _check(lib().mf_set_kernel_timing(1 if enable else 0))


def mf_kernel_times() -> dict[str, tuple[int, float]]:
    """{kernel name: (launches, total ms)} since the last read."""
    buf = C.create_string_buffer(1 << 16)
    _check(lib().mf_kernel_times(buf, len(buf)))
    out = {}
    for line in buf.value.decode().splitlines():
        name, cnt, ms = line.split()
        out[name] = (int(cnt), float(ms))
    return out


def mf_last_error() -> str:
    return lib().mf_last_error().decode()


# ---------------------------------------------------------------------------
# convenience: a generated problem on the GPU
# ---------------------------------------------------------------------------

class Problem:
    """Device copy of a ``gen`` problem with its mesh and pattern handles.

    ``values``/``d`` are torch tensors (float64) the assembly writes into;
    ``row_ptr``/``col`` are copies of the pattern's CSR arrays.
    """

    def __init__(self, prob: dict, device="cuda", stream=None):
        import numpy as np
        import torch

        self.prob = prob
        self.device = torch.device(device)
        dev = self.device

        def t(a, dt):
            return torch.from_numpy(np.ascontiguousarray(a)).to(dev, dt)

        self.form = FORM[prob["form"]]
        self.coords = t(prob["coords"], torch.float64)
        self.conn = t(prob["conn"], torch.int32)
        self.coef = t(prob["coef"], torch.float64)
        self.bc_mask = t(prob["bc_mask"], torch.uint8)
        self.bc_val = t(prob["bc_val"], torch.float64)
        flow = prob["form"] in ("oseen", "ns")
        self.pconn = t(prob["vconn"], torch.int32) if flow else None
        if prob["form"] == "ns":  # the state [u1 | u2 | p]
            n_state = 2 * prob["coords"].shape[0] + prob["vcoords"].shape[0]
            self.advect = t(prob["state"], torch.float64) if "state" in prob else \
                torch.zeros(n_state, dtype=torch.float64, device=dev)
        else:
            self.advect = t(prob["advect"], torch.float64) if flow else None
        self.desc = MeshDesc(dim=self.coords.shape[1], elem=ELEM[prob["elem"]], n_nodes=self.coords.shape[0],
                             n_elems=self.conn.shape[0], coords=_ptr(self.coords), conn=_ptr(self.conn),
                             n_pnodes=0 if self.pconn is None else prob["vcoords"].shape[0],
                             pconn=_ptr(self.pconn))
        self.mesh = mf_mesh_create(self.desc, stream)
        self.pattern = mf_pattern_build(self.mesh, self.form, stream)
        self.csr = mf_pattern_csr(self.pattern)
        self.n = self.csr.n_rows
        self.nnz = self.csr.nnz
        self.values = torch.empty(self.nnz, dtype=torch.float64, device=dev)
        self.d = torch.empty(self.n, dtype=torch.float64, device=dev)
        self.csr.values = _ptr(self.values)
        self.coeffs = self.make_coeffs()
        self.facets = None
        fac = prob.get("facets")
        if fac is not None:
            self.f_elem = t(fac["elem"], torch.int32)
            self.f_face = t(fac["face"], torch.uint8)
            self.f_h = t(fac["h"], torch.float64) if "h" in fac else None
            self.f_tenv = t(fac["t_env"], torch.float64) if "t_env" in fac else None
            self.f_stress = t(np.asarray(fac["stress"]).reshape(-1), torch.float64) if "stress" in fac else None
            self.facets = mf_facets_create(self.mesh, self.pattern, self.f_elem, self.f_face, stream)
            self.facet_coeffs = FacetCoeffs(h=_ptr(self.f_h), t_env=_ptr(self.f_tenv), stress=_ptr(self.f_stress),
                                            bc_mask=_ptr(self.bc_mask), bc_val=_ptr(self.bc_val))

    def make_coeffs(self, coef=None, bc=True) -> Coeffs:
        p = self.prob
        c = Coeffs()
        c.elem_coef = _ptr(self.coef if coef is None else coef)
        c.nu = p.get("nu", 0.0)
        c.visc = p.get("viscosity", 0.0)
        c.rho = p.get("rho", 0.0)
        if p["form"] == "thermal":
            c.source[0] = p.get("source", 1.0)
        elif p["form"] == "elastic":
            for i in range(3):
                c.source[i] = p["body"][i]
        c.advect = _ptr(self.advect)
        c.tau_m = p.get("tau_m", 0.0)
        c.tau_c = p.get("tau_c", 0.0)
        if bc:
            c.bc_mask = _ptr(self.bc_mask)
            c.bc_val = _ptr(self.bc_val)
        return c

    def csr_arrays(self, stream=None):
        import torch
        rp = torch.empty(self.n + 1, dtype=torch.int64, device=self.device)
        ci = torch.empty(self.nnz, dtype=torch.int32, device=self.device)
        mf_pattern_copy_csr(self.pattern, rp, ci, stream)
        return rp, ci

    def assemble(self, prec: int = MF_PREC_FP64, coeffs: Coeffs | None = None, stream=None):
        """Domain terms, then the boundary terms of ``prob["facets"]`` if any."""
        mf_assemble(self.form, self.mesh, self.pattern, coeffs or self.coeffs, prec, self.csr, self.d, stream)
        if self.facets:
            mf_assemble_boundary(self.facets, self.facet_coeffs, self.csr, self.d, stream)
        return self.values, self.d

    def newton(self, tol=1e-11, max_newton=30, lin_tol=1e-13, restart=50, max_iter=200000, flow_mg=None,
               check_every=10, stream=None):
        """Navier-Stokes form: Newton from the current state ``self.advect``
        (updated in place); the linear solves are GMRES, with the flow
        hierarchy ``flow_mg`` as preconditioner when given; returns (status,
        residual history, steps)."""
        lin = SolverOpts(solver=MF_SOLVER_GMRES if flow_mg is None else MF_SOLVER_GMRES_FLOW_MG, restart=restart,
                         tol=lin_tol, max_iter=max_iter, check_every=check_every,
                         flow_mg=flow_mg.value if flow_mg is not None else None)
        return mf_ns_newton(self.mesh, self.pattern, self.coeffs, self.advect, tol, max_newton, lin, stream)

    def pressure_mass_diag(self, stream=None):
        import torch
        out = torch.empty(self.desc.n_pnodes, dtype=torch.float64, device=self.device)
        mf_pressure_mass_diag(self.mesh, self.pattern, out, stream)
        return out

    def flow_precond(self, p_scale: float, stream=None):
        import torch
        out = torch.empty(self.n, dtype=torch.float64, device=self.device)
        mf_flow_precond(self.mesh, self.pattern, self.csr, self.bc_mask, p_scale, out, stream)
        return out

    def solve(self, x=None, solver=MF_SOLVER_PCG, tol=1e-10, max_iter=100000, restart=50, precond=None,
              check_every=50, inner_tol=0.0, flow_mg=None, stream=None):
        import torch
        if x is None:
            x = torch.zeros(self.n, dtype=torch.float64, device=self.device)
        opts = SolverOpts(solver=solver, restart=restart, tol=tol, max_iter=max_iter,
                          precond_diag=_ptr(precond), check_every=check_every, inner_tol=inner_tol,
                          flow_mg=flow_mg.value if flow_mg is not None else None)
        st, info = mf_solve(self.csr, self.d, x, opts, stream)
        return x, st, info

    def close(self):
        if getattr(self, "facets", None):
            mf_facets_destroy(self.facets)
            self.facets = None
        if getattr(self, "pattern", None):
            mf_pattern_destroy(self.pattern)
            self.pattern = None
        if getattr(self, "mesh", None):
            mf_mesh_destroy(self.mesh)
            self.mesh = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
