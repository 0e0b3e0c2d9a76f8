"""CPU FP64 oracle of the FEM assembly + Krylov hot path (MetaFEM, arXiv 2111.03541).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` use it; the product package never imports it.

The arithmetic lives in ``oracle.c`` (plain C, double precision, single
thread); this module compiles it with gcc and wraps it with ctypes.  It shares
no code with the CUDA library: both only receive the arrays made by ``gen``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "oracle.c")
LIB = os.path.join(HERE, "_oracle.so")
LIB_OMP = os.path.join(HERE, "_oracle_omp.so")  # the same source with OpenMP (all-core baseline)

P1, P2, Q1, Q2S, P2T, Q2Q = 0, 1, 2, 3, 4, 5
QTRI3, QTRI6, QHEX8, QHEX27, QTET64, QQUAD9 = 0, 1, 2, 3, 4, 5
THERMAL, ELASTIC, OSEEN, CAPACITY = 0, 1, 2, 3
ELEM = {"P1": P1, "P2": P2, "Q1": Q1, "Q2S": Q2S, "P2T": P2T, "Q2Q": Q2Q}
FORM = {"thermal": THERMAL, "elastic": ELASTIC, "oseen": OSEEN, "capacity": CAPACITY}

_lib = None


def build(force: bool = False) -> str:
    """Compiles oracle.c into _oracle.so (gcc, -O2, no fast-math), and the same
    source with -fopenmp into _oracle_omp.so for the all-core baseline (skipped
    when the compiler has no OpenMP)."""
    for out, extra in ((LIB, []), (LIB_OMP, ["-fopenmp"])):
        if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(SRC):
            tmp = out + ".%d.tmp" % os.getpid()
            try:
                subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-std=c11",
                                       "-ffp-contract=off", *extra, "-o", tmp, SRC, "-lm"])
            except subprocess.CalledProcessError:
                if extra:
                    continue
                raise
            os.replace(tmp, out)
    return LIB


class Problem(C.Structure):
    _fields_ = [("form", C.c_int), ("elem", C.c_int), ("quad", C.c_int),
                ("n_nodes", C.c_int64), ("n_el", C.c_int64), ("n_pnodes", C.c_int64),
                ("coords", C.c_void_p), ("conn", C.c_void_p), ("pconn", C.c_void_p),
                ("coef", C.c_void_p), ("nu", C.c_double), ("mu", C.c_double),
                ("rho", C.c_double), ("source", C.c_void_p), ("fnodal", C.c_void_p),
                ("advect", C.c_void_p), ("n_facets", C.c_int64), ("f_elem", C.c_void_p),
                ("f_face", C.c_void_p), ("f_h", C.c_void_p), ("f_tenv", C.c_void_p),
                ("f_stress", C.c_void_p)]


class Radiation(C.Structure):
    _fields_ = [("elem", C.c_int), ("dim", C.c_int), ("npe", C.c_int), ("coords", C.c_void_p),
                ("conn", C.c_void_p), ("n_facets", C.c_int64), ("f_elem", C.c_void_p), ("f_face", C.c_void_p),
                ("es", C.c_void_p), ("tenv", C.c_void_p)]


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        d, i64, vp, i = C.c_double, C.c_int64, C.c_void_p, C.c_int
        _lib.or_quad.argtypes = [i, vp, vp]
        _lib.or_shape.argtypes = [i, vp, vp, vp]
        _lib.or_elem_measure.argtypes = [i, i, vp]
        _lib.or_elem_measure.restype = d
        _lib.or_elem_thermal.argtypes = [i, i, vp, d, d, vp, vp, vp]
        _lib.or_elem_thermal.restype = d
        _lib.or_elem_elastic_q1.argtypes = [vp, d, d, vp, vp, vp]
        _lib.or_elem_elastic_q1.restype = d
        _lib.or_elem_elastic.argtypes = [i, vp, d, d, vp, vp, vp]
        _lib.or_elem_elastic.restype = d
        _lib.or_elem_oseen.argtypes = [vp, vp, d, d, vp, vp, vp, vp]
        _lib.or_elem_oseen.restype = d
        _lib.or_elem_ns.argtypes = [vp, vp, vp, d, d, d, d, vp, vp]
        _lib.or_elem_ns.restype = d
        _lib.or_ns_system.argtypes = [i64, i64, i64, vp, vp, vp, vp, vp, vp, d, d, d, d, vp, vp, vp, vp]
        _lib.or_elem_ns3.argtypes = [vp, vp, vp, d, d, d, d, vp, vp]
        _lib.or_elem_ns3.restype = d
        _lib.or_ns_system.restype = d
        _lib.or_elem_capacity.argtypes = [i, vp, d, vp]
        _lib.or_elem_capacity.restype = d
        _lib.or_genalpha.argtypes = [i64, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, d, d, d, d, d, d, i64, d, i, d,
                                     vp, C.POINTER(Radiation)]
        _lib.or_facet_radiation.argtypes = [i, vp, d, d, vp, vp, vp]
        _lib.or_genalpha.restype = i
        _lib.or_facet_nodes.argtypes = [i, i, vp]
        _lib.or_facet_thermal.argtypes = [i, vp, d, d, vp, vp]
        _lib.or_facet_thermal.restype = d
        _lib.or_facet_traction_q1.argtypes = [i, vp, vp, vp]
        _lib.or_facet_traction.argtypes = [i, i, vp, vp, vp]
        _lib.or_assemble.argtypes = [C.POINTER(Problem)] + [C.POINTER(i64)] * 2 + [C.POINTER(vp)] * 5
        _lib.or_assemble.restype = i
        _lib.or_assemble_filtered.argtypes = [C.POINTER(Problem), vp, vp] + [C.POINTER(i64)] * 2 + \
            [C.POINTER(vp)] * 5
        _lib.or_assemble_filtered.restype = i
        _lib.or_free.argtypes = [vp]
        _lib.or_dirichlet.argtypes = [i64, vp, vp, vp, vp, vp, vp]
        _lib.or_spmv.argtypes = [i64, vp, vp, vp, vp, vp]
        _lib.or_pcg.argtypes = [i64, vp, vp, vp, vp, vp, d, i64, C.POINTER(d)]
        _lib.or_pcg.restype = i64
        _lib.or_gmres.argtypes = [i64, vp, vp, vp, vp, vp, vp, i, d, i64, C.POINTER(d)]
        _lib.or_gmres.restype = i64
        _lib.or_conv3d_fwd.argtypes = [i64, i64, i64, i, i, vp, vp, vp, i, vp]
        _lib.or_conv3d_bwd_data.argtypes = [i64, i64, i64, i, i, vp, vp, vp]
        _lib.or_conv3d_bwd_weight.argtypes = [i64, i64, i64, i, i, vp, vp, vp, vp]
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data if a is not None else None


# ---------------------------------------------------------------------------
# element level
# ---------------------------------------------------------------------------

def quad(kind: int) -> tuple[np.ndarray, np.ndarray]:
    pts = np.zeros((64, 3))
    w = np.zeros(64)
    nq = lib().or_quad(kind, _p(pts), _p(w))
    dim = 3 if kind in (QHEX8, QHEX27, QTET64) else 2
    return pts.ravel()[: nq * dim].reshape(nq, dim).copy(), w[:nq].copy()


def shape(elem: int, xi) -> tuple[np.ndarray, np.ndarray]:
    dim = 3 if elem in (Q1, Q2S, P2T) else 2
    xi = np.ascontiguousarray(xi, dtype=np.float64)
    N = np.zeros(20)
    dN = np.zeros(60)
    npe = lib().or_shape(elem, _p(xi), _p(N), _p(dN))
    return N[:npe].copy(), dN[: npe * dim].reshape(npe, dim).copy()


def elem_measure(elem: int, quad_kind: int, X: np.ndarray) -> float:
    X = np.ascontiguousarray(X, dtype=np.float64)
    return lib().or_elem_measure(elem, quad_kind, _p(X))


def elem_thermal(elem: int, quad_kind: int, X, k: float, f: float = 1.0, fnodal=None):
    X = np.ascontiguousarray(X, dtype=np.float64)
    npe = X.shape[0]
    Ke = np.zeros((npe, npe))
    de = np.zeros(npe)
    fn = None if fnodal is None else np.ascontiguousarray(fnodal, dtype=np.float64)
    det = lib().or_elem_thermal(elem, quad_kind, _p(X), k, f, _p(fn), _p(Ke), _p(de))
    return Ke, de, det


def elem_elastic(X, E: float, nu: float, body=(0.0, 0.0, -1.0), elem: int = None):
    """Element stiffness [3 npe, 3 npe] (dof 3 a + c), load [3 npe] and min detJ;
    elem Q1 (the default, 8 nodes), Q2S (20 nodes) or P2T (10 nodes)."""
    X = np.ascontiguousarray(X, dtype=np.float64)
    b = np.ascontiguousarray(body, dtype=np.float64)
    if elem is None or elem == Q1:
        Ke = np.zeros((24, 24))
        de = np.zeros(24)
        det = lib().or_elem_elastic_q1(_p(X), E, nu, _p(b), _p(Ke), _p(de))
        return Ke, de, det
    if elem not in (Q2S, P2T):
        raise ValueError("elasticity takes the Q1 or Q2S brick or the P2T tetrahedron")
    m = 3 * (20 if elem == Q2S else 10)
    Ke = np.zeros((m, m))
    de = np.zeros(m)
    det = lib().or_elem_elastic(elem, _p(X), E, nu, _p(b), _p(Ke), _p(de))
    return Ke, de, det


def elem_oseen(X, aN, mu: float, rho: float):
    X = np.ascontiguousarray(X, dtype=np.float64)
    aN = np.ascontiguousarray(aN, dtype=np.float64)  # [6][2]
    A = np.zeros((6, 6))
    BT = np.zeros((2, 6, 3))
    B = np.zeros((2, 3, 6))
    Mp = np.zeros(3)
    det = lib().or_elem_oseen(_p(X), _p(aN), mu, rho, _p(A), _p(BT), _p(B), _p(Mp))
    return A, BT, B, Mp, det


def elem_ns(X, U, P, mu: float, rho: float, tau_m: float, tau_c: float):
    """Steady Navier-Stokes with SUPG on one Taylor-Hood triangle (Sec. 4.3):
    residual r[15] (velocity dof (a, i) at 2a + i, pressure vertex b at
    12 + b), tangent Ke[15, 15] by complex step, detJ.  U [6][2], P [3]."""
    X = np.ascontiguousarray(X, dtype=np.float64)
    U = np.ascontiguousarray(U, dtype=np.float64)
    P = np.ascontiguousarray(P, dtype=np.float64)
    r = np.zeros(15)
    Ke = np.zeros((15, 15))
    det = lib().or_elem_ns(_p(X), _p(U), _p(P), mu, rho, tau_m, tau_c, _p(r), _p(Ke))
    return r, Ke, det


def elem_ns3(X, U, P, mu: float, rho: float, tau_m: float, tau_c: float):
    """The Navier-Stokes form with SUPG on one Taylor-Hood tetrahedron:
    residual r[34] (velocity dof (a, i) at 3a + i, pressure vertex b at
    30 + b), tangent Ke[34, 34] by complex step, detJ.  X: the 4 vertices;
    U [10][3]; P [4]."""
    X = np.ascontiguousarray(X, dtype=np.float64)
    U = np.ascontiguousarray(U, dtype=np.float64)
    P = np.ascontiguousarray(P, dtype=np.float64)
    r = np.zeros(34)
    Ke = np.zeros((34, 34))
    det = lib().or_elem_ns3(_p(X), _p(U), _p(P), mu, rho, tau_m, tau_c, _p(r), _p(Ke))
    return r, Ke, det


def ns_system(prob: dict, x, tau_m: float, tau_c: float):
    """Residual R and tangent K (scipy CSR, duplicates summed) of the
    Navier-Stokes form with SUPG at the state x = [u1 | u2 | p] on a
    Taylor-Hood problem (``prob`` as gen.oseen_problem: coords, conn, vconn,
    viscosity, rho).  No Dirichlet elimination."""
    import scipy.sparse as sp
    coords = np.ascontiguousarray(prob["coords"], dtype=np.float64)
    conn = np.ascontiguousarray(prob["conn"], dtype=np.int32)
    pconn = np.ascontiguousarray(prob["vconn"], dtype=np.int32)
    n2, n1, ne = coords.shape[0], prob["vcoords"].shape[0], conn.shape[0]
    x = np.ascontiguousarray(x, dtype=np.float64)
    u1, u2, p = x[:n2].copy(), x[n2:2 * n2].copy(), x[2 * n2:].copy()
    R = np.zeros(2 * n2 + n1)
    rows = np.zeros(225 * ne, dtype=np.int64)
    cols = np.zeros(225 * ne, dtype=np.int32)
    vals = np.zeros(225 * ne)
    mindet = lib().or_ns_system(n2, n1, ne, _p(coords), _p(conn), _p(pconn), _p(u1), _p(u2), _p(p),
                                prob["viscosity"], prob["rho"], tau_m, tau_c, _p(R), _p(rows), _p(cols), _p(vals))
    if not mindet > 0:
        raise AssemblyError("element with detJ <= 0")
    n = 2 * n2 + n1
    K = sp.coo_matrix((vals, (rows, cols)), shape=(n, n)).tocsr()
    K.sum_duplicates()
    return R, K


def ns_newton(prob: dict, tau_m: float, tau_c: float, tol: float = 1e-11, maxit: int = 30, x0=None):
    """Newton-Raphson (Sec. 2.1) on the Navier-Stokes form with SUPG: from
    x0 (default: the Dirichlet values, zero elsewhere), dofs in bc_mask held
    at bc_val, K dx = -R on the free dofs (a sparse direct solve) until
    ||R_free|| <= tol max(1, ||R_free(x0)||).  Returns (x, residual norms)."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla
    mask = np.asarray(prob["bc_mask"]) > 0
    x = np.where(mask, prob["bc_val"], 0.0) if x0 is None else np.where(mask, prob["bc_val"], x0)
    free = np.flatnonzero(~mask)
    hist = []
    for _ in range(maxit):
        R, K = ns_system(prob, x, tau_m, tau_c)
        rn = np.linalg.norm(R[free])
        hist.append(rn)
        if rn <= tol * max(1.0, hist[0]):
            break
        Kff = K[free][:, free].tocsc()
        x[free] += spla.spsolve(Kff, -R[free])
    return x, hist


def elem_capacity(elem: int, X, C: float):
    """Capacity matrix C int N_a N_b of one element and its min detJ."""
    X = np.ascontiguousarray(X, dtype=np.float64)
    npe = X.shape[0]
    Me = np.zeros((npe, npe))
    det = lib().or_elem_capacity(elem, _p(X), C, _p(Me))
    return Me, det


def facet_nodes(elem: int, face: int) -> list[int]:
    """Local element nodes of a facet, in facet node order."""
    loc = np.zeros(8, dtype=np.int32)
    nf = lib().or_facet_nodes(elem, face, _p(loc))
    if nf < 0:
        raise ValueError("no such face")
    return loc[:nf].tolist()


def facet_thermal(elem: int, Xf, h: float, t_env: float):
    """Convection matrix and load of one facet: (Kf, df, measure)."""
    Xf = np.ascontiguousarray(Xf, dtype=np.float64)
    nf = Xf.shape[0]
    Kf = np.zeros((nf, nf))
    df = np.zeros(nf)
    meas = lib().or_facet_thermal(elem, _p(Xf), h, t_env, _p(Kf), _p(df))
    return Kf, df, meas


def facet_traction(face: int, Xf, sigma, elem: int = None) -> np.ndarray:
    """Loaded-boundary load of one brick face: [facet nodes][3] (4 for Q1,
    the default, 8 for Q2S)."""
    Xf = np.ascontiguousarray(Xf, dtype=np.float64)
    sg = np.ascontiguousarray(sigma, dtype=np.float64).reshape(9)
    if elem is None or elem == Q1:
        df = np.zeros((4, 3))
        lib().or_facet_traction_q1(face, _p(Xf), _p(sg), _p(df))
        return df
    df = np.zeros((8, 3))
    lib().or_facet_traction(elem, face, _p(Xf), _p(sg), _p(df))
    return df


# ---------------------------------------------------------------------------
# global level
# ---------------------------------------------------------------------------

class AssemblyError(RuntimeError):
    pass


def _default_quad(elem: str, form: str) -> int:
    if elem == "Q1":
        return QHEX8
    if elem == "Q2S":
        return QHEX27
    if elem == "P2T":
        return QTET64
    if elem == "Q2Q":
        return QQUAD9
    if form == "oseen":
        return QTRI6
    return QTRI3


def assemble(prob: dict, quad_kind: int | None = None, fnodal=None, dirichlet: bool = True,
             keep_nodes=None, keep_pnodes=None):
    """Assembles CSR K and d for a problem dict made by ``gen``.

    Returns dict(row_ptr int64, col int32, val f64, d f64[, pmass f64]).
    With ``dirichlet`` the strong elimination of ``bc_mask``/``bc_val`` is applied.
    ``keep_nodes`` (bool mask over nodes; ``keep_pnodes`` over flow pressure
    nodes) restricts the work to the elements touching them: only the rows of
    those nodes are then complete (use ``rows_of``).  ``prob["facets"]`` (from
    ``gen.convection_facets`` / ``gen.traction_facets``) adds the boundary terms.
    """
    form = prob["form"]
    elem = prob["elem"]
    keep = []

    def arr(a, dt):
        a = np.ascontiguousarray(a, dtype=dt)
        keep.append(a)
        return a

    coords = arr(prob["coords"], np.float64)
    conn = arr(prob["conn"], np.int32)
    coef = arr(prob["coef"], np.float64)
    pr = Problem()
    pr.form = FORM[form]
    pr.elem = ELEM[elem]
    pr.quad = _default_quad(elem, form) if quad_kind is None else quad_kind
    pr.n_nodes = coords.shape[0]
    pr.n_el = conn.shape[0]
    pr.coords = _p(coords)
    pr.conn = _p(conn)
    pr.coef = _p(coef)
    if form in ("thermal", "capacity"):
        src = arr([prob.get("source", 1.0), 0.0, 0.0], np.float64)
        pr.source = _p(src)
        if fnodal is not None:
            pr.fnodal = _p(arr(fnodal, np.float64))
    elif form == "elastic":
        pr.nu = prob["nu"]
        pr.source = _p(arr(prob["body"], np.float64))
    else:
        pconn = arr(prob["vconn"], np.int32)
        pr.pconn = _p(pconn)
        pr.n_pnodes = prob["vcoords"].shape[0]
        pr.mu = prob["viscosity"]
        pr.rho = prob["rho"]
        pr.advect = _p(arr(prob["advect"], np.float64))
    fac = prob.get("facets")
    if fac is not None and len(fac["elem"]) > 0:
        pr.n_facets = len(fac["elem"])
        pr.f_elem = _p(arr(fac["elem"], np.int32))
        pr.f_face = _p(arr(fac["face"], np.uint8))
        if "h" in fac:
            pr.f_h = _p(arr(fac["h"], np.float64))
            pr.f_tenv = _p(arr(fac["t_env"], np.float64))
        if "stress" in fac:
            pr.f_stress = _p(arr(fac["stress"], np.float64))
        if (form == "thermal" and "h" not in fac) or (form == "elastic" and "stress" not in fac):
            raise ValueError("facet data do not match the form")
    n_rows, nnz = C.c_int64(), C.c_int64()
    ptrs = [C.c_void_p() for _ in range(5)]
    if keep_nodes is None and keep_pnodes is None:
        rc = lib().or_assemble(C.byref(pr), C.byref(n_rows), C.byref(nnz), *[C.byref(x) for x in ptrs])
    else:
        kn = arr(np.zeros(coords.shape[0], np.uint8) if keep_nodes is None else keep_nodes, np.uint8)
        kp = None if keep_pnodes is None else arr(keep_pnodes, np.uint8)
        rc = lib().or_assemble_filtered(C.byref(pr), _p(kn), _p(kp), C.byref(n_rows), C.byref(nnz),
                                        *[C.byref(x) for x in ptrs])
    if rc == -2:
        raise AssemblyError("element with detJ <= 0")
    if rc == -3:
        raise AssemblyError("facet outside the mesh, a form without boundary terms, or an element the form does not take")
    if rc:
        raise MemoryError("oracle assembly failed")
    n, z = n_rows.value, nnz.value

    def take(ptr, count, ctype, dt):
        if not ptr.value:
            return None
        a = np.ctypeslib.as_array(C.cast(ptr, C.POINTER(ctype)), shape=(count,)).astype(dt, copy=True)
        lib().or_free(ptr)
        return a

    out = {"row_ptr": take(ptrs[0], n + 1, C.c_int64, np.int64),
           "col": take(ptrs[1], z, C.c_int32, np.int32),
           "val": take(ptrs[2], z, C.c_double, np.float64),
           "d": take(ptrs[3], n, C.c_double, np.float64)}
    pm = take(ptrs[4], int(pr.n_pnodes), C.c_double, np.float64)
    if pm is not None:
        out["pmass"] = pm
    if dirichlet:
        apply_dirichlet(out, prob["bc_mask"], prob["bc_val"])
    return out


_lib_omp = None


def assemble_threads(prob: dict, threads: int, dirichlet: bool = True) -> dict:
    """The assembly of ``assemble`` on ``threads`` host threads (OpenMP build
    of the same source; domain forms without facets).  Bit-identical to
    ``assemble``; used as the all-core CPU baseline."""
    global _lib_omp
    build()
    if _lib_omp is None:
        if not os.path.exists(LIB_OMP):
            raise RuntimeError("no OpenMP build of the oracle")
        _lib_omp = C.CDLL(LIB_OMP)
        vp, i64 = C.c_void_p, C.c_int64
        _lib_omp.or_assemble_threads.argtypes = [C.POINTER(Problem), C.c_int] + [C.POINTER(i64)] * 2 + \
            [C.POINTER(vp)] * 4
        _lib_omp.or_assemble_threads.restype = C.c_int
        _lib_omp.or_free.argtypes = [vp]
    keep = []

    def arr(a, dt):
        a = np.ascontiguousarray(a, dtype=dt)
        keep.append(a)
        return a

    form, elem = prob["form"], prob["elem"]
    coords = arr(prob["coords"], np.float64)
    conn = arr(prob["conn"], np.int32)
    pr = Problem()
    pr.form, pr.elem, pr.quad = FORM[form], ELEM[elem], _default_quad(elem, form)
    pr.n_nodes, pr.n_el = coords.shape[0], conn.shape[0]
    pr.coords, pr.conn, pr.coef = _p(coords), _p(conn), _p(arr(prob["coef"], np.float64))
    if form == "elastic":
        pr.nu = prob["nu"]
        pr.source = _p(arr(prob["body"], np.float64))
    else:
        pr.source = _p(arr([prob.get("source", 1.0), 0.0, 0.0], np.float64))
    n_rows, nnz = C.c_int64(), C.c_int64()
    ptrs = [C.c_void_p() for _ in range(4)]
    rc = _lib_omp.or_assemble_threads(C.byref(pr), int(threads), C.byref(n_rows), C.byref(nnz),
                                      *[C.byref(x) for x in ptrs])
    if rc == -2:
        raise AssemblyError("element with detJ <= 0")
    if rc:
        raise AssemblyError("threaded oracle assembly failed (%d)" % rc)
    n, z = n_rows.value, nnz.value

    def take(ptr, count, ctype, dt):
        a = np.ctypeslib.as_array(C.cast(ptr, C.POINTER(ctype)), shape=(count,)).astype(dt, copy=True)
        _lib_omp.or_free(ptr)
        return a

    out = {"row_ptr": take(ptrs[0], n + 1, C.c_int64, np.int64), "col": take(ptrs[1], z, C.c_int32, np.int32),
           "val": take(ptrs[2], z, C.c_double, np.float64), "d": take(ptrs[3], n, C.c_double, np.float64)}
    if dirichlet:
        apply_dirichlet(out, prob["bc_mask"], prob["bc_val"])
    return out


def rows_of(sys: dict, rows) -> list[tuple[np.ndarray, np.ndarray]]:
    """(columns, values) of the given rows of an assembled CSR system."""
    rp, col, val = sys["row_ptr"], sys["col"], sys["val"]
    return [(col[rp[r]:rp[r + 1]].copy(), val[rp[r]:rp[r + 1]].copy()) for r in rows]


def apply_dirichlet(sys: dict, mask, bval) -> None:
    mask = np.ascontiguousarray(mask, dtype=np.uint8)
    bval = np.ascontiguousarray(bval, dtype=np.float64)
    n = sys["d"].shape[0]
    lib().or_dirichlet(n, _p(sys["row_ptr"]), _p(sys["col"]), _p(sys["val"]), _p(sys["d"]),
                       _p(mask), _p(bval))


def spmv(sys: dict, x) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.zeros(sys["row_ptr"].shape[0] - 1)
    lib().or_spmv(y.shape[0], _p(sys["row_ptr"]), _p(sys["col"]), _p(sys["val"]), _p(x), _p(y))
    return y


def pcg(sys: dict, tol: float = 1e-10, maxit: int = 100000, x0=None):
    n = sys["d"].shape[0]
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64)
    rr = C.c_double()
    it = lib().or_pcg(n, _p(sys["row_ptr"]), _p(sys["col"]), _p(sys["val"]), _p(sys["d"]),
                      _p(x), tol, maxit, C.byref(rr))
    return x, int(it), rr.value


def gmres(sys: dict, pdiag, m: int = 50, tol: float = 1e-8, maxit: int = 20000, x0=None):
    n = sys["d"].shape[0]
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64)
    pdiag = np.ascontiguousarray(pdiag, dtype=np.float64)
    rr = C.c_double()
    it = lib().or_gmres(n, _p(sys["row_ptr"]), _p(sys["col"]), _p(sys["val"]), _p(sys["d"]),
                        _p(x), _p(pdiag), m, tol, maxit, C.byref(rr))
    return x, int(it), rr.value


def oseen_precond(sys: dict, prob: dict) -> np.ndarray:
    """Block-diagonal preconditioner diag(diag(A)_u1, diag(A)_u2, diag(M_p) / mu).

    Constrained dofs (velocity Dirichlet nodes, the pinned pressure) keep 1.
    """
    n = sys["d"].shape[0]
    rp, col, val = sys["row_ptr"], sys["col"], sys["val"]
    diag = np.zeros(n)
    for i in range(n):
        s = slice(rp[i], rp[i + 1])
        hit = np.nonzero(col[s] == i)[0]
        diag[i] = val[s][hit[0]]
    n2 = prob["coords"].shape[0]
    p = diag.copy()
    p[2 * n2:] = sys["pmass"] / prob["viscosity"]
    mask = prob["bc_mask"].astype(bool)
    p[mask] = 1.0
    return p


# ---------------------------------------------------------------------------
# generalised-alpha time stepping
# ---------------------------------------------------------------------------

def genalpha_params(rho_inf: float) -> dict:
    """Parameters of the first-order generalised-alpha method (Jansen,
    Whiting and Hulbert 2000) for the high-frequency spectral radius rho_inf,
    in the constraint/relaxation notation of Sec. 2.1: b1 = gamma,
    c1 = alpha_f, c2 = alpha_m; the second-rate level takes b2 = gamma,
    c3 = alpha_m (it does not enter a first-order residual)."""
    am = 0.5 * (3.0 - rho_inf) / (1.0 + rho_inf)
    af = 1.0 / (1.0 + rho_inf)
    g = 0.5 + am - af
    return {"b1": g, "b2": g, "c1": af, "c2": am, "c3": am}


def capacity(prob: dict, C) -> dict:
    """Capacity matrix sum_e C_e int N_a N_b of a thermal problem's mesh (no
    Dirichlet elimination); C is a per-element array."""
    p = dict(prob, form="capacity", coef=np.ascontiguousarray(C, dtype=np.float64))
    p.pop("facets", None)
    return assemble(p, dirichlet=False)


def initial_rate(K: dict, M: dict, F, mask, phi0) -> np.ndarray:
    """Consistent initial rate u0 with M u0 = F - K phi0 on the free rows,
    u0 = 0 on Dirichlet rows."""
    r = np.asarray(F, dtype=np.float64) - spmv(K, phi0)
    Mm = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in M.items()}
    Mm["d"] = r
    apply_dirichlet(Mm, mask, np.zeros_like(r))
    u0, _, _ = pcg(Mm, tol=1e-14)
    return u0


def facet_radiation(elem: int, Xf, es: float, t_env: float, Tf):
    """Radiation tangent and load of one facet at nodal temperatures Tf: (Kf, rf)."""
    Xf = np.ascontiguousarray(Xf, dtype=np.float64)
    Tf = np.ascontiguousarray(Tf, dtype=np.float64)
    nf = Xf.shape[0]
    Kf = np.zeros((nf, nf))
    rf = np.zeros(nf)
    lib().or_facet_radiation(elem, _p(Xf), es, t_env, _p(Tf), _p(Kf), _p(rf))
    return Kf, rf


def genalpha(K: dict, M: dict, F, mask, bval, phi, u, a, prm: dict, dt: float, steps: int,
             newton_tol: float = 1e-8, max_newton: int = 10, pcg_tol: float = 1e-13, prob=None, radiation=None):
    """Runs or_genalpha; returns (phi, u, a, newton solves per step).  With
    ``radiation`` (dict elem, face, es, t_env of facets of ``prob``'s mesh)
    the radiation terms enter the residual and the tangent."""
    n = K["d"].shape[0] if "d" in K else K["row_ptr"].shape[0] - 1
    phi = np.array(phi, dtype=np.float64)
    u = np.array(u, dtype=np.float64)
    a = np.array(a, dtype=np.float64)
    F = np.ascontiguousarray(F, dtype=np.float64)
    mask = np.ascontiguousarray(mask, dtype=np.uint8)
    bval = np.ascontiguousarray(bval, dtype=np.float64)
    its = np.zeros(max(steps, 1), dtype=np.int64)
    rad = None
    keep = []
    if radiation is not None:
        def arr(x, dt_):
            x = np.ascontiguousarray(x, dtype=dt_)
            keep.append(x)
            return x
        X = arr(prob["coords"], np.float64)
        cn = arr(prob["conn"], np.int32)
        rad = Radiation(elem=ELEM[prob["elem"]], dim=X.shape[1], npe=cn.shape[1], coords=_p(X), conn=_p(cn),
                        n_facets=len(radiation["elem"]), f_elem=_p(arr(radiation["elem"], np.int32)),
                        f_face=_p(arr(radiation["face"], np.uint8)), es=_p(arr(radiation["es"], np.float64)),
                        tenv=_p(arr(radiation["t_env"], np.float64)))
    rc = lib().or_genalpha(n, _p(K["row_ptr"]), _p(K["col"]), _p(K["val"]), _p(M["val"]), _p(F), _p(mask),
                           _p(bval), _p(phi), _p(u), _p(a), prm["b1"], prm["b2"], prm["c1"], prm["c2"], prm["c3"],
                           dt, steps, newton_tol, max_newton, pcg_tol, _p(its),
                           C.byref(rad) if rad is not None else None)
    if rc == -4:
        raise MemoryError("oracle generalised-alpha")
    if rc:
        raise RuntimeError("generalised-alpha: a step did not converge")
    return phi, u, a, its[:steps]


# ---------------------------------------------------------------------------
# 3x3x3 convolution layers (learned preconditioner correction)
# ---------------------------------------------------------------------------

def conv3d_fwd(x, w, b=None, relu=False):
    """x [nz, ny, nx, ci], w [co, ci, 27], b [co] -> [nz, ny, nx, co] (zero padding)."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    w = np.ascontiguousarray(w, dtype=np.float64)
    bb = None if b is None else np.ascontiguousarray(b, dtype=np.float64)
    nz, ny, nx, ci = x.shape
    co = w.shape[0]
    out = np.zeros((nz, ny, nx, co))
    lib().or_conv3d_fwd(nz, ny, nx, ci, co, _p(x), _p(w), _p(bb), int(relu), _p(out))
    return out


def conv3d_bwd_data(gout, w, ci):
    gout = np.ascontiguousarray(gout, dtype=np.float64)
    w = np.ascontiguousarray(w, dtype=np.float64)
    nz, ny, nx, co = gout.shape
    gin = np.zeros((nz, ny, nx, ci))
    lib().or_conv3d_bwd_data(nz, ny, nx, ci, co, _p(gout), _p(w), _p(gin))
    return gin


def conv3d_bwd_weight(x, gout):
    x = np.ascontiguousarray(x, dtype=np.float64)
    gout = np.ascontiguousarray(gout, dtype=np.float64)
    nz, ny, nx, ci = x.shape
    co = gout.shape[3]
    gw = np.zeros((co, ci, 27))
    gb = np.zeros(co)
    lib().or_conv3d_bwd_weight(nz, ny, nx, ci, co, _p(x), _p(gout), _p(gw), _p(gb))
    return gw, gb
