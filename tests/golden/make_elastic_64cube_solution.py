"""Writes elastic_q1_64cube_solution.txt: the oracle's tight solution of the
3D linear elasticity workload (Q1 hexahedra on the 64^3 box, Sec. 4.2 form,
seeded synthetic inputs), for the mixed-path refinement test.

Calls only the oracle (its FP64 assembly with the Dirichlet elimination) and
numpy/scipy: Jacobi-preconditioned conjugate gradients from x0 = 0 until the
true relative residual ||d - K x|| / ||d|| stops decreasing (the FP64
rounding floor), with the coefficients alpha_k, beta_k recorded; then
iterative refinement of that x with the residual d - K x formed in extended
precision (numpy longdouble, a 64-bit significand on x86) and each
correction solved by the same FP64 PCG to 1e-9, while a step gains a factor
10 and the extended-precision relative residual is above 1e-16.  The Lanczos tridiagonal matrix of the
first solve has the extreme eigenvalues of D^-1 K, so kappa_est =
lambda_max / lambda_min, and kappa_est * relres bounds the relative error of
x* (reading 12 requires it below 1e-9).

The file holds: dofs, iterations, relres, kappa_est, ||x*||_2, then 1024
sampled dofs (seeded, sorted) with their x* values (repr of the doubles).

Run: python tests/golden/make_elastic_64cube_solution.py  (a few minutes)
"""
import os
import sys

import numpy as np
import scipy.sparse as sp

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import gen  # noqa: E402
import oracle  # noqa: E402

OUT = os.path.join(HERE, "elastic_q1_64cube_solution.txt")
N_SAMPLES = 1024
SEED_SAMPLES = 2024


def pcg(K, dinv, b, tol, maxit=20000, record=None):
    """Jacobi-PCG from 0 on K x = b; stops when the true relative residual
    reaches tol or has not improved by 10% over 400 iterations."""
    x = np.zeros_like(b)
    r = b.copy()
    z = dinv * r
    p = z.copy()
    rz = r @ z
    bn = np.linalg.norm(b)
    best, xbest, kbest, stall = np.inf, x.copy(), 0, 0
    for k in range(1, maxit + 1):
        q = K @ p
        alpha = rz / (p @ q)
        x += alpha * p
        r -= alpha * q
        z = dinv * r
        rz_new = r @ z
        beta = rz_new / rz
        rz = rz_new
        p = z + beta * p
        if record is not None:
            record.append((alpha, beta))
        if k % 25 == 0:
            rel = np.linalg.norm(b - K @ x) / bn
            if rel < 0.9 * best:
                best, xbest, kbest, stall = rel, x.copy(), k, 0
            else:
                stall += 1
            if rel <= tol or stall >= 16:
                break
    return xbest, best, kbest


def main():
    prob = gen.elastic_problem(64)
    ref = oracle.assemble_threads(prob, os.cpu_count() or 1) if hasattr(oracle, "assemble_threads") \
        else oracle.assemble(prob)
    n = ref["row_ptr"].shape[0] - 1
    K = sp.csr_matrix((ref["val"], ref["col"], ref["row_ptr"]), shape=(n, n))
    d = ref["d"]
    dinv = 1.0 / K.diagonal()
    coef = []
    x, rel64, its = pcg(K, dinv, d, 1e-16, record=coef)
    # Lanczos tridiagonal of the first `its` steps
    a = np.array([c[0] for c in coef[:its]])
    b = np.array([c[1] for c in coef[:its]])
    diag = 1.0 / a
    diag[1:] += b[:-1] / a[:-1]
    off = np.sqrt(b[:-1]) / a[:-1]
    T = np.diag(diag) + np.diag(off, 1) + np.diag(off, -1)
    ev = np.linalg.eigvalsh(T)
    kappa = ev[-1] / ev[0]
    # refinement with the residual in extended precision
    ld = np.longdouble
    vals = ref["val"].astype(ld)
    rows = np.repeat(np.arange(n), np.diff(ref["row_ptr"]))
    dl = d.astype(ld)
    xl = x.astype(ld)
    dn = np.sqrt(np.sum(dl * dl))

    def resid(xl):
        kx = np.zeros(n, dtype=ld)
        np.add.at(kx, rows, vals * xl[ref["col"]])
        return dl - kx

    rl = resid(xl)
    relres = float(np.sqrt(np.sum(rl * rl)) / dn)
    print(f"FP64 PCG: {its} iterations, relres {rel64:.3e}; extended residual {relres:.3e}", flush=True)
    for step in range(3):  # stops at 1e-16 or when a step gains less than a factor 10
        if relres < 1e-16:
            break
        rn = float(np.sqrt(np.sum(rl * rl)))
        dx, _, _ = pcg(K, dinv, (rl / rn).astype(np.float64), 1e-9)
        xn = xl + ld(rn) * dx.astype(ld)
        rn_l = resid(xn)
        rel_n = float(np.sqrt(np.sum(rn_l * rn_l)) / dn)
        print(f"refinement {step + 1}: extended relres {rel_n:.3e}", flush=True)
        if rel_n > 0.1 * relres:
            break
        xl, rl, relres = xn, rn_l, rel_n
    xs = xl.astype(np.float64)
    idx = np.sort(np.random.default_rng(SEED_SAMPLES).choice(n, N_SAMPLES, replace=False))
    with open(OUT, "w") as f:
        f.write("# oracle tight solution, elasticity Q1 64^3 (gen.elastic_problem(64)); "
                "written by make_elastic_64cube_solution.py\n")
        f.write(f"dofs {n}\niterations {its}\nrelres {float(relres)!r}\nkappa_est {float(kappa)!r}\n")
        f.write(f"norm2 {float(np.linalg.norm(xs))!r}\n")
        for i in idx:
            f.write(f"{int(i)} {float(xs[i])!r}\n")
    print(f"dofs {n} iterations {its} relres {relres:.3e} kappa_est {kappa:.3e} kappa*relres {kappa * relres:.3e}")


if __name__ == "__main__":
    main()
