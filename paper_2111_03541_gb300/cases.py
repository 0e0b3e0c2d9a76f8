"""Run one workload's hot path a few times and print per-kernel device times,
for profiling (ncu, the kernel-timing hooks) without the whole benchmark.

    python -m paper_2111_03541_gb300.cases elastic --n 48 --prec mixed --reps 7
    python -m paper_2111_03541_gb300.cases thermal-grf --n 128 --reps 4 --pcg-iters 30
    python -m paper_2111_03541_gb300.cases cnn --n 129 --reps 5
    python -m paper_2111_03541_gb300.cases oseen --n 512 --reps 5
    python -m paper_2111_03541_gb300.cases batch --reps 5
    python -m paper_2111_03541_gb300.cases convection --n 128 --reps 5
    python -m paper_2111_03541_gb300.cases traction --n 64 --reps 5
    python -m paper_2111_03541_gb300.cases genalpha --n 96 --reps 3
    python -m paper_2111_03541_gb300.cases q2s --n 48 --reps 5
    python -m paper_2111_03541_gb300.cases q2s-elastic --n 48 --reps 5
    python -m paper_2111_03541_gb300.cases p2t --n 48 --reps 5

elastic: Q1 elasticity on an n^3 jittered box (gen.elastic_problem), assembled
reps times after one untimed call, then pcg-iters Jacobi-PCG iterations.  thermal-grf: Q1 thermal conduction with
k = exp(GRF) on an n^3 box (gen.grf_thermal_problem), assembled reps times,
then pcg-iters Jacobi-PCG iterations (graph of 50).  cnn: reps forward passes
of the preconditioner network on an n^3 node grid (package weights); with
--train also reps backward calls (each a forward and a backward pass,
random output gradient).  oseen:
the Taylor-Hood flow form on an n^2 grid (gen.oseen_problem), assembled reps
times.  batch: the 512-problem thermal batch (gen.batch_specs) in one graph,
default tiling, reps replays.  convection: the thermal-grf mesh with T = 0 on
x = 0 and convection (gen.convection_facets) on the other five sides, the
boundary terms added reps times.  traction: the elastic mesh with a random
stress load (gen.traction_facets) on the five sides away from the clamp.
q2s: thermal conduction on 20-node serendipity bricks (gen.thermal_q2s_problem),
assembled reps times.  q2s-elastic: linear elasticity on the same bricks
(gen.elastic_q2s_problem), assembled reps times.  p2t: thermal conduction on
quadratic tetrahedra (gen.thermal_p2t_problem: 6 n^3 elements), assembled reps
times.
genalpha: the convection case with capacity C = 1, reps generalised-alpha
steps (rho_inf = 0.5, dt = 1e-3) from T = 0 with the consistent initial rate.
Inputs are the seeded synthetic ones of `gen`; every step runs in libmf.
"""
from __future__ import annotations

import argparse
import os
import sys


def _times(mf):
    return {k: (c, round(t / c, 4)) for k, (c, t) in mf.mf_kernel_times().items()}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("case", choices=("elastic", "thermal-grf", "cnn", "oseen", "batch", "convection", "traction",
                                           "genalpha", "q2s", "q2s-elastic", "p2t"))
    ap.add_argument("--n", type=int, default=48)
    ap.add_argument("--prec", choices=("fp64", "mixed"), default="mixed")
    ap.add_argument("--reps", type=int, default=5)
    ap.add_argument("--pcg-iters", type=int, default=0)
    ap.add_argument("--train", action="store_true", help="cnn: also time forward + backward passes")
    a = ap.parse_args(argv)
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch

    import gen
    import paper_2111_03541_gb300 as mf
    if a.case == "elastic":
        P = mf.Problem(gen.elastic_problem(a.n))
        prec = mf.MF_PREC_MIXED if a.prec == "mixed" else mf.MF_PREC_FP64
        P.assemble(prec)
        torch.cuda.synchronize()
        mf.mf_set_kernel_timing(1)
        for _ in range(a.reps):
            P.assemble(prec)
        torch.cuda.synchronize()
        print("assembly", _times(mf))
        mf.mf_set_kernel_timing(0)
        if a.pcg_iters > 0:
            x, st, info = P.solve(tol=1e-12, max_iter=a.pcg_iters, check_every=50)
            torch.cuda.synchronize()
            print("pcg iterations", info.iterations, "residual", info.rel_residual)
    elif a.case in ("q2s", "q2s-elastic", "p2t"):
        P = mf.Problem(gen.thermal_q2s_problem(a.n) if a.case == "q2s"
                       else gen.elastic_q2s_problem(a.n) if a.case == "q2s-elastic" else gen.thermal_p2t_problem(a.n))
        P.assemble()
        torch.cuda.synchronize()
        mf.mf_set_kernel_timing(1)
        for _ in range(a.reps):
            P.assemble()
        torch.cuda.synchronize()
        print("assembly", _times(mf))
    elif a.case == "thermal-grf":
        P = mf.Problem(gen.grf_thermal_problem(a.n))
        P.assemble()
        torch.cuda.synchronize()
        mf.mf_set_kernel_timing(1)
        for _ in range(a.reps):
            P.assemble()
        torch.cuda.synchronize()
        print("assembly", _times(mf))
        mf.mf_set_kernel_timing(0)
        if a.pcg_iters > 0:
            x, st, info = P.solve(tol=1e-8, max_iter=a.pcg_iters, check_every=50)
            torch.cuda.synchronize()
            print("pcg iterations", info.iterations, "residual", info.rel_residual)
    elif a.case == "genalpha":
        import numpy as np
        prob = gen.grf_thermal_problem(a.n)
        left = prob["coords"][:, 0] <= 1e-14
        prob["bc_mask"] = left.astype(np.uint8)
        prob["bc_val"] = np.zeros(left.shape[0])
        prob["facets"] = gen.convection_facets(prob, ("x1", "y0", "y1", "z0", "z1"))
        P = mf.Problem(prob)
        mf.mf_assemble(P.form, P.mesh, P.pattern, P.make_coeffs(bc=False), mf.MF_PREC_FP64, P.csr, P.d)
        mf.mf_assemble_boundary(P.facets, mf.FacetCoeffs(h=P.facet_coeffs.h, t_env=P.facet_coeffs.t_env), P.csr, P.d)
        Mv = torch.empty(P.nnz, dtype=torch.float64, device="cuda")
        dz = torch.empty(P.n, dtype=torch.float64, device="cuda")
        csrM = mf.CSR(P.csr.n_rows, P.csr.nnz, P.csr.row_ptr, P.csr.col_idx, Mv.data_ptr())
        Cc = torch.ones(P.conn.shape[0], dtype=torch.float64, device="cuda")
        mf.mf_assemble(mf.MF_FORM_CAPACITY, P.mesh, P.pattern, P.make_coeffs(coef=Cc, bc=False), mf.MF_PREC_FP64,
                       csrM, dz)
        phi = torch.zeros(P.n, dtype=torch.float64, device="cuda")
        u = torch.empty_like(phi)
        acc = torch.zeros_like(phi)
        mf.mf_genalpha_initial_rate(P.csr, Mv, P.d, P.bc_mask, phi, u)
        prm = mf.mf_genalpha_params_from_rho(0.5)
        mf.mf_set_kernel_timing(1)
        st, nits, pits = mf.mf_genalpha_run(P.csr, Mv, P.d, P.bc_mask, P.bc_val, phi, u, acc, prm, 1e-3, a.reps,
                                            pcg_tol=1e-10)
        torch.cuda.synchronize()
        print("genalpha", _times(mf), "newton", nits.tolist(), "pcg", pits.tolist())
    elif a.case in ("convection", "traction"):
        import numpy as np
        sides = ("x1", "y0", "y1", "z0", "z1")
        if a.case == "convection":
            prob = gen.grf_thermal_problem(a.n)
            left = prob["coords"][:, 0] <= 1e-14
            prob["bc_mask"] = left.astype(np.uint8)
            prob["bc_val"] = np.zeros(left.shape[0])
            prob["facets"] = gen.convection_facets(prob, sides)
        else:
            prob = gen.elastic_problem(a.n)
            prob["facets"] = gen.traction_facets(prob, sides)
        P = mf.Problem(prob)
        P.assemble()
        torch.cuda.synchronize()
        mf.mf_set_kernel_timing(1)
        for _ in range(a.reps):
            mf.mf_assemble_boundary(P.facets, P.facet_coeffs, P.csr, P.d)
        torch.cuda.synchronize()
        print("boundary", _times(mf))
    elif a.case == "oseen":
        P = mf.Problem(gen.oseen_problem(a.n))
        P.assemble()
        torch.cuda.synchronize()
        mf.mf_set_kernel_timing(1)
        for _ in range(a.reps):
            P.assemble()
        torch.cuda.synchronize()
        print("assembly", _times(mf))
    elif a.case == "batch":
        Ps = [mf.Problem(gen.batch_problem(sp)) for sp in gen.batch_specs()]
        B = mf.mf_batch_create(Ps)
        mf.mf_batch_assemble(B)
        torch.cuda.synchronize()
        mf.mf_set_kernel_timing(1)
        for _ in range(a.reps):
            mf.mf_batch_assemble(B)
        torch.cuda.synchronize()
        print("batch", _times(mf))
        mf.mf_batch_destroy(B)
    else:
        from . import learned
        cnn = mf.mf_cnn_create(learned.load_params(os.path.join(os.path.dirname(os.path.abspath(__file__)), "weights",
                                                                "cnn_q1_thermal.f32")))
        nv = a.n ** 3
        g = torch.Generator(device="cuda").manual_seed(7)
        xin = torch.randn(2 * nv, device="cuda", generator=g).to(torch.bfloat16)
        y = torch.empty(nv, dtype=torch.float32, device="cuda")
        mf.mf_cnn_forward(cnn, 1, a.n, a.n, a.n, xin, y)
        torch.cuda.synchronize()
        mf.mf_set_kernel_timing(1)
        for _ in range(a.reps):
            mf.mf_cnn_forward(cnn, 1, a.n, a.n, a.n, xin, y)
        torch.cuda.synchronize()
        print("cnn forward", _times(mf))
        if a.train:
            gy = torch.randn(nv, device="cuda", generator=g)
            mf.mf_set_kernel_timing(0)
            mf.mf_cnn_backward(cnn, 1, a.n, a.n, a.n, xin, gy)
            torch.cuda.synchronize()
            mf.mf_set_kernel_timing(1)
            for _ in range(a.reps):  # the backward call runs its own forward pass first
                mf.mf_cnn_backward(cnn, 1, a.n, a.n, a.n, xin, gy)
            torch.cuda.synchronize()
            print("cnn forward + backward", _times(mf))
        mf.mf_cnn_destroy(cnn)
    mf.mf_set_kernel_timing(0)


if __name__ == "__main__":
    main()
