// Generalised-alpha time stepping of the linear conduction system with
// capacity (Sec. 2.1, Eq. time_constraints and time_effective; Blocks C and D
// of Sec. 2.2): per dof the value phi, its rate u and second rate a, with
// increments dphi, du, da tied by dphi = dt (u + b1 du), du = dt (a + b2 da).
// The residual of Block D-2 at the effective values phi~ = phi + c1 dphi,
// u~ = u + c2 du is d = F - K phi~ - M u~ (K, M positive: the paper's tangent
// negated); Block D-3's tangent is T = c1 K + c2 / (b1 dt) M.
//
// Every vector update is one elementwise kernel; the residual is one
// row-parallel pass over K and M (2 lanes per row) that also leaves per-block
// partial sums of the four norms Newton tests, summed in a fixed order in two
// levels, so a run is bit-reproducible; the tangent is one pass over
// the values with the Dirichlet rows and columns set as it goes.  The linear
// solves are the library's Jacobi-PCG.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "mf_internal.h"

namespace {

constexpr int TPB = 256;
// row kernels: lanes per row and entries per lane whose loads are in flight
// together (measured on the 128^3 Q1 system: the residual, FP64-heavier, is
// fastest with 2 x 8, the tangent with 4 x 4)
constexpr int RL = 2, RU = 8;         // residual
constexpr int TL = 4, TU = 4;         // tangent
constexpr int RPB = TPB / RL, TPBR = TPB / TL;  // rows per block

inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

// Dirichlet dofs hold phi = bc_val and u = a = 0; increments start at zero.
__global__ void k_ga_init(int64_t n, const uint8_t *__restrict__ mask, const double *__restrict__ bval, double *phi,
                          double *u, double *a, double *dphi, double *du, double *da)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (mask && mask[i]) {
        phi[i] = bval[i];
        u[i] = 0.0;
        a[i] = 0.0;
    }
    dphi[i] = du[i] = da[i] = 0.0;
}

// C-1: apply the last step's increments; with predict, C-2 (da = 0) and C-3:
// the increments that satisfy the constraints with da = 0.
__global__ void k_ga_begin(int64_t n, const uint8_t *__restrict__ mask, double *phi, double *u, double *a,
                           double *dphi, double *du, double *da, double dt, double b1, double b2, bool predict)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double p = phi[i] + dphi[i], v = u[i] + du[i], w = a[i] + da[i];
    phi[i] = p;
    u[i] = v;
    a[i] = w;
    double nda = 0.0, ndu = 0.0, ndp = 0.0;
    if (predict && !(mask && mask[i])) {
        ndu = dt * (w + b2 * nda);
        ndp = dt * (v + b1 * ndu);
    }
    da[i] = nda;
    du[i] = ndu;
    dphi[i] = ndp;
}

// D-1: the effective values
__global__ void k_ga_effective(int64_t n, const double *__restrict__ phi, const double *__restrict__ u,
                               const double *__restrict__ dphi, const double *__restrict__ du, double c1, double c2,
                               double *__restrict__ pt, double *__restrict__ ut)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    pt[i] = phi[i] + c1 * dphi[i];
    ut[i] = u[i] + c2 * du[i];
}

// fixed-order sum of v over the RL lanes of a row group
__device__ __forceinline__ double group_sum(double v)
{
#pragma unroll
    for (int o = RL / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o, RL);
    return v;
}

// D-2: d = F + R - K pt - M ut on free rows (0 on Dirichlet rows; R, the
// radiation loads at pt, may be null), one group of
// RL lanes per row and RPB rows per block, and per block the partial sums of
// d^2, (F + R)^2, (K pt)^2, (M ut)^2 over its free rows.
__global__ void __launch_bounds__(TPB) k_ga_residual(int64_t n, const int64_t *__restrict__ rp,
                                                     const int32_t *__restrict__ ci, const double *__restrict__ Kv,
                                                     const double *__restrict__ Mv, const double *__restrict__ F,
                                                     const double *__restrict__ R, const uint8_t *__restrict__ mask,
                                                     const double *__restrict__ pt, const double *__restrict__ ut,
                                                     double *__restrict__ d, double *__restrict__ part)
{
    __shared__ double sh[RPB][4];
    const int lane = threadIdx.x % RL, g = threadIdx.x / RL;
    const int64_t r = (int64_t)blockIdx.x * RPB + g;
    double kp = 0.0, mu = 0.0;
    if (r < n) {
        const int64_t t1 = rp[r + 1];
        for (int64_t tb = rp[r] + lane; tb < t1; tb += RL * RU) {
            int32_t c[RU];
            double kv[RU], mv[RU];
#pragma unroll
            for (int j = 0; j < RU; ++j) {
                const int64_t t = tb + j * RL;
                c[j] = t < t1 ? ci[t] : -1;
                kv[j] = t < t1 ? Kv[t] : 0.0;
                mv[j] = t < t1 ? Mv[t] : 0.0;
            }
#pragma unroll
            for (int j = 0; j < RU; ++j)
                if (c[j] >= 0) {
                    kp = fma(kv[j], pt[c[j]], kp);
                    mu = fma(mv[j], ut[c[j]], mu);
                }
        }
    }
    kp = group_sum(kp);
    mu = group_sum(mu);
    if (lane == 0) {
        double q[4] = {0.0, 0.0, 0.0, 0.0};
        if (r < n) {
            const bool fixed = mask && mask[r];
            const double f = R ? F[r] + R[r] : F[r];
            const double dr = fixed ? 0.0 : f - kp - mu;
            d[r] = dr;
            if (!fixed) {
                q[0] = dr * dr;
                q[1] = f * f;
                q[2] = kp * kp;
                q[3] = mu * mu;
            }
        }
        for (int k = 0; k < 4; ++k) sh[g][k] = q[k];
    }
    __syncthreads();
    if (threadIdx.x < 4) {  // fixed-order sum over the block's rows
        double s = 0.0;
        for (int j = 0; j < RPB; ++j) s += sh[j][threadIdx.x];
        part[4 * (int64_t)blockIdx.x + threadIdx.x] = s;
    }
}

// fixed-order sums of nb partial quadruples: block b adds its contiguous
// chunk of NCHUNK quadruples (thread k its k-th stride, then a fixed tree)
constexpr int NCHUNK = 4096;

__global__ void k_ga_sum4(int64_t nb, const double *__restrict__ part, double *__restrict__ out)
{
    __shared__ double sh[TPB][4];
    double s[4] = {0.0, 0.0, 0.0, 0.0};
    const int64_t b0 = (int64_t)blockIdx.x * NCHUNK, b1 = min(nb, b0 + NCHUNK);
    for (int64_t b = b0 + threadIdx.x; b < b1; b += TPB)
        for (int k = 0; k < 4; ++k) s[k] += part[4 * b + k];
    for (int k = 0; k < 4; ++k) sh[threadIdx.x][k] = s[k];
    __syncthreads();
    for (int o = TPB / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o)
            for (int k = 0; k < 4; ++k) sh[threadIdx.x][k] += sh[threadIdx.x + o][k];
        __syncthreads();
    }
    if (threadIdx.x < 4) out[4 * (int64_t)blockIdx.x + threadIdx.x] = sh[0][threadIdx.x];
}

// D-3: T = c1 K + s M, Dirichlet rows the identity, Dirichlet columns zero
// (the increments vanish there, so nothing is lifted)
__global__ void __launch_bounds__(TPB) k_ga_tangent(int64_t n, const int64_t *__restrict__ rp,
                                                    const int32_t *__restrict__ ci, const double *__restrict__ Kv,
                                                    const double *__restrict__ Mv, double c1, double s,
                                                    const uint8_t *__restrict__ mask, double *__restrict__ Tv)
{
    const int lane = threadIdx.x % TL;
    const int64_t r = (int64_t)blockIdx.x * TPBR + threadIdx.x / TL;
    if (r >= n) return;
    const bool fixed = mask && mask[r];
    const int64_t t1 = rp[r + 1];
    for (int64_t tb = rp[r] + lane; tb < t1; tb += TL * TU) {
        int32_t c[TU];
        double kv[TU], mv[TU];
        bool mc[TU];
#pragma unroll
        for (int j = 0; j < TU; ++j) {
            const int64_t t = tb + j * TL;
            c[j] = t < t1 ? ci[t] : -1;
            kv[j] = t < t1 ? Kv[t] : 0.0;
            mv[j] = t < t1 ? Mv[t] : 0.0;
        }
#pragma unroll
        for (int j = 0; j < TU; ++j) mc[j] = mask && c[j] >= 0 && mask[c[j]];
#pragma unroll
        for (int j = 0; j < TU; ++j) {
            if (c[j] < 0) continue;
            double v;
            if (fixed) v = c[j] == r ? 1.0 : 0.0;
            else if (mc[j]) v = 0.0;
            else v = fma(c1, kv[j], s * mv[j]);
            Tv[tb + j * TL] = v;
        }
    }
}

// D-4: dphi += x and the other increments from the constraints.  The host
// passes 1 / dt, 1 / b1, 1 / b2: an FP64 division costs tens of FP64
// instructions at 1/58 of the FP32 rate here.
__global__ void k_ga_correct(int64_t n, const uint8_t *__restrict__ mask, const double *__restrict__ x,
                             const double *__restrict__ u, const double *__restrict__ a, double *dphi, double *du,
                             double *da, double idt, double ib1, double ib2)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || (mask && mask[i])) return;
    const double p = dphi[i] + x[i];
    const double v = (p * idt - u[i]) * ib1;
    dphi[i] = p;
    du[i] = v;
    da[i] = (v * idt - a[i]) * ib2;
}

}  // namespace

mf_status mf_genalpha_params_from_rho_impl(double rho, mf_genalpha_params *out)
{
    // Jansen, Whiting and Hulbert (2000), first-order systems
    const double am = 0.5 * (3.0 - rho) / (1.0 + rho);
    const double af = 1.0 / (1.0 + rho);
    const double g = 0.5 + am - af;
    out->b1 = g;
    out->b2 = g;
    out->c1 = af;
    out->c2 = am;
    out->c3 = am;
    return MF_OK;
}

mf_status mf_genalpha_run_impl(const mf_csr *K, const double *Mv, const double *F, const uint8_t *mask,
                               const double *bval, const mf_facets *rad, const double *rad_es,
                               const double *rad_tenv, double *phi, double *u, double *a, const mf_genalpha_params *prm,
                               double dt, int64_t steps, double newton_tol, int32_t max_newton, double pcg_tol,
                               int64_t pcg_max_iter, int64_t *newton_its, int64_t *pcg_its, cudaStream_t st)
{
    const int64_t n = K->n_rows, nnz = K->nnz;
    const unsigned gv = nblk(n, TPB), gr = nblk(n, RPB), nc = nblk(gr, NCHUNK);
    if (nc > NCHUNK) return mf_fail(MF_ERR_UNSUPPORTED, "mf_genalpha_run: more than 2^34 rows");
    double *buf = nullptr, *Tv = nullptr, *part = nullptr, *part2 = nullptr, *norms = nullptr;
    const bool hasrad = rad && rad->n_bnodes > 0;
    MF_CUDA(cudaMallocAsync(&buf, sizeof(double) * 8 * n, st));
    double *dphi = buf, *du = buf + n, *da = buf + 2 * n, *pt = buf + 3 * n, *ut = buf + 4 * n, *d = buf + 5 * n,
           *x = buf + 6 * n, *R = hasrad ? buf + 7 * n : nullptr;
    if (hasrad && cudaMemsetAsync(R, 0, sizeof(double) * n, st) != cudaSuccess) {
        cudaFreeAsync(buf, st);
        return mf_cuda_check(cudaGetLastError(), "mf_genalpha_run");
    }
    mf_status rc = MF_OK;
    auto done = [&](mf_status s) {
        cudaFreeAsync(buf, st);
        cudaFreeAsync(Tv, st);
        cudaFreeAsync(part, st);
        cudaFreeAsync(part2, st);
        cudaFreeAsync(norms, st);
        return s;
    };
    if (cudaMallocAsync(&Tv, sizeof(double) * nnz, st) != cudaSuccess ||
        cudaMallocAsync(&part, sizeof(double) * 4 * gr, st) != cudaSuccess ||
        cudaMallocAsync(&part2, sizeof(double) * 4 * nc, st) != cudaSuccess ||
        cudaMallocAsync(&norms, sizeof(double) * 4, st) != cudaSuccess)
        return done(mf_fail(MF_ERR_OOM, "mf_genalpha_run: device allocation"));
    mf_csr T = *K;
    T.values = Tv;
    mf_solver_opts opts = {};
    opts.solver = MF_SOLVER_PCG;
    opts.tol = pcg_tol;
    opts.max_iter = pcg_max_iter;
    opts.check_every = 50;
    k_ga_init<<<gv, TPB, 0, st>>>(n, mask, bval, phi, u, a, dphi, du, da);
    if (cudaGetLastError() != cudaSuccess) return done(mf_cuda_check(cudaGetLastError(), "mf_genalpha_run"));
    const double s = prm->c2 / (prm->b1 * dt);
    for (int64_t m = 0; m < steps && rc == MF_OK; ++m) {
        k_ga_begin<<<gv, TPB, 0, st>>>(n, mask, phi, u, a, dphi, du, da, dt, prm->b1, prm->b2, true);
        double d0 = -1.0;
        int32_t it = 0;
        int64_t pits = 0;
        for (;;) {
            mf_prof_begin("ga_residual", st);
            k_ga_effective<<<gv, TPB, 0, st>>>(n, phi, u, dphi, du, prm->c1, prm->c2, pt, ut);
            if (hasrad) {
                const mf_status rs = mf_radiation_load(rad, rad_es, rad_tenv, pt, mask, R, st);
                if (rs != MF_OK) return done(rs);
            }
            k_ga_residual<<<gr, TPB, 0, st>>>(n, K->row_ptr, K->col_idx, K->values, Mv, F, R, mask, pt, ut, d, part);
            k_ga_sum4<<<nc, TPB, 0, st>>>(gr, part, part2);
            k_ga_sum4<<<1, TPB, 0, st>>>(nc, part2, norms);
            mf_prof_end(st);
            double h[4];
            if (cudaMemcpyAsync(h, norms, sizeof h, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                cudaStreamSynchronize(st) != cudaSuccess)
                return done(mf_cuda_check(cudaGetLastError(), "mf_genalpha_run"));
            const double r = sqrt(h[0]);
            if (!isfinite(r)) return done(mf_fail(MF_ERR_NONFINITE, "mf_genalpha_run: non-finite residual"));
            if (d0 < 0.0) d0 = r;
            if (r <= newton_tol * d0 || r <= 1e-13 * (sqrt(h[1]) + sqrt(h[2]) + sqrt(h[3]))) break;
            if (it == max_newton) {
                rc = mf_fail(MF_ERR_NOT_CONVERGED, "mf_genalpha_run: step %lld used %d Newton solves",
                             (long long)m, (int)max_newton);
                break;
            }
            mf_prof_begin("ga_tangent", st);
            k_ga_tangent<<<nblk(n, TPBR), TPB, 0, st>>>(n, K->row_ptr, K->col_idx, K->values, Mv, prm->c1, s, mask,
                                                        Tv);
            if (hasrad) {
                const mf_status rs = mf_radiation_tangent(rad, rad_es, pt, mask, prm->c1, Tv, st);
                if (rs != MF_OK) return done(rs);
            }
            mf_prof_end(st);
            if (cudaMemsetAsync(x, 0, sizeof(double) * n, st) != cudaSuccess)
                return done(mf_cuda_check(cudaGetLastError(), "mf_genalpha_run"));
            mf_solve_info info = {};
            const mf_status ss = mf_solve_impl(&T, d, x, &opts, &info, st);
            pits += info.iterations;
            if (ss != MF_OK) {
                rc = ss;
                break;
            }
            k_ga_correct<<<gv, TPB, 0, st>>>(n, mask, x, u, a, dphi, du, da, 1.0 / dt, 1.0 / prm->b1, 1.0 / prm->b2);
            ++it;
        }
        if (newton_its) newton_its[m] = it;
        if (pcg_its) pcg_its[m] = pits;
    }
    // C-1 of the next step: phi, u, a at t + steps dt
    k_ga_begin<<<gv, TPB, 0, st>>>(n, mask, phi, u, a, dphi, du, da, dt, prm->b1, prm->b2, false);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return done(mf_cuda_check(e, "mf_genalpha_run"));
    return done(rc);
}

mf_status mf_genalpha_initial_rate_impl(const mf_csr *K, const double *Mv, const double *F, const uint8_t *mask,
                                        const mf_facets *rad, const double *rad_es, const double *rad_tenv,
                                        const double *phi, double *u, double pcg_tol, int64_t pcg_max_iter,
                                        cudaStream_t st)
{
    // M u = F + R(phi) - K phi on the free rows, u = 0 on Dirichlet rows: the
    // residual kernel with u~ = 0 gives the right-hand side, the tangent
    // kernel with c1 = 0, s = 1 the matrix
    const int64_t n = K->n_rows, nnz = K->nnz;
    const unsigned gr = nblk(n, RPB);
    double *buf = nullptr, *Tv = nullptr, *part = nullptr;
    auto done = [&](mf_status s) {
        cudaFreeAsync(buf, st);
        cudaFreeAsync(Tv, st);
        cudaFreeAsync(part, st);
        return s;
    };
    const bool hasrad = rad && rad->n_bnodes > 0;
    if (cudaMallocAsync(&buf, sizeof(double) * 3 * n, st) != cudaSuccess ||
        cudaMallocAsync(&Tv, sizeof(double) * nnz, st) != cudaSuccess ||
        cudaMallocAsync(&part, sizeof(double) * 4 * gr, st) != cudaSuccess)
        return done(mf_fail(MF_ERR_OOM, "mf_genalpha_initial_rate: device allocation"));
    double *zero = buf, *rhs = buf + n, *R = hasrad ? buf + 2 * n : nullptr;
    if (cudaMemsetAsync(buf, 0, sizeof(double) * 3 * n, st) != cudaSuccess ||
        cudaMemsetAsync(u, 0, sizeof(double) * n, st) != cudaSuccess)
        return done(mf_cuda_check(cudaGetLastError(), "mf_genalpha_initial_rate"));
    if (hasrad) {
        const mf_status rs = mf_radiation_load(rad, rad_es, rad_tenv, phi, mask, R, st);
        if (rs != MF_OK) return done(rs);
    }
    k_ga_residual<<<gr, TPB, 0, st>>>(n, K->row_ptr, K->col_idx, K->values, Mv, F, R, mask, phi, zero, rhs, part);
    k_ga_tangent<<<nblk(n, TPBR), TPB, 0, st>>>(n, K->row_ptr, K->col_idx, K->values, Mv, 0.0, 1.0, mask, Tv);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return done(mf_cuda_check(e, "mf_genalpha_initial_rate"));
    mf_csr T = *K;
    T.values = Tv;
    mf_solver_opts opts = {};
    opts.solver = MF_SOLVER_PCG;
    opts.tol = pcg_tol;
    opts.max_iter = pcg_max_iter;
    opts.check_every = 50;
    mf_solve_info info = {};
    return done(mf_solve_impl(&T, rhs, u, &opts, &info, st));
}
