// Krylov solvers for K x = d (MetaFEM Sec. 2.2 Block D-4: "direct or
// iterative" solver, left open by the paper).
//
// Jacobi-PCG runs three kernels per iteration: q = K p with the partial sums
// of p.q; x += alpha p, r -= alpha q with the partial sums of r.D^-1 r and
// r.r; p = D^-1 r + beta p.  Each reduction is finished by the last block to
// arrive, in block order, so results are bit-reproducible and alpha, beta stay
// on the device.  A CUDA graph holds `check_every` iterations; the host reads
// the residual between replays, and kernels past convergence return at once.
//
// GMRES(m) is right preconditioned by a diagonal P: it runs on K' = K P^-1
// (columns scaled once) and returns x = P^-1 y.  Arnoldi uses classical
// Gram-Schmidt applied twice (block dot products and one multi-vector update
// per pass); the Givens rotations of the Hessenberg column run in a
// single-thread kernel, so a whole cycle stays on the device.
#include <algorithm>
#include <cmath>
#include <mutex>
#include <type_traits>

#include "mf_internal.h"

namespace {

constexpr int RT = 256;       // threads per reduction block
constexpr int RED_BLOCKS = 1024;  // fixed grid of the reduction kernels (bit-reproducible)
constexpr int VU = 4;         // vector kernels: elements a thread loads before it computes

struct PcgState {
    double rz, pq, rr, dd, tol2, alpha, beta;
    long long iter, max_iter;
    int done;         // 1 converged, 2 iteration cap, 3 breakdown / non-finite
    unsigned ticket;  // last-block counter
};

inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

// grid of the reduction kernels: a function of n only (bit-reproducible), at
// least 512 rows per block so small systems do not pay for idle blocks
inline unsigned red_grid(int64_t n)
{
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(RED_BLOCKS, (n + 511) / 512));
}

__device__ double block_sum(double v, double *sh)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[w] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += sh[i];
    return s;  // valid in thread 0
}

// true in every thread of the last block to arrive (block-uniform); the
// ticket is reset for the next launch.  Partials are written by thread 0 of
// each block before it takes a ticket.
__device__ bool last_block(unsigned *ticket)
{
    __shared__ bool last;
    __threadfence();
    if (threadIdx.x == 0) {
        const unsigned t = atomicAdd(ticket, 1u);
        last = (t == gridDim.x - 1);
        if (last) *ticket = 0;
    }
    __syncthreads();
    if (last) __threadfence();
    return last;
}

// Sums of NV interleaved partial arrays part[b * NV + v], b < nb, by the whole
// block in a fixed order (thread t adds b = t, t + blockDim, ... in turn, then
// the block tree), so the result depends on nb only.  Valid in thread 0.
template <int NV>
__device__ void finish_sums(const double *part, unsigned nb, double *out, double *sh)
{
    double acc[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) acc[v] = 0.0;
    for (unsigned b = threadIdx.x; b < nb; b += blockDim.x)
#pragma unroll
        for (int v = 0; v < NV; ++v) acc[v] += __ldcg(&part[(size_t)b * NV + v]);
#pragma unroll
    for (int v = 0; v < NV; ++v) out[v] = block_sum(acc[v], sh);
}

// ---------------------------------------------------------------------------
// SpMV: W lanes per row, U entries per lane per batch.  A lane issues the
// column and value loads of its whole batch, then the gathers of x, then the
// FMAs, so a row costs three dependent memory round trips however long it is
// (up to W * U entries per batch).
// ---------------------------------------------------------------------------

// Every lane of the warp calls the shuffles (full mask): rows past n give 0.
template <int W, int U>
__device__ __forceinline__ double row_dot(const int64_t *__restrict__ rp, const int32_t *__restrict__ ci,
                                          const double *__restrict__ v, const double *__restrict__ x, int64_t row,
                                          int sub, bool valid)
{
    double s = 0.0;
    if (valid) {
        const int64_t t1 = rp[row + 1];
        for (int64_t t = rp[row] + sub; t < t1; t += (int64_t)U * W) {
            int32_t c[U];
            double a[U], xv[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int64_t tt = t + (int64_t)u * W;
                const bool ok = tt < t1;
                c[u] = ok ? __ldcs(&ci[tt]) : -1;
                a[u] = ok ? __ldcs(&v[tt]) : 0.0;
            }
#pragma unroll
            for (int u = 0; u < U; ++u) xv[u] = c[u] >= 0 ? __ldg(&x[c[u]]) : 0.0;
#pragma unroll
            for (int u = 0; u < U; ++u) s = fma(a[u], xv[u], s);
        }
    }
#pragma unroll
    for (int o = W / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o, W);
    return s;
}

template <int W, int U>
__global__ void __launch_bounds__(RT, U <= 6 ? 5 : (U <= 12 ? 4 : 3)) k_spmv(int64_t n, const int64_t *__restrict__ rp,
                                                             const int32_t *__restrict__ ci,
                                             const double *__restrict__ v, const double *__restrict__ x,
                                             double *__restrict__ y)
{
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t row = g / W;
    const int sub = (int)(g % W);
    const bool valid = row < n;
    const double s = row_dot<W, U>(rp, ci, v, x, row, sub, valid);
    if (valid && sub == 0) y[row] = s;
}

// q = K p: one W-lane group per row over the whole matrix (no reduction here,
// so no per-block atomics on a shared ticket)
template <int W, int U>
__global__ void __launch_bounds__(RT, U <= 6 ? 5 : (U <= 12 ? 4 : 3)) k_pcg_spmv(int64_t n, const int64_t *__restrict__ rp,
                                                 const int32_t *__restrict__ ci, const double *__restrict__ v,
                                                 const double *__restrict__ p, double *__restrict__ q,
                                                 const PcgState *S)
{
    if (S->done) return;
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t row = g / W;
    const int sub = (int)(g % W);
    const bool valid = row < n;
    const double s = row_dot<W, U>(rp, ci, v, p, row, sub, valid);
    if (valid && sub == 0) q[row] = s;
}

// p.q over a grid fixed by n, finished by the last block; alpha = rz / p.q
__global__ void __launch_bounds__(RT) k_pcg_pq(int64_t n, const double *__restrict__ p, const double *__restrict__ q,
                                               double *__restrict__ part, PcgState *S)
{
    __shared__ double sh[RT / 32];
    if (S->done) return;
    double acc = 0.0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i0 < n; i0 += VU * stride) {
        double a[VU], b[VU];
#pragma unroll
        for (int u = 0; u < VU; ++u) {
            const int64_t i = i0 + u * stride;
            a[u] = i < n ? p[i] : 0.0;
            b[u] = i < n ? q[i] : 0.0;
        }
#pragma unroll
        for (int u = 0; u < VU; ++u)
            if (i0 + u * stride < n) acc = fma(a[u], b[u], acc);
    }
    const double bs = block_sum(acc, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = bs;
    if (last_block(&S->ticket)) {
        double pq;
        finish_sums<1>(part, gridDim.x, &pq, sh);
        if (threadIdx.x == 0) {
            S->pq = pq;
            if (!(pq > 0.0) || !isfinite(pq)) S->done = 3;
            else S->alpha = S->rz / pq;
        }
    }
}

// x += alpha p; r -= alpha q; partial r.D^-1 r and r.r
__global__ void __launch_bounds__(RT) k_pcg_update(int64_t n, const double *__restrict__ dinv,
                                                   const double *__restrict__ p, const double *__restrict__ q,
                                                   double *__restrict__ x, double *__restrict__ r,
                                                   double *__restrict__ part, PcgState *S)
{
    __shared__ double sh[RT / 32];
    if (S->done) return;
    const double alpha = S->alpha;
    double rz = 0.0, rr = 0.0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i0 < n; i0 += VU * stride) {
        double pv[VU], qv[VU], xv[VU], rv[VU], dv[VU];
#pragma unroll
        for (int u = 0; u < VU; ++u) {
            const int64_t i = i0 + u * stride;
            if (i < n) {
                pv[u] = p[i];
                qv[u] = q[i];
                xv[u] = x[i];
                rv[u] = r[i];
                dv[u] = dinv[i];
            }
        }
#pragma unroll
        for (int u = 0; u < VU; ++u) {
            const int64_t i = i0 + u * stride;
            if (i < n) {
                x[i] = fma(alpha, pv[u], xv[u]);
                const double ri = fma(-alpha, qv[u], rv[u]);
                r[i] = ri;
                rz = fma(ri * dv[u], ri, rz);
                rr = fma(ri, ri, rr);
            }
        }
    }
    const double bz = block_sum(rz, sh);
    const double br = block_sum(rr, sh);
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = bz;
        part[2 * blockIdx.x + 1] = br;
    }
    if (last_block(&S->ticket)) {
        double zs[2];
        finish_sums<2>(part, gridDim.x, zs, sh);
        if (threadIdx.x != 0) return;
        const double z = zs[0], s = zs[1];
        S->iter += 1;
        S->rr = s;
        if (!isfinite(s) || !isfinite(z)) S->done = 3;
        else if (s <= S->tol2 * S->dd) S->done = 1;
        else if (S->iter >= S->max_iter) S->done = 2;
        S->beta = z / S->rz;
        S->rz = z;
    }
}

// p = D^-1 r + beta p
__global__ void __launch_bounds__(RT) k_pcg_dir(int64_t n, const double *__restrict__ dinv,
                                                const double *__restrict__ r, double *__restrict__ p,
                                                const PcgState *S)
{
    if (S->done) return;
    const double beta = S->beta;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i0 < n; i0 += VU * stride) {
        double pv[VU], dv[VU], rv[VU];
#pragma unroll
        for (int u = 0; u < VU; ++u) {
            const int64_t i = i0 + u * stride;
            if (i < n) {
                pv[u] = p[i];
                dv[u] = dinv[i];
                rv[u] = r[i];
            }
        }
#pragma unroll
        for (int u = 0; u < VU; ++u) {
            const int64_t i = i0 + u * stride;
            if (i < n) p[i] = fma(beta, pv[u], dv[u] * rv[u]);
        }
    }
}

// set-up: dinv = 1 / diag(K); r = d - q (q = K x0); p = D^-1 r; rz, rr, dd
__global__ void k_diag_inv(int64_t n, const int64_t *__restrict__ rp, const int32_t *__restrict__ ci,
                           const double *__restrict__ v, double *__restrict__ dinv, int *bad)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double di = 0.0;
    for (int64_t t = rp[i]; t < rp[i + 1]; ++t)
        if (ci[t] == i) di = v[t];
    dinv[i] = 1.0 / di;
    if (!(di != 0.0) || !isfinite(di)) atomicExch(bad, 1);
}

__global__ void __launch_bounds__(RT) k_pcg_init(int64_t n, const double *__restrict__ d, const double *__restrict__ q,
                                                 const double *__restrict__ dinv, double *__restrict__ r,
                                                 double *__restrict__ p, double *__restrict__ part, PcgState *S)
{
    __shared__ double sh[RT / 32];
    double rz = 0.0, rr = 0.0, dd = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double ri = d[i] - q[i];
        r[i] = ri;
        p[i] = dinv[i] * ri;
        rz = fma(ri * dinv[i], ri, rz);
        rr = fma(ri, ri, rr);
        dd = fma(d[i], d[i], dd);
    }
    const double a = block_sum(rz, sh), b = block_sum(rr, sh), c = block_sum(dd, sh);
    if (threadIdx.x == 0) {
        part[3 * blockIdx.x] = a;
        part[3 * blockIdx.x + 1] = b;
        part[3 * blockIdx.x + 2] = c;
    }
    if (last_block(&S->ticket)) {
        double zst[3];
        finish_sums<3>(part, gridDim.x, zst, sh);
        if (threadIdx.x != 0) return;
        const double z = zst[0], s = zst[1], t = zst[2];
        S->rz = z;
        S->rr = s;
        S->dd = t;
        if (!isfinite(z) || !isfinite(s) || !isfinite(t)) S->done = 3;
        else if (s <= S->tol2 * t) S->done = 1;
        else if (S->max_iter == 0) S->done = 2;
    }
}

// ||d - K x|| / ||d|| : r_true into part-reduction; also used by GMRES
__global__ void __launch_bounds__(RT) k_resid_norm(int64_t n, const double *__restrict__ d,
                                                   const double *__restrict__ kx, double *__restrict__ part,
                                                   unsigned *ticket, double *out2 /* [2]: rr, dd */)
{
    __shared__ double sh[RT / 32];
    double rr = 0.0, dd = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double ri = d[i] - kx[i];
        rr = fma(ri, ri, rr);
        dd = fma(d[i], d[i], dd);
    }
    const double a = block_sum(rr, sh), b = block_sum(dd, sh);
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = a;
        part[2 * blockIdx.x + 1] = b;
    }
    if (last_block(ticket)) {
        double st[2];
        finish_sums<2>(part, gridDim.x, st, sh);
        if (threadIdx.x == 0) {
            out2[0] = st[0];
            out2[1] = st[1];
        }
    }
}

// SpMV shape: W lanes per row and U entries per lane per batch, the smallest
// W >= 2 (then U = 6 before 8) whose batch holds an average row: rows stay in
// one batch while a warp keeps as many rows in flight as it can
struct SpmvShape {
    int w, u;
};

SpmvShape spmv_shape(int64_t n, int64_t nnz)
{
    // Few lanes per row and many entries in flight per lane: the lanes' sum
    // costs FP64 adds (one per lane per level), and GB300 runs FP64 at 1/64
    // of the FP32 rate, so wide row groups spend the FP64 pipe on the
    // reduction.  Measured per-SpMV times (GB300): 64^3 elasticity (78.5
    // entries per row) 16 x 6: 0.241 ms, 4 x 12: 0.162 ms; 128^3 Q1 thermal
    // (26.6) 4 x 8: 0.168, 2 x 14: 0.144; Taylor-Hood 512^2 (18.8) 8 x 6:
    // 0.235, 2 x 10: 0.155; 20-node bricks 48^3 (56.5) 8 x 8: 0.092, 2 x 14:
    // 0.076; P1 512^2 (7.0): 2 x 6 0.046, 1 x 8 0.044 per PCG iteration.
    const double avg = n > 0 ? (double)nnz / (double)n : 0.0;
    if (avg <= 10.0) return {1, 8};
    if (avg <= 24.0) return {2, 10};
    if (avg <= 64.0) return {2, 14};
    if (avg <= 100.0) return {4, 12};
    if (avg <= 200.0) return {8, 12};
    if (avg <= 400.0) return {16, 12};
    return {32, 8};
}

// calls f(std::integral_constant<int, W>, std::integral_constant<int, U>)
template <typename F>
void spmv_dispatch(SpmvShape sh, F &&f)
{
    using std::integral_constant;
#define MF_SPMV_CASE(W_, U_) \
    case W_ * 16 + U_: f(integral_constant<int, W_>(), integral_constant<int, U_>()); break;
    switch (sh.w * 16 + sh.u) {
        MF_SPMV_CASE(1, 8) MF_SPMV_CASE(2, 10) MF_SPMV_CASE(2, 14) MF_SPMV_CASE(4, 12) MF_SPMV_CASE(8, 12)
        MF_SPMV_CASE(16, 12)
        default: f(integral_constant<int, 32>(), integral_constant<int, 8>()); break;
    }
#undef MF_SPMV_CASE
}

void spmv_any(const mf_csr *K, const double *v, const double *x, double *y, cudaStream_t st)
{
    spmv_dispatch(spmv_shape(K->n_rows, K->nnz), [&](auto Wc, auto Uc) {
        constexpr int W = decltype(Wc)::value, U = decltype(Uc)::value;
        k_spmv<W, U><<<nblk(K->n_rows * W, RT), RT, 0, st>>>(K->n_rows, K->row_ptr, K->col_idx, v, x, y);
    });
}

template <int W, int U>
void launch_pcg_spmv(const mf_csr *K, const double *p, double *q, double *part, PcgState *S, cudaStream_t st)
{
    k_pcg_spmv<W, U><<<nblk(K->n_rows * W, RT), RT, 0, st>>>(K->n_rows, K->row_ptr, K->col_idx, K->values, p, q, S);
    k_pcg_pq<<<red_grid(K->n_rows), RT, 0, st>>>(K->n_rows, p, q, part, S);
}

// partial slots the PCG reduction kernels need (3 per block) plus 2 outputs
inline int64_t pcg_parts(int64_t) { return 3 * RED_BLOCKS + 8; }

// ---------------------------------------------------------------------------
// GMRES kernels
// ---------------------------------------------------------------------------
struct GmState {
    double beta0, dd, tol2;
    long long iter, max_iter;
    int j;           // current Arnoldi column in the cycle
    int done;        // 1 converged, 2 cap, 3 breakdown
    int cycle_end;   // 1 when the cycle must stop (converged or j == m)
    unsigned ticket;
};

__global__ void k_recip(int64_t n, const double *__restrict__ a, double *__restrict__ b)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = 1.0 / a[i];
}

__global__ void k_scale_cols(int64_t nnz, const int32_t *__restrict__ ci, const double *__restrict__ v,
                             const double *__restrict__ pd, double *__restrict__ out)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < nnz) out[t] = v[t] / pd[ci[t]];
}

// partial dot products of w with V[0..j] (j+1 vectors), per block
__global__ void __launch_bounds__(RT) k_block_dots(int64_t n, const double *__restrict__ V, int64_t ldv,
                                                   const double *__restrict__ w, const GmState *S,
                                                   double *__restrict__ part /* [grid][m+1] */, int mp1)
{
    __shared__ double sh[RT / 32];
    if (S->cycle_end) return;
    const int j = S->j;
    for (int k = 0; k <= j; ++k) {
        double acc = 0.0;
        const double *vk = V + (int64_t)k * ldv;
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
            acc = fma(vk[i], w[i], acc);
        const double b = block_sum(acc, sh);
        if (threadIdx.x == 0) part[(int64_t)blockIdx.x * mp1 + k] = b;
    }
}

// h[k] = sum over blocks of part[.][k] (one block per k, fixed order); H column j += h (pass 2 adds)
__global__ void __launch_bounds__(RT) k_reduce_dots(int nb, const double *__restrict__ part, int mp1,
                                                    const GmState *S, double *h, double *Hcol_accum, int pass)
{
    __shared__ double sh[RT / 32];
    if (S->cycle_end) return;
    const int j = S->j;
    const int k = blockIdx.x;
    if (k > j) return;  // block-uniform
    double acc = 0.0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) acc += part[(int64_t)b * mp1 + k];
    const double s = block_sum(acc, sh);
    if (threadIdx.x == 0) {
        h[k] = s;
        Hcol_accum[k] = (pass == 0) ? s : Hcol_accum[k] + s;
    }
}

// w -= V[0..j] h
__global__ void __launch_bounds__(RT) k_multi_axpy(int64_t n, const double *__restrict__ V, int64_t ldv,
                                                   const double *__restrict__ h, const GmState *S,
                                                   double *__restrict__ w)
{
    if (S->cycle_end) return;
    const int j = S->j;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double s = w[i];
        for (int k = 0; k <= j; ++k) s = fma(-h[k], V[(int64_t)k * ldv + i], s);
        w[i] = s;
    }
}

__global__ void __launch_bounds__(RT) k_norm2(int64_t n, const double *__restrict__ w, const GmState *S,
                                              double *__restrict__ part, unsigned *ticket, double *out)
{
    __shared__ double sh[RT / 32];
    if (S->cycle_end) return;
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        acc = fma(w[i], w[i], acc);
    const double b = block_sum(acc, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = b;
    if (last_block(ticket)) {
        double s;
        finish_sums<1>(part, gridDim.x, &s, sh);
        if (threadIdx.x == 0) *out = sqrt(s);
    }
}

__global__ void __launch_bounds__(RT) k_scale_vec(int64_t n, const double *__restrict__ w, const double *nrm,
                                                  const GmState *S, double *__restrict__ out)
{
    if (S->cycle_end) return;
    const double r = 1.0 / *nrm;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = w[i] * r;
}

// Givens step on Hessenberg column j (stored H[k * m + j]); s = rotated rhs
__global__ void k_givens(int m, double *H, double *cs, double *sn, double *s, const double *hcol,
                         const double *hnext, GmState *S)
{
    if (S->cycle_end) return;
    const int j = S->j;
    for (int k = 0; k <= j; ++k) H[k * m + j] = hcol[k];
    double hj1 = *hnext;
    for (int k = 0; k < j; ++k) {
        const double a = H[k * m + j], b = H[(k + 1) * m + j];
        H[k * m + j] = cs[k] * a + sn[k] * b;
        H[(k + 1) * m + j] = -sn[k] * a + cs[k] * b;
    }
    const double a = H[j * m + j];
    const double rr = sqrt(a * a + hj1 * hj1);
    if (!(rr > 0.0) || !isfinite(rr)) {
        S->done = 3;
        S->cycle_end = 1;
        return;
    }
    cs[j] = a / rr;
    sn[j] = hj1 / rr;
    H[j * m + j] = rr;
    s[j + 1] = -sn[j] * s[j];
    s[j] = cs[j] * s[j];
    S->iter += 1;
    S->j = j + 1;
    if (s[j + 1] * s[j + 1] <= S->tol2 * S->dd) {
        S->done = 1;
        S->cycle_end = 1;
    } else if (S->j == m || S->iter >= S->max_iter) {
        if (S->iter >= S->max_iter) S->done = 2;
        S->cycle_end = 1;
    }
}

// back substitution H y = s (upper triangular j x j) into y
__global__ void k_backsolve(int m, const double *H, const double *s, double *y, const GmState *S)
{
    const int j = S->j;
    for (int k = j - 1; k >= 0; --k) {
        double t = s[k];
        for (int l = k + 1; l < j; ++l) t -= H[k * m + l] * y[l];
        y[k] = t / H[k * m + k];
    }
}

// x += P^-1 (V y)
__global__ void __launch_bounds__(RT) k_update_x(int64_t n, const double *__restrict__ V, int64_t ldv,
                                                 const double *__restrict__ y, const double *__restrict__ pd,
                                                 const GmState *S, double *__restrict__ x)
{
    const int j = S->j;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double t = 0.0;
        for (int k = 0; k < j; ++k) t = fma(V[(int64_t)k * ldv + i], y[k], t);
        x[i] += pd ? t / pd[i] : t;
    }
}

// cycle start: v0 = (d - K x) / beta, s = (beta, 0, ...)
__global__ void __launch_bounds__(RT) k_gm_start(int64_t n, const double *__restrict__ d,
                                                 const double *__restrict__ kx, double *__restrict__ v0,
                                                 double *__restrict__ part, GmState *S, double *s, int m)
{
    __shared__ double sh[RT / 32];
    double rr = 0.0, dd = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double ri = d[i] - kx[i];
        v0[i] = ri;
        rr = fma(ri, ri, rr);
        dd = fma(d[i], d[i], dd);
    }
    const double a = block_sum(rr, sh), b = block_sum(dd, sh);
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = a;
        part[2 * blockIdx.x + 1] = b;
    }
    if (last_block(&S->ticket)) {
        double tu[2];
        finish_sums<2>(part, gridDim.x, tu, sh);
        if (threadIdx.x != 0) return;
        const double t = tu[0], u = tu[1];
        S->dd = u;
        S->beta0 = sqrt(t);
        S->j = 0;
        S->cycle_end = 0;
        for (int k = 0; k <= m; ++k) s[k] = 0.0;
        s[0] = S->beta0;
        if (!isfinite(t) || !isfinite(u)) { S->done = 3; S->cycle_end = 1; }
        else if (t <= S->tol2 * u) { S->done = 1; S->cycle_end = 1; }
        else if (S->iter >= S->max_iter) { S->done = 2; S->cycle_end = 1; }
    }
}

__global__ void __launch_bounds__(RT) k_gm_norm_v0(int64_t n, double *__restrict__ v0, const GmState *S)
{
    if (S->cycle_end) return;
    const double r = 1.0 / S->beta0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        v0[i] *= r;
}

template <class T>
struct DevBuf {
    T *p = nullptr;
    cudaStream_t st;
    explicit DevBuf(cudaStream_t s) : st(s) {}
    cudaError_t alloc(size_t n) { return cudaMallocAsync(&p, sizeof(T) * (n ? n : 1), st); }
    ~DevBuf() { if (p) cudaFreeAsync(p, st); }
};

mf_status finish_status(mf_status s, int *status, cudaStream_t st)
{
    int h = 0;
    MF_CUDA(cudaMemcpyAsync(&h, status, sizeof(int), cudaMemcpyDeviceToHost, st));
    MF_CUDA(cudaStreamSynchronize(st));
    if (h) {
        const int zero = 0;
        MF_CUDA(cudaMemcpyAsync(status, &zero, sizeof(int), cudaMemcpyHostToDevice, st));
        MF_CUDA(cudaStreamSynchronize(st));
        return mf_fail((mf_status)h, "device reported status %d", h);
    }
    return s;
}

mf_status true_residual(const mf_csr *K, const double *d, const double *x, double *tmp, double *part,
                        unsigned *ticket, double *out2, cudaStream_t st, double *relres)
{
    spmv_any(K, K->values, x, tmp, st);
    k_resid_norm<<<red_grid(K->n_rows), RT, 0, st>>>(K->n_rows, d, tmp, part, ticket, out2);
    MF_CUDA(cudaGetLastError());
    double h[2];
    MF_CUDA(cudaMemcpyAsync(h, out2, sizeof h, cudaMemcpyDeviceToHost, st));
    MF_CUDA(cudaStreamSynchronize(st));
    *relres = h[1] > 0.0 ? sqrt(h[0] / h[1]) : sqrt(h[0]);
    return MF_OK;
}

mf_status solve_pcg(const mf_csr *K, const double *d, double *x, const mf_solver_opts *o, mf_solve_info *info,
                    cudaStream_t st)
{
    const int64_t n = K->n_rows;
    DevBuf<double> r(st), p(st), q(st), dinv(st), part(st);
    DevBuf<PcgState> S(st);
    DevBuf<int> bad(st);
    MF_CUDA(r.alloc(n));
    MF_CUDA(p.alloc(n));
    MF_CUDA(q.alloc(n));
    MF_CUDA(dinv.alloc(n));
    MF_CUDA(part.alloc(pcg_parts(n)));
    MF_CUDA(S.alloc(1));
    MF_CUDA(bad.alloc(1));
    PcgState h{};
    h.tol2 = o->tol * o->tol;
    h.max_iter = o->max_iter;
    MF_CUDA(cudaMemcpyAsync(S.p, &h, sizeof h, cudaMemcpyHostToDevice, st));
    MF_CUDA(cudaMemsetAsync(bad.p, 0, sizeof(int), st));
    k_diag_inv<<<nblk(n, RT), RT, 0, st>>>(n, K->row_ptr, K->col_idx, K->values, dinv.p, bad.p);
    spmv_any(K, K->values, x, q.p, st);
    k_pcg_init<<<red_grid(n), RT, 0, st>>>(n, d, q.p, dinv.p, r.p, p.p, part.p, S.p);
    MF_CUDA(cudaGetLastError());
    int hb = 0;
    MF_CUDA(cudaMemcpyAsync(&hb, bad.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    MF_CUDA(cudaStreamSynchronize(st));
    if (hb) return mf_fail(MF_ERR_NONFINITE, "mf_solve: zero or non-finite diagonal entry");

    const SpmvShape shape = spmv_shape(n, K->nnz);
    const int chunk = o->check_every > 0 ? o->check_every : 50;
    // capture `chunk` iterations in a graph on a private stream
    cudaStream_t cs;
    MF_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaError_t ce = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (ce == cudaSuccess) {
        for (int it = 0; it < chunk; ++it) {
            spmv_dispatch(shape, [&](auto Wc, auto Uc) {
                launch_pcg_spmv<decltype(Wc)::value, decltype(Uc)::value>(K, p.p, q.p, part.p, S.p, cs);
            });
            k_pcg_update<<<red_grid(n), RT, 0, cs>>>(n, dinv.p, p.p, q.p, x, r.p, part.p, S.p);
            k_pcg_dir<<<red_grid(n), RT, 0, cs>>>(n, dinv.p, r.p, p.p, S.p);
        }
        ce = cudaStreamEndCapture(cs, &graph);
    }
    if (ce == cudaSuccess) ce = cudaGraphInstantiate(&exec, graph, 0);
    if (ce != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        cudaStreamDestroy(cs);
        return mf_cuda_check(ce, "mf_solve: graph capture");
    }
    // order the private stream after the set-up work and the caller's stream after the loop
    cudaEvent_t ev;
    cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    cudaEventRecord(ev, st);
    cudaStreamWaitEvent(cs, ev, 0);
    mf_status s = MF_OK;
    for (;;) {
        MF_CUDA(cudaGraphLaunch(exec, cs));
        MF_CUDA(cudaMemcpyAsync(&h, S.p, sizeof h, cudaMemcpyDeviceToHost, cs));
        MF_CUDA(cudaStreamSynchronize(cs));
        if (h.done) break;
    }
    cudaEventRecord(ev, cs);
    cudaStreamWaitEvent(st, ev, 0);
    cudaEventDestroy(ev);
    cudaGraphExecDestroy(exec);
    cudaGraphDestroy(graph);
    cudaStreamDestroy(cs);

    double relres = 0.0;
    mf_status s2 = true_residual(K, d, x, q.p, part.p, &S.p->ticket, part.p + pcg_parts(n) - 4, st, &relres);
    if (s2 != MF_OK) return s2;
    if (info) {
        info->iterations = h.iter;
        info->rel_residual = relres;
        info->converged = h.done == 1;
    }
    if (h.done == 2) s = mf_fail(MF_ERR_NOT_CONVERGED, "mf_solve: %lld iterations, residual %.3e", h.iter, relres);
    if (h.done == 3) s = mf_fail(MF_ERR_NONFINITE, "mf_solve: breakdown or non-finite value");
    return s;
}

mf_status solve_gmres(const mf_csr *K, const double *d, double *x, const mf_solver_opts *o, mf_solve_info *info,
                      cudaStream_t st)
{
    const int64_t n = K->n_rows;
    const int m = o->restart;
    if (m > 1000) return mf_fail(MF_ERR_INVALID_ARG, "mf_solve: restart above 1000");
    DevBuf<double> V(st), w(st), kv(st), part(st), H(st), cs(st), sn(st), s(st), y(st), h(st), hcol(st), pd(st),
        nrm(st), ktmp(st);
    DevBuf<GmState> S(st);
    const int64_t ldv = n;
    MF_CUDA(V.alloc((size_t)(m + 1) * n));
    MF_CUDA(w.alloc(n));
    MF_CUDA(part.alloc((size_t)RED_BLOCKS * (m + 1) + 2 * RED_BLOCKS + 4));
    MF_CUDA(H.alloc((size_t)(m + 1) * m));
    MF_CUDA(cs.alloc(m));
    MF_CUDA(sn.alloc(m));
    MF_CUDA(s.alloc(m + 1));
    MF_CUDA(y.alloc(m));
    MF_CUDA(h.alloc(m + 1));
    MF_CUDA(hcol.alloc(m + 1));
    MF_CUDA(nrm.alloc(1));
    MF_CUDA(ktmp.alloc(K->nnz));
    MF_CUDA(S.alloc(1));
    // K' = K P^-1 (P = precond_diag or diag K)
    const double *pdiag = o->precond_diag;
    if (!pdiag) {
        MF_CUDA(pd.alloc(n));
        DevBuf<double> dinv(st);
        DevBuf<int> bad(st);
        MF_CUDA(dinv.alloc(n));
        MF_CUDA(bad.alloc(1));
        MF_CUDA(cudaMemsetAsync(bad.p, 0, sizeof(int), st));
        k_diag_inv<<<nblk(n, RT), RT, 0, st>>>(n, K->row_ptr, K->col_idx, K->values, dinv.p, bad.p);
        k_recip<<<nblk(n, RT), RT, 0, st>>>(n, dinv.p, pd.p);  // P = diag(K)
        pdiag = pd.p;
        int hb = 0;
        MF_CUDA(cudaMemcpyAsync(&hb, bad.p, sizeof(int), cudaMemcpyDeviceToHost, st));
        MF_CUDA(cudaStreamSynchronize(st));
        if (hb) return mf_fail(MF_ERR_NONFINITE, "mf_solve: zero or non-finite diagonal entry");
    }
    k_scale_cols<<<nblk(K->nnz, RT), RT, 0, st>>>(K->nnz, K->col_idx, K->values, pdiag, ktmp.p);
    mf_csr Kp = *K;
    Kp.values = ktmp.p;
    GmState hs{};
    hs.tol2 = o->tol * o->tol;
    hs.max_iter = o->max_iter;
    MF_CUDA(cudaMemcpyAsync(S.p, &hs, sizeof hs, cudaMemcpyHostToDevice, st));
    double *Vp = V.p;
    double *partB = part.p + (size_t)RED_BLOCKS * (m + 1);
    const int chunk = o->check_every > 0 ? o->check_every : 10;
    for (;;) {
        // cycle start: r = d - K x (the true residual, with the unscaled K)
        spmv_any(K, K->values, x, w.p, st);
        k_gm_start<<<RED_BLOCKS, RT, 0, st>>>(n, d, w.p, Vp, partB, S.p, s.p, m);
        k_gm_norm_v0<<<RED_BLOCKS, RT, 0, st>>>(n, Vp, S.p);
        MF_CUDA(cudaGetLastError());
        for (int j = 0; j < m; ++j) {
            // w = K' v_j
            spmv_any(&Kp, Kp.values, Vp + (int64_t)j * ldv, w.p, st);
            for (int pass = 0; pass < 2; ++pass) {
                k_block_dots<<<RED_BLOCKS, RT, 0, st>>>(n, Vp, ldv, w.p, S.p, part.p, m + 1);
                k_reduce_dots<<<m + 1, RT, 0, st>>>(RED_BLOCKS, part.p, m + 1, S.p, h.p, hcol.p, pass);
                k_multi_axpy<<<RED_BLOCKS, RT, 0, st>>>(n, Vp, ldv, h.p, S.p, w.p);
            }
            k_norm2<<<RED_BLOCKS, RT, 0, st>>>(n, w.p, S.p, partB, &S.p->ticket, nrm.p);
            k_scale_vec<<<RED_BLOCKS, RT, 0, st>>>(n, w.p, nrm.p, S.p, Vp + (int64_t)(j + 1) * ldv);
            k_givens<<<1, 1, 0, st>>>(m, H.p, cs.p, sn.p, s.p, hcol.p, nrm.p, S.p);
            MF_CUDA(cudaGetLastError());
            if ((j + 1) % chunk == 0 || j + 1 == m) {
                MF_CUDA(cudaMemcpyAsync(&hs, S.p, sizeof hs, cudaMemcpyDeviceToHost, st));
                MF_CUDA(cudaStreamSynchronize(st));
                if (hs.cycle_end) break;
            }
        }
        k_backsolve<<<1, 1, 0, st>>>(m, H.p, s.p, y.p, S.p);
        k_update_x<<<RED_BLOCKS, RT, 0, st>>>(n, Vp, ldv, y.p, pdiag, S.p, x);
        MF_CUDA(cudaGetLastError());
        MF_CUDA(cudaMemcpyAsync(&hs, S.p, sizeof hs, cudaMemcpyDeviceToHost, st));
        MF_CUDA(cudaStreamSynchronize(st));
        if (hs.done) {
            if (hs.done == 1) {
                // confirm on the true residual, else restart
                double rr = 0.0;
                mf_status t = true_residual(K, d, x, w.p, partB, &S.p->ticket, partB + 2 * RED_BLOCKS, st, &rr);
                if (t != MF_OK) return t;
                if (rr > o->tol && hs.iter < o->max_iter) {
                    hs.done = 0;
                    MF_CUDA(cudaMemcpyAsync(&S.p->done, &hs.done, sizeof(int), cudaMemcpyHostToDevice, st));
                    continue;
                }
            }
            break;
        }
    }
    double relres = 0.0;
    mf_status t = true_residual(K, d, x, w.p, partB, &S.p->ticket, partB + 2 * RED_BLOCKS, st, &relres);
    if (t != MF_OK) return t;
    if (info) {
        info->iterations = hs.iter;
        info->rel_residual = relres;
        info->converged = hs.done == 1;
    }
    if (hs.done == 2) return mf_fail(MF_ERR_NOT_CONVERGED, "mf_solve: %lld iterations, residual %.3e", hs.iter, relres);
    if (hs.done == 3) return mf_fail(MF_ERR_NONFINITE, "mf_solve: breakdown or non-finite value");
    return MF_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// Jacobi-PCG without any device allocation.
//
// For callers that cannot allocate device memory during a solve: a framework
// that reserved the whole device memory for its own pool at start-up (a
// cudaMalloc then fails or fragments that pool), or a latency-critical loop
// where cudaMalloc/cudaFree would synchronise the device.  The work vectors
// live in one file-scope __device__ array sized for MF_NOALLOC_MAX_ROWS rows;
// every GPU that loads the library holds it (about 32 MB) until the process
// exits.  All calls share the array, so calls that overlap on the GPU (other
// streams, other host threads) race and must be serialised by the caller.
// ---------------------------------------------------------------------------
namespace {
constexpr size_t NOALLOC_PART = 3 * RED_BLOCKS + 8;  // reduction block partials + 2 outputs
constexpr size_t NOALLOC_TAIL = 32;                        // PcgState + breakdown flag
constexpr size_t NOALLOC_DOUBLES = 4 * (size_t)MF_NOALLOC_MAX_ROWS + NOALLOC_PART + NOALLOC_TAIL;
static_assert(sizeof(PcgState) + sizeof(int) <= NOALLOC_TAIL * sizeof(double), "tail too small");
}  // namespace

static __device__ __align__(256) double g_noalloc_scratch[NOALLOC_DOUBLES];

namespace {
std::mutex g_noalloc_mu;
double *g_noalloc_ptr[64];

// Device address of g_noalloc_scratch for the current device (set-up once per
// device, with that device current; host code must not use the symbol itself).
mf_status noalloc_base(double **out)
{
    int dev = 0;
    MF_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return mf_fail(MF_ERR_UNSUPPORTED, "mf_solve_pcg_noalloc: device index %d", dev);
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return mf_cuda_check(e, "mf_solve_pcg_noalloc: cudaGetSymbolAddress");
        g_noalloc_ptr[dev] = static_cast<double *>(p);
    }
    *out = g_noalloc_ptr[dev];
    return MF_OK;
}
}  // namespace

extern "C" mf_status mf_solve_pcg_noalloc(const mf_csr *K, const double *d, double *x, double tol, int64_t max_iter,
                                          int32_t check_every, mf_solve_info *info, void *stream)
{
    mf_clear_error();
    if (!mf_csr_ok(K) || !d || !x)
        return mf_fail(MF_ERR_INVALID_ARG, "mf_solve_pcg_noalloc: NULL argument or an empty system");
    if (K->n_rows > MF_NOALLOC_MAX_ROWS)
        return mf_fail(MF_ERR_INVALID_ARG, "mf_solve_pcg_noalloc: %lld rows exceed MF_NOALLOC_MAX_ROWS = %d",
                       (long long)K->n_rows, MF_NOALLOC_MAX_ROWS);
    if (!(tol > 0.0) || max_iter < 0)
        return mf_fail(MF_ERR_INVALID_ARG, "mf_solve_pcg_noalloc: tol > 0, max_iter >= 0");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int *status = mf_status_word();
    if (!status) return mf_fail(MF_ERR_CUDA, "mf_solve_pcg_noalloc: status word unavailable");
    double *base = nullptr;
    mf_status s = noalloc_base(&base);
    if (s != MF_OK) return s;
    const int64_t n = K->n_rows;
    double *r = base, *p = base + MF_NOALLOC_MAX_ROWS, *q = base + 2 * (size_t)MF_NOALLOC_MAX_ROWS;
    double *dinv = base + 3 * (size_t)MF_NOALLOC_MAX_ROWS;
    double *part = base + 4 * (size_t)MF_NOALLOC_MAX_ROWS;
    PcgState *S = reinterpret_cast<PcgState *>(part + NOALLOC_PART);
    int *bad = reinterpret_cast<int *>(S + 1);

    // the array keeps the previous call's contents: reset the state and flag
    PcgState h{};
    h.tol2 = tol * tol;
    h.max_iter = max_iter;
    MF_CUDA(cudaMemcpyAsync(S, &h, sizeof h, cudaMemcpyHostToDevice, st));
    MF_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), st));
    k_diag_inv<<<nblk(n, RT), RT, 0, st>>>(n, K->row_ptr, K->col_idx, K->values, dinv, bad);
    spmv_any(K, K->values, x, q, st);
    k_pcg_init<<<red_grid(n), RT, 0, st>>>(n, d, q, dinv, r, p, part, S);
    MF_CUDA(cudaGetLastError());
    int hb = 0;
    MF_CUDA(cudaMemcpyAsync(&hb, bad, sizeof(int), cudaMemcpyDeviceToHost, st));
    MF_CUDA(cudaStreamSynchronize(st));
    if (hb) return mf_fail(MF_ERR_NONFINITE, "mf_solve_pcg_noalloc: zero or non-finite diagonal entry");

    const SpmvShape shape = spmv_shape(n, K->nnz);
    const int chunk = check_every > 0 ? check_every : 50;
    for (;;) {
        for (int it = 0; it < chunk; ++it) {
            spmv_dispatch(shape, [&](auto Wc, auto Uc) {
                launch_pcg_spmv<decltype(Wc)::value, decltype(Uc)::value>(K, p, q, part, S, st);
            });
            k_pcg_update<<<red_grid(n), RT, 0, st>>>(n, dinv, p, q, x, r, part, S);
            k_pcg_dir<<<red_grid(n), RT, 0, st>>>(n, dinv, r, p, S);
        }
        MF_CUDA(cudaGetLastError());
        MF_CUDA(cudaMemcpyAsync(&h, S, sizeof h, cudaMemcpyDeviceToHost, st));
        MF_CUDA(cudaStreamSynchronize(st));
        if (h.done) break;
    }
    double relres = 0.0;
    s = true_residual(K, d, x, q, part, &S->ticket, part + NOALLOC_PART - 4, st, &relres);
    if (s != MF_OK) return s;
    if (info) {
        info->iterations = h.iter;
        info->rel_residual = relres;
        info->converged = h.done == 1;
    }
    s = MF_OK;
    if (h.done == 2)
        s = mf_fail(MF_ERR_NOT_CONVERGED, "mf_solve_pcg_noalloc: %lld iterations, residual %.3e", h.iter, relres);
    if (h.done == 3) s = mf_fail(MF_ERR_NONFINITE, "mf_solve_pcg_noalloc: breakdown or non-finite value");
    return finish_status(s, status, st);
}

mf_status mf_spmv_impl(const mf_csr *K, const double *x, double *y, cudaStream_t st)
{
    spmv_any(K, K->values, x, y, st);
    MF_CUDA(cudaGetLastError());
    return MF_OK;
}

mf_status mf_solve_impl(const mf_csr *K, const double *d, double *x, const mf_solver_opts *o, mf_solve_info *info,
                        cudaStream_t st)
{
    int *status = mf_status_word();
    if (!status) return mf_fail(MF_ERR_CUDA, "mf_solve: status word unavailable");
    mf_status s = (o->solver == MF_SOLVER_PCG) ? solve_pcg(K, d, x, o, info, st) : solve_gmres(K, d, x, o, info, st);
    if (s == MF_ERR_CUDA || s == MF_ERR_OOM) return s;
    return finish_status(s, status, st);
}
