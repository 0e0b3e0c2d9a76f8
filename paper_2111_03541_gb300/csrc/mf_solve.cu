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

// FP32 SpMV shape (the refinement's inner solve): the lanes' sum costs FP32
// adds only, so W grows until one batch holds an average row (fewer
// dependent round trips per row).  64^3 elasticity (78.5 entries per row),
// 2,779 inner iterations: 8 x 12 0.353 s, 4 x 12 0.376 s.
SpmvShape spmv_shape32(int64_t n, int64_t nnz)
{
    const double avg = n > 0 ? (double)nnz / (double)n : 0.0;
    if (avg <= 8.0) return {1, 8};
    if (avg <= 20.0) return {2, 10};
    if (avg <= 28.0) return {2, 14};
    if (avg <= 48.0) return {4, 12};
    if (avg <= 96.0) return {8, 12};
    if (avg <= 192.0) return {16, 12};
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
        info->refinements = 0;
    }
    if (h.done == 2) s = mf_fail(MF_ERR_NOT_CONVERGED, "mf_solve: %lld iterations, residual %.3e", h.iter, relres);
    if (h.done == 3) s = mf_fail(MF_ERR_NONFINITE, "mf_solve: breakdown or non-finite value");
    return s;
}

// ---------------------------------------------------------------------------
// FP64 iterative refinement around an FP32 Jacobi-PCG (the mixed path's
// solve): the outer residual r = d - K x uses the FP64 K; each correction
// K32 z = r / ||r|| is solved in FP32 (values and vectors) to a relative
// residual inner_tol, and x += ||r|| z in FP64.  The refinement converges to
// K^-1 d as long as kappa(K) 2^-24 stays well below 1.
// ---------------------------------------------------------------------------
template <int W, int U>
__device__ __forceinline__ float row_dot32(const int64_t *__restrict__ rp, const int32_t *__restrict__ ci,
                                           const float *__restrict__ v, const float *__restrict__ x, int64_t row,
                                           int sub, bool valid)
{
    float s = 0.f;
    if (valid) {
        const int64_t t1 = rp[row + 1];
        for (int64_t t = rp[row] + sub; t < t1; t += (int64_t)U * W) {
            int32_t c[U];
            float a[U], xv[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int64_t tt = t + (int64_t)u * W;
                const bool ok = tt < t1;
                c[u] = ok ? __ldcs(&ci[tt]) : -1;
                a[u] = ok ? __ldcs(&v[tt]) : 0.f;
            }
#pragma unroll
            for (int u = 0; u < U; ++u) xv[u] = c[u] >= 0 ? __ldg(&x[c[u]]) : 0.f;
#pragma unroll
            for (int u = 0; u < U; ++u) s = fmaf(a[u], xv[u], s);
        }
    }
#pragma unroll
    for (int o = W / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o, W);
    return s;
}

template <int W, int U>
__global__ void __launch_bounds__(RT) k_pcg32_spmv(int64_t n, const int64_t *__restrict__ rp,
                                                   const int32_t *__restrict__ ci, const float *__restrict__ v,
                                                   const float *__restrict__ p, float *__restrict__ q,
                                                   const PcgState *S)
{
    if (S->done) return;
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t row = g / W;
    const int sub = (int)(g % W);
    const bool valid = row < n;
    const float s = row_dot32<W, U>(rp, ci, v, p, row, sub, valid);
    if (valid && sub == 0) q[row] = s;
}

__global__ void __launch_bounds__(RT) k_pcg32_pq(int64_t n, const float *__restrict__ p, const float *__restrict__ q,
                                                 double *__restrict__ part, PcgState *S)
{
    __shared__ double sh[RT / 32];
    if (S->done) return;
    float acc = 0.f;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        acc = fmaf(p[i], q[i], acc);
    const double bs = block_sum((double)acc, sh);
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

__global__ void __launch_bounds__(RT) k_pcg32_update(int64_t n, const float *__restrict__ dinv,
                                                     const float *__restrict__ p, const float *__restrict__ q,
                                                     float *__restrict__ x, float *__restrict__ r,
                                                     double *__restrict__ part, PcgState *S)
{
    __shared__ double sh[RT / 32];
    if (S->done) return;
    const float alpha = (float)S->alpha;
    float rz = 0.f, rr = 0.f;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        x[i] = fmaf(alpha, p[i], x[i]);
        const float ri = fmaf(-alpha, q[i], r[i]);
        r[i] = ri;
        rz = fmaf(ri * dinv[i], ri, rz);
        rr = fmaf(ri, ri, rr);
    }
    const double bz = block_sum((double)rz, sh);
    const double br = block_sum((double)rr, sh);
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = bz;
        part[2 * blockIdx.x + 1] = br;
    }
    if (last_block(&S->ticket)) {
        double zs[2];
        finish_sums<2>(part, gridDim.x, zs, sh);
        if (threadIdx.x != 0) return;
        const double z = zs[0], s2 = zs[1];
        S->iter += 1;
        S->rr = s2;
        if (!isfinite(s2) || !isfinite(z)) S->done = 3;
        else if (s2 <= S->tol2 * S->dd) S->done = 1;
        else if (S->iter >= S->max_iter) S->done = 2;
        S->beta = z / S->rz;
        S->rz = z;
    }
}

__global__ void __launch_bounds__(RT) k_pcg32_dir(int64_t n, const float *__restrict__ dinv,
                                                  const float *__restrict__ r, float *__restrict__ p,
                                                  const PcgState *S)
{
    if (S->done) return;
    const float beta = (float)S->beta;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = fmaf(beta, p[i], dinv[i] * r[i]);
}

// K32 = float(K), dinv32 = 1 / diag(K) (rounded once)
__global__ void k_to_f32(int64_t m, const double *__restrict__ a, float *__restrict__ b)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m) b[i] = (float)a[i];
}

// r = d - K x (FP64) with the partial sums of r.r and d.d; b = r / ||r|| is
// formed by the next kernel once the norm is known
__global__ void __launch_bounds__(RT) k_ref_resid(int64_t n, const double *__restrict__ d,
                                                  const double *__restrict__ kx, double *__restrict__ r,
                                                  double *__restrict__ part, unsigned *ticket, double *out2)
{
    __shared__ double sh[RT / 32];
    double rr = 0.0, dd = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double ri = d[i] - kx[i];
        r[i] = ri;
        rr = fma(ri, ri, rr);
        dd = fma(d[i], d[i], dd);
    }
    const double a = block_sum(rr, sh), b = block_sum(dd, sh);
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = a;
        part[2 * blockIdx.x + 1] = b;
    }
    if (last_block(ticket)) {
        double st2[2];
        finish_sums<2>(part, gridDim.x, st2, sh);
        if (threadIdx.x == 0) {
            out2[0] = st2[0];
            out2[1] = st2[1];
        }
    }
}

// inner start: b = r / ||r||, z = 0, rr = D^-1 b, p = D^-1 b; rz, rr, dd (= b.b)
__global__ void __launch_bounds__(RT) k_ref_start(int64_t n, const double *__restrict__ r, double inv_nrm,
                                                  const float *__restrict__ dinv, float *__restrict__ z,
                                                  float *__restrict__ ri, float *__restrict__ p,
                                                  double *__restrict__ part, PcgState *S)
{
    __shared__ double sh[RT / 32];
    float rz = 0.f, rr = 0.f;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float b = (float)(r[i] * inv_nrm);
        z[i] = 0.f;
        ri[i] = b;
        p[i] = dinv[i] * b;
        rz = fmaf(b * dinv[i], b, rz);
        rr = fmaf(b, b, rr);
    }
    const double a = block_sum((double)rz, sh), c = block_sum((double)rr, sh);
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = a;
        part[2 * blockIdx.x + 1] = c;
    }
    if (last_block(&S->ticket)) {
        double zs[2];
        finish_sums<2>(part, gridDim.x, zs, sh);
        if (threadIdx.x != 0) return;
        S->rz = zs[0];
        S->rr = zs[1];
        S->dd = zs[1];
        S->iter = 0;
        S->done = (!isfinite(zs[0]) || !isfinite(zs[1])) ? 3 : 0;
    }
}

// x += s z (FP64 update of the outer iterate)
__global__ void k_ref_update(int64_t n, double s, const float *__restrict__ z, double *__restrict__ x)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) x[i] = fma(s, (double)z[i], x[i]);
}

template <int W, int U>
void launch_pcg32_iter(const mf_csr *K, const float *v32, const float *dinv, float *z, float *r, float *p,
                       float *q, double *part, PcgState *S, cudaStream_t st)
{
    const int64_t n = K->n_rows;
    k_pcg32_spmv<W, U><<<nblk(n * W, RT), RT, 0, st>>>(n, K->row_ptr, K->col_idx, v32, p, q, S);
    k_pcg32_pq<<<red_grid(n), RT, 0, st>>>(n, p, q, part, S);
    k_pcg32_update<<<red_grid(n), RT, 0, st>>>(n, dinv, p, q, z, r, part, S);
    k_pcg32_dir<<<red_grid(n), RT, 0, st>>>(n, dinv, r, p, S);
}

mf_status solve_refined(const mf_csr *K, const double *d, double *x, const mf_solver_opts *o, mf_solve_info *info,
                        cudaStream_t st)
{
    const int64_t n = K->n_rows, nnz = K->nnz;
    const double inner_tol = o->inner_tol > 0.0 ? o->inner_tol : 1e-4;
    DevBuf<double> r64(st), kx(st), part(st), dinv64(st), out2(st);
    DevBuf<float> v32(st), dinv(st), z(st), r(st), p(st), q(st);
    DevBuf<PcgState> S(st);
    DevBuf<int> bad(st);
    MF_CUDA(r64.alloc(n));
    MF_CUDA(kx.alloc(n));
    MF_CUDA(part.alloc(pcg_parts(n)));
    MF_CUDA(dinv64.alloc(n));
    MF_CUDA(out2.alloc(2));
    MF_CUDA(v32.alloc(nnz));
    MF_CUDA(dinv.alloc(n));
    MF_CUDA(z.alloc(n));
    MF_CUDA(r.alloc(n));
    MF_CUDA(p.alloc(n));
    MF_CUDA(q.alloc(n));
    MF_CUDA(S.alloc(1));
    MF_CUDA(bad.alloc(1));
    MF_CUDA(cudaMemsetAsync(bad.p, 0, sizeof(int), st));
    MF_CUDA(cudaMemsetAsync(S.p, 0, sizeof(PcgState), st));
    k_diag_inv<<<nblk(n, RT), RT, 0, st>>>(n, K->row_ptr, K->col_idx, K->values, dinv64.p, bad.p);
    k_to_f32<<<nblk(n, RT), RT, 0, st>>>(n, dinv64.p, dinv.p);
    k_to_f32<<<nblk(nnz, RT), RT, 0, st>>>(nnz, K->values, v32.p);
    MF_CUDA(cudaGetLastError());
    int hb = 0;
    MF_CUDA(cudaMemcpyAsync(&hb, bad.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    MF_CUDA(cudaStreamSynchronize(st));
    if (hb) return mf_fail(MF_ERR_NONFINITE, "mf_solve: zero or non-finite diagonal entry");
    const SpmvShape shape = spmv_shape32(n, nnz);
    const int chunk = o->check_every > 0 ? o->check_every : 50;
    int64_t inner_total = 0, refinements = 0;
    double relres = 0.0, prev = 0.0;
    int stall = 0;  // refinements in a row that did not halve the residual
    int done = 0;   // 1 converged, 2 cap, 3 breakdown, 4 stagnated
    for (;;) {
        spmv_any(K, K->values, x, kx.p, st);
        k_ref_resid<<<red_grid(n), RT, 0, st>>>(n, d, kx.p, r64.p, part.p, &S.p->ticket, out2.p);
        MF_CUDA(cudaGetLastError());
        double h2[2];
        MF_CUDA(cudaMemcpyAsync(h2, out2.p, sizeof h2, cudaMemcpyDeviceToHost, st));
        MF_CUDA(cudaStreamSynchronize(st));
        const double rn = sqrt(h2[0]);
        relres = h2[1] > 0.0 ? rn / sqrt(h2[1]) : rn;
        if (!isfinite(relres)) { done = 3; break; }
        if (relres <= o->tol || rn == 0.0) { done = 1; break; }
        if (inner_total >= o->max_iter) { done = 2; break; }
        // the FP64 residual of a system has a rounding floor: below it the
        // corrections no longer reduce it, and the loop stops
        stall = (refinements > 0 && relres > 0.5 * prev) ? stall + 1 : 0;
        if (stall >= 3) { done = 4; break; }
        prev = relres;
        // inner FP32 Jacobi-PCG on K32 z = r / ||r|| from z = 0
        PcgState hs{};
        hs.tol2 = inner_tol * inner_tol;
        hs.max_iter = o->max_iter - inner_total;
        MF_CUDA(cudaMemcpyAsync(S.p, &hs, sizeof hs, cudaMemcpyHostToDevice, st));
        k_ref_start<<<red_grid(n), RT, 0, st>>>(n, r64.p, 1.0 / rn, dinv.p, z.p, r.p, p.p, part.p, S.p);
        MF_CUDA(cudaGetLastError());
        for (;;) {
            for (int it = 0; it < chunk; ++it)
                spmv_dispatch(shape, [&](auto Wc, auto Uc) {
                    launch_pcg32_iter<decltype(Wc)::value, decltype(Uc)::value>(K, v32.p, dinv.p, z.p, r.p, p.p,
                                                                                 q.p, part.p, S.p, st);
                });
            MF_CUDA(cudaGetLastError());
            MF_CUDA(cudaMemcpyAsync(&hs, S.p, sizeof hs, cudaMemcpyDeviceToHost, st));
            MF_CUDA(cudaStreamSynchronize(st));
            if (hs.done) break;
        }
        inner_total += hs.iter;
        if (hs.done == 3) { done = 3; break; }
        k_ref_update<<<nblk(n, RT), RT, 0, st>>>(n, rn, z.p, x);
        ++refinements;
    }
    if (info) {
        info->iterations = inner_total;
        info->rel_residual = relres;
        info->converged = done == 1;
        info->refinements = refinements;
    }
    if (done == 2)
        return mf_fail(MF_ERR_NOT_CONVERGED, "mf_solve: %lld inner iterations, residual %.3e", (long long)inner_total,
                       relres);
    if (done == 3) return mf_fail(MF_ERR_NONFINITE, "mf_solve: breakdown or non-finite value");
    if (done == 4)
        return mf_fail(MF_ERR_NOT_CONVERGED,
                       "mf_solve: refinement stagnated at residual %.3e after %lld refinements (the rounding floor "
                       "of the FP64 residual lies above the tolerance)",
                       relres, (long long)refinements);
    return MF_OK;
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
        info->refinements = 0;
    }
    if (hs.done == 2) return mf_fail(MF_ERR_NOT_CONVERGED, "mf_solve: %lld iterations, residual %.3e", hs.iter, relres);
    if (hs.done == 3) return mf_fail(MF_ERR_NONFINITE, "mf_solve: breakdown or non-finite value");
    return MF_OK;
}

// ---------------------------------------------------------------------------
// Flow system (Sec. 4.3 Picard form, Taylor-Hood P2-P1, [u1 | u2 | p]):
// right-preconditioned GMRES(m) with the block upper-triangular
//   M = [ A  B^T ]      M^-1 [v_u; v_p]:  z_p = S^-1 v_p,
//       [ 0   S  ]                       z_u = A^-1 (v_u - B^T z_p),
// S = diag(M_p) / nu (the pressure mass scaled by the viscosity, a spectrally
// equivalent stand-in for the Schur complement B A^-1 B^T of a viscous flow),
// and A^-1 (the same matrix for u1 and u2) replaced by one geometric
// multigrid V-cycle over the structured P2 grids of the hierarchy: damped
// Jacobi smoothing, P2 interpolation to the finer grid and its transpose
// back, operators rediscretised by the caller (its assembly on each grid).
// The preconditioner is a fixed linear operator, so plain right-
// preconditioned GMRES applies.
// ---------------------------------------------------------------------------

// rows [0, nv) of K restricted to columns < nv: entry counts, then the fill
__global__ void k_block_count(int64_t nv, const int64_t *__restrict__ rp, const int32_t *__restrict__ ci,
                              int64_t *__restrict__ cnt)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nv) return;
    int64_t c = 0;
    for (int64_t t = rp[i]; t < rp[i + 1]; ++t) c += ci[t] < nv;
    cnt[i] = c;
}
__global__ void k_block_fill(int64_t nv, const int64_t *__restrict__ rp, const int32_t *__restrict__ ci,
                             const double *__restrict__ v, const int64_t *__restrict__ orp, int32_t *__restrict__ oci,
                             double *__restrict__ ov)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nv) return;
    int64_t o = orp[i];
    for (int64_t t = rp[i]; t < rp[i + 1]; ++t)
        if (ci[t] < nv) {
            oci[o] = ci[t];
            ov[o] = v[t];
            ++o;
        }
}

// P2 interpolation from the grid of nc cells per side to the grid of 2 nc
// (the split-square Taylor-Hood meshes: P2 nodes on the (2n + 1)^2 lattice,
// x fastest; cell (i, j) split by its diagonal into (v00, v10, v11) and
// (v00, v11, v01)).  Fine node (fi, fj) sits at (fi / 4, fj / 4) in coarse
// cell units; row of P: the 6 coarse P2 basis values there (vertices
// l (2 l - 1), edge midpoints 4 la lb), columns ascending.
__global__ void k_p2_prolong(int64_t nc, int64_t *__restrict__ prp, int32_t *__restrict__ pci,
                             double *__restrict__ pv)
{
    const int64_t nfs = 4 * nc + 1;  // fine lattice side
    const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= nfs * nfs) return;
    const int64_t fi = id % nfs, fj = id / nfs;
    int64_t ic = fi / 4, jc = fj / 4;
    if (ic == nc) ic = nc - 1;
    if (jc == nc) jc = nc - 1;
    const double xi = 0.25 * (double)(fi - 4 * ic), eta = 0.25 * (double)(fj - 4 * jc);
    const int64_t ncs = 2 * nc + 1;  // coarse lattice side
    auto node = [&](int64_t a, int64_t b) { return (int32_t)((2 * jc + b) * ncs + 2 * ic + a); };
    int32_t c[6];
    double l0, l1, l2;
    if (xi >= eta) {  // (v00, v10, v11)
        l0 = 1.0 - xi; l1 = xi - eta; l2 = eta;
        c[0] = node(0, 0); c[1] = node(2, 0); c[2] = node(2, 2);
        c[3] = node(1, 0); c[4] = node(2, 1); c[5] = node(1, 1);
    } else {          // (v00, v11, v01)
        l0 = 1.0 - eta; l1 = xi; l2 = eta - xi;
        c[0] = node(0, 0); c[1] = node(2, 2); c[2] = node(0, 2);
        c[3] = node(1, 1); c[4] = node(1, 2); c[5] = node(0, 1);
    }
    double w[6] = {l0 * (2.0 * l0 - 1.0), l1 * (2.0 * l1 - 1.0), l2 * (2.0 * l2 - 1.0), 4.0 * l0 * l1, 4.0 * l1 * l2,
                   4.0 * l2 * l0};
    for (int a = 1; a < 6; ++a)  // ascending columns
        for (int b = a; b > 0 && c[b - 1] > c[b]; --b) {
            const int32_t tc = c[b]; c[b] = c[b - 1]; c[b - 1] = tc;
            const double tw = w[b]; w[b] = w[b - 1]; w[b - 1] = tw;
        }
    prp[id] = 6 * id;
    if (id == 0) prp[nfs * nfs] = 6 * nfs * nfs;
    for (int a = 0; a < 6; ++a) {
        pci[6 * id + a] = c[a];
        pv[6 * id + a] = w[a];
    }
}

// R = P^T: counts per column, then entries by an atomic cursor, then each
// row sorted by column (so the result does not depend on the atomics' order)
__global__ void k_tr_count(int64_t nnz, const int32_t *__restrict__ ci, int64_t *__restrict__ cnt)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < nnz) atomicAdd(reinterpret_cast<unsigned long long *>(cnt + ci[t]), 1ull);
}
__global__ void k_tr_fill(int64_t nrows, const int64_t *__restrict__ rp, const int32_t *__restrict__ ci,
                          const double *__restrict__ v, const int64_t *__restrict__ trp, int64_t *__restrict__ cur,
                          int32_t *__restrict__ tci, double *__restrict__ tv)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nrows) return;
    for (int64_t t = rp[i]; t < rp[i + 1]; ++t) {
        const int64_t o = trp[ci[t]] + (int64_t)atomicAdd(reinterpret_cast<unsigned long long *>(cur + ci[t]), 1ull);
        tci[o] = (int32_t)i;
        tv[o] = v[t];
    }
}
__global__ void k_tr_sort(int64_t n, const int64_t *__restrict__ trp, int32_t *__restrict__ tci,
                          double *__restrict__ tv)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int64_t a = trp[i] + 1; a < trp[i + 1]; ++a)
        for (int64_t b = a; b > trp[i] && tci[b - 1] > tci[b]; --b) {
            const int32_t c = tci[b]; tci[b] = tci[b - 1]; tci[b - 1] = c;
            const double w = tv[b]; tv[b] = tv[b - 1]; tv[b - 1] = w;
        }
}

// sum of squares, finished by the last block
__global__ void __launch_bounds__(RT) k_sumsq(int64_t n, const double *__restrict__ x, double *__restrict__ part,
                                              unsigned *ticket, double *out)
{
    __shared__ double sh[RT / 32];
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        acc = fma(x[i], x[i], acc);
    const double b = block_sum(acc, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = b;
    if (last_block(ticket)) {
        double s;
        finish_sums<1>(part, gridDim.x, &s, sh);
        if (threadIdx.x == 0) *out = s;
    }
}

__global__ void k_fill_pattern(int64_t n, double *__restrict__ x)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) x[i] = 1.0 + 0.125 * (double)(i % 7) - 0.0625 * (double)(i % 5);
}
__global__ void k_scale_into(int64_t n, const double *__restrict__ a, const double *__restrict__ b, double s,
                             double *__restrict__ out)  // out = s a b
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = s * a[i] * b[i];
}
// damped Jacobi step x += w D^-1 (b - A x) (t = A x); constrained rows x = b
__global__ void k_scal(int64_t n, double s, const double *__restrict__ a, double *__restrict__ out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = s * a[i];
}
__global__ void k_jacobi(int64_t n, const double *__restrict__ b, const double *__restrict__ t,
                         const double *__restrict__ dinv, const uint8_t *__restrict__ mask, double w,
                         double *__restrict__ x)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    x[i] = mask[i] ? b[i] : fma(w * dinv[i], b[i] - t[i], x[i]);
}
// first sweep from x = 0
__global__ void k_jacobi0(int64_t n, const double *__restrict__ b, const double *__restrict__ dinv,
                          const uint8_t *__restrict__ mask, double w, double *__restrict__ x)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) x[i] = mask[i] ? b[i] : w * dinv[i] * b[i];
}
// r = b - t elementwise; r may be t (the flow preconditioner forms its
// velocity right-hand side in place), so neither is declared restrict
__global__ void k_resid(int64_t n, const double *__restrict__ b, const double *t, double *r)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) r[i] = b[i] - t[i];
}
__global__ void k_zero_masked(int64_t n, const uint8_t *__restrict__ mask, double *__restrict__ x)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && mask[i]) x[i] = 0.0;
}
__global__ void k_add_unmasked(int64_t n, const uint8_t *__restrict__ mask, const double *__restrict__ t,
                               double *__restrict__ x)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && !mask[i]) x[i] += t[i];
}
// block-triangular pieces: w = [0; 0; S^-1 v_p], rhs_u = v_u - (K w)_u
__global__ void k_bt_pressure(int64_t nu, int64_t np, const double *__restrict__ v, const double *__restrict__ sinv,
                              double *__restrict__ w)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nu) w[i] = 0.0;
    else if (i < nu + np) w[i] = sinv[i - nu] * v[i];
}
// S^-1 = nu / Mp on pressure dofs, 1 on constrained ones
__global__ void k_sinv(int64_t n1, const double *__restrict__ pmass, const uint8_t *__restrict__ pmask, double nu,
                       double *__restrict__ sinv)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n1) sinv[i] = (pmask && pmask[i]) ? 1.0 : nu / pmass[i];
}
__global__ void k_axpy_vec(int64_t n, const double *__restrict__ a, double *__restrict__ x)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) x[i] += a[i];
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
        info->refinements = 0;
    }
    s = MF_OK;
    if (h.done == 2)
        s = mf_fail(MF_ERR_NOT_CONVERGED, "mf_solve_pcg_noalloc: %lld iterations, residual %.3e", h.iter, relres);
    if (h.done == 3) s = mf_fail(MF_ERR_NONFINITE, "mf_solve_pcg_noalloc: breakdown or non-finite value");
    return finish_status(s, status, st);
}

// ---------------------------------------------------------------------------
// Flow multigrid hierarchy (see the kernels above)
// ---------------------------------------------------------------------------
namespace {
constexpr int MG_MAX_LEVELS = 12;
struct MgLevel {
    int64_t n = 0, cells = 0;  // velocity dofs of one component (P2 nodes), grid cells per side
    mf_csr A{};                // the u1-u1 block (equal to the u2-u2 block)
    double *dinv = nullptr;
    double omega = 0.0;        // Jacobi damping 4 / (3 lambda_max(D^-1 A))
    uint8_t *mask = nullptr;   // constrained nodes
    mf_csr P{}, R{};           // to the next coarser level: P (n x n_coarse) and R = P^T
    double *x = nullptr, *b = nullptr, *r = nullptr, *t = nullptr;
};
}  // namespace

struct mf_flow_mg {
    int levels = 0;
    MgLevel L[MG_MAX_LEVELS];
    int64_t n2 = 0, n1 = 0;       // finest: velocity nodes, pressure nodes
    double *sinv = nullptr;       // [n1]: nu / Mp (1 on a constrained pressure dof)
    double *w = nullptr, *kw = nullptr;  // [2 n2 + n1] work of the block solve
    double *part = nullptr, *scal = nullptr;
    unsigned *ticket = nullptr;
    int pre = 2, post = 2, coarse = 60;
};

namespace {
void mg_free_csr(mf_csr &A)
{
    cudaFree(const_cast<int64_t *>(A.row_ptr));
    cudaFree(const_cast<int32_t *>(A.col_idx));
    cudaFree(A.values);
    A = mf_csr{};
}

mf_status mg_transpose(const mf_csr &P, int64_t ncols, mf_csr &R, cudaStream_t st)
{
    int64_t *trp = nullptr, *cur = nullptr;
    int32_t *tci = nullptr;
    double *tv = nullptr;
    MF_CUDA(cudaMallocAsync(&trp, sizeof(int64_t) * (ncols + 1), st));
    MF_CUDA(cudaMallocAsync(&cur, sizeof(int64_t) * ncols, st));
    MF_CUDA(cudaMallocAsync(&tci, sizeof(int32_t) * P.nnz, st));
    MF_CUDA(cudaMallocAsync(&tv, sizeof(double) * P.nnz, st));
    MF_CUDA(cudaMemsetAsync(trp, 0, sizeof(int64_t) * (ncols + 1), st));
    MF_CUDA(cudaMemsetAsync(cur, 0, sizeof(int64_t) * ncols, st));
    k_tr_count<<<nblk(P.nnz, RT), RT, 0, st>>>(P.nnz, P.col_idx, trp);
    MF_CUDA(mf_scan_i64(trp, ncols + 1, nullptr, st));
    k_tr_fill<<<nblk(P.n_rows, RT), RT, 0, st>>>(P.n_rows, P.row_ptr, P.col_idx, P.values, trp, cur, tci, tv);
    k_tr_sort<<<nblk(ncols, RT), RT, 0, st>>>(ncols, trp, tci, tv);
    MF_CUDA(cudaGetLastError());
    MF_CUDA(cudaFreeAsync(cur, st));
    R = mf_csr{ncols, P.nnz, trp, tci, tv};
    return MF_OK;
}

// one V-cycle for A x = b on level l (b, x given for level 0, own vectors below)
void mg_vcycle(mf_flow_mg &G, int l, const double *b, double *x, cudaStream_t st)
{
    MgLevel &L = G.L[l];
    const unsigned g = nblk(L.n, RT);
    const int sweeps = (l == G.levels - 1) ? G.coarse : G.pre;
    k_jacobi0<<<g, RT, 0, st>>>(L.n, b, L.dinv, L.mask, L.omega, x);
    for (int s = 1; s < sweeps; ++s) {
        spmv_any(&L.A, L.A.values, x, L.t, st);
        k_jacobi<<<g, RT, 0, st>>>(L.n, b, L.t, L.dinv, L.mask, L.omega, x);
    }
    if (l == G.levels - 1) return;
    MgLevel &C = G.L[l + 1];
    spmv_any(&L.A, L.A.values, x, L.t, st);
    k_resid<<<g, RT, 0, st>>>(L.n, b, L.t, L.r);
    spmv_any(&L.R, L.R.values, L.r, C.b, st);
    k_zero_masked<<<nblk(C.n, RT), RT, 0, st>>>(C.n, C.mask, C.b);
    mg_vcycle(G, l + 1, C.b, C.x, st);
    spmv_any(&L.P, L.P.values, C.x, L.t, st);
    k_add_unmasked<<<g, RT, 0, st>>>(L.n, L.mask, L.t, x);
    for (int s = 0; s < G.post; ++s) {
        spmv_any(&L.A, L.A.values, x, L.t, st);
        k_jacobi<<<g, RT, 0, st>>>(L.n, b, L.t, L.dinv, L.mask, L.omega, x);
    }
}

// z = M^-1 v for the block upper-triangular M (K: the finest flow system)
void flow_bt_apply(mf_flow_mg &G, const mf_csr *K, const double *v, double *z, cudaStream_t st)
{
    const int64_t nu = 2 * G.n2, nr = nu + G.n1;
    k_bt_pressure<<<nblk(nr, RT), RT, 0, st>>>(nu, G.n1, v, G.sinv, G.w);
    spmv_any(K, K->values, G.w, G.kw, st);
    k_resid<<<nblk(nu, RT), RT, 0, st>>>(nu, v, G.kw, G.kw);  // rhs_u = v_u - (K w)_u
    mg_vcycle(G, 0, G.kw, z, st);
    mg_vcycle(G, 0, G.kw + G.n2, z + G.n2, st);
    cudaMemcpyAsync(z + nu, G.w + nu, sizeof(double) * G.n1, cudaMemcpyDeviceToDevice, st);
}

mf_status solve_gmres_flow(const mf_csr *K, const double *d, double *x, const mf_solver_opts *o, mf_solve_info *info,
                           cudaStream_t st)
{
    mf_flow_mg &G = *const_cast<mf_flow_mg *>(o->flow_mg);
    const int64_t n = K->n_rows;
    if (n != 2 * G.n2 + G.n1) return mf_fail(MF_ERR_INVALID_ARG, "mf_solve: system does not match the hierarchy");
    const int m = o->restart;
    if (m > 1000) return mf_fail(MF_ERR_INVALID_ARG, "mf_solve: restart above 1000");
    DevBuf<double> V(st), w(st), zb(st), tb(st), part(st), H(st), cs(st), sn(st), s(st), y(st), h(st), hcol(st),
        nrm(st);
    DevBuf<GmState> S(st);
    const int64_t ldv = n;
    MF_CUDA(V.alloc((size_t)(m + 1) * n));
    MF_CUDA(w.alloc(n));
    MF_CUDA(zb.alloc(n));
    MF_CUDA(tb.alloc(n));
    MF_CUDA(part.alloc((size_t)RED_BLOCKS * (m + 1) + 2 * RED_BLOCKS + 4));
    MF_CUDA(H.alloc((size_t)(m + 1) * m));
    MF_CUDA(cs.alloc(m));
    MF_CUDA(sn.alloc(m));
    MF_CUDA(s.alloc(m + 1));
    MF_CUDA(y.alloc(m));
    MF_CUDA(h.alloc(m + 1));
    MF_CUDA(hcol.alloc(m + 1));
    MF_CUDA(nrm.alloc(1));
    MF_CUDA(S.alloc(1));
    GmState hs{};
    hs.tol2 = o->tol * o->tol;
    hs.max_iter = o->max_iter;
    MF_CUDA(cudaMemcpyAsync(S.p, &hs, sizeof hs, cudaMemcpyHostToDevice, st));
    double *Vp = V.p;
    double *partB = part.p + (size_t)RED_BLOCKS * (m + 1);
    for (;;) {
        spmv_any(K, K->values, x, w.p, st);
        k_gm_start<<<RED_BLOCKS, RT, 0, st>>>(n, d, w.p, Vp, partB, S.p, s.p, m);
        k_gm_norm_v0<<<RED_BLOCKS, RT, 0, st>>>(n, Vp, S.p);
        MF_CUDA(cudaGetLastError());
        MF_CUDA(cudaMemcpyAsync(&hs, S.p, sizeof hs, cudaMemcpyDeviceToHost, st));
        MF_CUDA(cudaStreamSynchronize(st));
        if (!hs.cycle_end)
            for (int j = 0; j < m; ++j) {
                // w = K M^-1 v_j
                flow_bt_apply(G, K, Vp + (int64_t)j * ldv, zb.p, st);
                spmv_any(K, K->values, zb.p, w.p, st);
                for (int pass = 0; pass < 2; ++pass) {
                    k_block_dots<<<RED_BLOCKS, RT, 0, st>>>(n, Vp, ldv, w.p, S.p, part.p, m + 1);
                    k_reduce_dots<<<m + 1, RT, 0, st>>>(RED_BLOCKS, part.p, m + 1, S.p, h.p, hcol.p, pass);
                    k_multi_axpy<<<RED_BLOCKS, RT, 0, st>>>(n, Vp, ldv, h.p, S.p, w.p);
                }
                k_norm2<<<RED_BLOCKS, RT, 0, st>>>(n, w.p, S.p, partB, &S.p->ticket, nrm.p);
                k_scale_vec<<<RED_BLOCKS, RT, 0, st>>>(n, w.p, nrm.p, S.p, Vp + (int64_t)(j + 1) * ldv);
                k_givens<<<1, 1, 0, st>>>(m, H.p, cs.p, sn.p, s.p, hcol.p, nrm.p, S.p);
                MF_CUDA(cudaGetLastError());
                MF_CUDA(cudaMemcpyAsync(&hs, S.p, sizeof hs, cudaMemcpyDeviceToHost, st));
                MF_CUDA(cudaStreamSynchronize(st));
                if (hs.cycle_end) break;
            }
        // x += M^-1 (V y)
        k_backsolve<<<1, 1, 0, st>>>(m, H.p, s.p, y.p, S.p);
        MF_CUDA(cudaMemsetAsync(tb.p, 0, sizeof(double) * n, st));
        k_update_x<<<RED_BLOCKS, RT, 0, st>>>(n, Vp, ldv, y.p, nullptr, S.p, tb.p);
        flow_bt_apply(G, K, tb.p, zb.p, st);
        k_axpy_vec<<<nblk(n, RT), RT, 0, st>>>(n, zb.p, x);
        MF_CUDA(cudaGetLastError());
        MF_CUDA(cudaMemcpyAsync(&hs, S.p, sizeof hs, cudaMemcpyDeviceToHost, st));
        MF_CUDA(cudaStreamSynchronize(st));
        if (hs.done) {
            if (hs.done == 1) {
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
        info->refinements = 0;
    }
    if (hs.done == 2) return mf_fail(MF_ERR_NOT_CONVERGED, "mf_solve: %lld iterations, residual %.3e", hs.iter, relres);
    if (hs.done == 3) return mf_fail(MF_ERR_NONFINITE, "mf_solve: breakdown or non-finite value");
    return MF_OK;
}
}  // namespace

mf_status mf_flow_mg_create_impl(int levels, const mf_csr *const *K, const int64_t *cells,
                                 const uint8_t *const *bc_mask, const double *pmass, double visc, cudaStream_t st,
                                 mf_flow_mg **out)
{
    mf_flow_mg *G = new (std::nothrow) mf_flow_mg();
    if (!G) return mf_fail(MF_ERR_OOM, "mf_flow_mg_create: host allocation");
    auto fail = [&](mf_status s) {
        mf_flow_mg_destroy_impl(G);
        return s;
    };
    G->levels = levels;
    for (int l = 0; l < levels; ++l) {
        const int64_t side = 2 * cells[l] + 1, n2 = side * side;
        if (K[l]->n_rows <= 2 * n2 || (l > 0 && cells[l - 1] != 2 * cells[l]) || cells[l] < 1)
            return fail(mf_fail(MF_ERR_INVALID_ARG, "mf_flow_mg_create: level %d does not halve the grid of level "
                                                   "%d or does not match its system", l, l - 1));
        MgLevel &L = G->L[l];
        L.n = n2;
        L.cells = cells[l];
        int64_t *rp = nullptr;
        MF_CUDA(cudaMallocAsync(&rp, sizeof(int64_t) * (n2 + 1), st));
        MF_CUDA(cudaMemsetAsync(rp + n2, 0, sizeof(int64_t), st));
        k_block_count<<<nblk(n2, RT), RT, 0, st>>>(n2, K[l]->row_ptr, K[l]->col_idx, rp);
        MF_CUDA(mf_scan_i64(rp, n2 + 1, nullptr, st));
        int64_t nnz = 0;
        MF_CUDA(cudaMemcpyAsync(&nnz, rp + n2, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
        MF_CUDA(cudaStreamSynchronize(st));
        int32_t *ci = nullptr;
        double *v = nullptr;
        MF_CUDA(cudaMallocAsync(&ci, sizeof(int32_t) * nnz, st));
        MF_CUDA(cudaMallocAsync(&v, sizeof(double) * nnz, st));
        k_block_fill<<<nblk(n2, RT), RT, 0, st>>>(n2, K[l]->row_ptr, K[l]->col_idx, K[l]->values, rp, ci, v);
        L.A = mf_csr{n2, nnz, rp, ci, v};
        MF_CUDA(cudaMallocAsync(&L.dinv, sizeof(double) * n2, st));
        MF_CUDA(cudaMallocAsync(&L.mask, n2, st));
        MF_CUDA(cudaMemcpyAsync(L.mask, bc_mask[l], n2, cudaMemcpyDeviceToDevice, st));
        for (double **p : {&L.x, &L.b, &L.r, &L.t}) MF_CUDA(cudaMallocAsync(p, sizeof(double) * n2, st));
        int *bad = nullptr;
        MF_CUDA(cudaMallocAsync(&bad, sizeof(int), st));
        MF_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), st));
        k_diag_inv<<<nblk(n2, RT), RT, 0, st>>>(n2, rp, ci, v, L.dinv, bad);
        int hb = 0;
        MF_CUDA(cudaMemcpyAsync(&hb, bad, sizeof(int), cudaMemcpyDeviceToHost, st));
        MF_CUDA(cudaFreeAsync(bad, st));
        MF_CUDA(cudaStreamSynchronize(st));
        if (hb) return fail(mf_fail(MF_ERR_NONFINITE, "mf_flow_mg_create: zero diagonal in level %d", l));
    }
    // lambda_max of D^-1 A per level (power iteration, 24 steps) -> omega
    MF_CUDA(cudaMallocAsync(&G->part, sizeof(double) * (RED_BLOCKS + 8), st));
    MF_CUDA(cudaMallocAsync(&G->scal, sizeof(double) * 2, st));
    MF_CUDA(cudaMallocAsync(&G->ticket, sizeof(unsigned), st));
    MF_CUDA(cudaMemsetAsync(G->ticket, 0, sizeof(unsigned), st));
    for (int l = 0; l < levels; ++l) {
        MgLevel &L = G->L[l];
        const unsigned g = nblk(L.n, RT);
        k_fill_pattern<<<g, RT, 0, st>>>(L.n, L.x);
        double lam = 1.0;
        for (int it = 0; it < 24; ++it) {
            double h2[2];
            k_sumsq<<<red_grid(L.n), RT, 0, st>>>(L.n, L.x, G->part, G->ticket, G->scal);
            spmv_any(&L.A, L.A.values, L.x, L.t, st);
            k_scale_into<<<g, RT, 0, st>>>(L.n, L.t, L.dinv, 1.0, L.r);  // r = D^-1 A x
            k_sumsq<<<red_grid(L.n), RT, 0, st>>>(L.n, L.r, G->part, G->ticket, G->scal + 1);
            MF_CUDA(cudaMemcpyAsync(h2, G->scal, sizeof h2, cudaMemcpyDeviceToHost, st));
            MF_CUDA(cudaStreamSynchronize(st));
            if (!(h2[0] > 0.0) || !(h2[1] > 0.0) || !std::isfinite(h2[1])) break;
            lam = sqrt(h2[1] / h2[0]);
            k_scal<<<g, RT, 0, st>>>(L.n, 1.0 / sqrt(h2[1]), L.r, L.x);  // x = r / ||r||
        }
        L.omega = 4.0 / (3.0 * lam);
    }
    // transfers
    for (int l = 0; l + 1 < levels; ++l) {
        MgLevel &L = G->L[l], &C = G->L[l + 1];
        const int64_t nf = L.n;
        int64_t *prp = nullptr;
        int32_t *pci = nullptr;
        double *pv = nullptr;
        MF_CUDA(cudaMallocAsync(&prp, sizeof(int64_t) * (nf + 1), st));
        MF_CUDA(cudaMallocAsync(&pci, sizeof(int32_t) * 6 * nf, st));
        MF_CUDA(cudaMallocAsync(&pv, sizeof(double) * 6 * nf, st));
        k_p2_prolong<<<nblk(nf, RT), RT, 0, st>>>(C.cells, prp, pci, pv);
        L.P = mf_csr{nf, 6 * nf, prp, pci, pv};
        mf_status s = mg_transpose(L.P, C.n, L.R, st);
        if (s != MF_OK) return fail(s);
    }
    // Schur stand-in and work vectors of the finest system
    G->n2 = G->L[0].n;
    G->n1 = K[0]->n_rows - 2 * G->n2;
    MF_CUDA(cudaMallocAsync(&G->sinv, sizeof(double) * G->n1, st));
    MF_CUDA(cudaMallocAsync(&G->w, sizeof(double) * K[0]->n_rows, st));
    MF_CUDA(cudaMallocAsync(&G->kw, sizeof(double) * K[0]->n_rows, st));
    k_sinv<<<nblk(G->n1, RT), RT, 0, st>>>(G->n1, pmass, bc_mask[0] + 2 * G->n2, visc, G->sinv);
    MF_CUDA(cudaGetLastError());
    MF_CUDA(cudaStreamSynchronize(st));
    *out = G;
    return MF_OK;
}

void mf_flow_mg_destroy_impl(mf_flow_mg *G)
{
    if (!G) return;
    for (int l = 0; l < G->levels; ++l) {
        MgLevel &L = G->L[l];
        mg_free_csr(L.A);
        mg_free_csr(L.P);
        mg_free_csr(L.R);
        cudaFree(L.dinv);
        cudaFree(L.mask);
        cudaFree(L.x);
        cudaFree(L.b);
        cudaFree(L.r);
        cudaFree(L.t);
    }
    cudaFree(G->sinv);
    cudaFree(G->w);
    cudaFree(G->kw);
    cudaFree(G->part);
    cudaFree(G->scal);
    cudaFree(G->ticket);
    delete G;
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
    if (info) info->refinements = 0;
    mf_status s = (o->solver == MF_SOLVER_PCG)       ? solve_pcg(K, d, x, o, info, st)
                  : (o->solver == MF_SOLVER_GMRES)   ? solve_gmres(K, d, x, o, info, st)
                  : (o->solver == MF_SOLVER_GMRES_FLOW_MG) ? solve_gmres_flow(K, d, x, o, info, st)
                                                     : solve_refined(K, d, x, o, info, st);
    if (s == MF_ERR_CUDA || s == MF_ERR_OOM) return s;
    return finish_status(s, status, st);
}
