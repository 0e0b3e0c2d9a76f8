// Steady Navier-Stokes with SUPG on Taylor-Hood P2-P1 triangles (Sec. 4.3),
// linearised by Newton-Raphson (Sec. 2.1): the element residual and its
// tangent in FP64, node-centric gathers into the full-block CSR pattern, and
// the Newton loop on the device.
//
// Element form (velocity test N_a e_i, pressure test M_b = l_b):
//   r_(a,i) = int -rho (g_a . u) u_i - g_a,i p + mu g_a . grad u_i
//             + tau_m rho (g_a . u) Rm_i + tau_c g_a,i Rc
//   r_b     = int l_b Rc + tau_m grad l_b . Rm
//   Rm_i = rho u . grad u_i + d_i p - mu lap u_i,   Rc = div u,
// with g_a = grad N_a.  The tangent is the exact derivative with respect to
// the element state (velocity dof (b, j): N_b e_j; pressure dof c: l_c):
//   d grad u_i / dU_bj = delta_ij g_b,  d lap u_i / dU_bj = delta_ij lap N_b,
//   dRm_i / dU_bj = rho (N_b d_j u_i + delta_ij u . g_b) - mu delta_ij lap N_b,
//   dRm_i / dP_c = d_i l_c,   dRc / dU_bj = g_b,j.
// Integrals by a collapsed 4 x 4 Gauss-Legendre rule on the reference
// triangle (xi = s, eta = t (1 - s), weight (1 - s)), exact for polynomials
// of total degree 6: every integrand on a straight-sided element (the SUPG
// terms reach degree 6).
#include "mf_internal.h"

namespace {

// 4-point Gauss-Legendre on [0, 1]: nodes (1 -+ z) / 2 and half weights of the
// published rule on [-1, 1] (z = 0.8611363115940526, 0.3399810435848563;
// weights 0.3478548451374536, 0.6521451548625464)
__device__ __forceinline__ double gl4_x(int i)
{
    return i == 0 ? 0.06943184420297371 : i == 1 ? 0.33000947820757187 : i == 2 ? 0.6699905217924281
                                                                                  : 0.9305681557970262;
}
__device__ __forceinline__ double gl4_w(int i)
{
    return (i == 0 || i == 3) ? 0.17392742256872679 : 0.3260725774312732;
}

constexpr int NS_EPB = 4;            // elements per block, 16 threads each
constexpr int NS_PT = 62;            // doubles of per-point data
constexpr int NS_EL = 240;           // scratch words per element: r (15), K (15 x 15)

// per point: wd, N[6], g[6][2], l[3], u[2], du[2][2], Rm[2], Rc, p, adv[6],
// dRm[i][j][b] = dRm_i / dU_bj (24)
enum {
    P_WD = 0, P_N = 1, P_G = 7, P_L = 19, P_U = 22, P_DU = 24, P_RM = 28, P_RC = 30, P_P = 31, P_ADV = 32,
    P_DRM = 38
};

__global__ void __launch_bounds__(NS_EPB * 16) k_elem_ns(int64_t n_el, int64_t n2, const double *__restrict__ X,
                                                         const int32_t *__restrict__ conn,
                                                         const int32_t *__restrict__ pconn,
                                                         const double *__restrict__ x, double mu, double rho,
                                                         double tm, double tc, double *__restrict__ out,
                                                         int *status)
{
    __shared__ double pts[NS_EPB][16][NS_PT];
    __shared__ double cst[NS_EPB][12];  // gl[3][2], lap[6]
    const int le = threadIdx.x >> 4, q = threadIdx.x & 15;
    const int64_t e = (int64_t)blockIdx.x * NS_EPB + le;
    const bool valid = e < n_el;
    const int64_t ee = valid ? e : n_el - 1;
    const int32_t *cn = conn + 6 * ee;
    const int32_t *pc = pconn + 3 * ee;
    // affine map of the vertices: J = [x1 - x0, x2 - x0]; gradients of the
    // barycentrics l1 = xi, l2 = eta, l0 = 1 - xi - eta
    const double x0 = X[2 * (int64_t)cn[0]], y0 = X[2 * (int64_t)cn[0] + 1];
    const double J00 = X[2 * (int64_t)cn[1]] - x0, J10 = X[2 * (int64_t)cn[1] + 1] - y0;
    const double J01 = X[2 * (int64_t)cn[2]] - x0, J11 = X[2 * (int64_t)cn[2] + 1] - y0;
    const double det = J00 * J11 - J01 * J10;
    if (valid && q == 0 && !(det > 0.0)) mf_dev_fail(status, MF_ERR_BAD_MESH);
    const double idet = 1.0 / det;
    const double gl[3][2] = {{(J10 - J11) * idet, (J01 - J00) * idet}, {J11 * idet, -J01 * idet}, {-J10 * idet, J00 * idet}};
    constexpr int ep[3][2] = {{0, 1}, {1, 2}, {2, 0}};
    double lap[6];
#pragma unroll
    for (int v = 0; v < 3; ++v) lap[v] = 4.0 * (gl[v][0] * gl[v][0] + gl[v][1] * gl[v][1]);
#pragma unroll
    for (int k = 0; k < 3; ++k)
        lap[3 + k] = 8.0 * (gl[ep[k][0]][0] * gl[ep[k][1]][0] + gl[ep[k][0]][1] * gl[ep[k][1]][1]);
    if (q == 0) {
#pragma unroll
        for (int v = 0; v < 3; ++v) {
            cst[le][2 * v] = gl[v][0];
            cst[le][2 * v + 1] = gl[v][1];
        }
#pragma unroll
        for (int a = 0; a < 6; ++a) cst[le][6 + a] = lap[a];
    }
    // element state
    double U[6][2], P[3];
#pragma unroll
    for (int a = 0; a < 6; ++a) {
        U[a][0] = x[cn[a]];
        U[a][1] = x[n2 + cn[a]];
    }
#pragma unroll
    for (int b = 0; b < 3; ++b) P[b] = x[2 * n2 + pc[b]];
    // phase 1: thread q evaluates point q
    {
        const double s = gl4_x(q >> 2), t = gl4_x(q & 3);
        const double xi = s, eta = t * (1.0 - s);
        const double wd = gl4_w(q >> 2) * gl4_w(q & 3) * (1.0 - s) * det;
        const double l[3] = {1.0 - xi - eta, xi, eta};
        double N[6], g[6][2];
#pragma unroll
        for (int v = 0; v < 3; ++v) {
            N[v] = l[v] * (2.0 * l[v] - 1.0);
            g[v][0] = (4.0 * l[v] - 1.0) * gl[v][0];
            g[v][1] = (4.0 * l[v] - 1.0) * gl[v][1];
        }
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const int a = ep[k][0], b = ep[k][1];
            N[3 + k] = 4.0 * l[a] * l[b];
            g[3 + k][0] = 4.0 * (gl[a][0] * l[b] + l[a] * gl[b][0]);
            g[3 + k][1] = 4.0 * (gl[a][1] * l[b] + l[a] * gl[b][1]);
        }
        double u[2] = {0.0, 0.0}, du[2][2] = {{0.0, 0.0}, {0.0, 0.0}}, lu[2] = {0.0, 0.0};
#pragma unroll
        for (int a = 0; a < 6; ++a)
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                u[i] += N[a] * U[a][i];
                du[i][0] += g[a][0] * U[a][i];
                du[i][1] += g[a][1] * U[a][i];
                lu[i] += lap[a] * U[a][i];
            }
        double ph = 0.0, dp[2] = {0.0, 0.0};
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            ph += l[b] * P[b];
            dp[0] += gl[b][0] * P[b];
            dp[1] += gl[b][1] * P[b];
        }
        double *o = pts[le][q];
        o[P_WD] = wd;
#pragma unroll
        for (int a = 0; a < 6; ++a) {
            o[P_N + a] = N[a];
            o[P_G + 2 * a] = g[a][0];
            o[P_G + 2 * a + 1] = g[a][1];
            o[P_ADV + a] = g[a][0] * u[0] + g[a][1] * u[1];
        }
#pragma unroll
        for (int v = 0; v < 3; ++v) o[P_L + v] = l[v];
        o[P_U] = u[0];
        o[P_U + 1] = u[1];
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            o[P_DU + 2 * i] = du[i][0];
            o[P_DU + 2 * i + 1] = du[i][1];
            o[P_RM + i] = rho * (u[0] * du[i][0] + u[1] * du[i][1]) + dp[i] - mu * lu[i];
        }
        o[P_RC] = du[0][0] + du[1][1];
        o[P_P] = ph;
        // dRm_i / dU_bj = rho (N_b d_j u_i + delta_ij u . g_b) - mu delta_ij lap N_b
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int j = 0; j < 2; ++j)
#pragma unroll
                for (int b = 0; b < 6; ++b) {
                    const double adv_b = g[b][0] * u[0] + g[b][1] * u[1];
                    o[P_DRM + 12 * i + 6 * j + b] =
                        i == j ? rho * (N[b] * du[i][j] + adv_b) - mu * lap[b] : rho * N[b] * du[i][j];
                }
    }
    __syncthreads();
    // phase 2: thread r < 15 forms row r of the residual and the tangent
    const int r = q;
    if (!valid || r >= 15) return;
    const double *cs = cst[le];
    double res = 0.0, K[15];
#pragma unroll
    for (int c = 0; c < 15; ++c) K[c] = 0.0;
    if (r < 12) {
        const int a = r >> 1, i = r & 1;
#pragma unroll 1
        for (int p = 0; p < 16; ++p) {
            const double *o = pts[le][p];
            const double wd = o[P_WD];
            const double ga0 = o[P_G + 2 * a], ga1 = o[P_G + 2 * a + 1], gai = i ? ga1 : ga0;
            const double adv = o[P_ADV + a], ui = o[P_U + i], rmi = o[P_RM + i], rc = o[P_RC];
            res += wd * (-rho * adv * ui - gai * o[P_P] + mu * (ga0 * o[P_DU + 2 * i] + ga1 * o[P_DU + 2 * i + 1]) +
                         tm * rho * adv * rmi + tc * gai * rc);
            // K[(a,i),(b,j)] = sum_q wd [ g_a,j N_b (-rho u_i + tm rho Rm_i) + tm rho adv_a dRm_ij(b)
            //                            + tc g_a,i g_b,j + delta_ij (-rho adv_a N_b + mu g_a . g_b) ]
            const double A = wd * rho * (tm * rmi - ui);
            const double c0 = ga0 * A, c1 = ga1 * A;
            const double T4 = wd * tm * rho * adv, T5 = wd * tc * gai, B = -wd * rho * adv, Mu = wd * mu;
            const double *dR = o + P_DRM + 12 * i;
#pragma unroll
            for (int b = 0; b < 6; ++b) {
                const double Nb = o[P_N + b], gb0 = o[P_G + 2 * b], gb1 = o[P_G + 2 * b + 1];
                const double diag = B * Nb + Mu * (ga0 * gb0 + ga1 * gb1);
                K[2 * b] += c0 * Nb + T4 * dR[b] + T5 * gb0 + (i == 0 ? diag : 0.0);
                K[2 * b + 1] += c1 * Nb + T4 * dR[6 + b] + T5 * gb1 + (i == 1 ? diag : 0.0);
            }
            const double T6 = wd * gai;
#pragma unroll
            for (int c = 0; c < 3; ++c) K[12 + c] += T4 * cs[2 * c + i] - T6 * o[P_L + c];
        }
    } else {
        const int bp = r - 12;
        const double gp0 = cs[2 * bp], gp1 = cs[2 * bp + 1];
        double area = 0.0;
#pragma unroll 1
        for (int p = 0; p < 16; ++p) {
            const double *o = pts[le][p];
            const double wd = o[P_WD];
            const double lb = o[P_L + bp];
            area += wd;
            res += wd * (lb * o[P_RC] + tm * (gp0 * o[P_RM] + gp1 * o[P_RM + 1]));
            // K[b',(b,j)] = sum_q wd [ l_b' g_b,j + tm sum_i grad l_b',i dRm_ij(b) ]
            const double L = wd * lb, G0 = wd * tm * gp0, G1 = wd * tm * gp1;
            const double *dR = o + P_DRM;
#pragma unroll
            for (int b = 0; b < 6; ++b)
#pragma unroll
                for (int j = 0; j < 2; ++j)
                    K[2 * b + j] += L * o[P_G + 2 * b + j] + G0 * dR[6 * j + b] + G1 * dR[12 + 6 * j + b];
        }
        // the pressure-pressure block: tm grad l_b' . grad l_c over the element
#pragma unroll
        for (int c = 0; c < 3; ++c) K[12 + c] = area * tm * (gp0 * cs[2 * c] + gp1 * cs[2 * c + 1]);
    }
    double *w = out + e * NS_EL;
    w[r] = res;
#pragma unroll
    for (int c = 0; c < 15; ++c) w[15 + 15 * r + c] = K[c];
}

// ---------------------------------------------------------------------------
// gathers: one warp per CSR row, the row's incident elements in ascending
// order; per element lanes 0..14 add its 15 contributions at distinct
// positions of a shared-memory row (fixed order: the sums are
// bit-reproducible).  Velocity row i n2 + n (P2 node n, component i):
// positions [u1: adj0 | u2: deg0 + adj0 | p: 2 deg0 + adj1]; pressure row
// 2 n2 + m (P1 node m): [u1: adj2 | u2: deg2 + adj2 | p: 2 deg2 + adj3].
// Then d = -r and the Dirichlet elimination with increment data
// bval - x: a constrained row becomes the identity row with d = bval - x; a
// constrained column's entry moves to d as -K (bval - x).
// ---------------------------------------------------------------------------
constexpr int NG_WARPS = 8;
constexpr int NG_ROW = 3 * MF_MAX_DEG;

__device__ __forceinline__ void ns_finish_row(int64_t row, int len, double *acc, double rsum, int lane,
                                              const int64_t *__restrict__ row_ptr,
                                              const int32_t *__restrict__ col_idx,
                                              const uint8_t *__restrict__ mask, const double *__restrict__ bval,
                                              const double *__restrict__ x, double *__restrict__ values,
                                              double *__restrict__ d)
{
    const int64_t rb = row_ptr[row];
    const bool rm = mask ? mask[row] != 0 : false;
    double lift = 0.0;
    for (int k = lane; k < len; k += 32) {
        double v = acc[k];
        if (mask) {
            const int32_t col = col_idx[rb + k];
            if (rm) v = (col == row) ? 1.0 : 0.0;
            else if (mask[col]) {
                lift -= v * (bval[col] - x[col]);
                v = 0.0;
            }
        }
        values[rb + k] = v;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) lift += __shfl_xor_sync(0xffffffffu, lift, o);
    if (lane == 0) d[row] = rm ? bval[row] - x[row] : -rsum + lift;
}

__global__ void __launch_bounds__(NG_WARPS * 32) k_gather_ns_u(
    int64_t n2, const int64_t *__restrict__ p0ptr, const int64_t *__restrict__ p1ptr,
    const int64_t *__restrict__ inc_ptr, const int32_t *__restrict__ inc, const uint8_t *__restrict__ inc_loc,
    const uint8_t *__restrict__ inc_slot, const uint8_t *__restrict__ inc_slot_pq, const double *__restrict__ sc,
    const int64_t *__restrict__ row_ptr, const int32_t *__restrict__ col_idx, const uint8_t *__restrict__ mask,
    const double *__restrict__ bval, const double *__restrict__ x, double *__restrict__ values,
    double *__restrict__ d)
{
    __shared__ double acc_all[NG_WARPS][NG_ROW];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t row = (int64_t)blockIdx.x * NG_WARPS + w;
    if (row >= 2 * n2) return;  // warp-uniform
    const int i = row >= n2 ? 1 : 0;
    const int64_t n = row - i * n2;
    double *acc = acc_all[w];
    const int deg0 = (int)(p0ptr[n + 1] - p0ptr[n]), deg1 = (int)(p1ptr[n + 1] - p1ptr[n]);
    const int len = 2 * deg0 + deg1;
    for (int k = lane; k < len; k += 32) acc[k] = 0.0;
    __syncwarp();
    double rsum = 0.0;  // lane 0: the residual in element order
    for (int64_t t = inc_ptr[n]; t < inc_ptr[n + 1]; ++t) {
        const int a = inc_loc[t];
        const double *E = sc + (int64_t)inc[t] * NS_EL;
        const int r = 2 * a + i;
        if (lane < 12) {
            const int b = lane >> 1, j = lane & 1;
            acc[j * deg0 + inc_slot[t * 6 + b]] += E[15 + 15 * r + lane];
        } else if (lane < 15) {
            acc[2 * deg0 + inc_slot_pq[t * 3 + (lane - 12)]] += E[15 + 15 * r + lane];
        }
        if (lane == 0) rsum += E[r];
        __syncwarp();
    }
    ns_finish_row(row, len, acc, rsum, lane, row_ptr, col_idx, mask, bval, x, values, d);
}

__global__ void __launch_bounds__(NG_WARPS * 32) k_gather_ns_p(
    int64_t n2, int64_t n1, const int64_t *__restrict__ p2ptr, const int64_t *__restrict__ p3ptr,
    const int64_t *__restrict__ pinc_ptr, const int32_t *__restrict__ pinc, const uint8_t *__restrict__ pinc_loc,
    const uint8_t *__restrict__ pinc_slot, const uint8_t *__restrict__ pinc_slot_pp, const double *__restrict__ sc,
    const int64_t *__restrict__ row_ptr, const int32_t *__restrict__ col_idx, const uint8_t *__restrict__ mask,
    const double *__restrict__ bval, const double *__restrict__ x, double *__restrict__ values,
    double *__restrict__ d)
{
    __shared__ double acc_all[NG_WARPS][NG_ROW];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t m = (int64_t)blockIdx.x * NG_WARPS + w;
    if (m >= n1) return;  // warp-uniform
    const int64_t row = 2 * n2 + m;
    double *acc = acc_all[w];
    const int deg2 = (int)(p2ptr[m + 1] - p2ptr[m]), deg3 = (int)(p3ptr[m + 1] - p3ptr[m]);
    const int len = 2 * deg2 + deg3;
    for (int k = lane; k < len; k += 32) acc[k] = 0.0;
    __syncwarp();
    double rsum = 0.0;
    for (int64_t t = pinc_ptr[m]; t < pinc_ptr[m + 1]; ++t) {
        const int a = pinc_loc[t];
        const double *E = sc + (int64_t)pinc[t] * NS_EL;
        const int r = 12 + a;
        if (lane < 12) {
            const int b = lane >> 1, j = lane & 1;
            acc[j * deg2 + pinc_slot[t * 6 + b]] += E[15 + 15 * r + lane];
        } else if (lane < 15) {
            acc[2 * deg2 + pinc_slot_pp[t * 3 + (lane - 12)]] += E[15 + 15 * r + lane];
        }
        if (lane == 0) rsum += E[r];
        __syncwarp();
    }
    ns_finish_row(row, len, acc, rsum, lane, row_ptr, col_idx, mask, bval, x, values, d);
}

// x[g] = bval[g] on the Dirichlet dofs
__global__ void k_ns_apply_bc(int64_t n, const uint8_t *__restrict__ mask, const double *__restrict__ bval,
                              double *__restrict__ x)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && mask[i]) x[i] = bval[i];
}

// sum of squares per block (fixed order within a block; the host adds the
// block partials in order): the same bits on every run
constexpr int NR_BLOCKS = 256, NR_T = 256;
__global__ void __launch_bounds__(NR_T) k_ns_sumsq(int64_t n, const double *__restrict__ v, double *__restrict__ part)
{
    __shared__ double sh[NR_T];
    double s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * NR_T + threadIdx.x; i < n; i += (int64_t)NR_BLOCKS * NR_T) s += v[i] * v[i];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = NR_T / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void k_ns_axpy(int64_t n, const double *__restrict__ dx, double *__restrict__ x)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) x[i] += dx[i];
}

inline unsigned nsblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

mf_status mf_assemble_ns(const mf_mesh *m, const mf_pattern *p, const mf_coeffs *c, double *values, double *d,
                         cudaStream_t st)
{
    if (!p->pinc_slot_pp || !c->advect)
        return mf_fail(MF_ERR_INVALID_ARG, "mf_assemble: the Navier-Stokes form needs its pattern and the state");
    int *status = mf_status_word();
    if (!status) return mf_fail(MF_ERR_CUDA, "mf_assemble: status word unavailable");
    const int64_t ne = m->n_elems, n2 = m->n_nodes, n1 = m->n_pnodes;
    mf_prof_begin("elem_ns", st);
    if (ne > 0)
        k_elem_ns<<<nsblk(ne, NS_EPB), NS_EPB * 16, 0, st>>>(ne, n2, m->coords, m->conn, m->pconn, c->advect,
                                                             c->visc, c->rho, c->tau_m, c->tau_c, p->scratch, status);
    mf_prof_end(st);
    MF_CUDA(cudaGetLastError());
    mf_prof_begin("gather_ns", st);
    k_gather_ns_u<<<nsblk(2 * n2, NG_WARPS), NG_WARPS * 32, 0, st>>>(
        n2, p->adj[0].ptr, p->adj[1].ptr, p->inc_ptr, p->inc, p->inc_loc, p->inc_slot, p->inc_slot_pq, p->scratch,
        p->row_ptr, p->col_idx, c->bc_mask, c->bc_val, c->advect, values, d);
    if (n1 > 0)
        k_gather_ns_p<<<nsblk(n1, NG_WARPS), NG_WARPS * 32, 0, st>>>(
            n2, n1, p->adj[2].ptr, p->adj[3].ptr, p->pinc_ptr, p->pinc, p->pinc_loc, p->pinc_slot, p->pinc_slot_pp,
            p->scratch, p->row_ptr, p->col_idx, c->bc_mask, c->bc_val, c->advect, values, d);
    mf_prof_end(st);
    MF_CUDA(cudaGetLastError());
    return MF_OK;
}

// ||v||_2, deterministic (device partials, summed on the host in order)
static mf_status ns_norm(int64_t n, const double *v, double *part, cudaStream_t st, double *out)
{
    k_ns_sumsq<<<NR_BLOCKS, NR_T, 0, st>>>(n, v, part);
    MF_CUDA(cudaGetLastError());
    double h[NR_BLOCKS];
    MF_CUDA(cudaMemcpyAsync(h, part, sizeof h, cudaMemcpyDeviceToHost, st));
    MF_CUDA(cudaStreamSynchronize(st));
    double s = 0.0;
    for (int i = 0; i < NR_BLOCKS; ++i) s += h[i];
    *out = sqrt(s);
    return MF_OK;
}

mf_status mf_ns_newton_impl(const mf_mesh *m, const mf_pattern *p, const mf_coeffs *coeffs, double *x,
                            double newton_tol, int32_t max_newton, const mf_solver_opts *lin, double *hist,
                            int32_t *n_steps, cudaStream_t st)
{
    const int64_t n = p->n_rows, nnz = p->nnz;
    double *values = nullptr, *d = nullptr, *dx = nullptr, *part = nullptr;
    mf_status s = MF_OK;
    auto cleanup = [&]() {
        cudaFreeAsync(values, st);
        cudaFreeAsync(d, st);
        cudaFreeAsync(dx, st);
        cudaFreeAsync(part, st);
        cudaStreamSynchronize(st);
    };
    if (cudaMallocAsync(&values, sizeof(double) * nnz, st) != cudaSuccess ||
        cudaMallocAsync(&d, sizeof(double) * n, st) != cudaSuccess ||
        cudaMallocAsync(&dx, sizeof(double) * n, st) != cudaSuccess ||
        cudaMallocAsync(&part, sizeof(double) * NR_BLOCKS, st) != cudaSuccess) {
        cleanup();
        return mf_fail(MF_ERR_OOM, "mf_ns_newton: device allocation");
    }
    if (coeffs->bc_mask) k_ns_apply_bc<<<nsblk(n, 256), 256, 0, st>>>(n, coeffs->bc_mask, coeffs->bc_val, x);
    mf_coeffs c = *coeffs;
    c.advect = x;
    mf_csr K{n, nnz, p->row_ptr, p->col_idx, values};
    double r0 = 0.0;
    int32_t steps = 0;
    bool converged = false;
    for (int32_t k = 0;; ++k) {
        s = mf_assemble_ns(m, p, &c, values, d, st);
        if (s != MF_OK) break;
        // with x on the Dirichlet data, d holds -r on the free rows and 0 on the others
        double rn = 0.0;
        s = ns_norm(n, d, part, st, &rn);
        if (s != MF_OK) break;
        if (hist) hist[k] = rn;
        if (k == 0) r0 = rn;
        if (!isfinite(rn)) {
            s = mf_fail(MF_ERR_NONFINITE, "mf_ns_newton: non-finite residual");
            break;
        }
        if (rn <= newton_tol * fmax(1.0, r0)) {
            converged = true;
            break;
        }
        if (k >= max_newton) break;
        if (cudaMemsetAsync(dx, 0, sizeof(double) * n, st) != cudaSuccess) {
            s = mf_fail(MF_ERR_CUDA, "mf_ns_newton: memset");
            break;
        }
        mf_solve_info info{};
        s = mf_solve_impl(&K, d, dx, lin, &info, st);
        if (s != MF_OK) break;
        k_ns_axpy<<<nsblk(n, 256), 256, 0, st>>>(n, dx, x);
        ++steps;
    }
    if (n_steps) *n_steps = steps;
    cleanup();
    if (s != MF_OK) return s;
    if (!converged) return mf_fail(MF_ERR_NOT_CONVERGED, "mf_ns_newton: %d Newton steps", steps);
    return MF_OK;
}
