// Steady Navier-Stokes with SUPG on Taylor-Hood P2-P1 triangles (Sec. 4.3),
// linearised by Newton-Raphson (Sec. 2.1): the element residual and its
// tangent in double-float (FP32 pairs, about 47 bits: FP32 runs at 64 times
// the FP64 rate on GB300), node-centric gathers into the full-block CSR
// pattern in FP64, and the Newton loop on the device.
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
#include "mf_fem.cuh"

namespace {

__device__ __forceinline__ float2 dfma2(float2 a, float2 b, float2 c) { return df_add(df_mul(a, b), c); }
__device__ __forceinline__ float2 dsub2(float2 a, float2 b) { return df_add(a, df_neg(b)); }

// 4-point Gauss-Legendre on [0, 1]: nodes (1 -+ z) / 2 and half weights of the
// published rule on [-1, 1] (z = 0.8611363115940526, 0.3399810435848563;
// weights 0.3478548451374536, 0.6521451548625464)
__device__ __forceinline__ float2 gl4_x(int i)
{
    return i == 0 ? DFC(0.06943184420297371)
                  : i == 1 ? DFC(0.33000947820757187) : i == 2 ? DFC(0.6699905217924281) : DFC(0.9305681557970262);
}
__device__ __forceinline__ float2 gl4_w(int i)
{
    return (i == 0 || i == 3) ? DFC(0.17392742256872679) : DFC(0.3260725774312732);
}

constexpr int NS_EPB = 4;            // elements per block, 16 threads each
constexpr int NS_PT = 62;            // pairs of per-point data
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
                                                         const double *__restrict__ x, double mu_d, double rho_d,
                                                         double tm_d, double tc_d, double *__restrict__ out,
                                                         int *status)
{
    __shared__ float2 pts[NS_EPB][16][NS_PT];
    __shared__ float2 cst[NS_EPB][12];  // gl[3][2], lap[6]
    const int le = threadIdx.x >> 4, q = threadIdx.x & 15;
    const int64_t e = (int64_t)blockIdx.x * NS_EPB + le;
    const bool valid = e < n_el;
    const int64_t ee = valid ? e : n_el - 1;
    const int32_t *cn = conn + 6 * ee;
    const int32_t *pc = pconn + 3 * ee;
    const float2 mu = f64_to_df(mu_d), rho = f64_to_df(rho_d), tm = f64_to_df(tm_d), tc = f64_to_df(tc_d);
    const float2 one = make_float2(1.f, 0.f), two = make_float2(2.f, 0.f), four = make_float2(4.f, 0.f);
    // affine map of the vertices: J = [x1 - x0, x2 - x0] (differences in FP64,
    // then pairs); gradients of the barycentrics l1 = xi, l2 = eta, l0 = 1 - xi - eta
    const double x0 = X[2 * (int64_t)cn[0]], y0 = X[2 * (int64_t)cn[0] + 1];
    const double J00d = X[2 * (int64_t)cn[1]] - x0, J10d = X[2 * (int64_t)cn[1] + 1] - y0;
    const double J01d = X[2 * (int64_t)cn[2]] - x0, J11d = X[2 * (int64_t)cn[2] + 1] - y0;
    if (valid && q == 0 && !(J00d * J11d - J01d * J10d > 0.0)) mf_dev_fail(status, MF_ERR_BAD_MESH);
    const float2 J00 = f64_to_df(J00d), J10 = f64_to_df(J10d), J01 = f64_to_df(J01d), J11 = f64_to_df(J11d);
    const float2 det = df_det2(J00, J11, J01, J10);
    const float2 idet = df_recip(det);
    const float2 gl[3][2] = {{df_mul(dsub2(J10, J11), idet), df_mul(dsub2(J01, J00), idet)},
                             {df_mul(J11, idet), df_neg(df_mul(J01, idet))},
                             {df_neg(df_mul(J10, idet)), df_mul(J00, idet)}};
    constexpr int ep[3][2] = {{0, 1}, {1, 2}, {2, 0}};
    float2 lap[6];
#pragma unroll
    for (int v = 0; v < 3; ++v)
        lap[v] = df_mul(four, dfma2(gl[v][0], gl[v][0], df_mul(gl[v][1], gl[v][1])));
#pragma unroll
    for (int k = 0; k < 3; ++k)
        lap[3 + k] = df_mul(make_float2(8.f, 0.f), dfma2(gl[ep[k][0]][0], gl[ep[k][1]][0],
                                                         df_mul(gl[ep[k][0]][1], gl[ep[k][1]][1])));
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
    float2 U[6][2], P[3];
#pragma unroll
    for (int a = 0; a < 6; ++a) {
        U[a][0] = f64_to_df(x[cn[a]]);
        U[a][1] = f64_to_df(x[n2 + cn[a]]);
    }
#pragma unroll
    for (int b = 0; b < 3; ++b) P[b] = f64_to_df(x[2 * n2 + pc[b]]);
    // phase 1: thread q evaluates point q
    {
        const float2 s = gl4_x(q >> 2), t = gl4_x(q & 3);
        const float2 oms = dsub2(one, s);
        const float2 xi = s, eta = df_mul(t, oms);
        const float2 wd = df_mul(df_mul(df_mul(gl4_w(q >> 2), gl4_w(q & 3)), oms), det);
        const float2 l[3] = {dsub2(dsub2(one, xi), eta), xi, eta};
        float2 N[6], g[6][2];
#pragma unroll
        for (int v = 0; v < 3; ++v) {
            N[v] = df_mul(l[v], dsub2(df_mul(two, l[v]), one));
            const float2 f = dsub2(df_mul(four, l[v]), one);
            g[v][0] = df_mul(f, gl[v][0]);
            g[v][1] = df_mul(f, gl[v][1]);
        }
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const int a = ep[k][0], b = ep[k][1];
            N[3 + k] = df_mul(four, df_mul(l[a], l[b]));
            g[3 + k][0] = df_mul(four, dfma2(gl[a][0], l[b], df_mul(l[a], gl[b][0])));
            g[3 + k][1] = df_mul(four, dfma2(gl[a][1], l[b], df_mul(l[a], gl[b][1])));
        }
        const float2 z = make_float2(0.f, 0.f);
        float2 u[2] = {z, z}, du[2][2] = {{z, z}, {z, z}}, lu[2] = {z, z};
#pragma unroll
        for (int a = 0; a < 6; ++a)
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                u[i] = dfma2(N[a], U[a][i], u[i]);
                du[i][0] = dfma2(g[a][0], U[a][i], du[i][0]);
                du[i][1] = dfma2(g[a][1], U[a][i], du[i][1]);
                lu[i] = dfma2(lap[a], U[a][i], lu[i]);
            }
        float2 ph = z, dp[2] = {z, z};
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            ph = dfma2(l[b], P[b], ph);
            dp[0] = dfma2(gl[b][0], P[b], dp[0]);
            dp[1] = dfma2(gl[b][1], P[b], dp[1]);
        }
        float2 *o = pts[le][q];
        o[P_WD] = wd;
        float2 adv[6];
#pragma unroll
        for (int a = 0; a < 6; ++a) {
            adv[a] = dfma2(g[a][0], u[0], df_mul(g[a][1], u[1]));
            o[P_N + a] = N[a];
            o[P_G + 2 * a] = g[a][0];
            o[P_G + 2 * a + 1] = g[a][1];
            o[P_ADV + a] = adv[a];
        }
#pragma unroll
        for (int v = 0; v < 3; ++v) o[P_L + v] = l[v];
        o[P_U] = u[0];
        o[P_U + 1] = u[1];
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            o[P_DU + 2 * i] = du[i][0];
            o[P_DU + 2 * i + 1] = du[i][1];
            // Rm_i = rho (u . grad u_i) + d_i p - mu lap u_i
            o[P_RM + i] = dsub2(df_add(df_mul(rho, dfma2(u[0], du[i][0], df_mul(u[1], du[i][1]))), dp[i]),
                                df_mul(mu, lu[i]));
        }
        o[P_RC] = df_add(du[0][0], du[1][1]);
        o[P_P] = ph;
        // dRm_i / dU_bj = rho (N_b d_j u_i + delta_ij u . g_b) - mu delta_ij lap N_b
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int j = 0; j < 2; ++j)
#pragma unroll
                for (int b = 0; b < 6; ++b)
                    o[P_DRM + 12 * i + 6 * j + b] =
                        i == j ? dsub2(df_mul(rho, dfma2(N[b], du[i][j], adv[b])), df_mul(mu, lap[b]))
                               : df_mul(rho, df_mul(N[b], du[i][j]));
    }
    __syncthreads();
    // phase 2: thread r < 12 forms velocity row r = (a, i) of the residual and
    // the tangent and also column (a, i) of the three pressure rows (so the
    // warps do not run the pressure rows' loop after the velocity rows');
    // thread 12 + b' forms the pressure residual r_b' and the row's p-p block
    const int r = q;
    if (!valid || r >= 15) return;
    const float2 *cs = cst[le];
    const float2 z = make_float2(0.f, 0.f);
    float2 res = z, K[15], Kp[3] = {z, z, z};
#pragma unroll
    for (int c = 0; c < 15; ++c) K[c] = z;
    const float2 rtm = df_mul(rho, tm);
    double *w = out + e * NS_EL;
    if (r < 12) {
        const int a = r >> 1, i = r & 1;
        // pressure rows' gradients times tau_m
        float2 tg[3][2];
#pragma unroll
        for (int bp = 0; bp < 3; ++bp) {
            tg[bp][0] = df_mul(tm, cs[2 * bp]);
            tg[bp][1] = df_mul(tm, cs[2 * bp + 1]);
        }
#pragma unroll 1
        for (int p = 0; p < 16; ++p) {
            const float2 *o = pts[le][p];
            const float2 wd = o[P_WD];
            const float2 ga0 = o[P_G + 2 * a], ga1 = o[P_G + 2 * a + 1], gai = i ? ga1 : ga0;
            const float2 adv = o[P_ADV + a], ui = o[P_U + i], rmi = o[P_RM + i], rc = o[P_RC];
            // -rho adv u_i - g_a,i p + mu (g_a . grad u_i) + tau_m rho adv Rm_i + tau_c g_a,i Rc
            float2 tt = df_neg(df_mul(rho, df_mul(adv, ui)));
            tt = dsub2(tt, df_mul(gai, o[P_P]));
            tt = dfma2(mu, dfma2(ga0, o[P_DU + 2 * i], df_mul(ga1, o[P_DU + 2 * i + 1])), tt);
            tt = dfma2(rtm, df_mul(adv, rmi), tt);
            tt = dfma2(tc, df_mul(gai, rc), tt);
            res = dfma2(wd, tt, res);
            // K[(a,i),(b,j)] = sum_q wd [ g_a,j N_b (-rho u_i + tm rho Rm_i) + tm rho adv_a dRm_ij(b)
            //                            + tc g_a,i g_b,j + delta_ij (-rho adv_a N_b + mu g_a . g_b) ]
            const float2 A = df_mul(wd, df_mul(rho, dsub2(df_mul(tm, rmi), ui)));
            const float2 c0 = df_mul(ga0, A), c1 = df_mul(ga1, A);
            const float2 T4 = df_mul(wd, df_mul(rtm, adv)), T5 = df_mul(wd, df_mul(tc, gai));
            const float2 Bn = df_neg(df_mul(wd, df_mul(rho, adv))), Mu = df_mul(wd, mu);
            const float2 *dR = o + P_DRM + 12 * i;
#pragma unroll
            for (int b = 0; b < 6; ++b) {
                const float2 Nb = o[P_N + b], gb0 = o[P_G + 2 * b], gb1 = o[P_G + 2 * b + 1];
                const float2 diag = dfma2(Bn, Nb, df_mul(Mu, dfma2(ga0, gb0, df_mul(ga1, gb1))));
                float2 k0 = dfma2(c0, Nb, dfma2(T4, dR[b], df_mul(T5, gb0)));
                float2 k1 = dfma2(c1, Nb, dfma2(T4, dR[6 + b], df_mul(T5, gb1)));
                if (i == 0) k0 = df_add(k0, diag);
                else k1 = df_add(k1, diag);
                K[2 * b] = df_add(K[2 * b], k0);
                K[2 * b + 1] = df_add(K[2 * b + 1], k1);
            }
            const float2 T6 = df_mul(wd, gai);
#pragma unroll
            for (int c = 0; c < 3; ++c) K[12 + c] = df_add(K[12 + c], dsub2(df_mul(T4, cs[2 * c + i]), df_mul(T6, o[P_L + c])));
            // K[b',(a,i)] = sum_q wd [ l_b' g_a,i + tm sum_k grad l_b',k dRm_k,i(a) ]
            const float2 d0 = o[P_DRM + 6 * i + a], d1 = o[P_DRM + 12 + 6 * i + a];
#pragma unroll
            for (int bp = 0; bp < 3; ++bp)
                Kp[bp] = dfma2(wd, dfma2(o[P_L + bp], gai, dfma2(tg[bp][0], d0, df_mul(tg[bp][1], d1))), Kp[bp]);
        }
#pragma unroll
        for (int bp = 0; bp < 3; ++bp) w[15 + 15 * (12 + bp) + r] = df_to_double_int(Kp[bp]);
    } else {
        const int bp = r - 12;
        const float2 gp0 = cs[2 * bp], gp1 = cs[2 * bp + 1];
        float2 area = z;
#pragma unroll 1
        for (int p = 0; p < 16; ++p) {
            const float2 *o = pts[le][p];
            const float2 wd = o[P_WD];
            area = df_add(area, wd);
            res = dfma2(wd, dfma2(o[P_L + bp], o[P_RC], df_mul(tm, dfma2(gp0, o[P_RM], df_mul(gp1, o[P_RM + 1])))),
                        res);
        }
        // the pressure-pressure block: tm grad l_b' . grad l_c over the element
#pragma unroll
        for (int c = 0; c < 3; ++c)
            K[12 + c] = df_mul(df_mul(area, tm), dfma2(gp0, cs[2 * c], df_mul(gp1, cs[2 * c + 1])));
        w[r] = df_to_double_int(res);
#pragma unroll
        for (int c = 0; c < 3; ++c) w[15 + 15 * r + 12 + c] = df_to_double_int(K[12 + c]);
        return;
    }
    w[r] = df_to_double_int(res);
#pragma unroll
    for (int c = 0; c < 15; ++c) w[15 + 15 * r + c] = df_to_double_int(K[c]);
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

// flag[r] = 1 for every constrained dof s and each column r of row s (in a
// structurally symmetric pattern with its diagonal: the rows holding s)
__global__ void k_ns_mark_rows(int64_t n_rows, const int64_t *__restrict__ row_ptr,
                               const int32_t *__restrict__ col_idx, const uint8_t *__restrict__ mask,
                               uint8_t *__restrict__ flag)
{
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n_rows || !mask[s]) return;
    for (int64_t q = row_ptr[s]; q < row_ptr[s + 1]; ++q) flag[col_idx[q]] = 1;
}

__global__ void __launch_bounds__(NG_WARPS * 32) k_gather_ns_u(
    int64_t n2, const int64_t *__restrict__ p0ptr, const int64_t *__restrict__ p1ptr,
    const int64_t *__restrict__ inc_ptr, const int32_t *__restrict__ inc, const uint8_t *__restrict__ inc_loc,
    const uint8_t *__restrict__ inc_slot, const uint8_t *__restrict__ inc_slot_pq, const double *__restrict__ sc,
    const int64_t *__restrict__ row_ptr, const int32_t *__restrict__ col_idx, const uint8_t *__restrict__ mask,
    const uint8_t *__restrict__ bcrow, const double *__restrict__ bval, const double *__restrict__ x,
    double *__restrict__ values, double *__restrict__ d)
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
    // the Dirichlet tests (column loads) only on rows next to a constrained dof
    ns_finish_row(row, len, acc, rsum, lane, row_ptr, col_idx, (mask && bcrow[row]) ? mask : nullptr, bval, x,
                  values, d);
}

__global__ void __launch_bounds__(NG_WARPS * 32) k_gather_ns_p(
    int64_t n2, int64_t n1, const int64_t *__restrict__ p2ptr, const int64_t *__restrict__ p3ptr,
    const int64_t *__restrict__ pinc_ptr, const int32_t *__restrict__ pinc, const uint8_t *__restrict__ pinc_loc,
    const uint8_t *__restrict__ pinc_slot, const uint8_t *__restrict__ pinc_slot_pp, const double *__restrict__ sc,
    const int64_t *__restrict__ row_ptr, const int32_t *__restrict__ col_idx, const uint8_t *__restrict__ mask,
    const uint8_t *__restrict__ bcrow, const double *__restrict__ bval, const double *__restrict__ x,
    double *__restrict__ values, double *__restrict__ d)
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
    // the Dirichlet tests (column loads) only on rows next to a constrained dof
    ns_finish_row(row, len, acc, rsum, lane, row_ptr, col_idx, (mask && bcrow[row]) ? mask : nullptr, bval, x,
                  values, d);
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
    if (c->bc_mask) {  // rows next to a constrained dof: the pattern is structurally symmetric
        MF_CUDA(cudaMemsetAsync(p->bcrow, 0, (size_t)p->n_rows, st));
        k_ns_mark_rows<<<nsblk(p->n_rows, NR_T), NR_T, 0, st>>>(p->n_rows, p->row_ptr, p->col_idx, c->bc_mask,
                                                               p->bcrow);
    }
    k_gather_ns_u<<<nsblk(2 * n2, NG_WARPS), NG_WARPS * 32, 0, st>>>(
        n2, p->adj[0].ptr, p->adj[1].ptr, p->inc_ptr, p->inc, p->inc_loc, p->inc_slot, p->inc_slot_pq, p->scratch,
        p->row_ptr, p->col_idx, c->bc_mask, p->bcrow, c->bc_val, c->advect, values, d);
    if (n1 > 0)
        k_gather_ns_p<<<nsblk(n1, NG_WARPS), NG_WARPS * 32, 0, st>>>(
            n2, n1, p->adj[2].ptr, p->adj[3].ptr, p->pinc_ptr, p->pinc, p->pinc_loc, p->pinc_slot, p->pinc_slot_pp,
            p->scratch, p->row_ptr, p->col_idx, c->bc_mask, p->bcrow, c->bc_val, c->advect, values, d);
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
