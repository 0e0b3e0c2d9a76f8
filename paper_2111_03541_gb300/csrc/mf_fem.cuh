// Device routines shared by the single-problem and the batched assembly:
// quadrature constants, reference elements, geometry, and the thermal
// element kernels of Sec. 4.1 (one element per call, FP64).
#pragma once

#include <cstring>

#include "mf_internal.h"

namespace {

constexpr double QG = 0.57735026918962576451;  // 2-point Gauss abscissa 1/sqrt(3)
// symmetric 6-point degree-4 triangle rule (two orbits (a, a, 1-2a)); weights
// normalised to area 1
constexpr double T6A1 = 0.44594849091596488632, T6W1 = 0.22338158967801146570;
constexpr double T6A2 = 0.091576213509770743460, T6W2 = 0.10995174365532186764;

// reference derivative dN_a/dxi_j of the trilinear basis at Gauss point q
__device__ __forceinline__ double q1_dref(int q, int a, int j)
{
    const double xs[3] = {(q & 1) ? QG : -QG, (q & 2) ? QG : -QG, (q & 4) ? QG : -QG};
    const double s[3] = {(a & 1) ? 1.0 : -1.0, (a & 2) ? 1.0 : -1.0, (a & 4) ? 1.0 : -1.0};
    double v = 0.125 * s[j];
    for (int i = 0; i < 3; ++i)
        if (i != j) v *= 1.0 + s[i] * xs[i];
    return v;
}

__device__ __forceinline__ double q1_n(int q, int a)
{
    const double xs[3] = {(q & 1) ? QG : -QG, (q & 2) ? QG : -QG, (q & 4) ? QG : -QG};
    const double s[3] = {(a & 1) ? 1.0 : -1.0, (a & 2) ? 1.0 : -1.0, (a & 4) ? 1.0 : -1.0};
    return 0.125 * (1.0 + s[0] * xs[0]) * (1.0 + s[1] * xs[1]) * (1.0 + s[2] * xs[2]);
}

// Coefficients of the trilinear map x(xi) = sum_a x_a N_a(xi) = sum_S c_S
// prod_{k in S} xi_k, from a fast Walsh-Hadamard transform over the corners:
// H[S] = sum_a (-1)^popc(a & S) x_a, c_S = (-1)^popc(S) H[S] / 8 (S a bit set
// of xi = 1, eta = 2, zeta = 4).  Returns H (the caller tests H[3], H[5],
// H[6], H[7] = 0 for a parallelepiped).
__device__ __forceinline__ void q1_wht(const double (&x)[8][3], double (&H)[8][3])
{
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        double v[8];
#pragma unroll
        for (int a = 0; a < 8; ++a) v[a] = x[a][i];
#pragma unroll
        for (int m = 1; m < 8; m <<= 1)
#pragma unroll
            for (int a = 0; a < 8; ++a)
                if (!(a & m)) {
                    const double t = v[a], u = v[a | m];
                    v[a] = t + u;
                    v[a | m] = t - u;
                }
#pragma unroll
        for (int a = 0; a < 8; ++a) H[a][i] = v[a];
    }
}

// J^-1 and detJ at Gauss point q from the map coefficients c (c[S][i] as
// above): column j of J is d x / d xi_j = sum_{S containing j} c_S prod_{k in
// S, k != j} xi_k, three FMAs per entry.
__device__ __forceinline__ double q1_jac_at(const double (&c)[8][3], double xs, double ys, double zs,
                                            double (&Ji)[3][3])
{
    double J[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        J[i][0] = fma(zs, fma(ys, c[7][i], c[5][i]), fma(ys, c[3][i], c[1][i]));
        J[i][1] = fma(zs, fma(xs, c[7][i], c[6][i]), fma(xs, c[3][i], c[2][i]));
        J[i][2] = fma(ys, fma(xs, c[7][i], c[6][i]), fma(xs, c[5][i], c[4][i]));
    }
    const double c00 = J[1][1] * J[2][2] - J[1][2] * J[2][1];
    const double c01 = J[1][2] * J[2][0] - J[1][0] * J[2][2];
    const double c02 = J[1][0] * J[2][1] - J[1][1] * J[2][0];
    const double det = J[0][0] * c00 + J[0][1] * c01 + J[0][2] * c02;
    const double r = 1.0 / det;
    Ji[0][0] = c00 * r;
    Ji[1][0] = c01 * r;
    Ji[2][0] = c02 * r;
    Ji[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) * r;
    Ji[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) * r;
    Ji[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) * r;
    Ji[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) * r;
    Ji[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) * r;
    Ji[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) * r;
    return det;
}

// q1_jac_at at the 2 x 2 x 2 Gauss point q
__device__ __forceinline__ double q1_jac_coef(const double (&c)[8][3], int q, double (&Ji)[3][3])
{
    return q1_jac_at(c, (q & 1) ? QG : -QG, (q & 2) ? QG : -QG, (q & 4) ? QG : -QG, Ji);
}

// affine triangle from its first three nodes: detJ and grad lambda_k
__device__ __forceinline__ double tri_affine(const double *__restrict__ X, const int32_t *__restrict__ c,
                                             double (&gl)[3][2])
{
    const double x0 = X[2 * (int64_t)c[0]], y0 = X[2 * (int64_t)c[0] + 1];
    const double j00 = X[2 * (int64_t)c[1]] - x0, j10 = X[2 * (int64_t)c[1] + 1] - y0;
    const double j01 = X[2 * (int64_t)c[2]] - x0, j11 = X[2 * (int64_t)c[2] + 1] - y0;
    const double det = j00 * j11 - j01 * j10;
    const double r = 1.0 / det;
    // J^{-1} = [[j11, -j01], [-j10, j00]] / det ; grad lambda = J^{-T} gradref lambda
    const double i00 = j11 * r, i01 = -j01 * r, i10 = -j10 * r, i11 = j00 * r;
    gl[1][0] = i00; gl[1][1] = i01;   // gradref lambda_1 = (1, 0)
    gl[2][0] = i10; gl[2][1] = i11;   // gradref lambda_2 = (0, 1)
    gl[0][0] = -i00 - i10; gl[0][1] = -i01 - i11;
    return det;
}

// P2 basis values and physical gradients at barycentric point l
__device__ __forceinline__ void p2_basis(const double (&l)[3], const double (&gl)[3][2], double (&N)[6],
                                         double (&g)[6][2])
{
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        N[i] = l[i] * (2.0 * l[i] - 1.0);
        g[i][0] = (4.0 * l[i] - 1.0) * gl[i][0];
        g[i][1] = (4.0 * l[i] - 1.0) * gl[i][1];
    }
    const int ep[3][2] = {{0, 1}, {1, 2}, {2, 0}};
#pragma unroll
    for (int e = 0; e < 3; ++e) {
        const int p = ep[e][0], q = ep[e][1];
        N[3 + e] = 4.0 * l[p] * l[q];
        g[3 + e][0] = 4.0 * (gl[p][0] * l[q] + l[p] * gl[q][0]);
        g[3 + e][1] = 4.0 * (gl[p][1] * l[q] + l[p] * gl[q][1]);
    }
}

__device__ __forceinline__ void tri6_point(int q, double (&l)[3], double &w)
{
    const double a = q < 3 ? T6A1 : T6A2;
    const double b = 1.0 - 2.0 * a;
    const int k = q % 3;
    l[0] = (k == 0) ? b : a;
    l[1] = (k == 1) ? b : a;
    l[2] = (k == 2) ? b : a;
    w = 0.5 * (q < 3 ? T6W1 : T6W2);  // reference triangle area 1/2
}

__device__ __forceinline__ int upair(int a, int b) { return a * (15 - a) / 2 + b; }  // a <= b < 8

// Reference sums of degree-2 P2 integrands over the 6-point rule, in
// barycentric derivatives dN_a/dl_i of the P2 basis (pair p of (i, j):
// (0,0), (1,1), (2,2), (0,1), (0,2), (1,2); off-diagonal pairs hold ij + ji):
//   c_Ms[p][a][b] = sum_q w_q (dN_a/dl_i dN_b/dl_j + [i != j] dN_a/dl_j dN_b/dl_i)(q)
//   c_R[j][a1][b] = sum_q w_q l_a1(q) dN_b/dl_j(q)
// With G_ij = grad l_i . grad l_j, the viscous block
// D_ab = det sum_p G_p c_Ms[p][a][b] and the divergence blocks
// B_i[a1][b] = det sum_j (grad l_j)_i c_R[j][a1][b] are the same finite sums
// as their quadrature, reordered (the integrands have degree 2).
__constant__ double c_Ms[6][6][6];
// 10-node tetrahedron (vertices, then edges (0,1), (1,2), (2,0), (0,3),
// (1,3), (2,3)): c_Mt[u][s] for the pairs u = (a, b), a <= b (row-major) and
// the entries s = 00, 11, 22, 01, 02, 12 of G = J^-1 J^-T:
//   c_Mt[u][s] = int_ref d_p N_a d_q N_b (+ d_q N_a d_p N_b for p != q),
// exact by the 4-point degree-2 rule (the integrand is quadratic), so that
// K_ab = k detJ sum_s G_s c_Mt[u][s] on the affine element; kept as FP32
// pairs (hi, lo) for the double-float contraction
__constant__ float2 c_Mt[55][6];
__constant__ double c_R[3][3][6];

// 20-node serendipity brick: shape function a and its reference gradient at
// xi.  Vertex a = i + 2j + 4k at (2i-1, 2j-1, 2k-1):
// N = (1 + x xa)(1 + y ya)(1 + z za)(x xa + y ya + z za - 2) / 8; edge
// midpoints (x edges 8 + j + 2k, y edges 12 + i + 2k, z edges 16 + i + 2j)
// with zero coordinate along their edge: N = (1 - u^2)(1 + v1 s1)(1 + v2 s2) / 4,
// v1, v2 the other two coordinates in increasing axis order.
__host__ __device__ inline double q2s_shape(int a, const double (&xi)[3], double (&g)[3])
{
    if (a < 8) {
        const double xa = (a & 1) ? 1.0 : -1.0, ya = (a & 2) ? 1.0 : -1.0, za = (a & 4) ? 1.0 : -1.0;
        const double A = 1.0 + xi[0] * xa, B = 1.0 + xi[1] * ya, Cz = 1.0 + xi[2] * za;
        const double S = xi[0] * xa + xi[1] * ya + xi[2] * za - 2.0;
        g[0] = 0.125 * xa * B * Cz * (S + A);
        g[1] = 0.125 * ya * A * Cz * (S + B);
        g[2] = 0.125 * za * A * B * (S + Cz);
        return 0.125 * A * B * Cz * S;
    }
    const int axis = (a - 8) >> 2, t = (a - 8) & 3;
    const int d1 = axis == 0 ? 1 : 0, d2 = axis == 2 ? 1 : 2;
    const double s1 = (t & 1) ? 1.0 : -1.0, s2 = (t & 2) ? 1.0 : -1.0;
    const double u = xi[axis], Q = 1.0 - u * u, P1 = 1.0 + xi[d1] * s1, P2 = 1.0 + xi[d2] * s2;
    g[axis] = -0.5 * u * P1 * P2;
    g[d1] = 0.25 * Q * s1 * P2;
    g[d2] = 0.25 * Q * P1 * s2;
    return 0.25 * Q * P1 * P2;
}

// Double-float arithmetic on FP32 pairs (hi, lo), |lo| <= ulp(hi) / 2, about
// 48 significant bits (Dekker's product with an FMA, Knuth's two-sum): FP32
// runs at 64 times the FP64 rate here.
__host__ __device__ __forceinline__ float2 df_mul(float2 a, float2 b)
{
    const float p = a.x * b.x;
    const float e = fmaf(a.x, b.y, fmaf(a.y, b.x, fmaf(a.x, b.x, -p)));
    const float h = p + e;
    return make_float2(h, e - (h - p));
}

__host__ __device__ __forceinline__ float2 df_add(float2 a, float2 b)
{
    const float s = a.x + b.x;
    const float z = s - a.x;
    const float e = ((a.x - (s - z)) + (b.x - z)) + (a.y + b.y);
    const float h = s + e;
    return make_float2(h, e - (h - s));
}

__host__ __device__ __forceinline__ float2 df_neg(float2 a) { return make_float2(-a.x, -a.y); }

// 1 / a: an FP32 seed and one Newton step r0 + r0 (1 - a r0), the residual
// from the exact product a.x r0 (FMA) and the low part
__host__ __device__ __forceinline__ float2 df_recip(float2 a)
{
    const float r0 = 1.0f / a.x;
    const float ph = a.x * r0;
    const float pl = fmaf(a.x, r0, -ph);
    const float e = ((1.0f - ph) - pl) - a.y * r0;
    const float d = r0 * e;
    const float h = r0 + d;
    return make_float2(h, d - (h - r0));
}

// sqrt(a), a > 0: an FP32 seed and one Newton step s0 + (a - s0^2) / (2 s0)
__host__ __device__ __forceinline__ float2 df_sqrt(float2 a)
{
    const float s0 = sqrtf(a.x);
    const float ph = s0 * s0;
    const float pl = fmaf(s0, s0, -ph);
    const float e = ((a.x - ph) - pl) + a.y;
    const float d = e * (0.5f / s0);
    const float h = s0 + d;
    return make_float2(h, d - (h - s0));
}

// Exact FP32 -> FP64 conversion by integer operations on the IEEE-754 fields
// (FP32 subnormals, below 1.2e-38 in magnitude, become zero; infinities and
// NaN keep their class), and a pair's value as one FP64 add
__host__ __device__ __forceinline__ double f32_to_f64_exact(float f)
{
    unsigned u;
    memcpy(&u, &f, 4);
    const unsigned ex = (u >> 23) & 0xffu, sg = u & 0x80000000u, mt = u & 0x7fffffu;
    unsigned long long b = (unsigned long long)sg << 32;
    if (ex != 0u)
        b |= ((unsigned long long)(ex == 0xffu ? 0x7ffu : ex + 896u) << 52) | ((unsigned long long)mt << 29);
    double r;
    memcpy(&r, &b, 8);
    return r;
}

__host__ __device__ __forceinline__ double df_to_double(float2 a) { return f32_to_f64_exact(a.x) + f32_to_f64_exact(a.y); }

// FP64 -> pair: the nearest FP32 and the nearest FP32 of the exact remainder
__device__ __forceinline__ float2 f64_to_df(double x)
{
    const float h = __double2float_rn(x);
    return make_float2(h, __double2float_rn(x - (double)h));
}

// A normalised pair's value as FP64 by integer operations only (no FP64
// instruction, so nothing lands on GB300's narrow FP64 pipe): the high word's
// 24-bit significand followed by the low word's bits aligned below it (those
// under the 53-bit significand are truncated toward -inf, at most one ulp).
// A zero or subnormal high word gives a signed zero, an infinite or NaN one
// its own FP64 value.
__device__ __forceinline__ double df_to_double_int(float2 a)
{
    const unsigned hb = __float_as_uint(a.x);
    const int eh = (int)((hb >> 23) & 0xffu);
    if (eh == 0) return __longlong_as_double((long long)((unsigned long long)(hb & 0x80000000u) << 32));
    if (eh == 0xff) return f32_to_f64_exact(a.x);
    long long M = (long long)((hb & 0x7fffffu) | 0x800000u) << 29;  // units of 2^(eh - 127 - 52)
    const unsigned lb = __float_as_uint(a.y);
    const int el = (int)((lb >> 23) & 0xffu);
    if (el != 0) {
        const long long L = (long long)((lb & 0x7fffffu) | 0x800000u);  // units of 2^(el - 150)
        int sh = eh - 29 - el;  // >= -5 for a normalised pair, |lo| <= ulp(hi) / 2
        sh = sh < -5 ? -5 : sh;
        const long long add = sh >= 63 ? 0 : (sh >= 0 ? (L >> sh) : (L << -sh));
        M = ((hb ^ lb) >> 31) ? M - add : M + add;
    }
    long long e = eh - 127 + 1023;
    if (M >= (1ll << 53)) {
        M >>= 1;
        ++e;
    } else if (M < (1ll << 52)) {
        M <<= 1;
        --e;
    }
    const unsigned long long bits = ((unsigned long long)(hb >> 31) << 63) | ((unsigned long long)e << 52) |
                                    ((unsigned long long)M & ((1ull << 52) - 1));
    return __longlong_as_double((long long)bits);
}

// a double constant as an FP32 pair (folded at compile time)
#define DFC(x) make_float2((float)(x), (float)((x) - (double)(float)(x)))

// a b - c d in double-float
__host__ __device__ __forceinline__ float2 df_det2(float2 a, float2 b, float2 c, float2 d)
{
    return df_add(df_mul(a, b), df_neg(df_mul(c, d)));
}

// Geometry of the 20-node brick (the vertices' trilinear map) at point
// q = i + 3 j + 9 k of the 3 x 3 x 3 Gauss rule, in double-float: c holds the
// map coefficients of q1_jac_at as FP32 pairs; the Jacobian, its cofactors
// and determinant follow q1_jac_at; Mq[3 i + j] = sqrt(w detJ) (J^-1)_ji;
// returns w detJ.  About 47 bits against FP64's 53, at FP32 issue rates.
__host__ __device__ __forceinline__ float2 q2s_point_df(const float2 (&c)[8][3], int q, float2 (&Mq)[9])
{
    constexpr double G3 = 0.77459666924148337704;  // sqrt(3/5)
    constexpr double W5 = 5.0 / 9.0, W8 = 8.0 / 9.0;
    const float2 g = make_float2((float)G3, (float)(G3 - (double)(float)G3));
    const float2 w5 = make_float2((float)W5, (float)(W5 - (double)(float)W5));
    const float2 w8 = make_float2((float)W8, (float)(W8 - (double)(float)W8));
    const int qi = q % 3, qj = (q / 3) % 3, qk = q / 9;
    const float2 zero = make_float2(0.0f, 0.0f);
    const float2 xs = qi == 1 ? zero : (qi == 0 ? df_neg(g) : g);
    const float2 ys = qj == 1 ? zero : (qj == 0 ? df_neg(g) : g);
    const float2 zs = qk == 1 ? zero : (qk == 0 ? df_neg(g) : g);
    float2 J[3][3];
    for (int i = 0; i < 3; ++i) {
        J[i][0] = df_add(df_mul(zs, df_add(df_mul(ys, c[7][i]), c[5][i])), df_add(df_mul(ys, c[3][i]), c[1][i]));
        J[i][1] = df_add(df_mul(zs, df_add(df_mul(xs, c[7][i]), c[6][i])), df_add(df_mul(xs, c[3][i]), c[2][i]));
        J[i][2] = df_add(df_mul(ys, df_add(df_mul(xs, c[7][i]), c[6][i])), df_add(df_mul(xs, c[5][i]), c[4][i]));
    }
    float2 C[3][3];  // C[j][i] = detJ (J^-1)_ji
    C[0][0] = df_det2(J[1][1], J[2][2], J[1][2], J[2][1]);
    C[1][0] = df_det2(J[1][2], J[2][0], J[1][0], J[2][2]);
    C[2][0] = df_det2(J[1][0], J[2][1], J[1][1], J[2][0]);
    C[0][1] = df_det2(J[0][2], J[2][1], J[0][1], J[2][2]);
    C[1][1] = df_det2(J[0][0], J[2][2], J[0][2], J[2][0]);
    C[2][1] = df_det2(J[0][1], J[2][0], J[0][0], J[2][1]);
    C[0][2] = df_det2(J[0][1], J[1][2], J[0][2], J[1][1]);
    C[1][2] = df_det2(J[0][2], J[1][0], J[0][0], J[1][2]);
    C[2][2] = df_det2(J[0][0], J[1][1], J[0][1], J[1][0]);
    const float2 det = df_add(df_add(df_mul(J[0][0], C[0][0]), df_mul(J[0][1], C[1][0])), df_mul(J[0][2], C[2][0]));
    const float2 wv = df_mul(df_mul(qi == 1 ? w8 : w5, qj == 1 ? w8 : w5), qk == 1 ? w8 : w5);
    const float2 wd = df_mul(wv, det);
    const float2 sr = df_mul(df_sqrt(wd), df_recip(det));  // sqrt(w detJ) / detJ
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) Mq[3 * i + j] = df_mul(sr, C[j][i]);
    return wd;
}

// 20-node brick at the 27 points of the 3 x 3 x 3 Gauss rule (point q = i +
// 3 j + 9 k at ((i - 1), (j - 1), (k - 1)) sqrt(3/5)): [q][a] = N_a, then the
// reference gradient (global memory: lanes read different nodes)
__device__ double c_q2s_tab[27][20][4];
// the reference gradients again, each as an FP32 pair (hi, lo) with hi + lo
// within 2^-48 of the FP64 value
__device__ float2 c_q2s_tabf[27][20][3];

// Host: the reference sums, uploaded to this translation unit's copy of c_Ms,
// c_R and c_q2s_tab on the current device (each file that includes this
// header and launches a kernel using them uploads its own copy).
inline mf_status fem_consts_upload()
{
    double Ms[6][6][6] = {}, R[3][3][6] = {};
    const int pi[6] = {0, 1, 2, 0, 0, 1}, pj[6] = {0, 1, 2, 1, 2, 2};
    const int ep[3][2] = {{0, 1}, {1, 2}, {2, 0}};
    for (int q = 0; q < 6; ++q) {
        const double a = q < 3 ? T6A1 : T6A2, b = 1.0 - 2.0 * a;
        const int k = q % 3;
        const double l[3] = {k == 0 ? b : a, k == 1 ? b : a, k == 2 ? b : a};
        const double w = 0.5 * (q < 3 ? T6W1 : T6W2);
        double dN[6][3] = {};  // dN_a / dl_i
        for (int v = 0; v < 3; ++v) dN[v][v] = 4.0 * l[v] - 1.0;
        for (int e = 0; e < 3; ++e) {
            dN[3 + e][ep[e][0]] = 4.0 * l[ep[e][1]];
            dN[3 + e][ep[e][1]] = 4.0 * l[ep[e][0]];
        }
        for (int p = 0; p < 6; ++p)
            for (int x = 0; x < 6; ++x)
                for (int y = 0; y < 6; ++y) {
                    double t = dN[x][pi[p]] * dN[y][pj[p]];
                    if (pi[p] != pj[p]) t += dN[x][pj[p]] * dN[y][pi[p]];
                    Ms[p][x][y] += w * t;
                }
        for (int j = 0; j < 3; ++j)
            for (int a1 = 0; a1 < 3; ++a1)
                for (int y = 0; y < 6; ++y) R[j][a1][y] += w * l[a1] * dN[y][j];
    }
    MF_CUDA(cudaMemcpyToSymbol(c_Ms, Ms, sizeof Ms));
    {
        // 4-point rule on the reference tetrahedron (volume 1/6), degree 2:
        // barycentric (al, be, be, be) and permutations, weight 1/24 each
        const double al = (5.0 + 3.0 * sqrt(5.0)) / 20.0, be = (5.0 - sqrt(5.0)) / 20.0;
        const int ed[6][2] = {{0, 1}, {1, 2}, {2, 0}, {0, 3}, {1, 3}, {2, 3}};
        const int sp[6] = {0, 1, 2, 0, 0, 1}, sq[6] = {0, 1, 2, 1, 2, 2};
        double Mt[55][6] = {};
        for (int q = 0; q < 4; ++q) {
            double l[4];
            for (int i = 0; i < 4; ++i) l[i] = i == q ? al : be;
            double dN[10][4] = {};  // dN_a / dlambda_i
            for (int v = 0; v < 4; ++v) dN[v][v] = 4.0 * l[v] - 1.0;
            for (int k = 0; k < 6; ++k) {
                dN[4 + k][ed[k][0]] = 4.0 * l[ed[k][1]];
                dN[4 + k][ed[k][1]] = 4.0 * l[ed[k][0]];
            }
            double g[10][3];  // reference gradient: lambda_0 = 1 - x - y - z, lambda_{j+1} = x_j
            for (int a = 0; a < 10; ++a)
                for (int j = 0; j < 3; ++j) g[a][j] = dN[a][j + 1] - dN[a][0];
            int u = 0;
            for (int a = 0; a < 10; ++a)
                for (int b = a; b < 10; ++b, ++u)
                    for (int s2 = 0; s2 < 6; ++s2) {
                        double t = g[a][sp[s2]] * g[b][sq[s2]];
                        if (sp[s2] != sq[s2]) t += g[a][sq[s2]] * g[b][sp[s2]];
                        Mt[u][s2] += t / 24.0;
                    }
        }
        float2 Mtf[55][6];
        for (int u = 0; u < 55; ++u)
            for (int s2 = 0; s2 < 6; ++s2) {
                const float hi = (float)Mt[u][s2];
                Mtf[u][s2] = make_float2(hi, (float)(Mt[u][s2] - (double)hi));
            }
        MF_CUDA(cudaMemcpyToSymbol(c_Mt, Mtf, sizeof Mtf));

    }
    MF_CUDA(cudaMemcpyToSymbol(c_R, R, sizeof R));
    static double tab[27][20][4];
    const double g3 = 0.77459666924148337704;  // sqrt(3/5)
    for (int q = 0; q < 27; ++q) {
        const double xi[3] = {(q % 3 - 1) * g3, ((q / 3) % 3 - 1) * g3, (q / 9 - 1) * g3};
        for (int a = 0; a < 20; ++a) {
            double g[3];
            tab[q][a][0] = q2s_shape(a, xi, g);
            for (int i = 0; i < 3; ++i) tab[q][a][1 + i] = g[i];
        }
    }
    MF_CUDA(cudaMemcpyToSymbol(c_q2s_tab, tab, sizeof tab));
    static float2 tabf[27][20][3];
    for (int q = 0; q < 27; ++q)
        for (int a = 0; a < 20; ++a)
            for (int i = 0; i < 3; ++i) {
                const float hi = (float)tab[q][a][1 + i];
                tabf[q][a][i] = make_float2(hi, (float)(tab[q][a][1 + i] - (double)hi));
            }
    MF_CUDA(cudaMemcpyToSymbol(c_q2s_tabf, tabf, sizeof tabf));
    return MF_OK;
}

// Output of a thermal element routine.  With an incidence map, row a of
// element e goes to incidence entry t = map[e * NPE + a] of node conn[e][a] as
// [K_e[a][0..NPE), d_e[a]], so that a node's rows are contiguous; without one
// (map == nullptr), in element order [K_e (NPE x NPE, row-major), d_e (NPE)].
template <int NPE>
struct ThOut {
    int64_t base[NPE];  // offset of row a
    int64_t ld[NPE];    // offset of load entry a
    __device__ __forceinline__ ThOut(const int32_t *__restrict__ map, int64_t e)
    {
#pragma unroll
        for (int a = 0; a < NPE; ++a) {
            if (map) {
                base[a] = (int64_t)map[e * NPE + a] * mf_th_rs(NPE);
                ld[a] = base[a] + NPE;
            } else {
                base[a] = e * (NPE * NPE + NPE) + a * NPE;
                ld[a] = e * (NPE * NPE + NPE) + NPE * NPE + a;
            }
        }
    }
};

__device__ __forceinline__ void elem_thermal_p1(int64_t e, const double *__restrict__ X, const int32_t *__restrict__ conn,
                                  const double *__restrict__ kc, double f, const int32_t *__restrict__ map,
                                  double *__restrict__ out, int *status)
{
    const double k = kc[e];
    if (!isfinite(k)) mf_dev_fail(status, MF_ERR_NONFINITE);
    double gl[3][2];
    const double det = tri_affine(X, conn + 3 * e, gl);
    // the integrand is constant: the 3 point weights sum to 1/2
    const double s = 0.5 * det * k;
    const ThOut<3> W(map, e);
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) out[W.base[a] + b] = s * (gl[a][0] * gl[b][0] + gl[a][1] * gl[b][1]);
    // 3-point rule: sum_q w_q lambda_a(q) = 1/6
    const double l = det * f * (1.0 / 6.0);
#pragma unroll
    for (int a = 0; a < 3; ++a) out[W.ld[a]] = l;
}

__device__ __forceinline__ void elem_thermal_p2(int64_t e, const double *__restrict__ X, const int32_t *__restrict__ conn,
                                  const double *__restrict__ kc, double f, const int32_t *__restrict__ map,
                                  double *__restrict__ out, int *status)
{
    const double k = kc[e];
    if (!isfinite(k)) mf_dev_fail(status, MF_ERR_NONFINITE);
    double gl[3][2];
    const double det = tri_affine(X, conn + 6 * e, gl);
    // K_e = k det sum_p G_p c_Ms[p] (the integrand grad N_a . grad N_b has
    // degree 2: the quadrature sum reordered, see c_Ms); the load of a vertex
    // node integrates to 0, of an edge node to det / 6 (exact sums of the
    // degree-2 rule)
    double Gs[6];
    Gs[0] = fma(gl[0][0], gl[0][0], gl[0][1] * gl[0][1]);
    Gs[1] = fma(gl[1][0], gl[1][0], gl[1][1] * gl[1][1]);
    Gs[2] = fma(gl[2][0], gl[2][0], gl[2][1] * gl[2][1]);
    Gs[3] = fma(gl[0][0], gl[1][0], gl[0][1] * gl[1][1]);
    Gs[4] = fma(gl[0][0], gl[2][0], gl[0][1] * gl[2][1]);
    Gs[5] = fma(gl[1][0], gl[2][0], gl[1][1] * gl[2][1]);
    const double kd = k * det;
    const ThOut<6> W(map, e);
#pragma unroll
    for (int a = 0; a < 6; ++a)
#pragma unroll
        for (int b = a; b < 6; ++b) {
            double v = 0.0;
#pragma unroll
            for (int p = 0; p < 6; ++p) v = fma(Gs[p], c_Ms[p][a][b], v);
            out[W.base[a] + b] = kd * v;
            out[W.base[b] + a] = kd * v;
        }
    const double le = f * det * (1.0 / 6.0);
#pragma unroll
    for (int a = 0; a < 6; ++a) out[W.ld[a]] = a < 3 ? 0.0 : le;
}

// 10-node tetrahedron, thermal form: the affine map of the vertices, then
// K_e = k detJ sum_s G_s c_Mt[s] (G = J^-1 J^-T, exact; the contraction in
// double-float); the load of a vertex node integrates to -f detJ / 120, of an
// edge node to f detJ / 30 (the moments -V/20 and V/5 of the quadratic
// simplex, V = detJ / 6).  One thread per element; returns the metric as
// FP32 pairs and the two load values (vertex, edge); false for a lane
// without an element.
__device__ __forceinline__ bool p2t_metric(int64_t e, int64_t n_el, const double *__restrict__ X,
                                           const int32_t *__restrict__ conn, const double *__restrict__ kc,
                                           double f, float2 (&G)[6], double &lv, double &le, int *status)
{
    if (e >= n_el) return false;
    const double k = kc[e];
    if (!isfinite(k)) mf_dev_fail(status, MF_ERR_NONFINITE);
    const int32_t *c = conn + 10 * e;
    double J[3][3];
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
        for (int i = 0; i < 3; ++i) J[i][j] = X[3 * (int64_t)c[j + 1] + i] - X[3 * (int64_t)c[0] + i];
    // inverse by cofactors (as q1_jac_at): Ji[p][i] = d xi_p / d x_i
    double Ji[3][3];
    Ji[0][0] = J[1][1] * J[2][2] - J[1][2] * J[2][1];
    Ji[1][0] = J[1][2] * J[2][0] - J[1][0] * J[2][2];
    Ji[2][0] = J[1][0] * J[2][1] - J[1][1] * J[2][0];
    const double det = J[0][0] * Ji[0][0] + J[0][1] * Ji[1][0] + J[0][2] * Ji[2][0];
    const double r = 1.0 / det;
    Ji[0][0] *= r;
    Ji[1][0] *= r;
    Ji[2][0] *= r;
    Ji[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) * r;
    Ji[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) * r;
    Ji[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) * r;
    Ji[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) * r;
    Ji[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) * r;
    Ji[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) * r;
    const int sp[6] = {0, 1, 2, 0, 0, 1}, sq[6] = {0, 1, 2, 1, 2, 2};
    const double kd = k * det;
#pragma unroll
    for (int s = 0; s < 6; ++s) {
        const double g =
            kd * fma(Ji[sp[s]][0], Ji[sq[s]][0], fma(Ji[sp[s]][1], Ji[sq[s]][1], Ji[sp[s]][2] * Ji[sq[s]][2]));
        const float hi = __double2float_rn(g);
        G[s] = make_float2(hi, __double2float_rn(g - (double)hi));
    }
    lv = -f * det * (1.0 / 120.0);
    le = f * det * (1.0 / 30.0);
    return true;
}

// K_ab of the tetrahedron from its metric: pair u = (min, max) of the upper
// triangle (row-major), so that K_ab and K_ba are the same bits
__device__ __forceinline__ double p2t_entry(const float2 (&G)[6], int a, int b)
{
    const int lo = a < b ? a : b, hi = a < b ? b : a;
    const int u = lo * (19 - lo) / 2 + hi;
    float2 v = df_mul(G[0], c_Mt[u][0]);
#pragma unroll
    for (int s = 1; s < 6; ++s) v = df_add(v, df_mul(G[s], c_Mt[u][s]));
    return df_to_double(v);
}

// 8-node serendipity quadrilateral, thermal form: the vertices' bilinear map
// at the 3 x 3 Gauss points; reference gradients of the 8-node basis
// (vertex a at (sa, ta): N = (1 + x sa)(1 + y ta)(x sa + y ta - 1) / 4; x edge
// 4 + j at y = tj: N = (1 - x^2)(1 + y tj) / 2; y edge 6 + i at x = si:
// N = (1 - y^2)(1 + x si) / 2); K_e = k sum_q w detJ grad N_a . grad N_b,
// d_e = f sum_q w detJ N_a.  FP64, one thread per element.
__device__ __forceinline__ void elem_thermal_q2q(int64_t e, const double *__restrict__ X,
                                                 const int32_t *__restrict__ conn, const double *__restrict__ kc,
                                                 double f, const int32_t *__restrict__ map, double *__restrict__ out,
                                                 int *status)
{
    const double k = kc[e];
    if (!isfinite(k)) mf_dev_fail(status, MF_ERR_NONFINITE);
    const int32_t *c = conn + 8 * e;
    double x[4][2];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int i = 0; i < 2; ++i) x[a][i] = X[2 * (int64_t)c[a] + i];
    double K[36] = {}, dl[8] = {};
    const double g3 = 0.77459666924148337704;  // sqrt(3/5)
#pragma unroll 1
    for (int q = 0; q < 9; ++q) {
        const double xs = (q % 3 - 1) * g3, ys = (q / 3 - 1) * g3;
        const double w = (q % 3 == 1 ? 8.0 / 9.0 : 5.0 / 9.0) * (q / 3 == 1 ? 8.0 / 9.0 : 5.0 / 9.0);
        double N[8], dN[8][2];
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            const double sa = (a & 1) ? 1.0 : -1.0, ta = (a & 2) ? 1.0 : -1.0;
            const double A = 1.0 + xs * sa, B = 1.0 + ys * ta;
            N[a] = 0.25 * A * B * (xs * sa + ys * ta - 1.0);
            dN[a][0] = 0.25 * sa * B * (2.0 * xs * sa + ys * ta);
            dN[a][1] = 0.25 * ta * A * (xs * sa + 2.0 * ys * ta);
        }
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const double t = j ? 1.0 : -1.0;
            N[4 + j] = 0.5 * (1.0 - xs * xs) * (1.0 + ys * t);
            dN[4 + j][0] = -xs * (1.0 + ys * t);
            dN[4 + j][1] = 0.5 * t * (1.0 - xs * xs);
            N[6 + j] = 0.5 * (1.0 - ys * ys) * (1.0 + xs * t);
            dN[6 + j][0] = 0.5 * t * (1.0 - ys * ys);
            dN[6 + j][1] = -ys * (1.0 + xs * t);
        }
        // the bilinear map of the vertices: J[i][r] = sum_a x_a,i dN1_a / dxi_r
        double J[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            const double sa = (a & 1) ? 1.0 : -1.0, ta = (a & 2) ? 1.0 : -1.0;
            const double d0 = 0.25 * sa * (1.0 + ta * ys), d1 = 0.25 * ta * (1.0 + sa * xs);
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                J[i][0] = fma(x[a][i], d0, J[i][0]);
                J[i][1] = fma(x[a][i], d1, J[i][1]);
            }
        }
        const double det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
        const double r = 1.0 / det, wd = w * det;
        // grad N = J^-T gradref N, J^-1 = [[J11, -J01], [-J10, J00]] / det
        double g[8][2];
#pragma unroll
        for (int a = 0; a < 8; ++a) {
            g[a][0] = (J[1][1] * dN[a][0] - J[1][0] * dN[a][1]) * r;
            g[a][1] = (J[0][0] * dN[a][1] - J[0][1] * dN[a][0]) * r;
            dl[a] = fma(wd, N[a], dl[a]);
        }
        int u = 0;
#pragma unroll
        for (int a = 0; a < 8; ++a)
#pragma unroll
            for (int b = a; b < 8; ++b, ++u) K[u] = fma(wd, fma(g[a][0], g[b][0], g[a][1] * g[b][1]), K[u]);
    }
    const ThOut<8> W(map, e);
    int u = 0;
#pragma unroll
    for (int a = 0; a < 8; ++a) {
#pragma unroll
        for (int b = a; b < 8; ++b, ++u) {
            out[W.base[a] + b] = k * K[u];
            if (b != a) out[W.base[b] + a] = k * K[u];
        }
        out[W.ld[a]] = f * dl[a];
    }
}

__device__ __forceinline__ void elem_thermal_q1(int64_t e, const double *__restrict__ X,
                                                         const int32_t *__restrict__ conn,
                                                         const double *__restrict__ kc, double f,
                                                         const int32_t *__restrict__ map, double *__restrict__ out,
                                                         int *status)
{
    const double k = kc[e];
    if (!isfinite(k)) mf_dev_fail(status, MF_ERR_NONFINITE);
    double x[8][3];
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int i = 0; i < 3; ++i) x[a][i] = X[3 * (int64_t)conn[8 * e + a] + i];
    // Parallelepiped test: the bilinear and trilinear coefficients of the map
    // x(xi) = sum_a x_a N_a(xi) vanish exactly.  Then J is constant and the
    // Gauss sums factor: sum_q dN_a/dxi_i dN_b/dxi_j = R_ab[i][j] (closed form
    // below), so Ke[a][b] = k detJ sum_ij R_ab[i][j] (J^-1 J^-T)_ij and
    // de[a] = f detJ sum_q N_a(q) with sum_q N_a(q) = 1.
    double c[8][3];  // map coefficients c_S (q1_wht)
    q1_wht(x, c);
    bool affine = true;
#pragma unroll
    for (int i = 0; i < 3; ++i)
        affine = affine && c[3][i] == 0.0 && c[5][i] == 0.0 && c[6][i] == 0.0 && c[7][i] == 0.0;
#pragma unroll
    for (int S = 1; S < 8; ++S)
#pragma unroll
        for (int i = 0; i < 3; ++i) c[S][i] *= (__popc(S) & 1) ? -0.125 : 0.125;
    if (affine) {
        double Ji[3][3];
        const double det = q1_jac_coef(c, 0, Ji);  // constant over the element
        double G[3][3];
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) G[i][j] = Ji[i][0] * Ji[j][0] + Ji[i][1] * Ji[j][1] + Ji[i][2] * Ji[j][2];
        const ThOut<8> W(map, e);
        const double kd = k * det;
#pragma unroll
        for (int a = 0; a < 8; ++a) {
#pragma unroll
            for (int b = a; b < 8; ++b) {
                // R_ab[i][j]: product over the three directions of the 2-point
                // sums of the 1D factors: sum (1 + s x)(1 + s' x) = 2 (1 + s s' / 3),
                // sum (1 + s x) s' = 2 s', sum s s' = 2 s s'; then / 64
                const double s[2][3] = {{(a & 1) ? 1.0 : -1.0, (a & 2) ? 1.0 : -1.0, (a & 4) ? 1.0 : -1.0},
                                        {(b & 1) ? 1.0 : -1.0, (b & 2) ? 1.0 : -1.0, (b & 4) ? 1.0 : -1.0}};
                double v = 0.0;
#pragma unroll
                for (int i = 0; i < 3; ++i)
#pragma unroll
                    for (int j = 0; j < 3; ++j) {
                        double r = 1.0 / 8.0;  // (2 * 2 * 2) / 64
#pragma unroll
                        for (int d = 0; d < 3; ++d) {
                            if (d == i && d == j) r *= s[0][d] * s[1][d];
                            else if (d == i) r *= s[0][d];
                            else if (d == j) r *= s[1][d];
                            else r *= 1.0 + s[0][d] * s[1][d] / 3.0;
                        }
                        v = fma(r, G[i][j], v);
                    }
                out[W.base[a] + b] = kd * v;
                out[W.base[b] + a] = kd * v;
            }
            out[W.ld[a]] = f * det;
        }
        return;
    }
    double Ke[36] = {}, m[8] = {};
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        double Ji[3][3];
        const double wd = q1_jac_coef(c, q, Ji);  // Gauss weights are 1
        double g[8][3];
#pragma unroll
        for (int a = 0; a < 8; ++a)
#pragma unroll
            for (int i = 0; i < 3; ++i)
                g[a][i] = q1_dref(q, a, 0) * Ji[0][i] + q1_dref(q, a, 1) * Ji[1][i] + q1_dref(q, a, 2) * Ji[2][i];
        int t = 0;
#pragma unroll
        for (int a = 0; a < 8; ++a) {
            const double ga0 = wd * g[a][0], ga1 = wd * g[a][1], ga2 = wd * g[a][2];
#pragma unroll
            for (int b = a; b < 8; ++b, ++t) Ke[t] = fma(ga0, g[b][0], fma(ga1, g[b][1], fma(ga2, g[b][2], Ke[t])));
            m[a] = fma(wd, q1_n(q, a), m[a]);
        }
    }
    const ThOut<8> W(map, e);
    int t = 0;
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int b = a; b < 8; ++b, ++t) {
            out[W.base[a] + b] = k * Ke[t];
            out[W.base[b] + a] = k * Ke[t];
        }
#pragma unroll
    for (int a = 0; a < 8; ++a) out[W.ld[a]] = f * m[a];
}



// Capacity (the rate term -C(T, T_t) of Sec. 4.1, tangent negated):
// M_e[a][b] = C int_e N_a N_b, no load.  P1: C |e| (1 + delta_ab) / 12.  P2:
// C det R[a][b], R the integrals of the quadratic basis over the reference
// triangle per unit det = 2|e| (vertices, then the midpoints of edges (0,1),
// (1,2), (2,0)).  Q1: 2 x 2 x 2 Gauss with detJ from the map coefficients,
// exact on parallelepipeds.
__device__ __forceinline__ void elem_capacity_p1(int64_t e, const double *__restrict__ X,
                                                 const int32_t *__restrict__ conn, const double *__restrict__ kc,
                                                 const int32_t *__restrict__ map, double *__restrict__ out,
                                                 int *status)
{
    const double C = kc[e];
    if (!isfinite(C)) mf_dev_fail(status, MF_ERR_NONFINITE);
    double gl[3][2];
    const double s = C * tri_affine(X, conn + 3 * e, gl) * (1.0 / 24.0);
    const ThOut<3> W(map, e);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
#pragma unroll
        for (int b = 0; b < 3; ++b) out[W.base[a] + b] = a == b ? 2.0 * s : s;
        out[W.ld[a]] = 0.0;
    }
}

__device__ __forceinline__ void elem_capacity_p2(int64_t e, const double *__restrict__ X,
                                                 const int32_t *__restrict__ conn, const double *__restrict__ kc,
                                                 const int32_t *__restrict__ map, double *__restrict__ out,
                                                 int *status)
{
    constexpr double R[6][6] = {{6, -1, -1, 0, -4, 0},  {-1, 6, -1, 0, 0, -4},  {-1, -1, 6, -4, 0, 0},
                                {0, 0, -4, 32, 16, 16}, {-4, 0, 0, 16, 32, 16}, {0, -4, 0, 16, 16, 32}};
    const double C = kc[e];
    if (!isfinite(C)) mf_dev_fail(status, MF_ERR_NONFINITE);
    double gl[3][2];
    const double s = C * tri_affine(X, conn + 6 * e, gl) * (1.0 / 360.0);
    const ThOut<6> W(map, e);
#pragma unroll
    for (int a = 0; a < 6; ++a) {
#pragma unroll
        for (int b = 0; b < 6; ++b) out[W.base[a] + b] = s * R[a][b];
        out[W.ld[a]] = 0.0;
    }
}

// 10-node tetrahedron: the consistent mass matrix of the affine element in
// closed form, C V / 420 [vertex-vertex 6 (diagonal) or 1, vertex-edge -4
// (the edge touches the vertex) or -6, edge-edge 32 (diagonal), 16 (a shared
// vertex) or 8], V = detJ / 6; zero load.  Incidence layout (map required).
__device__ __forceinline__ void elem_capacity_p2t(int64_t e, const double *__restrict__ X,
                                                  const int32_t *__restrict__ conn, const double *__restrict__ kc,
                                                  const int32_t *__restrict__ map, double *__restrict__ out,
                                                  int *status)
{
    const double C = kc[e];
    if (!isfinite(C)) mf_dev_fail(status, MF_ERR_NONFINITE);
    const int32_t *c = conn + 10 * e;
    double J[3][3];
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
        for (int i = 0; i < 3; ++i) J[i][j] = X[3 * (int64_t)c[j + 1] + i] - X[3 * (int64_t)c[0] + i];
    const double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) +
                       J[0][1] * (J[1][2] * J[2][0] - J[1][0] * J[2][2]) +
                       J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
    const double s = C * det * (1.0 / 2520.0);
    const int ep[6][2] = {{0, 1}, {1, 2}, {2, 0}, {0, 3}, {1, 3}, {2, 3}};
    constexpr int RS = mf_th_rs(10);
#pragma unroll 1
    for (int a = 0; a < 10; ++a) {
        double *row = out + (int64_t)map[e * 10 + a] * RS;
#pragma unroll
        for (int b = 0; b < 10; ++b) {
            double m;
            if (a < 4 && b < 4) {
                m = a == b ? 6.0 : 1.0;
            } else if (a < 4 || b < 4) {
                const int v = a < 4 ? a : b, k = (a < 4 ? b : a) - 4;
                m = (ep[k][0] == v || ep[k][1] == v) ? -4.0 : -6.0;
            } else {
                const int k = a - 4, l = b - 4;
                const int sh = (ep[k][0] == ep[l][0]) + (ep[k][0] == ep[l][1]) + (ep[k][1] == ep[l][0]) +
                               (ep[k][1] == ep[l][1]);
                m = k == l ? 32.0 : (sh == 1 ? 16.0 : 8.0);
            }
            row[b] = s * m;
        }
        row[10] = 0.0;
    }
}

// 8-node serendipity quadrilateral: C sum_q w detJ N_a N_b at the 3 x 3 Gauss
// points of the vertices' bilinear map (the basis of elem_thermal_q2q); zero load.
__device__ __forceinline__ void elem_capacity_q2q(int64_t e, const double *__restrict__ X,
                                                  const int32_t *__restrict__ conn, const double *__restrict__ kc,
                                                  const int32_t *__restrict__ map, double *__restrict__ out,
                                                  int *status)
{
    const double C = kc[e];
    if (!isfinite(C)) mf_dev_fail(status, MF_ERR_NONFINITE);
    const int32_t *c = conn + 8 * e;
    double x[4][2];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int i = 0; i < 2; ++i) x[a][i] = X[2 * (int64_t)c[a] + i];
    double Me[36] = {};
    const double g3 = 0.77459666924148337704;  // sqrt(3/5)
#pragma unroll 1
    for (int q = 0; q < 9; ++q) {
        const double xs = (q % 3 - 1) * g3, ys = (q / 3 - 1) * g3;
        const double w = (q % 3 == 1 ? 8.0 / 9.0 : 5.0 / 9.0) * (q / 3 == 1 ? 8.0 / 9.0 : 5.0 / 9.0);
        double N[8];
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            const double sa = (a & 1) ? 1.0 : -1.0, ta = (a & 2) ? 1.0 : -1.0;
            N[a] = 0.25 * (1.0 + xs * sa) * (1.0 + ys * ta) * (xs * sa + ys * ta - 1.0);
        }
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const double t = j ? 1.0 : -1.0;
            N[4 + j] = 0.5 * (1.0 - xs * xs) * (1.0 + ys * t);
            N[6 + j] = 0.5 * (1.0 - ys * ys) * (1.0 + xs * t);
        }
        double J[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            const double sa = (a & 1) ? 1.0 : -1.0, ta = (a & 2) ? 1.0 : -1.0;
            const double d0 = 0.25 * sa * (1.0 + ta * ys), d1 = 0.25 * ta * (1.0 + sa * xs);
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                J[i][0] = fma(x[a][i], d0, J[i][0]);
                J[i][1] = fma(x[a][i], d1, J[i][1]);
            }
        }
        const double wd = w * (J[0][0] * J[1][1] - J[0][1] * J[1][0]);
        int t = 0;
#pragma unroll
        for (int a = 0; a < 8; ++a) {
            const double na = wd * N[a];
#pragma unroll
            for (int b = a; b < 8; ++b, ++t) Me[t] = fma(na, N[b], Me[t]);
        }
    }
    const ThOut<8> W(map, e);
    int t = 0;
#pragma unroll
    for (int a = 0; a < 8; ++a) {
#pragma unroll
        for (int b = a; b < 8; ++b, ++t) {
            out[W.base[a] + b] = C * Me[t];
            out[W.base[b] + a] = C * Me[t];
        }
        out[W.ld[a]] = 0.0;
    }
}

__device__ __forceinline__ void elem_capacity_q1(int64_t e, const double *__restrict__ X,
                                                 const int32_t *__restrict__ conn, const double *__restrict__ kc,
                                                 const int32_t *__restrict__ map, double *__restrict__ out,
                                                 int *status)
{
    const double C = kc[e];
    if (!isfinite(C)) mf_dev_fail(status, MF_ERR_NONFINITE);
    double x[8][3];
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int i = 0; i < 3; ++i) x[a][i] = X[3 * (int64_t)conn[8 * e + a] + i];
    double c[8][3];
    q1_wht(x, c);
#pragma unroll
    for (int S = 1; S < 8; ++S)
#pragma unroll
        for (int i = 0; i < 3; ++i) c[S][i] *= (__popc(S) & 1) ? -0.125 : 0.125;
    double Me[36] = {};
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        double Ji[3][3];
        const double wd = q1_jac_coef(c, q, Ji);  // Gauss weights are 1
        int t = 0;
#pragma unroll
        for (int a = 0; a < 8; ++a) {
            const double na = wd * q1_n(q, a);
#pragma unroll
            for (int b = a; b < 8; ++b, ++t) Me[t] = fma(na, q1_n(q, b), Me[t]);
        }
    }
    const ThOut<8> W(map, e);
    int t = 0;
#pragma unroll
    for (int a = 0; a < 8; ++a) {
#pragma unroll
        for (int b = a; b < 8; ++b, ++t) {
            out[W.base[a] + b] = C * Me[t];
            out[W.base[b] + a] = C * Me[t];
        }
        out[W.ld[a]] = 0.0;
    }
}

// Thermal translate shortcut (Q1): true when element e is a translate of
// element 0, whose unit matrices stand in for its own (the gather takes k_e
// from the coefficients); k_e is still checked here.
__device__ __forceinline__ bool q1_translate(int64_t e, const uint8_t *__restrict__ tr, const double *__restrict__ kc,
                                             int *status)
{
    if (!tr || !tr[e]) return false;
    if (!isfinite(kc[e])) mf_dev_fail(status, MF_ERR_NONFINITE);
    return true;
}

// Lanes per node of the thermal gather: 4 for P1, 8 for P2 and Q1, a warp for
// the 20-node brick.
template <int NPE>
constexpr int th_lanes() { return NPE <= 4 ? 4 : (NPE <= 8 ? 8 : (NPE <= 16 ? 16 : 32)); }

// Thermal row of node n by a group of th_lanes<NPE>() lanes (`sub` = lane in
// the group, `gmask` = the group's lanes; groups of a warp are independent).
// The scratch is in incidence layout: incidence entry t of the node (element
// e = inc[t], local index a) holds row a of K_e and d_e[a].  A translate
// (bit 7 of inc_loc) stores nothing: it takes k_e Kref[a][b] and f dref[a].
// Lane b fetches entry b of each of the node's rows (ascending elements) and
// its slot among the node's neighbours; the loads of up to 4 rows, the row's
// columns and their Dirichlet flags do not depend on one another.  The adds
// into the shared-memory row `acc` (MF_MAX_DEG doubles) run element by
// element, so every entry is a sum in ascending element order.  d_n: lane j
// adds the load entries of incidence entries j, j + L, ... in turn, then the
// group sums its lanes in a fixed tree.  Dirichlet rows become identity rows;
// constrained columns move to the right-hand side (lifting).  FP64 is the
// scarce pipe here, so every FP64 instruction of the loop does useful work in
// all lanes.
// Loads of values that the same launch wrote (element rows, coefficient
// pairs): L2 only when a kernel both writes and reads them (the batch's single
// persistent launch), plain loads otherwise.
template <bool L2ONLY, typename T>
__device__ __forceinline__ T ld_fresh(const T *p)
{
    if constexpr (L2ONLY) return __ldcg(p);
    else return *p;
}

template <int NPE, bool L2ONLY = false>
__device__ __forceinline__ void gather_row_th(int64_t n, int sub, unsigned gmask, double *acc,
                                              const int64_t *__restrict__ adj_ptr, const int32_t *__restrict__ adj_col,
                                              const int64_t *__restrict__ inc_ptr, const int32_t *__restrict__ inc,
                                              const uint8_t *__restrict__ inc_loc,
                                              const uint8_t *__restrict__ inc_slot, const double *__restrict__ sc,
                                              const double *__restrict__ kref, const double *__restrict__ kc,
                                              double f, const uint8_t *__restrict__ mask,
                                              const double *__restrict__ bval, const int64_t *__restrict__ row_ptr,
                                              double *__restrict__ values, double *__restrict__ d)
{
    constexpr int L = th_lanes<NPE>();
    constexpr int U = 4;   // rows whose loads are in flight together
    constexpr int KM = 4;  // prefetched columns per lane (the rest: plain loop)
    constexpr int RS = mf_th_rs(NPE);
    const int64_t p0 = adj_ptr[n];
    const int deg = (int)(adj_ptr[n + 1] - p0);
    const int64_t i0 = inc_ptr[n], i1 = inc_ptr[n + 1];
    const bool rm = mask ? mask[n] != 0 : false;
    const int64_t rb = row_ptr[n];
    int32_t mc[KM];
    unsigned cmask = 0;  // bit i: column sub + L i is constrained
#pragma unroll
    for (int i = 0; i < KM; ++i) mc[i] = (sub + L * i < deg) ? adj_col[p0 + sub + L * i] : -1;
    if (mask)
#pragma unroll
        for (int i = 0; i < KM; ++i)
            if (mc[i] >= 0 && mask[mc[i]]) cmask |= 1u << i;
    for (int i = sub; i < deg; i += L) acc[i] = 0.0;
    __syncwarp(gmask);
    const int b = sub;
    const bool act = b < NPE;
    double dsum = 0.0;
    // load vector: lane sub takes incidence entries i0 + sub, i0 + sub + L, ...
    for (int64_t t = i0 + sub; t < i1; t += L) {
        const int loc = inc_loc[t];
        dsum += (loc & 0x80) ? f * __ldg(&kref[NPE * NPE + (loc & 0x7f)]) : ld_fresh<L2ONLY>(&sc[t * RS + NPE]);
    }
    for (int64_t cb = i0; cb < i1; cb += U) {
        const int cnt = (int)min((int64_t)U, i1 - cb);
        double mul[U], val[U];
        int s[U];
#pragma unroll
        for (int j = 0; j < U; ++j) {
            mul[j] = 1.0;
            val[j] = 0.0;
            s[j] = 0;
            if (j < cnt && act) {
                const int64_t t = cb + j;
                const int loc = inc_loc[t];
                s[j] = inc_slot[t * NPE + b];
                if (loc & 0x80) {
                    mul[j] = kc[inc[t]];
                    val[j] = __ldg(&kref[(loc & 0x7f) * NPE + b]);
                } else {
                    val[j] = ld_fresh<L2ONLY>(&sc[t * RS + b]);
                }
            }
        }
#pragma unroll
        for (int j = 0; j < U; ++j) {
            if (j < cnt) {  // group-uniform
                if (act) acc[s[j]] = fma(mul[j], val[j], acc[s[j]]);  // exact product when mul = 1
                __syncwarp(gmask);
            }
        }
    }
    double lift = 0.0;
#pragma unroll
    for (int i = 0; i < KM; ++i) {
        if (mc[i] < 0) continue;
        const int k = sub + L * i;
        double v = acc[k];
        if (mask) {
            if (rm) {
                v = (mc[i] == n) ? 1.0 : 0.0;
            } else if (cmask & (1u << i)) {
                lift -= v * bval[mc[i]];
                v = 0.0;
            }
        }
        values[rb + k] = v;
    }
    for (int k = sub + L * KM; k < deg; k += L) {  // rows longer than L * KM
        const int64_t mcol = adj_col[p0 + k];
        double v = acc[k];
        if (mask) {
            if (rm) {
                v = (mcol == n) ? 1.0 : 0.0;
            } else if (mask[mcol]) {
                lift -= v * bval[mcol];
                v = 0.0;
            }
        }
        values[rb + k] = v;
    }
#pragma unroll
    for (int o = L / 2; o > 0; o >>= 1) dsum += __shfl_xor_sync(gmask, dsum, o, L);
    if (__any_sync(gmask, lift != 0.0))  // rows next to a constrained node only
#pragma unroll
        for (int o = L / 2; o > 0; o >>= 1) lift += __shfl_xor_sync(gmask, lift, o, L);
    if (sub == 0) d[n] = rm ? bval[n] : dsum + lift;
    __syncwarp(gmask);
}

// One node's row of the thermal Q1 form (or its capacity form: cls = m_cls,
// zero load) on a lexicographic box of translates of a rectangular cell
// (mf_pattern::box).  The reference entry of two corners depends only on the
// axes in which they differ, so entry (n, m) = cls[axes] x (sum of k_e over
// the elements holding n and m): with the node's 8 incident coefficients k
// (zero past the box edge), the 27 sums come from 19 FP64 adds (pairs along
// z, y, x, then faces, then all 8), one product per entry.  The load is f
// dref times the number of incident elements.  The entries go out in
// ascending column order through emit(k, value), k = 0, 1, ... over the
// existing neighbours (slot (dz + 1) 9 + (dy + 1) 3 + (dx + 1) order), so no
// row is held in registers; the load entry is returned.
// With near_bc (the node or a neighbour constrained; any row may pass true)
// Dirichlet rows become identity rows and constrained columns move to the
// right-hand side (lifting, in ascending column order); other rows give the
// same values either way.
template <typename Emit>
__device__ __forceinline__ double box_row_q1(int n, int nx1, int ny1, int nz1, const double *__restrict__ cls,
                                             double dref_f, const double *__restrict__ kc, bool near_bc,
                                             const uint8_t *__restrict__ mask, const double *__restrict__ bval,
                                             Emit emit)
{
    const int S = nx1 * ny1;
    const int z = n / S, y = (n - z * S) / nx1, x = n - z * S - y * nx1;
    const int nx = nx1 - 1, ny = ny1 - 1, nz = nz1 - 1;
    double k[2][2][2];  // [ez][ey][ex]: element (x - 1 + ex, y - 1 + ey, z - 1 + ez)
    int cnt = 0;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const int ex = c & 1, ey = (c >> 1) & 1, ez = c >> 2;
        const int cx = x - 1 + ex, cy = y - 1 + ey, cz = z - 1 + ez;
        const bool ok = cx >= 0 && cx < nx && cy >= 0 && cy < ny && cz >= 0 && cz < nz;
        k[ez][ey][ex] = ok ? kc[cx + nx * (cy + ny * cz)] : 0.0;
        cnt += ok ? 1 : 0;
    }
    // s[iz][iy][ix]: index 0 / 1 one element layer (the - / + side), 2 both
    double sm[3][3][3];
#pragma unroll
    for (int ez = 0; ez < 2; ++ez)
#pragma unroll
        for (int ey = 0; ey < 2; ++ey)
#pragma unroll
            for (int ex = 0; ex < 2; ++ex) sm[ez][ey][ex] = k[ez][ey][ex];
#pragma unroll
    for (int ey = 0; ey < 2; ++ey)
#pragma unroll
        for (int ex = 0; ex < 2; ++ex) sm[2][ey][ex] = k[0][ey][ex] + k[1][ey][ex];
#pragma unroll
    for (int ez = 0; ez < 2; ++ez)
#pragma unroll
        for (int ex = 0; ex < 2; ++ex) sm[ez][2][ex] = k[ez][0][ex] + k[ez][1][ex];
#pragma unroll
    for (int ez = 0; ez < 2; ++ez)
#pragma unroll
        for (int ey = 0; ey < 2; ++ey) sm[ez][ey][2] = k[ez][ey][0] + k[ez][ey][1];
#pragma unroll
    for (int ex = 0; ex < 2; ++ex) sm[2][2][ex] = sm[2][0][ex] + sm[2][1][ex];
#pragma unroll
    for (int ey = 0; ey < 2; ++ey) sm[2][ey][2] = sm[2][ey][0] + sm[2][ey][1];
#pragma unroll
    for (int ez = 0; ez < 2; ++ez) sm[ez][2][2] = sm[ez][2][0] + sm[ez][2][1];
    sm[2][2][2] = sm[2][2][0] + sm[2][2][1];
    int col = 0;
    const bool chk = near_bc && mask != nullptr;
    const bool rm = chk ? mask[n] != 0 : false;
    double lift = 0.0;
#pragma unroll
    for (int sl = 0; sl < 27; ++sl) {
        const int dx = sl % 3 - 1, dy = (sl / 3) % 3 - 1, dz = sl / 9 - 1;
        const int xx = x + dx, yy = y + dy, zz = z + dz;
        // neighbour offset -1 -> the - side layer (index 0), +1 -> index 1, 0 -> both (2)
        const int ix = dx < 0 ? 0 : (dx > 0 ? 1 : 2), iy = dy < 0 ? 0 : (dy > 0 ? 1 : 2),
                  iz = dz < 0 ? 0 : (dz > 0 ? 1 : 2);
        const int axes = (dx != 0 ? 1 : 0) | (dy != 0 ? 2 : 0) | (dz != 0 ? 4 : 0);
        if (xx < 0 || xx > nx || yy < 0 || yy > ny || zz < 0 || zz > nz) continue;
        double val = cls[axes] * sm[iz][iy][ix];
        if (chk) {
            const int mcol = xx + nx1 * (yy + ny1 * zz);
            if (rm) val = (sl == 13) ? 1.0 : 0.0;
            else if (mask[mcol]) {
                lift -= val * bval[mcol];
                val = 0.0;
            }
        }
        emit(col++, val);
    }
    const double dl = dref_f * (double)cnt;
    return rm ? bval[n] : (lift != 0.0 ? dl + lift : dl);
}

// One node's row of the thermal Q1 form on a mesh whose elements are all
// translates of element 0, in double-float: every entry of element e is k_e
// times a reference entry, so the row is a sum of at most 64 products, formed
// and summed as FP32 pairs (the FP32 pipe runs 64 times the FP64 one on
// GB300) in the same fixed order as gather_row_th (lane b adds column b of
// each incident element, elements ascending), then converted once per value
// to FP64 by integer operations.  L = 8 lanes per node; acc holds MF_MAX_DEG
// pairs.  near_bc: the node or a neighbour is constrained (only then are the
// columns read for the Dirichlet elimination; the FP64 lifting lives in that
// branch alone, so an interior row issues no FP64 instruction).
template <bool L2ONLY = false>
__device__ __forceinline__ void gather_row_th_q1df(int64_t n, int sub, unsigned gmask, float2 *acc, bool near_bc,
                                                   const int64_t *__restrict__ adj_ptr,
                                                   const int32_t *__restrict__ adj_col,
                                                   const int64_t *__restrict__ inc_ptr, const int32_t *__restrict__ inc,
                                                   const uint8_t *__restrict__ inc_loc,
                                                   const uint8_t *__restrict__ inc_slot,
                                                   const float2 *__restrict__ kref_df,
                                                   const float2 *__restrict__ kc_df, float2 f_df,
                                                   const uint8_t *__restrict__ mask, const double *__restrict__ bval,
                                                   const int64_t *__restrict__ row_ptr, double *__restrict__ values,
                                                   double *__restrict__ d)
{
    constexpr int NPE = 8, L = 8, U = 1;  // one element at a time: 32 registers, full occupancy (measured
                                          // fastest against 2, 4 and 8 elements' loads in flight)
    const int64_t p0 = adj_ptr[n];
    const int deg = (int)(adj_ptr[n + 1] - p0);
    // incidence entries number below 2^31 (checked when the pattern is built)
    const int32_t i0 = (int32_t)inc_ptr[n], i1 = (int32_t)inc_ptr[n + 1];
    const int64_t rb = row_ptr[n];
    for (int i = sub; i < deg; i += L) acc[i] = make_float2(0.f, 0.f);
    __syncwarp(gmask);
    // load vector: lane sub takes incidence entries i0 + sub, i0 + sub + L, ...
    float2 dsum = make_float2(0.f, 0.f);
    for (int32_t t = i0 + sub; t < i1; t += L)
        dsum = df_add(dsum, df_mul(f_df, kref_df[NPE * NPE + (inc_loc[t] & 0x7f)]));
    for (int32_t cb = i0; cb < i1; cb += U) {
        const int cnt = min(U, i1 - cb);
        float2 val[U];
        int s[U];
#pragma unroll
        for (int j = 0; j < U; ++j) {
            val[j] = make_float2(0.f, 0.f);
            s[j] = 0;
            if (j < cnt) {
                const int32_t t = cb + j;
                s[j] = inc_slot[(uint32_t)t * NPE + sub];
                val[j] = df_mul(ld_fresh<L2ONLY>(&kc_df[inc[t]]), kref_df[(inc_loc[t] & 0x7f) * NPE + sub]);
            }
        }
#pragma unroll
        for (int j = 0; j < U; ++j) {
            if (j < cnt) {  // group-uniform
                acc[s[j]] = df_add(acc[s[j]], val[j]);
                __syncwarp(gmask);
            }
        }
    }
#pragma unroll
    for (int o = L / 2; o > 0; o >>= 1)
        dsum = df_add(dsum, make_float2(__shfl_xor_sync(gmask, dsum.x, o, L), __shfl_xor_sync(gmask, dsum.y, o, L)));
    if (!near_bc) {
        for (int k = sub; k < deg; k += L) values[rb + k] = df_to_double_int(acc[k]);
        if (sub == 0) d[n] = df_to_double_int(dsum);
    } else {
        double lift = 0.0;
        const bool rm = mask[n] != 0;
        for (int k = sub; k < deg; k += L) {
            double v = df_to_double_int(acc[k]);
            const int32_t mcol = adj_col[p0 + k];
            if (rm) v = (mcol == n) ? 1.0 : 0.0;
            else if (mask[mcol]) {
                lift -= v * bval[mcol];
                v = 0.0;
            }
            values[rb + k] = v;
        }
#pragma unroll
        for (int o = L / 2; o > 0; o >>= 1) lift += __shfl_xor_sync(gmask, lift, o, L);
        if (sub == 0) d[n] = rm ? bval[n] : (lift != 0.0 ? df_to_double_int(dsum) + lift : df_to_double_int(dsum));
    }
    __syncwarp(gmask);
}

}  // namespace
