// Mixed-precision assembly of Q1 elasticity (tensor-core element contraction).
//
// The element matrix of linear elasticity (Sec. 4.2, -(d_i,j, sigma_ij) with
// the tangent negated) is, per block pair (a, b) of nodes,
//   K_ab[c][c'] = lambda A_ab[c][c'] + mu A_ab[c'][c] + mu delta_cc' tr A_ab,
//   A_ab[c][c'] = sum_q w_q detJ_q d_c N_a(q) d_c' N_b(q).
// With mu_e = E_e / (2 (1 + nu)) and lambda / mu = r = 2 nu / (1 - 2 nu) (the
// same for every element), scale the gradients
//   G[(a,c), q] = sqrt(mu_e w_q detJ_q) d_c N_a(q)                  (24 x 8)
// so that A'' = G G^T and K_e = r A'' + swap(A'') + I tr(A''); that map is
// linear, so it is applied once per CSR block after the element sums, with r
// held exactly as a 53-bit integer times a power of two (any nu).
//
// Precision plan (GB300 runs FP64 at 1/64 of FP32):
//  * geometry (Jacobian, cofactors, detJ, scale, gradients) in double-float
//    arithmetic (pairs of FP32, ~44 bits), one lane per (element, Gauss point),
//    from FP64 coordinate differences;
//  * the rows of G are ordered component-major (8 c + a) and split into 5
//    BF16 slices of 8 bits with one exponent per (element, component)
//    (Ozaki, Ogita, Oishi & Rump 2012): every slice product summed over the 8
//    points is an exact integer in FP32, so each level L = s + t of the slice
//    pairs accumulates exactly on the tensor cores (mma.sync m16n8k16, bf16
//    in, fp32 accumulate; fragments by ldmatrix.trans);
//  * the levels are combined into 64-bit fixed point at a global scale 2^S,
//    chosen per assembly by an FP32 pre-pass over the current coordinates and
//    coefficients so that no sum can overflow, and added with integer atomics
//    into one 3x3 block per node pair (n <= m; the lower pairs are
//    transposes): integer sums are exact, so the result does not depend on
//    the order the atomics land in; a node-centric finishing pass applies
//    r A + A^T + I tr A once per CSR block, converts each value once to FP64
//    and eliminates the Dirichlet dofs.
// The dropped levels (s + t > 4) bound the error at about 2^-40 of the
// element's scale; the solution error against the FP64 path is measured per
// run.
#include <cuda_bf16.h>

#include <algorithm>

#include "mf_internal.h"

namespace {

constexpr int MX_WARPS = 4;          // warps per block; each warp: 4 elements
constexpr int MX_ELEMS = 4 * MX_WARPS;
constexpr int NSL = 5;               // BF16 slices of G
constexpr int SL_ROWS = 24;          // rows (a, c) of G; the second m16 row tile's rows 24..31 are zero

struct MixedState {
    int S;         // global fixed-point exponent of K
    int mx_bits;   // max over elements of max_row sum_q G^2 (float bits, >= 0)
    int Sd;        // fixed-point exponent of the load vector d
    int vol_bits;  // max over elements of sum_q detJ_q (float bits, > 0)
};

// ---------------------------------------------------------------------------
// double-float arithmetic: value = h + l with |l| <= ulp(h) / 2
// ---------------------------------------------------------------------------
struct f2 {
    float h, l;
};

__device__ __forceinline__ f2 two_sum(float a, float b)
{
    const float s = a + b;
    const float bb = s - a;
    return {s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ f2 fast_two_sum(float a, float b)
{
    const float s = a + b;
    return {s, b - (s - a)};
}
__device__ __forceinline__ f2 dadd(f2 a, f2 b)
{
    f2 s = two_sum(a.h, b.h);
    s.l += a.l + b.l;
    return fast_two_sum(s.h, s.l);
}
__device__ __forceinline__ f2 dneg(f2 a) { return {-a.h, -a.l}; }
__device__ __forceinline__ f2 dsgn(f2 a, bool neg) { return neg ? dneg(a) : a; }
__device__ __forceinline__ f2 dsub(f2 a, f2 b) { return dadd(a, dneg(b)); }
__device__ __forceinline__ f2 dmul(f2 a, f2 b)
{
    const float p = a.h * b.h;
    float e = fmaf(a.h, b.h, -p);
    e = fmaf(a.h, b.l, e);
    e = fmaf(a.l, b.h, e);
    return fast_two_sum(p, e);
}
__device__ __forceinline__ f2 dmulf(f2 a, float b)
{
    const float p = a.h * b;
    float e = fmaf(a.h, b, -p);
    e = fmaf(a.l, b, e);
    return fast_two_sum(p, e);
}
__device__ __forceinline__ f2 ddiv(f2 a, f2 b)
{
    const float q1 = __fdiv_rn(a.h, b.h);
    const f2 r = dsub(a, dmulf(b, q1));
    return fast_two_sum(q1, __fdiv_rn(r.h, b.h));
}
__device__ __forceinline__ f2 dsqrt(f2 a)
{
    const float s = sqrtf(a.h);
    const float p = s * s;
    const float pe = fmaf(s, s, -p);  // s^2 = p + pe exactly
    const float r = ((a.h - p) - pe) + a.l;
    return fast_two_sum(s, __fdiv_rn(r, 2.0f * s));
}
__device__ __forceinline__ f2 from_double(double x)
{
    const float h = __double2float_rn(x);
    return {h, __double2float_rn(x - (double)h)};
}
__device__ __forceinline__ f2 shfl_xor(f2 v, int m)
{
    return {__shfl_xor_sync(0xffffffffu, v.h, m), __shfl_xor_sync(0xffffffffu, v.l, m)};
}
__device__ __forceinline__ f2 shfl(f2 v, int src)
{
    return {__shfl_sync(0xffffffffu, v.h, src), __shfl_sync(0xffffffffu, v.l, src)};
}

#define DF(x) f2{(float)(x), (float)((x) - (double)(float)(x))}

// 2-point Gauss abscissa G = 1/sqrt(3); factors P = 1 + G, M = 1 - G
constexpr double GD = 0.57735026918962576450914878050196;
// d_j N_a(q) = (1/8) s_a^j prod_{k != j} F_k, F_k in {P, M}:  products / 8
constexpr double KPP = 1.0 / 6.0 + GD / 4.0;   // P^2 / 8
constexpr double KPM = 1.0 / 12.0;             // P M / 8 = (1 - 1/3) / 8
constexpr double KMM = 1.0 / 6.0 - GD / 4.0;   // M^2 / 8
// N_a(q) = (1/8) prod_k F_k: P^3/8, P^2 M/8, P M^2/8, M^3/8 (3, 2, 1, 0 matches)
// one axis of N_a at a Gauss point: (1 + s_a s_q G) / 2, signs equal or opposite
constexpr double NEQ = (1.0 + GD) / 2.0;
constexpr double NOP = (1.0 - GD) / 2.0;


__device__ __forceinline__ int f2i_exact(float x)  // |x| < 2^22, integer valued
{
    return __float_as_int(x + 12582912.0f) - 0x4B400000;
}

__device__ __forceinline__ void mma_bf16(float (&c)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// ---------------------------------------------------------------------------
// pre-pass (per assembly, from the current coordinates and coefficients):
// bound of the fixed-point values, FP32 geometry is enough for a bound
// ---------------------------------------------------------------------------
// an FP64 value as FP32 by its bits, toward zero (integer operations only; the
// FP64 pipe runs at 1/64 of the FP32 rate): |x| below 2^-126 gives a signed
// zero, above the FP32 range an infinity (the bound then reports non-finite)
__device__ __forceinline__ float trunc_to_float(double x)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned sgn = (unsigned)(b >> 32) & 0x80000000u;
    const int e = (int)((b >> 52) & 0x7ff) - 1023 + 127;
    if (e <= 0) return __uint_as_float(sgn);
    if (e >= 255) return __uint_as_float(sgn | 0x7f800000u);
    return __uint_as_float(sgn | ((unsigned)e << 23) | (unsigned)((b >> 29) & 0x7fffffull));
}

// mx = max over elements of mu_e max_row sum_q G^2 / mu_e-free geometry,
// vol = max over elements of sum_q |detJ_q| (float bits, atomicMax on
// non-negative floats orders like the integers); one thread per element
constexpr int BOUND_THREADS = 256;
__global__ void __launch_bounds__(BOUND_THREADS) k_mixed_bound(int64_t n_el, const double *__restrict__ X,
                                                               const int32_t *__restrict__ conn,
                                                               const double *__restrict__ Ec, float cmu,
                                                               MixedState *st, int *status)
{
    __shared__ float red[2][BOUND_THREADS / 32];
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    float mx = 0.f, vol = 0.f;
    if (e < n_el) {
        float x[8][3];
        const int32_t *cn = conn + 8 * e;
        for (int a = 0; a < 8; ++a)
            for (int i = 0; i < 3; ++i)
                x[a][i] = trunc_to_float(X[3 * (int64_t)cn[a] + i] - X[3 * (int64_t)cn[0] + i]);
        const float g = (float)GD;
        float rowsum[24] = {};
        for (int q = 0; q < 8; ++q) {
            const float xs[3] = {(q & 1) ? g : -g, (q & 2) ? g : -g, (q & 4) ? g : -g};
            float J[3][3] = {}, dN[8][3];
            for (int a = 0; a < 8; ++a) {
                const float s[3] = {(a & 1) ? 1.f : -1.f, (a & 2) ? 1.f : -1.f, (a & 4) ? 1.f : -1.f};
                const float f[3] = {1.f + s[0] * xs[0], 1.f + s[1] * xs[1], 1.f + s[2] * xs[2]};
                dN[a][0] = 0.125f * s[0] * f[1] * f[2];
                dN[a][1] = 0.125f * f[0] * s[1] * f[2];
                dN[a][2] = 0.125f * f[0] * f[1] * s[2];
                for (int i = 0; i < 3; ++i)
                    for (int j = 0; j < 3; ++j) J[i][j] += x[a][i] * dN[a][j];
            }
            float C[3][3];
            C[0][0] = J[1][1] * J[2][2] - J[1][2] * J[2][1];
            C[0][1] = J[1][2] * J[2][0] - J[1][0] * J[2][2];
            C[0][2] = J[1][0] * J[2][1] - J[1][1] * J[2][0];
            C[1][0] = J[0][2] * J[2][1] - J[0][1] * J[2][2];
            C[1][1] = J[0][0] * J[2][2] - J[0][2] * J[2][0];
            C[1][2] = J[0][1] * J[2][0] - J[0][0] * J[2][1];
            C[2][0] = J[0][1] * J[1][2] - J[0][2] * J[1][1];
            C[2][1] = J[0][2] * J[1][0] - J[0][0] * J[1][2];
            C[2][2] = J[0][0] * J[1][1] - J[0][1] * J[1][0];
            const float det = J[0][0] * C[0][0] + J[0][1] * C[0][1] + J[0][2] * C[0][2];
            vol += fabsf(det);
            const float sc = 1.0f / fabsf(det);  // G^2 = (mu / det) (sum_j dN_j C[c][j])^2 per mu
            for (int a = 0; a < 8; ++a)
                for (int c = 0; c < 3; ++c) {
                    const float v = dN[a][0] * C[c][0] + dN[a][1] * C[c][1] + dN[a][2] * C[c][2];
                    rowsum[3 * a + c] += sc * v * v;
                }
        }
        for (int r = 0; r < 24; ++r) mx = fmaxf(mx, rowsum[r]);
        const double E = Ec[e];
        if (!isfinite(E) || !(E > 0.0)) {
            mf_dev_fail(status, MF_ERR_NONFINITE);
            mx = 0.f;
        } else {
            mx *= (float)E * cmu;
        }
    }
    // each thread tests its own values (fmaxf drops a NaN next to a number),
    // then block maxima: one atomic per block and quantity
    if (!isfinite(mx) || !isfinite(vol)) {
        mf_dev_fail(status, MF_ERR_NONFINITE);
        mx = vol = 0.f;
    }
    for (int o = 16; o > 0; o >>= 1) {
        mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        vol = fmaxf(vol, __shfl_xor_sync(0xffffffffu, vol, o));
    }
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        red[0][w] = mx;
        red[1][w] = vol;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int i = 1; i < BOUND_THREADS / 32; ++i) {
            mx = fmaxf(mx, red[0][i]);
            vol = fmaxf(vol, red[1][i]);
        }
        if (mx > 0.f) atomicMax(&st->mx_bits, __float_as_int(mx));
        if (vol > 0.f) atomicMax(&st->vol_bits, __float_as_int(vol));
    }
}

// S = floor(62 - log2(MF_MAX_INC (|r| + 4) Mx 1.25)): every element value
// |K_e| <= (|r| + 4) Mx 2^S and a CSR entry sums at most MF_MAX_INC of them,
// below 2^62.  The load entries are |b_c| sum_q detJ_q N_a(q) <= |b|max vol:
// Sd likewise.
__global__ void k_mixed_scale(MixedState *st, double rabs, double bmax)
{
    const float mx = __int_as_float(st->mx_bits);
    st->S = (int)floor(62.0 - log2((double)MF_MAX_INC * (rabs + 4.0) * (double)mx * 1.25));
    const double bv = bmax * (double)__int_as_float(st->vol_bits);
    st->Sd = bv > 0.0 ? (int)floor(62.0 - log2((double)MF_MAX_INC * bv * 1.25)) : 0;
}

// ---------------------------------------------------------------------------
// element kernel
// ---------------------------------------------------------------------------
struct WarpSmem {
    __nv_bfloat16 sl[4][NSL][8][SL_ROWS];  // slices of G per element: [slice][point][row (a,c)]
    int ex[4][3];                           // exponents per (element, component)
    int32_t tgt[4][36];                     // accumulator pair of block (a <= b); bit 31: transposed
};

__global__ void __launch_bounds__(MX_WARPS * 32, 6) k_mixed_elem(
    int64_t e0, int64_t e1, const double *__restrict__ X, const int32_t *__restrict__ conn,
    const double *__restrict__ Ec,
    double cmu, double b0, double b1, double b2, const MixedState *__restrict__ st,
    const int32_t *__restrict__ etgt, unsigned long long *__restrict__ kacc,
    unsigned long long *__restrict__ dacc, int *status)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];  // WarpSmem per warp (16-byte rows)
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    WarpSmem &W = reinterpret_cast<WarpSmem *>(smem_raw)[w];
    const int j = lane >> 3;   // element slot of this lane
    const int qp = lane & 7;   // Gauss point (and node for loads) of this lane
    const int gb = lane & ~7;  // first lane of the element group
    const int64_t e_raw = e0 + ((int64_t)blockIdx.x * MX_WARPS + w) * 4 + j;
    const bool valid = e_raw < e1;
    const int64_t e = valid ? e_raw : e1 - 1;

    // --- coordinates: d = x_q - x_0 in FP64, then double-float ---
    const int32_t *cn = conn + 8 * e;
    const int64_t n0 = cn[0], nq = cn[qp];
    f2 d[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) d[i] = from_double(X[3 * nq + i] - X[3 * n0 + i]);
    // Walsh-Hadamard transform over the 8 corners: lane k of the group gets
    // H[k] = sum_a (-1)^popcount(k & a) d_a; the trilinear coefficient of the
    // monomial with index k is (-1)^popcount(k) H[k] / 8.
#pragma unroll
    for (int m = 1; m < 8; m <<= 1)
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const f2 o = shfl_xor(d[i], m);
            d[i] = (qp & m) ? dsub(o, d[i]) : dadd(d[i], o);
        }
    {
        // pre-scale: k = 1,2,4 (linear) by 1/8; k = 3,5,6 by G/8; k = 7 by 1/24 (G^2 = 1/3)
        const int pc = __popc(qp);
        const f2 kf = (pc == 2) ? DF(GD / 8.0) : ((pc == 3) ? DF(1.0 / 24.0) : DF(1.0 / 8.0));
#pragma unroll
        for (int i = 0; i < 3; ++i) d[i] = dsgn(dmul(d[i], kf), pc & 1);
    }
    f2 C1[3], C2[3], C4[3], C3[3], C5[3], C6[3], C7[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        C1[i] = shfl(d[i], gb + 1);  // xi
        C2[i] = shfl(d[i], gb + 2);  // eta
        C4[i] = shfl(d[i], gb + 4);  // zeta
        C3[i] = shfl(d[i], gb + 3);  // xi eta    (x G)
        C5[i] = shfl(d[i], gb + 5);  // xi zeta   (x G)
        C6[i] = shfl(d[i], gb + 6);  // eta zeta  (x G)
        C7[i] = shfl(d[i], gb + 7);  // xi eta zeta (x 1/3)
    }
    // --- Jacobian at this lane's Gauss point ---
    const bool nx = !(qp & 1), ny = !(qp & 2), nz = !(qp & 4);  // sign of xi, eta, zeta is negative
    f2 J[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        J[i][0] = dadd(dadd(C1[i], dsgn(C3[i], ny)), dadd(dsgn(C5[i], nz), dsgn(C7[i], ny != nz)));
        J[i][1] = dadd(dadd(C2[i], dsgn(C3[i], nx)), dadd(dsgn(C6[i], nz), dsgn(C7[i], nx != nz)));
        J[i][2] = dadd(dadd(C4[i], dsgn(C6[i], ny)), dadd(dsgn(C5[i], nx), dsgn(C7[i], nx != ny)));
    }
    f2 Cf[3][3];
    Cf[0][0] = dsub(dmul(J[1][1], J[2][2]), dmul(J[1][2], J[2][1]));
    Cf[0][1] = dsub(dmul(J[1][2], J[2][0]), dmul(J[1][0], J[2][2]));
    Cf[0][2] = dsub(dmul(J[1][0], J[2][1]), dmul(J[1][1], J[2][0]));
    Cf[1][0] = dsub(dmul(J[0][2], J[2][1]), dmul(J[0][1], J[2][2]));
    Cf[1][1] = dsub(dmul(J[0][0], J[2][2]), dmul(J[0][2], J[2][0]));
    Cf[1][2] = dsub(dmul(J[0][1], J[2][0]), dmul(J[0][0], J[2][1]));
    Cf[2][0] = dsub(dmul(J[0][1], J[1][2]), dmul(J[0][2], J[1][1]));
    Cf[2][1] = dsub(dmul(J[0][2], J[1][0]), dmul(J[0][0], J[1][2]));
    Cf[2][2] = dsub(dmul(J[0][0], J[1][1]), dmul(J[0][1], J[1][0]));
    const f2 det = dadd(dadd(dmul(J[0][0], Cf[0][0]), dmul(J[0][1], Cf[0][1])), dmul(J[0][2], Cf[0][2]));

    // --- load vector: m_a = sum_q detJ_q N_a(q) ---
    {
        // N_a(q) is a product over the three axes of (1 + s_a s_q G) / 2, so
        // three butterflies over the point lanes (one per axis) turn detJ_q in
        // lane q into m_a in lane a
        f2 mine = det;
#pragma unroll
        for (int m = 1; m < 8; m <<= 1) {
            const f2 o = shfl_xor(mine, m);
            mine = dadd(dmul(mine, DF(NEQ)), dmul(o, DF(NOP)));
        }
        if (valid) {
            // d_(3 n + c) += b_c m_a, n = conn[e][a], in fixed point at 2^Sd
            const double mv = (double)mine.h + (double)mine.l;
            const double scl = ldexp(1.0, st->Sd);
            const double bb[3] = {b0, b1, b2};
#pragma unroll
            for (int cc = 0; cc < 3; ++cc) {
                const long long v = __double2ll_rn(bb[cc] * mv * scl);
                if (v != 0) atomicAdd(&dacc[3 * (int64_t)nq + cc], (unsigned long long)v);
            }
        }
    }
    __syncwarp();

    // --- scale sqrt(mu_e / det), mu_e = E cmu ---
    const double E = Ec[e];
    if (valid && !isfinite(E)) mf_dev_fail(status, MF_ERR_NONFINITE);
    const f2 sig = dsqrt(ddiv(from_double(E * cmu), det));
    // rows of G component-major, row 8 c + a:
    //   G[(c, a), qp] = sig sum_j d_j N_a(qp) Cf[c][j],
    // sum-factorised over the three factor products P^2/8, PM/8, M^2/8; one
    // component at a time, each with its own exponent: 2^(ex - 1) <= max over
    // the element's 8 x 8 values of component c < 2^ex.  The 8-bit digits of
    // x 2^-ex (exact) are rounded to nearest (magic-number rounding: |x| <
    // 2^22), digits 0..2 from the high word, the low word folded in before
    // digits 3 and 4.  A digit is an integer of at most 8 significant bits, so
    // its bfloat16 is the top half of its float: the 8 rows of a component
    // pack into one 16-byte store per slice in the [slice][point][row] layout.
    constexpr float RND = 12582912.0f;  // 1.5 2^23
    uint32_t *slw = reinterpret_cast<uint32_t *>(&W.sl[j][0][qp][0]);
#pragma unroll 1
    for (int c = 0; c < 3; ++c) {  // rolled: one copy of the code, the cofactor row picked by selects
        f2 T[3][3];  // T[j][k]: (sig Cf[c][j]) x {PP, PM, MM}
#pragma unroll
        for (int jj = 0; jj < 3; ++jj) {
            const f2 cf = c == 0 ? Cf[0][jj] : (c == 1 ? Cf[1][jj] : Cf[2][jj]);
            const f2 u = dmul(sig, cf);
            T[jj][0] = dmul(u, DF(KPP));
            T[jj][1] = dmul(u, DF(KPM));
            T[jj][2] = dmul(u, DF(KMM));
        }
        f2 G[8];
        float gmx = 0.f;
#pragma unroll
        for (int a = 0; a < 8; ++a) {
            const int match = ~(a ^ qp) & 7;  // bit k: s_a^k equals the sign of the point
            f2 acc = {0.f, 0.f};
#pragma unroll
            for (int jj = 0; jj < 3; ++jj) {
                const int others = match & ~(1 << jj) & 7;
                const int k = 2 - __popc(others);  // 2 matches -> PP, 1 -> PM, 0 -> MM
                const f2 t = (k == 0) ? T[jj][0] : ((k == 1) ? T[jj][1] : T[jj][2]);
                acc = jj == 0 ? dsgn(t, !(a & 1)) : dadd(acc, dsgn(t, !((a >> jj) & 1)));
            }
            G[a] = acc;
            gmx = fmaxf(gmx, fabsf(acc.h));
        }
        gmx = fmaxf(gmx, __shfl_xor_sync(0xffffffffu, gmx, 1));
        gmx = fmaxf(gmx, __shfl_xor_sync(0xffffffffu, gmx, 2));
        gmx = fmaxf(gmx, __shfl_xor_sync(0xffffffffu, gmx, 4));
        const int ex = (gmx > 0.f) ? (((__float_as_int(gmx) >> 23) & 0xff) - 126) : -200;
        if (qp == 0) W.ex[j][c] = ex;
        const float sc = (gmx > 0.f) ? __int_as_float((127 - ex) << 23) : 0.f;
        uint32_t pk[NSL][4];
#pragma unroll
        for (int pr = 0; pr < 4; ++pr) {
            float dgt[2][NSL];
#pragma unroll
            for (int h2 = 0; h2 < 2; ++h2) {
                float h = G[2 * pr + h2].h * sc, l = G[2 * pr + h2].l * sc;
#pragma unroll
                for (int sl = 0; sl < NSL; ++sl) {
                    h *= 256.f;
                    if (sl >= 3) {
                        l *= (sl == 3) ? 4294967296.0f : 256.f;  // the low word at the digit's scale
                        const f2 r = two_sum(h, l);
                        h = r.h;
                        l = r.l;
                    }
                    const float dg = (h + RND) - RND;
                    h -= dg;
                    dgt[h2][sl] = dg;
                }
            }
#pragma unroll
            for (int sl = 0; sl < NSL; ++sl)
                pk[sl][pr] = __byte_perm(__float_as_uint(dgt[0][sl]), __float_as_uint(dgt[1][sl]), 0x7632);
        }
#pragma unroll
        for (int sl = 0; sl < NSL; ++sl)
            *reinterpret_cast<uint4 *>(slw + sl * (8 * SL_ROWS / 2) + 4 * c) =
                make_uint4(pk[sl][0], pk[sl][1], pk[sl][2], pk[sl][3]);
    }
    // --- accumulator block of each upper block pair (a <= b) of the warp's 4
    // elements (precomputed with the pattern; bit 31: stored transposed) ---
    {
        const int64_t ebase = e0 + ((int64_t)blockIdx.x * MX_WARPS + w) * 4;
        for (int i = lane; i < 4 * 36; i += 32) {
            const int el = i / 36;
            W.tgt[el][i - 36 * el] = (ebase + el < e1) ? __ldg(etgt + ebase * 36 + i) : 0;
        }
    }
    __syncwarp();

    // --- tensor cores: A'' = G G^T by levels, per element of the warp;
    // fragments by ldmatrix.trans from the [point][row] slice layout ---
    const int g = lane >> 2, t = lane & 3;
    const int S = st->S;
    const uint32_t sl_base = (uint32_t)__cvta_generic_to_shared(&W.sl[0][0][0][0]);
    constexpr uint32_t PTB = SL_ROWS * 2, SLB = 8 * PTB, ELB = NSL * SLB;  // bytes per point, slice, element
    // the accumulator entries of this lane's outputs, the same for every
    // element.  Output (rho, sig2) of tile (m, n) is A''[(c, a), (c', b)],
    // c = rho / 8, a = rho % 8, c' = sig2 / 8 = n, b = sig2 % 8; the tiles
    // cover the component blocks (0,0), (1,0), (0,1), (1,1), (0,2), (1,2) and
    // (2,2).  Blocks (0,2) and (1,2) are taken whole (their a > b half is the
    // symmetric (2,0), (2,1) entry of the pair (b, a)), the others on a < b
    // and, for a = b, on c <= c'.  item: u = block pair (lo, hi) of the
    // element's nodes (u = lo (15 - lo) / 2 + hi), bits 6..9 the entry (row
    // component of lo, column component of hi), bits 10..13 the same entry
    // of the transposed block; 0xffff: not taken.
    uint32_t item[4][2];
#pragma unroll
    for (int tl = 0; tl < 4; ++tl) {  // tiles (m, n): (0,0), (0,1), (0,2), (1,2)
        const int mt = tl == 3 ? 1 : 0, nt = tl == 3 ? 2 : tl;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int rho = mt * 16 + g + 8 * (k >> 1);
            const int sig2 = nt * 8 + 2 * t + (k & 1);
            const int c = rho >> 3, a = rho & 7, cp = sig2 >> 3, b = sig2 & 7;
            uint32_t it = 0xffffu;
            if (c < 3) {
                int lo = a, hi = b, x = c, y = cp;
                bool ok;
                if (cp == 2 && c < 2) {
                    ok = true;
                    if (a > b) {
                        lo = b;
                        hi = a;
                        x = cp;
                        y = c;
                    }
                } else {
                    ok = a < b || (a == b && c <= cp);
                }
                if (ok) it = (uint32_t)((lo * (15 - lo) / 2 + hi) | ((3 * x + y) << 6) | ((3 * y + x) << 10));
            }
            if (k & 1) item[tl][k >> 1] |= it << 16;
            else item[tl][k >> 1] = it;
        }
    }
#pragma unroll 1
    for (int el = 0; el < 4; ++el) {
        const int64_t eo = e0 + ((int64_t)blockIdx.x * MX_WARPS + w) * 4 + el;
        if (eo >= e1) break;  // warp-uniform
        const uint32_t eb = sl_base + el * ELB;
        // fixed-point shift of entry (c, c'): G_c G_c'^T = T 2^(ex_c + ex_c' - 48)
        const int ex0 = W.ex[el][0], ex1 = W.ex[el][1], ex2 = W.ex[el][2];
#pragma unroll 1
        for (int tl = 0; tl < 4; ++tl) {
            const int mt = tl == 3 ? 1 : 0, nt = tl == 3 ? 2 : tl;
            const int shn = (nt == 0 ? ex0 : (nt == 1 ? ex1 : ex2)) + S - 48;
            const int sh_lo = (mt ? ex2 : ex0) + shn, sh_hi = ex1 + shn;  // rows c = 2 m, 2 m + 1
            const uint32_t iw0 = tl == 0 ? item[0][0] : (tl == 1 ? item[1][0] : (tl == 2 ? item[2][0] : item[3][0]));
            const uint32_t iw1 = tl == 0 ? item[0][1] : (tl == 1 ? item[1][1] : (tl == 2 ? item[2][1] : item[3][1]));
            uint32_t A[3][4], B[NSL][2];
            // A = slices (s0, s0 + 1) of rows mt 16 + ..; the second row tile
            // has 8 real rows (16..23), rows 24..31 are zero
#pragma unroll
            for (int sp = 0; sp < 3; ++sp) {  // slice pairs (0,1), (2,3), (4,-)
                const int s0 = 2 * sp, s1 = s0 + 1 < NSL ? s0 + 1 : s0;
                if (mt == 0) {
                    // matrices (rows 0-7 | 8-15) x (slice s0 | s1), stored as
                    // 8 point rows of 8 consecutive G rows
                    const int mi = lane >> 3;
                    const uint32_t ad = eb + ((mi >> 1) ? s1 : s0) * SLB + (lane & 7) * PTB + (mi & 1) * 16;
                    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                                 : "=r"(A[sp][0]), "=r"(A[sp][1]), "=r"(A[sp][2]), "=r"(A[sp][3]) : "r"(ad));
                } else {
                    // rows 16-23 of slice s0 (-> a0) and s1 (-> a2)
                    const uint32_t ad = eb + ((lane & 8) ? s1 : s0) * SLB + (lane & 7) * PTB + 32;
                    asm volatile("ldmatrix.sync.aligned.m8n8.x2.trans.shared.b16 {%0,%1}, [%2];\n"
                                 : "=r"(A[sp][0]), "=r"(A[sp][2]) : "r"(ad));
                    A[sp][1] = 0u;
                    A[sp][3] = 0u;
                }
                if (s0 + 1 >= NSL) {  // no slice s0 + 1: the second k half is zero
                    A[sp][2] = 0u;
                    A[sp][3] = 0u;
                }
            }
#pragma unroll
            for (int tp = 0; tp < NSL; ++tp) {  // B pairs (slice t', slice t' - 1), rows nt 8 + ..
                const int sb = ((lane >> 3) & 1) ? (tp > 0 ? tp - 1 : 0) : tp;
                const uint32_t ad = eb + sb * SLB + (lane & 7) * PTB + nt * 16;
                asm volatile("ldmatrix.sync.aligned.m8n8.x2.trans.shared.b16 {%0,%1}, [%2];\n"
                             : "=r"(B[tp][0]), "=r"(B[tp][1]) : "r"(ad));
                if (tp == 0) B[tp][1] = 0u;
            }
            float acc[5][4];
#pragma unroll
            for (int L = 0; L < 5; ++L)
#pragma unroll
                for (int k = 0; k < 4; ++k) acc[L][k] = 0.f;
            // level L = sum over s0 = 0, 2, 4 <= L of [slice s0 | s0 + 1] x [slice L - s0 | L - s0 - 1]
#pragma unroll
            for (int L = 0; L < 5; ++L)
#pragma unroll
                for (int s0 = 0; s0 <= L; s0 += 2)
                    mma_bf16(acc[L], A[s0 / 2][0], A[s0 / 2][1], A[s0 / 2][2], A[s0 / 2][3], B[L - s0][0],
                             s0 + 1 <= L ? B[L - s0][1] : 0u);
            // levels -> 64-bit fixed point at scale 2^S, added into the node-pair
            // block accumulator (exact integer sums: any order gives the same
            // bits); the r finishing is linear and is applied once per CSR
            // block after all elements
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const uint32_t it = ((k >> 1 ? iw1 : iw0) >> (16 * (k & 1))) & 0xffffu;
                if (it == 0xffffu) continue;
                const int sh = (k >> 1) ? sh_hi : sh_lo;
                // T = sum_L acc[L] 256^(4 - L): each level is an integer below
                // 2^22 in magnitude (at most 5 digit products of 2^16, 8 points),
                // so the pairs (0, 1) and (2, 3) combine exactly in int32 and two
                // wide multiply-adds finish the int64 value
                const int hi = f2i_exact(acc[0][k]) * 256 + f2i_exact(acc[1][k]);
                const int mid = f2i_exact(acc[2][k]) * 256 + f2i_exact(acc[3][k]);
                const long long T = (long long)hi * 16777216ll + ((long long)mid * 256ll + f2i_exact(acc[4][k]));
                long long v;
                if (sh >= 0) v = T << sh;
                else if (sh > -62) v = (T + (1ll << (-sh - 1))) >> (-sh);
                else v = 0;
                const int32_t tg = W.tgt[el][it & 63];
                const int64_t pr = tg & 0x7fffffff;
                const int q = tg < 0 ? (int)(it >> 10) & 15 : (int)(it >> 6) & 15;
                if (v != 0) atomicAdd(&kacc[pr * 9 + q], (unsigned long long)v);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// finishing: one warp per node.  Lane k takes neighbour k's 3x3 block from the
// accumulator (its own pair (n, m) for m > n, the transpose of (m, n) for
// m < n, the upper triangle of the diagonal block for m = n; the load
// offsets are picked per lane), applies K = r A + A^T + I tr A in int64,
// converts each value once to FP64 and eliminates the Dirichlet dofs (blocks
// with no constrained row or column skip those tests); the three rows are
// staged in shared memory and written with coalesced stores.
// ---------------------------------------------------------------------------
// floor(A R / 2^s), 1 <= s <= 63: bits s .. s + 63 of the 128-bit product
__device__ __forceinline__ long long mul_r(long long A, long long R, int s)
{
    const long long hi = __mul64hi(A, R);
    const unsigned long long lo = (unsigned long long)A * (unsigned long long)R;
    return (long long)((lo >> s) | ((unsigned long long)hi << (64 - s)));
}
// r A with r = R 2^-s exactly; a short multiplier (|R| < 2^20, e.g. r = 3/2
// for nu = 0.3) takes one 64 x 32-bit product (|A| < 2^42 then: the scale
// keeps r A below 2^62)
__device__ __forceinline__ long long times_r(long long A, long long R, int s)
{
    if (R > -(1ll << 20) && R < (1ll << 20)) return (A * R) >> s;
    return mul_r(A, R, s);
}

// v 2^-S as FP64, rounded to nearest even (values below the normal range
// flush to signed zero): the hardware conversion of the integer, then the
// exponent lowered by S
__device__ __forceinline__ double fixed_to_double(long long v, int S)
{
    if (v == 0) return 0.0;
    const long long bits = __double_as_longlong(__ll2double_rn(v));
    const long long ex = ((bits >> 52) & 0x7ff) - S;
    if (ex <= 0) return __longlong_as_double(bits & (1ll << 63));
    return __longlong_as_double(bits - ((long long)S << 52));
}

// flag[n] = 1 for every node n holding a constrained dof or adjacent to one
// (the adjacency includes each node itself)
__global__ void k_mark_bc_nodes(int64_t n_nodes, const int64_t *__restrict__ adj_ptr,
                                const int32_t *__restrict__ adj_col, const uint8_t *__restrict__ mask,
                                uint8_t *__restrict__ flag)
{
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= 3 * n_nodes || !mask[s]) return;
    const int64_t m = s / 3;
    for (int64_t q = adj_ptr[m]; q < adj_ptr[m + 1]; ++q) flag[adj_col[q]] = 1;
}

constexpr int FN_WARPS = 8;

__global__ void __launch_bounds__(FN_WARPS * 32, 4) k_mixed_finish(
    int64_t n_begin, int64_t n_nodes, const int64_t *__restrict__ adj_ptr, const int32_t *__restrict__ adj_col,
    const int32_t *__restrict__ tpos, const long long *__restrict__ kacc, const long long *__restrict__ dacc,
    const MixedState *__restrict__ st, long long rR, int rs, const uint8_t *__restrict__ mask_all,
    const uint8_t *__restrict__ bcnode, const double *__restrict__ bval, const int64_t *__restrict__ row_ptr,
    double *__restrict__ values, double *__restrict__ d)
{
    __shared__ double rows_all[FN_WARPS][3][3 * MF_MAX_DEG];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t n = n_begin + (int64_t)blockIdx.x * FN_WARPS + w;
    if (n >= n_nodes) return;  // warp-uniform
    double(*rows)[3 * MF_MAX_DEG] = rows_all[w];
    // the Dirichlet tests only on nodes with a constrained dof at or next to them
    const uint8_t *mask = (mask_all && bcnode[n]) ? mask_all : nullptr;
    const int S = st->S, Sd = st->Sd;
    const int64_t p0 = adj_ptr[n];
    const int deg = (int)(adj_ptr[n + 1] - p0);
    bool rm[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) rm[c] = mask ? mask[3 * n + c] != 0 : false;
    const bool rm_any = rm[0] || rm[1] || rm[2];
    double lift[3] = {0.0, 0.0, 0.0};
    for (int k = lane; k < deg; k += 32) {
        const int32_t mcol = adj_col[p0 + k];
        const int64_t src = tpos[p0 + k];  // the accumulator block of pair (n, mcol)
        const long long *B = kacc + src * 9;
        // A[c][c'] = B[3 c + c'] (m > n), B[3 c' + c] (m < n), the upper
        // triangle of the diagonal block (m = n): offsets picked per lane
        const int orient = mcol > n ? 0 : (mcol < n ? 1 : 2);
        long long A[3][3];
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int cp = 0; cp < 3; ++cp) {
                const int o0 = 3 * c + cp, o1 = 3 * cp + c, o2 = 3 * (c < cp ? c : cp) + (c < cp ? cp : c);
                A[c][cp] = B[orient == 0 ? o0 : (orient == 1 ? o1 : o2)];
            }
        const long long tr = A[0][0] + A[1][1] + A[2][2];
        unsigned cm = 0;
        if (mask)
#pragma unroll
            for (int cp = 0; cp < 3; ++cp) cm |= (mask[3 * (int64_t)mcol + cp] != 0 ? 1u : 0u) << cp;
        if (!rm_any && cm == 0) {  // no constrained row or column: the plain block
#pragma unroll
            for (int c = 0; c < 3; ++c)
#pragma unroll
                for (int cp = 0; cp < 3; ++cp) {
                    long long kv = times_r(A[c][cp], rR, rs) + A[cp][c];
                    if (c == cp) kv += tr;
                    rows[c][3 * k + cp] = fixed_to_double(kv, S);
                }
        } else {
#pragma unroll
            for (int c = 0; c < 3; ++c)
#pragma unroll
                for (int cp = 0; cp < 3; ++cp) {
                    long long kv = times_r(A[c][cp], rR, rs) + A[cp][c];
                    if (c == cp) kv += tr;
                    double v = fixed_to_double(kv, S);
                    const int64_t sdof = 3 * (int64_t)mcol + cp;
                    if (rm[c]) v = (3 * n + c == sdof) ? 1.0 : 0.0;
                    else if ((cm >> cp) & 1u) {
                        lift[c] -= v * bval[sdof];
                        v = 0.0;
                    }
                    rows[c][3 * k + cp] = v;
                }
        }
    }
    __syncwarp();
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const int64_t r = 3 * n + c;
        const int64_t rb = row_ptr[r];
        for (int j = lane; j < 3 * deg; j += 32) values[rb + j] = rows[c][j];
        double l = lift[c];
        if (__any_sync(0xffffffffu, l != 0.0))  // rows next to a constrained dof only
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
        if (lane == 0) d[r] = rm[c] ? bval[r] : fixed_to_double(dacc[r], Sd) + l;
    }
}

}  // namespace

mf_status mf_assemble_mixed(int form, const mf_mesh *m, const mf_pattern *p, const mf_coeffs *c, double *values,
                            double *d, cudaStream_t st)
{
    if (form != MF_FORM_ELASTIC || m->elem != MF_Q1_HEX || !p->slot || !p->mixed_state)
        return mf_fail(MF_ERR_UNSUPPORTED, "mf_assemble: the mixed path covers Q1 elasticity");
    const double nu = c->nu;
    if (!(nu > -1.0 && nu < 0.5)) return mf_fail(MF_ERR_INVALID_ARG, "mf_assemble: Poisson ratio outside (-1, 0.5)");
    // lambda / mu = r = 2 nu / (1 - 2 nu) exactly as rR 2^-rs (a 53-bit integer)
    const double r = 2.0 * nu / (1.0 - 2.0 * nu);
    long long rR = 0;
    int rs = 1;
    if (r != 0.0) {
        int ex = 0;
        const double fr = frexp(r, &ex);  // r = fr 2^ex, 0.5 <= |fr| < 1
        rR = (long long)ldexp(fr, 53);
        rs = 53 - ex;
        while (rs > 1 && (rR & 1) == 0) {
            rR /= 2;
            --rs;
        }
        if (rs > 63) {  // |r| < 2^-11: the bits of r below 2^-63 are dropped (r A is tiny next to A^T)
            rR /= (1ll << std::min(rs - 63, 62));
            rs = 63;
        }
        if (rs < 1) return mf_fail(MF_ERR_UNSUPPORTED, "mf_assemble: Poisson ratio out of the mixed path's range");
    }
    int *status = mf_status_word();
    if (!status) return mf_fail(MF_ERR_CUDA, "mf_assemble: status word unavailable");
    const double cmu = 1.0 / (2.0 * (1.0 + nu));
    MixedState *ms = static_cast<MixedState *>(p->mixed_state);
    const int64_t ne = m->n_elems;
    // element blocks go straight into the int64 block accumulator (atomics:
    // exact, so order-free); the finishing gather then writes each CSR row once.
    // The accumulator clears (HBM writes) and the node flags run on the
    // pattern's clear stream beside the bound pass (latency-bound gathers);
    // the element kernel waits for both.
    MF_CUDA(cudaEventRecord(p->clr_fork, st));
    MF_CUDA(cudaStreamWaitEvent(p->clr_side, p->clr_fork, 0));
    MF_CUDA(cudaMemsetAsync(p->kacc, 0, sizeof(long long) * 9 * p->n_upper, p->clr_side));
    MF_CUDA(cudaMemsetAsync(p->dacc, 0, sizeof(long long) * 3 * m->n_nodes, p->clr_side));
    if (c->bc_mask) {  // nodes at or next to a constrained dof
        MF_CUDA(cudaMemsetAsync(p->bcrow, 0, (size_t)m->n_nodes, p->clr_side));
        k_mark_bc_nodes<<<(unsigned)((3 * m->n_nodes + 255) / 256), 256, 0, p->clr_side>>>(
            m->n_nodes, p->adj[0].ptr, p->adj[0].col, c->bc_mask, p->bcrow);
    }
    MF_CUDA(cudaEventRecord(p->clr_join, p->clr_side));
    mf_prof_begin("mixed_bound", st);
    MF_CUDA(cudaMemsetAsync(ms, 0, sizeof(MixedState), st));
    if (ne > 0)
        k_mixed_bound<<<(unsigned)((ne + BOUND_THREADS - 1) / BOUND_THREADS), BOUND_THREADS, 0, st>>>(
            ne, m->coords, m->conn, c->elem_coef, (float)cmu, ms, status);
    const double bmax = fmax(fabs(c->source[0]), fmax(fabs(c->source[1]), fabs(c->source[2])));
    k_mixed_scale<<<1, 1, 0, st>>>(ms, fabs(r), bmax);
    mf_prof_end(st);
    MF_CUDA(cudaStreamWaitEvent(st, p->clr_join, 0));
    const size_t smem = sizeof(WarpSmem) * MX_WARPS;
    MF_CUDA(cudaFuncSetAttribute(k_mixed_elem, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    // element chunks on the caller's stream; with more than one chunk the
    // finishing of the nodes a chunk completes runs on the side stream
    // (MF_SLABS: one chunk measured fastest)
    return mf_slab_pipeline(
        p, st,
        [&](size_t k, cudaStream_t s2) -> mf_status {
            const int64_t e0 = p->slab_e[k], e1 = p->slab_e[k + 1];
            mf_prof_begin("mixed_elem", s2);
            k_mixed_elem<<<(unsigned)((e1 - e0 + MX_ELEMS - 1) / MX_ELEMS), MX_WARPS * 32, smem, s2>>>(
                e0, e1, m->coords, m->conn, c->elem_coef, cmu, c->source[0], c->source[1], c->source[2], ms,
                p->etgt, reinterpret_cast<unsigned long long *>(p->kacc),
                reinterpret_cast<unsigned long long *>(p->dacc), status);
            mf_prof_end(s2);
            MF_CUDA(cudaGetLastError());
            return MF_OK;
        },
        [&](size_t k, cudaStream_t s2) -> mf_status {
            const int64_t n0 = p->slab_n[k], n1 = p->slab_n[k + 1];
            if (n1 > n0) {
                mf_prof_begin("mixed_finish", s2);
                k_mixed_finish<<<(unsigned)((n1 - n0 + FN_WARPS - 1) / FN_WARPS), FN_WARPS * 32, 0, s2>>>(
                    n0, n1, p->adj[0].ptr, p->adj[0].col, p->tpos, p->kacc, p->dacc, ms, rR, rs, c->bc_mask,
                    p->bcrow, c->bc_val, p->row_ptr, values, d);
                mf_prof_end(s2);
            }
            MF_CUDA(cudaGetLastError());
            return MF_OK;
        });
}
