// FP64 assembly of K and d (MetaFEM Sec. 2.2 Block D-2 / D-3).
//
// Two kernels per form.  The element kernel evaluates the quadrature of the
// form (Sec. 2.1) for one element per thread and writes the element blocks
// to a scratch array.  The gather kernel then builds every CSR row node by
// node: it walks the node's incident elements in ascending order and adds
// their rows into a shared-memory row through the pattern's slot maps, so the
// contributions of one entry are summed in ascending element order (the
// paper increments K with atomics in Block D-3; a fixed order makes K
// bit-reproducible); the strong Dirichlet elimination is applied, and every
// value of K and d is written exactly once, so no separate clearing pass is
// needed.  (The mixed elasticity path, mf_mixed.cu, adds exact integer
// blocks with atomics instead.)
//
// Forms (K positive; Sec. 4.1-4.3):
//   thermal   Ke[a][b] = sum_q w detJ k gradN_a . gradN_b,  de[a] = sum_q w detJ f N_a
//   elastic   Ke[(a,c),(b,c')] = lambda A_ab[c][c'] + mu A_ab[c'][c] + mu delta_cc' tr A_ab
//             with A_ab = sum_q w detJ gradN_a gradN_b^T,   de[(a,c)] = body_c sum_q w detJ N_a
//   flow      A[a][b] = sum_q w detJ (mu gradN_a.gradN_b - rho (a_h.gradN_a) N_b),
//             B_i[a][b] = sum_q w detJ M_a d_i N_b; the u-p block is -B_i^T.
#include "mf_fem.cuh"

namespace {

inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }



// ---------------------------------------------------------------------------
// element kernels
// ---------------------------------------------------------------------------
__global__ void k_elem_thermal_p1(int64_t n_el, const double *__restrict__ X, const int32_t *__restrict__ conn,
                                  const double *__restrict__ kc, double f, const int32_t *__restrict__ map,
                                  double *__restrict__ out, int *status)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n_el) elem_thermal_p1(e, X, conn, kc, f, map, out, status);
}

// 10-node tetrahedra: one element per thread; its incidence rows go out one
// row index a at a time through a per-warp stage in shared memory, so that
// the warp stores whole 96-byte rows (about three per store instruction)
// instead of 32 scattered words
__global__ void __launch_bounds__(128) k_elem_thermal_p2t(int64_t n_el, const double *__restrict__ X,
                                                          const int32_t *__restrict__ conn,
                                                          const double *__restrict__ kc, double f,
                                                          const int32_t *__restrict__ map, double *__restrict__ out,
                                                          int *status)
{
    constexpr int RS = mf_th_rs(10);       // 12 words per row
    __shared__ double stage[4][32][13];    // row of each lane (stride 13: no bank conflicts)
    __shared__ int32_t rows[4][32][11];    // incidence entries of each lane's element
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    float2 G[6];
    double lv = 0.0, le = 0.0;
    const bool has = p2t_metric(e, n_el, X, conn, kc, f, G, lv, le, status);
    if (has)
#pragma unroll
        for (int a = 0; a < 10; ++a) rows[w][lane][a] = map[e * 10 + a];
    // lanes of the warp that hold an element (the last block's tail)
    const int64_t w0 = (int64_t)blockIdx.x * blockDim.x + 32 * w;
    const int nl = (int)(n_el - w0 < 32 ? (n_el - w0 > 0 ? n_el - w0 : 0) : 32);
#pragma unroll 1
    for (int a = 0; a < 10; ++a) {
        if (has) {
#pragma unroll
            for (int b = 0; b < 10; ++b) stage[w][lane][b] = p2t_entry(G, a, b);
            stage[w][lane][10] = a < 4 ? lv : le;
            stage[w][lane][11] = 0.0;
        }
        __syncwarp();
        for (int i = lane; i < nl * RS; i += 32) {
            const int L = i / RS, j = i - RS * L;
            out[(int64_t)rows[w][L][a] * RS + j] = stage[w][L][j];
        }
        __syncwarp();
    }
}

__global__ void __launch_bounds__(128) k_elem_thermal_q2q(int64_t n_el, const double *__restrict__ X,
                                                          const int32_t *__restrict__ conn,
                                                          const double *__restrict__ kc, double f,
                                                          const int32_t *__restrict__ map, double *__restrict__ out,
                                                          int *status)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n_el) elem_thermal_q2q(e, X, conn, kc, f, map, out, status);
}

__global__ void k_elem_thermal_p2(int64_t n_el, const double *__restrict__ X, const int32_t *__restrict__ conn,
                                  const double *__restrict__ kc, double f, const int32_t *__restrict__ map,
                                  double *__restrict__ out, int *status)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n_el) elem_thermal_p2(e, X, conn, kc, f, map, out, status);
}

__global__ void __launch_bounds__(128) k_elem_thermal_q1(int64_t n_el, const double *__restrict__ X,
                                                         const int32_t *__restrict__ conn,
                                                         const double *__restrict__ kc, double f,
                                                         const uint8_t *__restrict__ tr,
                                                         const int32_t *__restrict__ map, double *__restrict__ out,
                                                         int *status)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n_el && !q1_translate(e, tr, kc, status)) elem_thermal_q1(e, X, conn, kc, f, map, out, status);
}

__global__ void k_elem_capacity(int elem, int64_t n_el, const double *__restrict__ X,
                                const int32_t *__restrict__ conn, const double *__restrict__ kc,
                                const uint8_t *__restrict__ tr, const int32_t *__restrict__ map,
                                double *__restrict__ out, int *status)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n_el) return;
    if (elem == MF_P1_TRI) elem_capacity_p1(e, X, conn, kc, map, out, status);
    else if (elem == MF_P2_TRI) elem_capacity_p2(e, X, conn, kc, map, out, status);
    else if (elem == MF_P2_TET) elem_capacity_p2t(e, X, conn, kc, map, out, status);
    else if (elem == MF_Q2S_QUAD) elem_capacity_q2q(e, X, conn, kc, map, out, status);
    else if (!q1_translate(e, tr, kc, status)) elem_capacity_q1(e, X, conn, kc, map, out, status);
}

// 20-node serendipity brick, thermal form (Sec. 4.1), 3 x 3 x 3 Gauss: one
// warp per element, every phase spread over all 32 lanes.  FP64 is the scarce
// pipe (1/64 of the FP32 rate here): the shape values and reference gradients
// at the 27 points come from a table, and everything but the map
// coefficients and the load runs in double-float (FP32 pairs, about 47
// bits).  (0) lanes < 24 load the element's map coefficients (cached by the
// pattern); (1) lanes
// q < 27 the geometry of Gauss point q from the trilinear map (q2s_point_df):
// w detJ, and sqrt(w detJ) J^-T (detJ > 0 at every point is checked when the
// mesh is made); (2) the 540 (node,
// point) items form sqrt(w detJ) times the physical gradients, 9 points at a
// time (less shared memory, more resident warps); (3) the 210 pairs a <= b of
// K_e = k sum_q w detJ grad N_a . grad N_b are spread over the lanes (6 or 7
// each), summed over the chunks in double-float and written to rows a and b;
// lanes a < 20 add d_e[a] = f sum_q w detJ N_a (FP64).  Output as the other
// thermal elements (incidence layout).
constexpr int Q2W = 4;  // elements (warps) per block
constexpr int QCH = 9;  // Gauss points per chunk of gradients in shared memory

__global__ void __launch_bounds__(Q2W * 32) k_elem_thermal_q2s(int64_t n_el, const float2 *__restrict__ gmap,
                                                               const double *__restrict__ kc, double f,
                                                               const int32_t *__restrict__ map,
                                                               double *__restrict__ out, int *status)
{
    __shared__ double wdet[Q2W][27];         // w detJ
    __shared__ float2 Mq[Q2W][27][9];        // sqrt(w detJ) (J^-1)_ji at [i][j], FP32 pairs
    __shared__ float2 cw[Q2W][8][3];         // map coefficients, FP32 pairs
    __shared__ float2 grd[Q2W][QCH][20][3];  // sqrt(w detJ) times the physical gradients, one chunk of points
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t e = (int64_t)blockIdx.x * Q2W + w;
    if (e >= n_el) return;  // warp-uniform
    if (lane < 24) cw[w][lane / 3][lane % 3] = gmap[e * 24 + lane];  // map coefficient c_S[i], S = lane / 3
    __syncwarp();
    if (lane < 27) {
        float2 c[8][3], M9[9];
#pragma unroll
        for (int S = 0; S < 8; ++S)
#pragma unroll
            for (int i = 0; i < 3; ++i) c[S][i] = cw[w][S][i];
        wdet[w][lane] = df_to_double(q2s_point_df(c, lane, M9));
#pragma unroll
        for (int k = 0; k < 9; ++k) Mq[w][lane][k] = M9[k];
    }
    // pairs p = lane + 32 t (t < 7, p < 210) of the upper triangle, row-major
    int pa[7], pb[7];
#pragma unroll
    for (int t = 0; t < 7; ++t) {
        const int p = lane + 32 * t;
        int a = 0, rem = p < 210 ? p : 0;
        while (rem >= 20 - a) {
            rem -= 20 - a;
            ++a;
        }
        pa[t] = p < 210 ? a : -1;
        pb[t] = a + rem;
    }
    float sh[7], sl[7];
#pragma unroll
    for (int t = 0; t < 7; ++t) sh[t] = sl[t] = 0.0f;
    for (int q0 = 0; q0 < 27; q0 += QCH) {
        __syncwarp();  // geometry written / the last chunk's gradients read
        for (int it = lane; it < QCH * 20; it += 32) {  // grad N = J^-T gradref N, in FP32 pairs
            const int qq = it / 20, a = it - 20 * qq, q = q0 + qq;
            const float2 *T = c_q2s_tabf[q][a];
            const float2 t0 = T[0], t1 = T[1], t2 = T[2];
#pragma unroll
            for (int i = 0; i < 3; ++i)
                grd[w][qq][a][i] = df_add(df_add(df_mul(Mq[w][q][3 * i], t0), df_mul(Mq[w][q][3 * i + 1], t1)),
                                          df_mul(Mq[w][q][3 * i + 2], t2));
        }
        __syncwarp();
        // double-float Gram sums (exact products of the high parts by FMA,
        // cross terms of the low parts, two-sum accumulation)
#pragma unroll
        for (int t = 0; t < 7; ++t) {
            if (pa[t] < 0) continue;
            for (int qq = 0; qq < QCH; ++qq)
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    const float2 x = grd[w][qq][pa[t]][i], y = grd[w][qq][pb[t]][i];
                    const float p = x.x * y.x;
                    const float ep = fmaf(x.x, y.x, -p) + fmaf(x.x, y.y, x.y * y.x);
                    const float tt = sh[t] + p;  // two-sum of sh and p
                    const float z = tt - sh[t];
                    sl[t] += ((sh[t] - (tt - z)) + (p - z)) + ep;
                    sh[t] = tt;
                }
        }
    }
    const double k = kc[e];
    if (!isfinite(k)) mf_dev_fail(status, MF_ERR_NONFINITE);
#pragma unroll
    for (int t = 0; t < 7; ++t) {
        if (pa[t] < 0) continue;
        const double kv = k * (f32_to_f64_exact(sh[t]) + f32_to_f64_exact(sl[t]));
        out[(int64_t)map[e * 20 + pa[t]] * 21 + pb[t]] = kv;
        out[(int64_t)map[e * 20 + pb[t]] * 21 + pa[t]] = kv;
    }
    if (lane < 20) {
        double m = 0.0;
        for (int q = 0; q < 27; ++q) m = fma(wdet[w][q], c_q2s_tab[q][lane][0], m);
        out[(int64_t)map[e * 20 + lane] * 21 + 20] = f * m;
    }
}

// 20-node serendipity brick, linear elasticity (Sec. 4.2, the element of the
// cantilever beams), 3 x 3 x 3 Gauss: one block per element, from the map
// coefficients cached by the pattern.  The geometry (q2s_point_df) and the
// gradients sqrt(w detJ) grad N_a(q) are formed in
// double-float as in the thermal brick (all 27 points at once, [q][i][a] so
// that the threads of a warp read consecutive nodes); thread p < 210 then
// takes the pair a <= b (row-major upper triangle), sums the nine entries of
// M_ab[i][j] = sum_q w detJ d_i N_a d_j N_b and finishes
// K_ab = lambda M_ab + mu M_ab^T + mu tr(M_ab) I, all in double-float (FP64
// runs at 1/64 of the FP32 rate here; lambda and mu are formed once per
// element).  Row a of element e is incidence entry t = map[e * 20 + a] of
// EQ_ROW 8-byte words: K_ab for b < 20 (3 x 3, row-major) as FP32 pairs
// (hi, lo), then d_e(a) (3 doubles); K_ba = K_ab^T goes to row b.
constexpr int EQ_T = 224;  // 7 warps: one thread per pair a <= b (210)
constexpr int EQ_ROW = 20 * 9 + 3;

__global__ void __launch_bounds__(EQ_T) k_elem_elastic_q2s(int64_t n_el, const float2 *__restrict__ gmap,
                                                           const double *__restrict__ Ec, double nu, double b0,
                                                           double b1, double b2, const int32_t *__restrict__ map,
                                                           double *__restrict__ out, int *status)
{
    __shared__ float2 cw[8][3];         // map coefficients, FP32 pairs
    __shared__ float2 lmu[2];           // lambda, mu
    __shared__ double wdet[27];         // w detJ
    __shared__ float2 Mq[27][9];        // J[q][i][j], then sqrt(w detJ) (J^-1)_ji at [q][3 i + j]
    __shared__ float2 Cq[27][9];        // cofactors: detJ (J^-1)_ji at [q][3 j + i]
    __shared__ float2 grd[27][3][20];   // sqrt(w detJ) d_i N_a at [q][i][a]
    __shared__ int32_t tmap[20];
    const int tid = threadIdx.x;
    const int64_t e = blockIdx.x;
    if (e >= n_el) return;  // block-uniform
    if (tid < 24) {
        cw[tid / 3][tid % 3] = gmap[e * 24 + tid];  // map coefficient c_S[i], S = tid / 3
    } else if (tid >= 32 && tid < 52) {
        tmap[tid - 32] = map[e * 20 + tid - 32];
    } else if (tid == 64) {
        const double E = Ec[e];
        if (!isfinite(E)) mf_dev_fail(status, MF_ERR_NONFINITE);
        const double lm[2] = {E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu)), E / (2.0 * (1.0 + nu))};
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const float hi = __double2float_rn(lm[k]);
            lmu[k] = make_float2(hi, __double2float_rn(lm[k] - (double)hi));
        }
    }
    // the geometry of q2s_point_df spread over the block in three short
    // phases (the Jacobian entries, the cofactors, then per point detJ,
    // sqrt(w detJ) / detJ and the scaled inverse), so that the warps do not
    // wait on one long dependent chain
    constexpr double G3 = 0.77459666924148337704;  // sqrt(3/5)
    constexpr double W5 = 5.0 / 9.0, W8 = 8.0 / 9.0;
    const float2 g3 = make_float2((float)G3, (float)(G3 - (double)(float)G3));
    __syncthreads();
    for (int it = tid; it < 27 * 9; it += EQ_T) {  // J[q][i][j]
        const int q = it / 9, i = (it - 9 * q) / 3, j = it - 9 * q - 3 * i;
        const int qd[3] = {q % 3, (q / 3) % 3, q / 9};
        float2 xyz[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) xyz[d] = qd[d] == 1 ? make_float2(0.0f, 0.0f) : (qd[d] == 0 ? df_neg(g3) : g3);
        // J[i][0] = z (y c7 + c5) + (y c3 + c1), J[i][1] = z (x c7 + c6) + (x c3 + c2),
        // J[i][2] = y (x c7 + c6) + (x c5 + c4)
        const float2 u = j == 2 ? xyz[1] : xyz[2], v = j == 0 ? xyz[1] : xyz[0];
        const int A = j == 0 ? 5 : 6, B = j == 2 ? 5 : 3, C = j == 0 ? 1 : (j == 1 ? 2 : 4);
        Mq[q][3 * i + j] = df_add(df_mul(u, df_add(df_mul(v, cw[7][i]), cw[A][i])), df_add(df_mul(v, cw[B][i]), cw[C][i]));
    }
    __syncthreads();
    for (int it = tid; it < 27 * 9; it += EQ_T) {  // Cq[q][3 j + i] = J[i1][j1] J[i2][j2] - J[i1][j2] J[i2][j1]
        const int q = it / 9, j = (it - 9 * q) / 3, i = it - 9 * q - 3 * j;
        const int i1 = i == 2 ? 0 : i + 1, i2 = i == 0 ? 2 : i - 1, j1 = j == 2 ? 0 : j + 1, j2 = j == 0 ? 2 : j - 1;
        Cq[q][3 * j + i] = df_det2(Mq[q][3 * i1 + j1], Mq[q][3 * i2 + j2], Mq[q][3 * i1 + j2], Mq[q][3 * i2 + j1]);
    }
    __syncthreads();
    if (tid < 27) {
        const int q = tid, qi = q % 3, qj = (q / 3) % 3, qk = q / 9;
        const float2 w5 = make_float2((float)W5, (float)(W5 - (double)(float)W5));
        const float2 w8 = make_float2((float)W8, (float)(W8 - (double)(float)W8));
        const float2 det = df_add(df_add(df_mul(Mq[q][0], Cq[q][0]), df_mul(Mq[q][1], Cq[q][3])),
                                  df_mul(Mq[q][2], Cq[q][6]));
        const float2 wv = df_mul(df_mul(qi == 1 ? w8 : w5, qj == 1 ? w8 : w5), qk == 1 ? w8 : w5);
        const float2 wd = df_mul(wv, det);
        const float2 sr = df_mul(df_sqrt(wd), df_recip(det));  // sqrt(w detJ) / detJ
        wdet[q] = df_to_double(wd);
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) Mq[q][3 * i + j] = df_mul(sr, Cq[q][3 * j + i]);
    }
    __syncthreads();
    for (int it = tid; it < 27 * 20; it += EQ_T) {  // grad N = J^-T gradref N, in FP32 pairs
        const int q = it / 20, a = it - 20 * q;
        const float2 *T = c_q2s_tabf[q][a];
        const float2 t0 = T[0], t1 = T[1], t2 = T[2];
#pragma unroll
        for (int i = 0; i < 3; ++i)
            grd[q][i][a] = df_add(df_add(df_mul(Mq[q][3 * i], t0), df_mul(Mq[q][3 * i + 1], t1)),
                                  df_mul(Mq[q][3 * i + 2], t2));
    }
    __syncthreads();
    if (tid < 210) {
        int pa = 0, rem = tid;
        while (rem >= 20 - pa) {
            rem -= 20 - pa;
            ++pa;
        }
        const int pb = pa + rem;
        // double-float sums (exact products of the high parts by FMA,
        // cross terms of the low parts, two-sum accumulation)
        float sh[9], sl[9];
#pragma unroll
        for (int k = 0; k < 9; ++k) sh[k] = sl[k] = 0.0f;
#pragma unroll 3
        for (int q = 0; q < 27; ++q) {
            float2 x[3], y[3];
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                x[i] = grd[q][i][pa];
                y[i] = grd[q][i][pb];
            }
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    const int k = 3 * i + j;
                    const float p = x[i].x * y[j].x;
                    const float ep = fmaf(x[i].x, y[j].x, -p);  // exact error of p
                    const float tt = sh[k] + p;                 // two-sum of sh and p
                    const float z = tt - sh[k];
                    const float es = (sh[k] - (tt - z)) + (p - z);
                    sl[k] = fmaf(x[i].x, y[j].y, fmaf(x[i].y, y[j].x, sl[k] + (es + ep)));  // + cross terms
                    sh[k] = tt;
                }
        }
        float2 M[9];
#pragma unroll
        for (int k = 0; k < 9; ++k) {  // renormalise (fast two-sum)
            const float h = sh[k] + sl[k];
            M[k] = make_float2(h, sl[k] - (h - sh[k]));
        }
        const float2 L = lmu[0], U = lmu[1];
        const float2 mtr = df_mul(U, df_add(df_add(M[0], M[4]), M[8]));
        float2 *ra = reinterpret_cast<float2 *>(out + (int64_t)tmap[pa] * EQ_ROW + 9 * pb);
        float2 *rb = reinterpret_cast<float2 *>(out + (int64_t)tmap[pb] * EQ_ROW + 9 * pa);
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                float2 kv = df_add(df_mul(L, M[3 * i + j]), df_mul(U, M[3 * j + i]));
                if (i == j) kv = df_add(kv, mtr);
                ra[3 * i + j] = kv;
                if (pb != pa) rb[3 * j + i] = kv;
            }
    }
    if (tid < 20) {  // d_e[3 a + c] = b_c sum_q w detJ N_a (FP64)
        double m = 0.0;
        for (int q = 0; q < 27; ++q) m = fma(wdet[q], c_q2s_tab[q][tid][0], m);
        double *o = out + (int64_t)tmap[tid] * EQ_ROW + 180;
        o[0] = b0 * m;
        o[1] = b1 * m;
        o[2] = b2 * m;
    }
}

// Q1 elasticity, one element per thread.  The scaled gradients
// sqrt(w detJ) gradN_a(q) of all 8 points go to shared memory (each thread its
// own column, no synchronisation), then every block pair a <= b contracts
// them into A_ab and finishes K_ab with lambda, mu.
constexpr int EL_T = 64;

__global__ void __launch_bounds__(EL_T) k_elem_elastic_q1(int64_t e0, int64_t e1, const double *__restrict__ X,
                                                          const int32_t *__restrict__ conn,
                                                          const double *__restrict__ Ec, double nu, double b0,
                                                          double b1, double b2, double *__restrict__ out,
                                                          int *status)
{
    extern __shared__ double sg[];  // [q][a][i][EL_T]
    const int tid = threadIdx.x;
    const int64_t e = e0 + (int64_t)blockIdx.x * EL_T + tid;
    if (e >= e1) return;
    const double E = Ec[e];
    if (!isfinite(E)) mf_dev_fail(status, MF_ERR_NONFINITE);
    const double lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
    const double mu = E / (2.0 * (1.0 + nu));
    double x[8][3];
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int i = 0; i < 3; ++i) x[a][i] = X[3 * (int64_t)conn[8 * e + a] + i];
    // map coefficients (q1_wht), so that J at a Gauss point costs 27 FMAs
    double c[8][3];
    q1_wht(x, c);
#pragma unroll
    for (int S = 1; S < 8; ++S)
#pragma unroll
        for (int i = 0; i < 3; ++i) c[S][i] *= (__popc(S) & 1) ? -0.125 : 0.125;
    double m[8] = {};
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        double Ji[3][3];
        const double wd = q1_jac_coef(c, q, Ji);
        const double sw = sqrt(wd);
#pragma unroll
        for (int a = 0; a < 8; ++a) {
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                const double gi = q1_dref(q, a, 0) * Ji[0][i] + q1_dref(q, a, 1) * Ji[1][i] +
                                  q1_dref(q, a, 2) * Ji[2][i];
                sg[((q * 8 + a) * 3 + i) * EL_T + tid] = sw * gi;
            }
            m[a] = fma(wd, q1_n(q, a), m[a]);
        }
    }
    double *o = out + e * (36 * 9 + 24);
#pragma unroll 1
    for (int a = 0; a < 8; ++a) {
#pragma unroll 1
        for (int b = a; b < 8; ++b) {
            double A[3][3] = {};
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                double ga[3], gb[3];
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    ga[i] = sg[((q * 8 + a) * 3 + i) * EL_T + tid];
                    gb[i] = sg[((q * 8 + b) * 3 + i) * EL_T + tid];
                }
#pragma unroll
                for (int c = 0; c < 3; ++c)
#pragma unroll
                    for (int cp = 0; cp < 3; ++cp) A[c][cp] = fma(ga[c], gb[cp], A[c][cp]);
            }
            const double tr = A[0][0] + A[1][1] + A[2][2];
            double *blk = o + upair(a, b) * 9;
#pragma unroll
            for (int c = 0; c < 3; ++c)
#pragma unroll
                for (int cp = 0; cp < 3; ++cp)
                    blk[3 * c + cp] = lam * A[c][cp] + mu * A[cp][c] + (c == cp ? mu * tr : 0.0);
        }
    }
#pragma unroll
    for (int a = 0; a < 8; ++a) {
        o[324 + 3 * a + 0] = b0 * m[a];
        o[324 + 3 * a + 1] = b1 * m[a];
        o[324 + 3 * a + 2] = b2 * m[a];
    }
}

// Taylor-Hood flow, one element per thread: A (6x6) then B_1, B_2 (3x6), in
// double-float (FP32 pairs, about 47 bits): FP64 only for the vertex
// differences, the finiteness checks and the per-block conversion of the
// reference sums; each output converts once (integer-only).
__device__ __forceinline__ float2 dfma_(float2 a, float2 b, float2 c) { return df_add(df_mul(a, b), c); }

__global__ void __launch_bounds__(128) k_elem_oseen(int64_t n_el, int64_t n2, const double *__restrict__ X,
                                                    const int32_t *__restrict__ conn, const double *__restrict__ adv,
                                                    double mu_d, double rho_d, double *__restrict__ out, int *status)
{
    __shared__ float2 sMs[6][6][6], sR[3][3][6];
    for (int i = threadIdx.x; i < 216; i += blockDim.x) (&sMs[0][0][0])[i] = f64_to_df((&c_Ms[0][0][0])[i]);
    for (int i = threadIdx.x; i < 54; i += blockDim.x) (&sR[0][0][0])[i] = f64_to_df((&c_R[0][0][0])[i]);
    __syncthreads();
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n_el) return;
    const int32_t *c = conn + 6 * e;
    const float2 mu = f64_to_df(mu_d), rho = f64_to_df(rho_d);
    // affine triangle (as tri_affine): J^-1 = [[j11, -j01], [-j10, j00]] / det,
    // grad lambda = J^-T gradref lambda
    const double x0 = X[2 * (int64_t)c[0]], y0 = X[2 * (int64_t)c[0] + 1];
    const float2 j00 = f64_to_df(X[2 * (int64_t)c[1]] - x0), j10 = f64_to_df(X[2 * (int64_t)c[1] + 1] - y0);
    const float2 j01 = f64_to_df(X[2 * (int64_t)c[2]] - x0), j11 = f64_to_df(X[2 * (int64_t)c[2] + 1] - y0);
    const float2 det = df_det2(j00, j11, j01, j10);
    const float2 r = df_recip(det);
    const float2 i00 = df_mul(j11, r), i01 = df_neg(df_mul(j01, r)), i10 = df_neg(df_mul(j10, r)),
                 i11 = df_mul(j00, r);
    const float2 gl[3][2] = {{df_neg(df_add(i00, i10)), df_neg(df_add(i01, i11))}, {i00, i01}, {i10, i11}};
    float2 aN[6][2];
#pragma unroll
    for (int a = 0; a < 6; ++a) {
        const double v0 = adv[c[a]], v1 = adv[n2 + c[a]];
        if (!isfinite(v0) || !isfinite(v1)) mf_dev_fail(status, MF_ERR_NONFINITE);
        aN[a][0] = f64_to_df(v0);
        aN[a][1] = f64_to_df(v1);
    }
    double *o = out + e * 72;
    const float2 z = make_float2(0.f, 0.f), one = make_float2(1.f, 0.f), two = make_float2(2.f, 0.f),
                 four = make_float2(4.f, 0.f);
    {
        // A = mu D + C: the viscous part D from the reference sums, the
        // advection part C[a][b] = -rho sum_q w detJ (a_h . grad N_a) N_b by
        // the 6-point rule (a_h varies over the element)
        float2 Cv[36];
#pragma unroll
        for (int k = 0; k < 36; ++k) Cv[k] = z;
        const float2 rdet = df_mul(rho, det);
#pragma unroll 1
        for (int q = 0; q < 6; ++q) {
            const float2 la = q < 3 ? DFC(T6A1) : DFC(T6A2), lb = q < 3 ? DFC(1.0 - 2.0 * T6A1) : DFC(1.0 - 2.0 * T6A2);
            const int kq = q % 3;
            const float2 l[3] = {kq == 0 ? lb : la, kq == 1 ? lb : la, kq == 2 ? lb : la};
            const float2 w = q < 3 ? DFC(0.5 * T6W1) : DFC(0.5 * T6W2);
            float2 N[6], g[6][2];
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                N[i] = df_mul(l[i], df_add(df_mul(two, l[i]), df_neg(one)));
                const float2 f = df_add(df_mul(four, l[i]), df_neg(one));
                g[i][0] = df_mul(f, gl[i][0]);
                g[i][1] = df_mul(f, gl[i][1]);
            }
            const int ep[3][2] = {{0, 1}, {1, 2}, {2, 0}};
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const int pa = ep[k][0], pb = ep[k][1];
                N[3 + k] = df_mul(four, df_mul(l[pa], l[pb]));
                g[3 + k][0] = df_mul(four, dfma_(gl[pa][0], l[pb], df_mul(l[pa], gl[pb][0])));
                g[3 + k][1] = df_mul(four, dfma_(gl[pa][1], l[pb], df_mul(l[pa], gl[pb][1])));
            }
            const float2 wrho = df_mul(w, rdet);
            float2 ah0 = z, ah1 = z;
#pragma unroll
            for (int b = 0; b < 6; ++b) {
                ah0 = dfma_(aN[b][0], N[b], ah0);
                ah1 = dfma_(aN[b][1], N[b], ah1);
            }
#pragma unroll
            for (int a = 0; a < 6; ++a) {
                const float2 nsa = df_neg(df_mul(wrho, dfma_(ah0, g[a][0], df_mul(ah1, g[a][1]))));
#pragma unroll
                for (int b = 0; b < 6; ++b) Cv[6 * a + b] = dfma_(nsa, N[b], Cv[6 * a + b]);
            }
        }
        float2 Gs[6];
        Gs[0] = dfma_(gl[0][0], gl[0][0], df_mul(gl[0][1], gl[0][1]));
        Gs[1] = dfma_(gl[1][0], gl[1][0], df_mul(gl[1][1], gl[1][1]));
        Gs[2] = dfma_(gl[2][0], gl[2][0], df_mul(gl[2][1], gl[2][1]));
        Gs[3] = dfma_(gl[0][0], gl[1][0], df_mul(gl[0][1], gl[1][1]));
        Gs[4] = dfma_(gl[0][0], gl[2][0], df_mul(gl[0][1], gl[2][1]));
        Gs[5] = dfma_(gl[1][0], gl[2][0], df_mul(gl[1][1], gl[2][1]));
        const float2 mdet = df_mul(mu, det);
#pragma unroll
        for (int a = 0; a < 6; ++a)
#pragma unroll
            for (int b = a; b < 6; ++b) {
                float2 Dab = z;
#pragma unroll
                for (int pp = 0; pp < 6; ++pp) Dab = dfma_(Gs[pp], sMs[pp][a][b], Dab);
                const float2 vd = df_mul(mdet, Dab);
                o[6 * a + b] = df_to_double_int(df_add(vd, Cv[6 * a + b]));
                if (b != a) o[6 * b + a] = df_to_double_int(df_add(vd, Cv[6 * b + a]));
            }
    }
    {
        // B_i[a1][b] = det sum_j (grad l_j)_i c_R[j][a1][b]
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int a = 0; a < 3; ++a)
#pragma unroll
                for (int b = 0; b < 6; ++b) {
                    float2 v = z;
#pragma unroll
                    for (int j = 0; j < 3; ++j) v = dfma_(gl[j][i], sR[j][a][b], v);
                    o[36 + 18 * i + 6 * a + b] = df_to_double_int(df_mul(det, v));
                }
    }
}

// ---------------------------------------------------------------------------
// thermal gather: one warp per node (gather_row_th)
// ---------------------------------------------------------------------------
constexpr int GT_WARPS = 8;

template <int NPE>
__global__ void __launch_bounds__(GT_WARPS * 32, 3) k_gather_th(
    int64_t n_nodes, const int64_t *__restrict__ adj_ptr, const int32_t *__restrict__ adj_col,
    const int64_t *__restrict__ inc_ptr, const int32_t *__restrict__ inc, const uint8_t *__restrict__ inc_loc,
    const uint8_t *__restrict__ inc_slot, const double *__restrict__ sc, const double *__restrict__ kref,
    const double *__restrict__ kc, double f, const uint8_t *__restrict__ mask,
    const double *__restrict__ bval, const int64_t *__restrict__ row_ptr, double *__restrict__ values,
    double *__restrict__ d)
{
    constexpr int L = th_lanes<NPE>(), G = 32 / L;  // G nodes per warp
    __shared__ double acc_all[GT_WARPS * G][NPE > 8 ? MF_MAX_DEG_HO : MF_MAX_DEG];
    const int lane = threadIdx.x & 31, grp = threadIdx.x / L;
    const int64_t n = (int64_t)blockIdx.x * (GT_WARPS * G) + grp;
    if (n >= n_nodes) return;  // group-uniform
    const unsigned gmask = (L == 32 ? 0xffffffffu : ((1u << L) - 1u)) << (lane & ~(L - 1));
    gather_row_th<NPE>(n, lane & (L - 1), gmask, acc_all[grp], adj_ptr, adj_col, inc_ptr, inc, inc_loc, inc_slot, sc,
                       kref, kc, f, mask, bval, row_ptr, values, d);
}

// ---------------------------------------------------------------------------
// thermal Q1 with translate elements: the gather in double-float.  Every
// entry of a translate is k_e times a reference entry, so a node's row is a
// sum of at most 64 such products; they are formed and summed as FP32 pairs
// (the FP32 pipe runs 64 times the FP64 one here) in the same fixed order as
// the FP64 gather, and each CSR value is converted once to FP64 by integer
// operations.  Only rows flagged as next to a constrained node read their
// columns for the Dirichlet elimination.  Used when every element is a
// translate; a mesh with other elements takes the FP64 gather.
// ---------------------------------------------------------------------------
// the translates' coefficients as pairs, checked finite
__global__ void k_kc_split(int64_t n_el, const double *__restrict__ kc, const uint8_t *__restrict__ tr,
                           float2 *__restrict__ kc_df, int *status)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n_el || !tr[e]) return;
    const double k = kc[e];
    if (!isfinite(k)) mf_dev_fail(status, MF_ERR_NONFINITE);
    kc_df[e] = f64_to_df(k);
}

// flag[n] = 1 for every constrained node m and each of its neighbours n
__global__ void k_mark_bc_rows(int64_t n_nodes, const int64_t *__restrict__ adj_ptr,
                               const int32_t *__restrict__ adj_col, const uint8_t *__restrict__ mask,
                               uint8_t *__restrict__ flag)
{
    const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= n_nodes || !mask[m]) return;
    for (int64_t q = adj_ptr[m]; q < adj_ptr[m + 1]; ++q) flag[adj_col[q]] = 1;
}

constexpr int GD_WARPS = 8;

__global__ void __launch_bounds__(GD_WARPS * 32, 8) k_gather_th_q1df(
    int64_t n_nodes, const int64_t *__restrict__ adj_ptr, const int32_t *__restrict__ adj_col,
    const int64_t *__restrict__ inc_ptr, const int32_t *__restrict__ inc, const uint8_t *__restrict__ inc_loc,
    const uint8_t *__restrict__ inc_slot, const float2 *__restrict__ kref_df, const float2 *__restrict__ kc_df,
    float2 f_df, const uint8_t *__restrict__ mask, const uint8_t *__restrict__ bcrow,
    const double *__restrict__ bval, const int64_t *__restrict__ row_ptr, double *__restrict__ values,
    double *__restrict__ d)
{
    constexpr int L = 8, G = 4;  // 8 lanes per node, 4 nodes per warp
    __shared__ float2 acc_all[GD_WARPS * G][MF_MAX_DEG];
    const int lane = threadIdx.x & 31, grp = threadIdx.x / L;
    const int64_t n = (int64_t)blockIdx.x * (GD_WARPS * G) + grp;
    if (n >= n_nodes) return;  // group-uniform
    const unsigned gmask = 0xffu << (lane & ~(L - 1));
    gather_row_th_q1df(n, lane & (L - 1), gmask, acc_all[grp], mask != nullptr && bcrow[n] != 0, adj_ptr, adj_col,
                       inc_ptr, inc, inc_loc, inc_slot, kref_df, kc_df, f_df, mask, bval, row_ptr, values, d);
}

// Thermal Q1 (or capacity) rows on a lexicographic box of translates of a
// rectangular cell (box_row_q1): one thread per node; a warp's 32 rows are
// consecutive in the CSR arrays, so each warp stages them in its part of
// shared memory and stores them with coalesced writes (no block barrier: a
// warp with rows next to the constrained boundary delays only itself).
constexpr int QB = 128;  // nodes (threads) per block

__global__ void __launch_bounds__(QB) k_rows_q1box(int n_nodes, int nx1, int ny1, int nz1, mf_box_classes C,
                                                   int capacity, double f, const double *__restrict__ kc,
                                                   const uint8_t *__restrict__ mask, const uint8_t *__restrict__ bcrow,
                                                   const double *__restrict__ bval,
                                                   const int64_t *__restrict__ row_ptr, double *__restrict__ values,
                                                   double *__restrict__ d, int64_t n_el, int *status)
{
    // the coefficients are read straight from kc: check them here
    for (int64_t e = (int64_t)blockIdx.x * QB + threadIdx.x; e < n_el; e += (int64_t)gridDim.x * QB)
        if (!isfinite(kc[e])) mf_dev_fail(status, MF_ERR_NONFINITE);
    __shared__ double stage[QB * 27];
    __shared__ double cls[8];
    if (threadIdx.x < 8) cls[threadIdx.x] = capacity ? C.m_cls[threadIdx.x] : C.k_cls[threadIdx.x];
    __syncthreads();
    const int lane = threadIdx.x & 31, wbase = blockIdx.x * QB + (threadIdx.x & ~31), n = wbase + lane;
    if (wbase >= n_nodes) return;  // warp-uniform
    const int nend = min(n_nodes, wbase + 32);
    const int64_t r0 = row_ptr[wbase];
    double *wst = stage + (threadIdx.x & ~31) * 27;  // this warp's 32 rows
    if (n < n_nodes) {
        double *row = wst + (row_ptr[n] - r0);
        d[n] = box_row_q1(n, nx1, ny1, nz1, cls, capacity ? 0.0 : f * C.dref, kc, mask != nullptr && bcrow[n] != 0,
                          mask, bval, [row](int k, double v) { row[k] = v; });
    }
    __syncwarp();
    const int64_t cnt = row_ptr[nend] - r0;
    for (int64_t i = lane; i < cnt; i += 32) values[r0 + i] = wst[i];
}

// ---------------------------------------------------------------------------
// elasticity gather: one warp per node, walking the node's incident elements in
// ascending order.  Each element's 8 blocks (a_n, b) of the node's rows (72
// values, stored as the upper blocks a <= b) are added into a shared-memory
// row accumulator at the neighbour slot of node b; after the last element the
// three CSR rows of the node are written once, coalesced.  T = double (FP64
// path) or long long (fixed-point mixed path: exact sums, converted once).
// ---------------------------------------------------------------------------
constexpr int GEL_WARPS = 8;

template <typename T>
__device__ __forceinline__ double to_double(T v, int S);

template <>
__device__ __forceinline__ double to_double<double>(double v, int)
{
    return v;
}

// x * 2^-S for a fixed-point integer x (mf_fixed_to_double)
template <>
__device__ __forceinline__ double to_double<long long>(long long v, int S)
{
    return mf_fixed_to_double(v, S);
}

template <typename T>
__global__ void __launch_bounds__(GEL_WARPS * 32, 5) k_gather_el(
    int64_t n0, int64_t n1, const int64_t *__restrict__ adj_ptr, const int32_t *__restrict__ adj_col,
    const int64_t *__restrict__ inc_ptr, const int32_t *__restrict__ inc, const uint8_t *__restrict__ inc_loc,
    const uint8_t *__restrict__ slot, const double *__restrict__ sc, int64_t stride, const int *__restrict__ scale,
    int fp, int fq, const uint8_t *__restrict__ mask, const double *__restrict__ bval,
    const int64_t *__restrict__ row_ptr, double *__restrict__ values, double *__restrict__ d)
{
    __shared__ T acc_all[GEL_WARPS][MF_MAX_DEG * 9];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t n = n0 + (int64_t)blockIdx.x * GEL_WARPS + w;
    if (n >= n1) return;  // warp-uniform
    T *acc = acc_all[w];
    constexpr bool fixed = sizeof(T) == 8 && T(0.5) == T(0);  // integer accumulator
    const int64_t p0 = adj_ptr[n];
    const int deg = (int)(adj_ptr[n + 1] - p0);
    for (int i = lane; i < 9 * deg; i += 32) acc[i] = T(0);
    // load vector: lane 3 j + c (j < 8) holds component c of incidence entry
    // j, j + 8, ... in turn; the 8 partial sums of component c are added in a
    // fixed tree below
    double dsum = 0.0;
    __syncwarp();
    const int64_t i0 = inc_ptr[n], i1 = inc_ptr[n + 1];
    // incident elements in chunks of 8: element ids and the local index of n
    // are fetched by lanes 0..7 at once, then the values
    for (int64_t cb = i0; cb < i1; cb += 8) {
        const int cnt = (int)min((int64_t)8, i1 - cb);
        int64_t my_e = 0;
        int my_a = 0;
        if (lane < cnt) {
            my_e = inc[cb + lane];
            my_a = inc_loc[cb + lane];
        }
        {
            const int jd = lane / 3, cd = lane - 3 * (lane / 3);
            const int64_t ed = __shfl_sync(0xffffffffu, my_e, jd < 8 ? jd : 0);
            const int ad = __shfl_sync(0xffffffffu, my_a, jd < 8 ? jd : 0);
            if (jd < cnt) dsum += sc[ed * stride + 324 + 3 * ad + cd];
        }
        if constexpr (fixed) {
            // exact integer sums: order is irrelevant, so every value of the
            // chunk streams through shared-memory integer atomics
            const int items = cnt * 72;
            constexpr int IU = 6;  // items per lane whose loads are in flight together
            for (int it0 = 0; it0 < (items + 31) / 32; it0 += IU) {  // warp-uniform trip count
                T v[IU];
                int ad[IU];
#pragma unroll
                for (int u = 0; u < IU; ++u) {
                    const int item = lane + 32 * (it0 + u);
                    const bool act = item < items;
                    const int j = act ? item / 72 : 0;
                    const int64_t e = __shfl_sync(0xffffffffu, my_e, j);
                    const int a = __shfl_sync(0xffffffffu, my_a, j);
                    v[u] = T(0);
                    ad[u] = -1;
                    if (act) {
                        const int idx = item - 72 * j;
                        const int b = idx / 9, cc = idx - 9 * b;
                        const int c = cc / 3, cp = cc - 3 * c;
                        const T *blk = reinterpret_cast<const T *>(sc + e * stride);
                        v[u] = (a <= b) ? blk[upair(a, b) * 9 + cc] : blk[upair(b, a) * 9 + 3 * cp + c];
                        ad[u] = slot[e * 64 + a * 8 + b] * 9 + cc;
                    }
                }
#pragma unroll
                for (int u = 0; u < IU; ++u)
                    if (ad[u] >= 0)
                        atomicAdd(reinterpret_cast<unsigned long long *>(&acc[ad[u]]), (unsigned long long)v[u]);
            }
        } else {
            // FP64 sums in ascending element order (bit-reproducible)
            for (int j = 0; j < cnt; ++j) {
                const int64_t e = __shfl_sync(0xffffffffu, my_e, j);
                const int a = __shfl_sync(0xffffffffu, my_a, j);
                const T *blk = reinterpret_cast<const T *>(sc + e * stride);
                for (int idx = lane; idx < 72; idx += 32) {
                    const int b = idx / 9, cc = idx - 9 * b;
                    const int c = cc / 3, cp = cc - 3 * c;
                    const T v = (a <= b) ? blk[upair(a, b) * 9 + cc] : blk[upair(b, a) * 9 + 3 * cp + c];
                    acc[slot[e * 64 + a * 8 + b] * 9 + cc] += v;
                }
                __syncwarp();
            }
        }
        __syncwarp();
    }
    // component c of the load: lanes c, c + 3, ..., c + 21 (fixed tree)
    dsum += __shfl_down_sync(0xffffffffu, dsum, 12);  // lanes c + 3 j, j < 4, take j + 4
    dsum += __shfl_down_sync(0xffffffffu, dsum, 6);   // j < 2 take j + 2
    dsum += __shfl_down_sync(0xffffffffu, dsum, 3);   // j = 0 takes j = 1
    const int S = scale ? *scale : 0;
    // neighbour k's column node and Dirichlet flags, loaded once by lane k
    // (and k - 32 for rows with more than 32 neighbours), read by shuffle
    int32_t mcol_l[2] = {0, 0};
    unsigned cm_l[2] = {0u, 0u};
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int k = lane + 32 * h;
        if (k < deg) {
            mcol_l[h] = adj_col[p0 + k];
            if (mask)
#pragma unroll
                for (int cp = 0; cp < 3; ++cp) cm_l[h] |= (mask[3 * (int64_t)mcol_l[h] + cp] != 0 ? 1u : 0u) << cp;
        }
    }
#pragma unroll 1
    for (int c = 0; c < 3; ++c) {
        const int64_t r = 3 * n + c;
        const bool rm = mask ? mask[r] != 0 : false;
        const int64_t rb = row_ptr[r];
        double lift = 0.0;
        for (int j0 = 0; j0 < 3 * deg; j0 += 32) {  // warp-uniform
            const int j = j0 + lane;
            const int k = (j < 3 * deg ? j : 0) / 3, cp = j - 3 * (j / 3);
            const int kk = k & 31;
            const int32_t mc0 = __shfl_sync(0xffffffffu, mcol_l[0], kk), mc1 = __shfl_sync(0xffffffffu, mcol_l[1], kk);
            const unsigned f0 = __shfl_sync(0xffffffffu, cm_l[0], kk), f1 = __shfl_sync(0xffffffffu, cm_l[1], kk);
            if (j >= 3 * deg) continue;
            const int32_t mcol = k < 32 ? mc0 : mc1;
            const bool cmk = ((k < 32 ? f0 : f1) >> cp) & 1u;
            T kv = acc[k * 9 + 3 * c + cp];
            if (fq) {  // fixed-point path: K = p A + q A^T + q I tr(A) per node-pair block
                kv = (T)fp * kv + (T)fq * acc[k * 9 + 3 * cp + c];
                if (c == cp) kv += (T)fq * (acc[k * 9] + acc[k * 9 + 4] + acc[k * 9 + 8]);
            }
            double v = to_double<T>(kv, S);
            if (mask) {
                const int64_t sdof = 3 * (int64_t)mcol + cp;
                if (rm) v = (r == sdof) ? 1.0 : 0.0;
                else if (cmk) { lift -= v * bval[sdof]; v = 0.0; }
            }
            values[rb + j] = v;
        }
        if (__any_sync(0xffffffffu, lift != 0.0))  // rows next to a constrained dof only
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) lift += __shfl_xor_sync(0xffffffffu, lift, o);
        const double dc = __shfl_sync(0xffffffffu, dsum, c);
        if (lane == 0) d[r] = rm ? bval[r] : dc + lift;
    }
}

// elasticity gather for the serendipity brick: one warp per node.  Row a of
// each incident element is incidence entry t (ascending, so the sums run in
// element order: bit-reproducible); its 180 values (FP32 pairs) are added in
// double-float at the neighbour slot inc_slot[t * 20 + b] of node b in a
// shared-memory row accumulator (up to MF_MAX_DEG_HO neighbours); the node's
// three CSR rows are then written once in FP64 (one exact conversion and one
// FP64 add per entry), with Dirichlet elimination and lifting.
constexpr int GQ_WARPS = 4;

// shared memory of one warp of k_gather_el_q2s for rows of up to maxd neighbours
__host__ __device__ constexpr size_t gq_warp_bytes(int maxd) { return (size_t)maxd * (9 * sizeof(float2) + 8); }

__global__ void __launch_bounds__(GQ_WARPS * 32, 8) k_gather_el_q2s(
    int64_t n_nodes, int maxd, const int64_t *__restrict__ adj_ptr, const int32_t *__restrict__ adj_col,
    const int64_t *__restrict__ inc_ptr, const uint8_t *__restrict__ inc_slot, const double *__restrict__ sc,
    const uint8_t *__restrict__ mask, const double *__restrict__ bval, const int64_t *__restrict__ row_ptr,
    double *__restrict__ values, double *__restrict__ d)
{
    extern __shared__ float2 gq_smem[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t n = (int64_t)blockIdx.x * GQ_WARPS + w;
    if (n >= n_nodes) return;  // warp-uniform
    // per warp: the row accumulator [maxd][9], then the neighbours' column
    // nodes and Dirichlet flags [maxd] each
    float2 *acc = reinterpret_cast<float2 *>(reinterpret_cast<char *>(gq_smem) + w * gq_warp_bytes(maxd));
    int32_t *ncol = reinterpret_cast<int32_t *>(acc + 9 * maxd);
    int32_t *nflag = ncol + maxd;
    const float2 *scf = reinterpret_cast<const float2 *>(sc);
    const int64_t p0 = adj_ptr[n];
    const int deg = (int)(adj_ptr[n + 1] - p0);
    for (int i = lane; i < 9 * deg; i += 32) acc[i] = make_float2(0.0f, 0.0f);
    for (int k = lane; k < deg; k += 32) {
        const int32_t mc = adj_col[p0 + k];
        int f = 0;
        if (mask)
#pragma unroll
            for (int cp = 0; cp < 3; ++cp) f |= (mask[3 * (int64_t)mc + cp] != 0 ? 1 : 0) << cp;
        ncol[k] = mc;
        nflag[k] = f;
    }
    const int64_t i0 = inc_ptr[n], i1 = inc_ptr[n + 1];
    double dsum = 0.0;  // lane c < 3: component c of the load, element order
    if (lane < 3)
        for (int64_t t = i0; t < i1; ++t) dsum += sc[t * EQ_ROW + 180 + lane];
    __syncwarp();
    constexpr int IU = (180 + 31) / 32;  // items per lane and incidence entry
    for (int64_t cb = i0; cb < i1; cb += 2) {
        const int cnt = (int)min((int64_t)2, i1 - cb);
        float2 v[2][IU];
        int ad[2][IU];
#pragma unroll
        for (int j = 0; j < 2; ++j)
#pragma unroll
            for (int u = 0; u < IU; ++u) {
                const int idx = lane + 32 * u;
                v[j][u] = make_float2(0.0f, 0.0f);
                ad[j][u] = -1;
                if (j < cnt && idx < 180) {
                    const int64_t t = cb + j;
                    const int b = idx / 9;
                    v[j][u] = scf[t * EQ_ROW + idx];
                    ad[j][u] = inc_slot[t * 20 + b] * 9 + (idx - 9 * b);
                }
            }
#pragma unroll
        for (int j = 0; j < 2; ++j) {
#pragma unroll
            for (int u = 0; u < IU; ++u)
                if (ad[j][u] >= 0) acc[ad[j][u]] = df_add(acc[ad[j][u]], v[j][u]);
            __syncwarp();
        }
    }
#pragma unroll 1
    for (int c = 0; c < 3; ++c) {
        const int64_t r = 3 * n + c;
        const bool rm = mask ? mask[r] != 0 : false;
        const int64_t rb = row_ptr[r];
        double lift = 0.0;
        for (int j = lane; j < 3 * deg; j += 32) {
            const int k = j / 3, cp = j - 3 * k;
            double v = df_to_double(acc[k * 9 + 3 * c + cp]);
            if (mask) {
                const int64_t sdof = 3 * (int64_t)ncol[k] + cp;
                if (rm) v = (r == sdof) ? 1.0 : 0.0;
                else if ((nflag[k] >> cp) & 1) { lift -= v * bval[sdof]; v = 0.0; }
            }
            values[rb + j] = v;
        }
        if (__any_sync(0xffffffffu, lift != 0.0))  // rows next to a constrained dof only
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) lift += __shfl_xor_sync(0xffffffffu, lift, o);
        const double dc = __shfl_sync(0xffffffffu, dsum, c);
        if (lane == 0) d[r] = rm ? bval[r] : dc + lift;
    }
}

// flow rows, node-centric (groups of 16 lanes per node, 2 nodes per warp):
//   u_i(n) = [A over the P2 neighbours | -B_i^T over the P1 neighbours],
//   p(n1)  = [B_1 | B_2 over the P2 neighbours | 0 on the diagonal].
// The element scratch holds A (6 x 6) at 0 and B_i[a1][b2] at 36 + 18 i +
// 6 a1 + b2.  Each entry is a sum over the incident elements in ascending
// order (the node's incidence list), the adds into shared-memory rows run
// element by element; Dirichlet rows become identity rows and constrained
// columns move to the right-hand side (f = 0, so d is the lifting alone).
constexpr int GO_GROUPS = 16;  // node groups per block (8 warps)

__device__ __forceinline__ void flow_put(double &v, double &lift, bool rm, int64_t r, int64_t sdof,
                                         const uint8_t *__restrict__ mask, const double *__restrict__ bval)
{
    if (mask) {
        if (rm) v = (r == sdof) ? 1.0 : 0.0;
        else if (mask[sdof]) { lift -= v * bval[sdof]; v = 0.0; }
    }
}

__global__ void __launch_bounds__(GO_GROUPS * 16) k_gather_oseen_u(
    int64_t n2, mf_adj pp, mf_adj pq, const int64_t *__restrict__ inc_ptr, const uint8_t *__restrict__ inc_loc,
    const int32_t *__restrict__ inc, const uint8_t *__restrict__ slot_pp, const uint8_t *__restrict__ slot_pq,
    const double *__restrict__ sc, const uint8_t *__restrict__ mask, const uint8_t *__restrict__ bcrow,
    const double *__restrict__ bval, const int64_t *__restrict__ row_ptr, double *__restrict__ values,
    double *__restrict__ d)
{
    __shared__ double accA_all[GO_GROUPS][MF_MAX_DEG];
    __shared__ double accB_all[GO_GROUPS][2][MF_MAX_DEG];
    const int lane = threadIdx.x & 31, grp = threadIdx.x >> 4, sub = threadIdx.x & 15;
    const unsigned gmask = 0xffffu << (lane & 16);
    const int64_t n = (int64_t)blockIdx.x * GO_GROUPS + grp;
    if (n >= n2) return;  // group-uniform
    double *accA = accA_all[grp];
    double(*accB)[MF_MAX_DEG] = accB_all[grp];
    const int64_t pa0 = pp.ptr[n], pb0 = pq.ptr[n];
    const int da = (int)(pp.ptr[n + 1] - pa0), db = (int)(pq.ptr[n + 1] - pb0);
    for (int k = sub; k < da; k += 16) accA[k] = 0.0;
    for (int k = sub; k < db; k += 16) accB[0][k] = accB[1][k] = 0.0;
    __syncwarp(gmask);
    // lanes 0..5: A[a][b]; lanes 6..11: B_i[a1][a] with i = (sub - 6) / 3, a1 = (sub - 6) % 3
    const bool isA = sub < 6, isB = sub >= 6 && sub < 12;
    const int bi = isB ? (sub - 6) / 3 : 0, ba1 = isB ? (sub - 6) % 3 : 0;
    const int64_t i0 = inc_ptr[n], i1 = inc_ptr[n + 1];
    for (int64_t cb = i0; cb < i1; cb += 4) {
        const int cnt = (int)min((int64_t)4, i1 - cb);
        double v[4];
        int s[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            v[j] = 0.0;
            s[j] = 0;
            if (j < cnt && (isA || isB)) {
                const int64_t t = cb + j;
                const double *se = sc + (int64_t)inc[t] * 72;
                const int a = inc_loc[t];
                if (isA) {
                    v[j] = se[6 * a + sub];
                    s[j] = slot_pp[t * 6 + sub];
                } else {
                    v[j] = se[36 + 18 * bi + 6 * ba1 + a];
                    s[j] = slot_pq[t * 3 + ba1];
                }
            }
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (j < cnt) {  // group-uniform
                if (isA) accA[s[j]] += v[j];
                else if (isB) accB[bi][s[j]] -= v[j];
                __syncwarp(gmask);
            }
        }
    }
    // rows u_1(n), u_2(n): A part (columns i n2 + m), then -B_i^T (columns 2 n2 + m1)
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const int64_t r = i * n2 + n;
        // the Dirichlet tests (column loads) only on rows next to a constrained dof
        const uint8_t *mk = (mask && bcrow[r]) ? mask : nullptr;
        const bool rm = mk ? mk[r] != 0 : false;
        const int64_t rb = row_ptr[r];
        double lift = 0.0;
        for (int k = sub; k < da; k += 16) {
            double val = accA[k];
            if (mk) flow_put(val, lift, rm, r, i * n2 + pp.col[pa0 + k], mk, bval);
            values[rb + k] = val;
        }
        for (int k = sub; k < db; k += 16) {
            double val = accB[i][k];
            if (mk) flow_put(val, lift, rm, r, 2 * n2 + pq.col[pb0 + k], mk, bval);
            values[rb + da + k] = val;
        }
        if (__any_sync(gmask, lift != 0.0))
#pragma unroll
            for (int o = 8; o > 0; o >>= 1) lift += __shfl_xor_sync(gmask, lift, o, 16);
        if (sub == 0) d[r] = rm ? bval[r] : lift;
    }
}

__global__ void __launch_bounds__(GO_GROUPS * 16) k_gather_oseen_p(
    int64_t n2, int64_t n1, mf_adj qp, const int64_t *__restrict__ pinc_ptr, const int32_t *__restrict__ pinc,
    const uint8_t *__restrict__ pinc_loc, const uint8_t *__restrict__ pslot, const double *__restrict__ sc,
    const uint8_t *__restrict__ mask, const uint8_t *__restrict__ bcrow, const double *__restrict__ bval,
    const int64_t *__restrict__ row_ptr, double *__restrict__ values, double *__restrict__ d)
{
    __shared__ double acc_all[GO_GROUPS][2][MF_MAX_DEG];
    const int lane = threadIdx.x & 31, grp = threadIdx.x >> 4, sub = threadIdx.x & 15;
    const unsigned gmask = 0xffffu << (lane & 16);
    const int64_t n = (int64_t)blockIdx.x * GO_GROUPS + grp;
    if (n >= n1) return;  // group-uniform
    double(*acc)[MF_MAX_DEG] = acc_all[grp];
    const int64_t q0 = qp.ptr[n];
    const int dq = (int)(qp.ptr[n + 1] - q0);
    for (int k = sub; k < dq; k += 16) acc[0][k] = acc[1][k] = 0.0;
    __syncwarp(gmask);
    // lanes 0..11: B_i[a1][b] with i = sub / 6, b = sub % 6
    const bool act = sub < 12;
    const int bi = act ? sub / 6 : 0, bb = act ? sub % 6 : 0;
    const int64_t i0 = pinc_ptr[n], i1 = pinc_ptr[n + 1];
    for (int64_t cb = i0; cb < i1; cb += 4) {
        const int cnt = (int)min((int64_t)4, i1 - cb);
        double v[4];
        int s[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            v[j] = 0.0;
            s[j] = 0;
            if (j < cnt && act) {
                const int64_t t = cb + j;
                v[j] = sc[(int64_t)pinc[t] * 72 + 36 + 18 * bi + 6 * pinc_loc[t] + bb];
                s[j] = pslot[t * 6 + bb];
            }
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (j < cnt) {  // group-uniform
                if (act) acc[bi][s[j]] += v[j];
                __syncwarp(gmask);
            }
        }
    }
    const int64_t r = 2 * n2 + n;
    // the Dirichlet tests (column loads) only on rows next to a constrained dof
    const uint8_t *mk = (mask && bcrow[r]) ? mask : nullptr;
    const bool rm = mk ? mk[r] != 0 : false;
    const int64_t rb = row_ptr[r];
    double lift = 0.0;
#pragma unroll
    for (int i = 0; i < 2; ++i)
        for (int k = sub; k < dq; k += 16) {
            double val = acc[i][k];
            if (mk) flow_put(val, lift, rm, r, i * n2 + qp.col[q0 + k], mk, bval);
            values[rb + i * dq + k] = val;
        }
    if (sub == 0) {
        double val = 0.0;
        if (mk) flow_put(val, lift, rm, r, r, mk, bval);
        values[rb + 2 * dq] = val;
    }
    if (__any_sync(gmask, lift != 0.0))
#pragma unroll
        for (int o = 8; o > 0; o >>= 1) lift += __shfl_xor_sync(gmask, lift, o, 16);
    if (sub == 0) d[r] = rm ? bval[r] : lift;
}

// pressure-mass diagonal: one thread per P1 node, incident elements ascending
__global__ void k_pmass(int64_t n1, const int64_t *__restrict__ pinc_ptr, const int32_t *__restrict__ pinc,
                        const int32_t *__restrict__ pconn, const int32_t *__restrict__ conn,
                        const double *__restrict__ X, double *__restrict__ out)
{
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= n1) return;
    double s = 0.0;
    for (int64_t t = pinc_ptr[n]; t < pinc_ptr[n + 1]; ++t) {
        const int64_t e = pinc[t];
        int a = 0;
        while (a < 2 && pconn[3 * e + a] != n) ++a;
        double gl[3][2];
        const double det = tri_affine(X, conn + 6 * e, gl);
        double m = 0.0;
        for (int q = 0; q < 6; ++q) {
            double l[3], w;
            tri6_point(q, l, w);
            m = fma(w * det, l[a] * l[a], m);
        }
        s += m;
    }
    out[n] = s;
}

// flow preconditioner: velocity rows diag(K), pressure rows p_scale * Mp (written by k_pmass
// into out[2 n2 ..] beforehand), constrained dofs 1
__global__ void k_flow_precond(int64_t n2, int64_t n_rows, const int64_t *__restrict__ rp,
                               const int32_t *__restrict__ ci, const double *__restrict__ v,
                               const uint8_t *__restrict__ mask, double p_scale, double *__restrict__ out)
{
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n_rows) return;
    double val;
    if (r < 2 * n2) {
        val = 0.0;
        for (int64_t t = rp[r]; t < rp[r + 1]; ++t)
            if (ci[t] == r) val = v[t];
    } else {
        val = p_scale * out[r];
    }
    if (mask && mask[r]) val = 1.0;
    out[r] = val;
}

}  // namespace

// Host: the reference sums (c_Ms, c_R) in this file's constant memory
mf_status mf_flow_consts_upload() { return fem_consts_upload(); }

void mf_launch_gather_elastic(bool fixed_point, int fp, int fq, int64_t n0, int64_t n1, const mf_mesh *m,
                              const mf_pattern *p, const mf_coeffs *c, double *values, double *d, cudaStream_t st)
{
    if (n1 <= n0) return;
    const mf_adj &A = p->adj[0];
    const unsigned grid = nblk(n1 - n0, GEL_WARPS);
    if (fixed_point)
        k_gather_el<long long><<<grid, GEL_WARPS * 32, 0, st>>>(
            n0, n1, A.ptr, A.col, p->inc_ptr, p->inc, p->inc_loc, p->slot, p->scratch, p->scratch_stride,
            static_cast<const int *>(p->mixed_state), fp, fq, c->bc_mask, c->bc_val, p->row_ptr, values, d);
    else
        k_gather_el<double><<<grid, GEL_WARPS * 32, 0, st>>>(
            n0, n1, A.ptr, A.col, p->inc_ptr, p->inc, p->inc_loc, p->slot, p->scratch, p->scratch_stride, nullptr,
            0, 0, c->bc_mask, c->bc_val, p->row_ptr, values, d);
}

mf_status mf_flow_precond_impl(const mf_mesh *m, const mf_pattern *p, const mf_csr *K, const uint8_t *mask,
                               double p_scale, double *out, cudaStream_t st)
{
    const int64_t n2 = m->n_nodes;
    k_pmass<<<nblk(m->n_pnodes, 128), 128, 0, st>>>(m->n_pnodes, p->pinc_ptr, p->pinc, m->pconn, m->conn,
                                                    m->coords, out + 2 * n2);
    k_flow_precond<<<nblk(p->n_rows, 256), 256, 0, st>>>(n2, p->n_rows, K->row_ptr, K->col_idx, K->values, mask,
                                                         p_scale, out);
    MF_CUDA(cudaGetLastError());
    return MF_OK;
}

mf_status mf_assemble_fp64(int form, const mf_mesh *m, const mf_pattern *p, const mf_coeffs *c, double *values,
                           double *d, cudaStream_t st)
{
    int *status = mf_status_word();
    if (!status) return mf_fail(MF_ERR_CUDA, "mf_assemble: status word unavailable");
    const int64_t ne = m->n_elems;
    if (form == MF_FORM_THERMAL || form == MF_FORM_CAPACITY) {
        const bool cap = form == MF_FORM_CAPACITY;
        const double f = cap ? 0.0 : c->source[0];
        // the translate shortcut of the capacity form takes element 0's unit-C
        // capacity matrix (and its zero load) stored after the stiffness's
        const double *kref = (cap && p->kref) ? p->kref + 73 : p->kref;
        mf_prof_begin(cap ? "elem_capacity"
                      : m->elem == MF_P1_TRI ? "elem_thermal_p1"
                      : m->elem == MF_P2_TRI ? "elem_thermal_p2"
                      : m->elem == MF_Q1_HEX ? "elem_thermal_q1"
                      : m->elem == MF_P2_TET ? "elem_thermal_p2t"
                      : m->elem == MF_Q2S_QUAD ? "elem_thermal_q2q"
                                             : "elem_thermal_q2s",
                      st);
        if (cap && (m->elem == MF_Q2S_QUAD || m->elem == MF_P2_TET))
            k_elem_capacity<<<nblk(ne, 128), 128, 0, st>>>(m->elem, ne, m->coords, m->conn, c->elem_coef, p->tr,
                                                           p->elem_inc, p->scratch, status);
        else if (m->elem == MF_Q2S_QUAD)
            k_elem_thermal_q2q<<<nblk(ne, 128), 128, 0, st>>>(ne, m->coords, m->conn, c->elem_coef, f, p->elem_inc,
                                                              p->scratch, status);
        else if (m->elem == MF_P2_TET)
            k_elem_thermal_p2t<<<nblk(ne, 128), 128, 0, st>>>(ne, m->coords, m->conn, c->elem_coef, f, p->elem_inc,
                                                              p->scratch, status);
        else if (m->elem == MF_Q2S_HEX)
            k_elem_thermal_q2s<<<nblk(ne, Q2W), Q2W * 32, 0, st>>>(ne, p->q2s_map, c->elem_coef, f, p->elem_inc,
                                                                   p->scratch, status);
        else if (cap)
            k_elem_capacity<<<nblk(ne, 128), 128, 0, st>>>(m->elem, ne, m->coords, m->conn, c->elem_coef, p->tr,
                                                           p->elem_inc, p->scratch, status);
        else if (m->elem == MF_P1_TRI)
            k_elem_thermal_p1<<<nblk(ne, 128), 128, 0, st>>>(ne, m->coords, m->conn, c->elem_coef, f, p->elem_inc,
                                                             p->scratch, status);
        else if (m->elem == MF_P2_TRI)
            k_elem_thermal_p2<<<nblk(ne, 128), 128, 0, st>>>(ne, m->coords, m->conn, c->elem_coef, f, p->elem_inc,
                                                             p->scratch, status);
        else if (!p->kc_df || p->n_translate < ne)
            k_elem_thermal_q1<<<nblk(ne, 128), 128, 0, st>>>(ne, m->coords, m->conn, c->elem_coef, f, p->tr,
                                                             p->elem_inc, p->scratch, status);
        // Q1 with translates: their coefficients as pairs for the double-float
        // gather (the element kernel only runs for the other elements); a
        // lexicographic box of a rectangular cell takes its rows straight from
        // the FP64 coefficients
        const bool q1df = m->elem == MF_Q1_HEX && p->kc_df && p->kref_df && p->bcrow && p->n_translate == ne;
        const bool q1box = q1df && p->box[0] > 0;
        if (q1df && !q1box && ne > 0)
            k_kc_split<<<nblk(ne, 256), 256, 0, st>>>(ne, c->elem_coef, p->tr, p->kc_df, status);
        mf_prof_end(st);
        MF_CUDA(cudaGetLastError());
        const mf_adj &A = p->adj[0];
        mf_prof_begin("gather_scalar", st);
        if (q1df) {
            if (c->bc_mask) {
                MF_CUDA(cudaMemsetAsync(p->bcrow, 0, (size_t)A.n_rows, st));
                k_mark_bc_rows<<<nblk(A.n_rows, 256), 256, 0, st>>>(A.n_rows, A.ptr, A.col, c->bc_mask, p->bcrow);
            }
            if (q1box) {
                k_rows_q1box<<<nblk(A.n_rows, QB), QB, 0, st>>>((int)A.n_rows, p->box[0], p->box[1], p->box[2],
                                                                p->box_cls, cap ? 1 : 0, f, c->elem_coef, c->bc_mask,
                                                                p->bcrow, c->bc_val, p->row_ptr, values, d, ne,
                                                                status);
                mf_prof_end(st);
                MF_CUDA(cudaGetLastError());
                return MF_OK;
            }
            const float fh = (float)f;
            const float2 f_df = make_float2(fh, (float)(f - (double)fh));  // as f64_to_df
            k_gather_th_q1df<<<nblk(A.n_rows, GD_WARPS * 4), GD_WARPS * 32, 0, st>>>(
                A.n_rows, A.ptr, A.col, p->inc_ptr, p->inc, p->inc_loc, p->inc_slot,
                cap ? p->kref_df + 73 : p->kref_df, p->kc_df, f_df, c->bc_mask, p->bcrow, c->bc_val, p->row_ptr,
                values, d);
            mf_prof_end(st);
            MF_CUDA(cudaGetLastError());
            return MF_OK;
        }
#define MF_GATHER_TH(NPE)                                                                                         \
    k_gather_th<NPE><<<nblk(A.n_rows, GT_WARPS * (32 / th_lanes<NPE>())), GT_WARPS * 32, 0, st>>>(                 \
        A.n_rows, A.ptr, A.col, p->inc_ptr, p->inc, p->inc_loc, p->inc_slot, p->scratch, kref, c->elem_coef, f,     \
        c->bc_mask, c->bc_val, p->row_ptr, values, d)
        if (m->elem == MF_P1_TRI) MF_GATHER_TH(3);
        else if (m->elem == MF_P2_TRI) MF_GATHER_TH(6);
        else if (m->elem == MF_Q1_HEX || m->elem == MF_Q2S_QUAD) MF_GATHER_TH(8);
        else if (m->elem == MF_P2_TET) MF_GATHER_TH(10);
        else MF_GATHER_TH(20);
#undef MF_GATHER_TH
        mf_prof_end(st);
    } else if (form == MF_FORM_ELASTIC && m->elem == MF_Q2S_HEX) {
        mf_prof_begin("elem_elastic_q2s", st);
        if (ne > 0)
            k_elem_elastic_q2s<<<(unsigned)ne, EQ_T, 0, st>>>(ne, p->q2s_map, c->elem_coef, c->nu, c->source[0],
                                                              c->source[1], c->source[2], p->elem_inc, p->scratch,
                                                              status);
        mf_prof_end(st);
        MF_CUDA(cudaGetLastError());
        mf_prof_begin("gather_elastic_q2s", st);
        const mf_adj &A = p->adj[0];
        const int maxd = A.max_deg > 0 ? A.max_deg : 1;
        const size_t smem = GQ_WARPS * gq_warp_bytes(maxd);
        MF_CUDA(cudaFuncSetAttribute(k_gather_el_q2s, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_gather_el_q2s<<<nblk(m->n_nodes, GQ_WARPS), GQ_WARPS * 32, smem, st>>>(
            m->n_nodes, maxd, A.ptr, A.col, p->inc_ptr, p->inc_slot, p->scratch, c->bc_mask, c->bc_val, p->row_ptr,
            values, d);
        mf_prof_end(st);
    } else if (form == MF_FORM_ELASTIC) {
        const size_t smem = sizeof(double) * 8 * 8 * 3 * EL_T;
        MF_CUDA(cudaFuncSetAttribute(k_elem_elastic_q1, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        // one launch pair over the whole mesh: both kernels are bound by the
        // FP64 pipe, so chunks would not overlap usefully
        mf_prof_begin("elem_elastic_q1_fp64", st);
        k_elem_elastic_q1<<<nblk(ne, EL_T), EL_T, smem, st>>>(0, ne, m->coords, m->conn, c->elem_coef, c->nu,
                                                             c->source[0], c->source[1], c->source[2], p->scratch,
                                                             status);
        mf_prof_end(st);
        MF_CUDA(cudaGetLastError());
        mf_prof_begin("gather_elastic", st);
        mf_launch_gather_elastic(false, 0, 0, 0, m->n_nodes, m, p, c, values, d, st);
        mf_prof_end(st);
    } else {
        mf_prof_begin("elem_oseen", st);
        k_elem_oseen<<<nblk(ne, 128), 128, 0, st>>>(ne, m->n_nodes, m->coords, m->conn, c->advect, c->visc, c->rho,
                                                    p->scratch, status);
        mf_prof_end(st);
        MF_CUDA(cudaGetLastError());
        mf_prof_begin("gather_oseen", st);
        if (c->bc_mask) {  // rows next to a constrained dof: the pattern is structurally symmetric
            MF_CUDA(cudaMemsetAsync(p->bcrow, 0, (size_t)p->n_rows, st));
            k_mark_bc_rows<<<nblk(p->n_rows, 256), 256, 0, st>>>(p->n_rows, p->row_ptr, p->col_idx, c->bc_mask,
                                                                 p->bcrow);
        }
        k_gather_oseen_u<<<nblk(m->n_nodes, GO_GROUPS), GO_GROUPS * 16, 0, st>>>(
            m->n_nodes, p->adj[0], p->adj[1], p->inc_ptr, p->inc_loc, p->inc, p->inc_slot, p->inc_slot_pq,
            p->scratch, c->bc_mask, p->bcrow, c->bc_val, p->row_ptr, values, d);
        k_gather_oseen_p<<<nblk(m->n_pnodes, GO_GROUPS), GO_GROUPS * 16, 0, st>>>(
            m->n_nodes, m->n_pnodes, p->adj[2], p->pinc_ptr, p->pinc, p->pinc_loc, p->pinc_slot, p->scratch,
            c->bc_mask, p->bcrow, c->bc_val, p->row_ptr, values, d);
        mf_prof_end(st);
    }
    MF_CUDA(cudaGetLastError());
    return MF_OK;
}

mf_status mf_pmass_impl(const mf_mesh *m, const mf_pattern *p, double *out, cudaStream_t st)
{
    k_pmass<<<nblk(m->n_pnodes, 128), 128, 0, st>>>(m->n_pnodes, p->pinc_ptr, p->pinc, m->pconn, m->conn,
                                                    m->coords, out);
    MF_CUDA(cudaGetLastError());
    return MF_OK;
}
