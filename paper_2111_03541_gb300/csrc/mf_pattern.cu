// Mesh validation and sparsity pattern (MetaFEM Sec. 2.2 Block B).
//
// Block B-1 collects the unique control-point pairs of every element, Block
// B-4 gives each (symbol pair, control-point pair) one sparse id.  Here the
// unique pairs of a row node space and a column node space form an adjacency
// (CSR over row nodes, ascending columns) built without hashing: per row node
// the incident elements are gathered and their nodes sorted and de-duplicated
// in registers.  The gathers walk a node's incident elements in ascending
// order and place each entry through a slot map (the position of the column
// node among the row node's neighbours), which fixes the summation order of
// the assembly.  The dof-level CSR of a form is then laid out from its blocks.
#include <algorithm>
#include <cmath>
#include <cstdio>

#include "mf_fem.cuh"

namespace {

constexpr int TPB = 256;

inline unsigned nblk(int64_t n, int t = TPB) { return (unsigned)((n + t - 1) / t); }

// ---------------------------------------------------------------------------
// mesh validation: indices in range, finite coordinates, detJ > 0 at every
// quadrature point of the rules the assembly uses
// ---------------------------------------------------------------------------
__global__ void k_validate(int elem, int64_t n_el, int64_t n_nodes, const double *__restrict__ X,
                           const int32_t *__restrict__ conn, int64_t n_p, const int32_t *__restrict__ pconn,
                           int *status)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n_el) return;
    const int npe = elem == MF_P1_TRI ? 3
                  : elem == MF_P2_TRI ? 6
                  : (elem == MF_Q1_HEX || elem == MF_Q2S_QUAD) ? 8
                  : elem == MF_Q2S_HEX ? 20 : 10;
    for (int a = 0; a < npe; ++a) {
        const int32_t v = conn[e * npe + a];
        if (v < 0 || v >= n_nodes) { mf_dev_fail(status, MF_ERR_BAD_MESH); return; }
    }
    if (pconn)
        for (int a = 0; a < 3; ++a) {
            const int32_t v = pconn[e * 3 + a];
            if (v < 0 || v >= n_p) { mf_dev_fail(status, MF_ERR_BAD_MESH); return; }
        }
    if (elem == MF_P1_TRI || elem == MF_P2_TRI) {
        const int32_t *c = conn + e * npe;
        const double x0 = X[2 * c[0]], y0 = X[2 * c[0] + 1];
        const double x1 = X[2 * c[1]], y1 = X[2 * c[1] + 1];
        const double x2 = X[2 * c[2]], y2 = X[2 * c[2] + 1];
        const double det = (x1 - x0) * (y2 - y0) - (x2 - x0) * (y1 - y0);
        if (!isfinite(det)) { mf_dev_fail(status, MF_ERR_NONFINITE); return; }
        if (!(det > 0.0)) mf_dev_fail(status, MF_ERR_BAD_MESH);
        return;
    }
    if (elem == MF_Q2S_QUAD) {  // the bilinear map of the 4 vertices at the 3 x 3 Gauss points
        const int32_t *c = conn + e * npe;
        double x[4][2];
        for (int a = 0; a < 4; ++a)
            for (int i = 0; i < 2; ++i) x[a][i] = X[2 * (int64_t)c[a] + i];
        const double g3 = 0.77459666924148337704;  // sqrt(3/5)
        for (int q = 0; q < 9; ++q) {
            const double xs = (q % 3 - 1) * g3, ys = (q / 3 - 1) * g3;
            double J[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
            for (int a = 0; a < 4; ++a) {
                const double sa = (a & 1) ? 1.0 : -1.0, ta = (a & 2) ? 1.0 : -1.0;
                const double dx = 0.25 * sa * (1.0 + ta * ys), dy = 0.25 * ta * (1.0 + sa * xs);
                for (int i = 0; i < 2; ++i) {
                    J[i][0] += x[a][i] * dx;
                    J[i][1] += x[a][i] * dy;
                }
            }
            const double det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
            if (!isfinite(det)) { mf_dev_fail(status, MF_ERR_NONFINITE); return; }
            if (!(det > 0.0)) { mf_dev_fail(status, MF_ERR_BAD_MESH); return; }
        }
        return;
    }
    if (elem == MF_P2_TET) {  // the affine map of the 4 vertices
        const int32_t *c = conn + e * npe;
        double J[3][3];
        for (int j = 0; j < 3; ++j)
            for (int i = 0; i < 3; ++i) J[i][j] = X[3 * (int64_t)c[j + 1] + i] - X[3 * (int64_t)c[0] + i];
        const double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) +
                           J[0][1] * (J[1][2] * J[2][0] - J[1][0] * J[2][2]) +
                           J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
        if (!isfinite(det)) { mf_dev_fail(status, MF_ERR_NONFINITE); return; }
        if (!(det > 0.0)) mf_dev_fail(status, MF_ERR_BAD_MESH);
        return;
    }
    // hexahedra: the trilinear map of the 8 vertices (also the geometry of a
    // straight-edged serendipity brick) at the 2 x 2 x 2 (Q1) or 3 x 3 x 3
    // (Q2S) Gauss points
    double x[8][3];
    for (int a = 0; a < 8; ++a)
        for (int i = 0; i < 3; ++i) x[a][i] = X[3 * (int64_t)conn[e * npe + a] + i];
    const double g = 0.57735026918962576451;  // 1/sqrt(3)
    const double g3 = 0.77459666924148337704;  // sqrt(3/5)
    const int nq = elem == MF_Q1_HEX ? 8 : 27;
    for (int q = 0; q < nq; ++q) {
        double xi[3];
        if (elem == MF_Q1_HEX) {
            xi[0] = (q & 1) ? g : -g;
            xi[1] = (q & 2) ? g : -g;
            xi[2] = (q & 4) ? g : -g;
        } else {
            xi[0] = (q % 3 - 1) * g3;
            xi[1] = ((q / 3) % 3 - 1) * g3;
            xi[2] = (q / 9 - 1) * g3;
        }
        double J[3][3] = {};
        for (int a = 0; a < 8; ++a) {
            const double s[3] = {(a & 1) ? 1.0 : -1.0, (a & 2) ? 1.0 : -1.0, (a & 4) ? 1.0 : -1.0};
            const double f[3] = {1.0 + s[0] * xi[0], 1.0 + s[1] * xi[1], 1.0 + s[2] * xi[2]};
            const double dN[3] = {0.125 * s[0] * f[1] * f[2], 0.125 * f[0] * s[1] * f[2], 0.125 * f[0] * f[1] * s[2]};
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) J[i][j] += x[a][i] * dN[j];
        }
        const double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
                           J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                           J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
        if (!isfinite(det)) { mf_dev_fail(status, MF_ERR_NONFINITE); return; }
        if (!(det > 0.0)) { mf_dev_fail(status, MF_ERR_BAD_MESH); return; }
    }
}

// ---------------------------------------------------------------------------
// incidence: elements of every node, ascending
// ---------------------------------------------------------------------------
__global__ void k_inc_count(int64_t n_el, int npe, const int32_t *__restrict__ conn, int64_t *cnt)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_el * npe) return;
    atomicAdd(reinterpret_cast<unsigned long long *>(&cnt[conn[t]]), 1ull);
}

__global__ void k_inc_fill(int64_t n_el, int npe, const int32_t *__restrict__ conn, const int64_t *ptr,
                           int64_t *cursor, int32_t *inc)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_el * npe) return;
    const int32_t v = conn[t];
    const int64_t pos = ptr[v] + (int64_t)atomicAdd(reinterpret_cast<unsigned long long *>(&cursor[v]), 1ull);
    inc[pos] = (int32_t)(t / npe);
}

// position of node n within each of its incident elements
__global__ void k_inc_local(int64_t n_nodes, int npe, const int32_t *__restrict__ conn, const int64_t *__restrict__ ptr,
                            const int32_t *__restrict__ inc, uint8_t *__restrict__ loc)
{
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= n_nodes) return;
    for (int64_t t = ptr[n]; t < ptr[n + 1]; ++t) {
        const int32_t *ce = conn + (int64_t)inc[t] * npe;
        int a = 0;
        for (int k = 0; k < npe; ++k)
            if (ce[k] == (int32_t)n) a = k;
        loc[t] = (uint8_t)a;
    }
}

__global__ void k_sort_segments_i32(int64_t n, const int64_t *__restrict__ ptr, int32_t *v, int *status)
{
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    const int64_t b = ptr[r], e = ptr[r + 1];
    if (e - b > 4 * MF_MAX_INC) { mf_dev_fail(status, MF_ERR_UNSUPPORTED); return; }
    for (int64_t i = b + 1; i < e; ++i) {  // insertion sort of a short segment
        const int32_t x = v[i];
        int64_t j = i - 1;
        while (j >= b && v[j] > x) { v[j + 1] = v[j]; --j; }
        v[j + 1] = x;
    }
}

// ---------------------------------------------------------------------------
// adjacency between row space (conn_r, npe_r) and column space (conn_c, npe_c)
// ---------------------------------------------------------------------------
template <bool FILL, int MAXD>
__global__ void k_adj(int64_t n_rows, const int64_t *__restrict__ inc_ptr, const int32_t *__restrict__ inc,
                      int npe_c, const int32_t *__restrict__ conn_c, bool self, int64_t *cnt,
                      const int64_t *__restrict__ ptr, int32_t *col, int *status)
{
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n_rows) return;
    int32_t nb[MAXD];
    int deg = 0;
    if (self) nb[deg++] = (int32_t)r;  // square adjacency: the diagonal is always present
    const int64_t b = inc_ptr[r], e = inc_ptr[r + 1];
    if (e - b > MF_MAX_INC) { mf_dev_fail(status, MF_ERR_UNSUPPORTED); return; }
    for (int64_t t = b; t < e; ++t) {
        const int32_t el = inc[t];
        for (int a = 0; a < npe_c; ++a) {
            const int32_t m = conn_c[(int64_t)el * npe_c + a];
            int pos = 0;
            while (pos < deg && nb[pos] < m) ++pos;
            if (pos < deg && nb[pos] == m) continue;
            if (deg == MAXD) { mf_dev_fail(status, MF_ERR_UNSUPPORTED); return; }
            for (int s = deg; s > pos; --s) nb[s] = nb[s - 1];
            nb[pos] = m;
            ++deg;
        }
    }
    if (!FILL) {
        cnt[r] = deg;
    } else {
        int32_t *out = col + ptr[r];
        for (int s = 0; s < deg; ++s) out[s] = nb[s];
    }
}

__device__ __forceinline__ int64_t find_pair(const int64_t *ptr, const int32_t *col, int32_t n, int32_t m)
{
    int64_t lo = ptr[n], hi = ptr[n + 1] - 1;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (col[mid] < m) lo = mid + 1; else hi = mid;
    }
    return lo;  // the pair exists by construction
}

// last (largest) incident element of every node
__global__ void k_node_ready(int64_t n, const int64_t *__restrict__ inc_ptr, const int32_t *__restrict__ inc,
                             int32_t *ready)
{
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    ready[v] = inc_ptr[v + 1] > inc_ptr[v] ? inc[inc_ptr[v + 1] - 1] : -1;
}

// Upper node pairs (n, m >= n) in a compact numbering: they are the tail of
// n's sorted neighbour list from the diagonal on, so upper pair (n, slot k)
// is number cbase[n] + k with cbase[n] = (upper pairs of nodes < n) - the
// diagonal's slot.  First the count of each node's upper pairs:
__global__ void k_upper_count(int64_t n_nodes, const int64_t *__restrict__ ptr, const int32_t *__restrict__ col,
                              int64_t *__restrict__ cnt, int64_t *__restrict__ kdiag)
{
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= n_nodes) return;
    int64_t kd = 0;
    for (int64_t p = ptr[n]; p < ptr[n + 1]; ++p)
        if (col[p] == (int32_t)n) kd = p - ptr[n];
    kdiag[n] = kd;
    cnt[n] = (ptr[n + 1] - ptr[n]) - kd;
}

__global__ void k_upper_base(int64_t n_nodes, const int64_t *__restrict__ scan, int64_t *__restrict__ cbase)
{
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= n_nodes) return;
    cbase[n] = scan[n] - cbase[n];  // cbase holds the diagonal slots on entry
}

// tpos[p] = compact number of the upper pair (m, n) for a lower pair p = (n, m < n)
__global__ void k_tpos(int64_t n_nodes, const int64_t *__restrict__ ptr, const int32_t *__restrict__ col,
                       const int64_t *__restrict__ cbase, int32_t *__restrict__ tpos)
{
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= n_nodes) return;
    for (int64_t p = ptr[n]; p < ptr[n + 1]; ++p) {
        const int32_t m = col[p];
        tpos[p] = m < n ? (int32_t)(cbase[m] + (find_pair(ptr, col, m, (int32_t)n) - ptr[m]))
                        : (int32_t)(cbase[n] + (p - ptr[n]));
    }
}

// the accumulator block of each upper block pair (a <= b) of every element:
// (n_a, n_b) when n_a <= n_b, else (n_b, n_a) holding the transpose (bit 31)
__global__ void k_mixed_etgt(int64_t ne, const int32_t *__restrict__ conn, const int64_t *__restrict__ cbase,
                             const uint8_t *__restrict__ slot, int32_t *__restrict__ etgt)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ne * 36) return;
    const int64_t e = i / 36;
    const int u = (int)(i - 36 * e);
    int a = 0, rem = u;
    while (rem >= 8 - a) {
        rem -= 8 - a;
        ++a;
    }
    const int b = a + rem;
    const int32_t na = conn[8 * e + a], nb = conn[8 * e + b];
    etgt[i] = na <= nb ? (int32_t)(cbase[na] + slot[e * 64 + a * 8 + b])
                       : (int32_t)((cbase[nb] + slot[e * 64 + b * 8 + a]) | 0x80000000ll);
}

// incidence slot map: for incidence entry t of row node n (element e),
// inc_slot[t * npe_c + b] = position of column node conn_c[e][b] among the
// neighbours of n in the adjacency (ptr, col)
__global__ void k_inc_slot(int64_t n_nodes, int npe_c, const int32_t *__restrict__ conn_c,
                           const int64_t *__restrict__ inc_ptr, const int32_t *__restrict__ inc,
                           const int64_t *__restrict__ ptr, const int32_t *__restrict__ col, uint8_t *inc_slot)
{
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= n_nodes) return;
    for (int64_t t = inc_ptr[n]; t < inc_ptr[n + 1]; ++t) {
        const int32_t *ce = conn_c + (int64_t)inc[t] * npe_c;
        for (int b = 0; b < npe_c; ++b)
            inc_slot[t * npe_c + b] = (uint8_t)(find_pair(ptr, col, (int32_t)n, ce[b]) - ptr[n]);
    }
}

// elem_inc[e * npe + a] = incidence entry of (e, a)
__global__ void k_elem_inc(int64_t n_nodes, int npe, const int64_t *__restrict__ inc_ptr,
                           const int32_t *__restrict__ inc, const uint8_t *__restrict__ loc, int32_t *elem_inc)
{
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= n_nodes) return;
    for (int64_t t = inc_ptr[n]; t < inc_ptr[n + 1]; ++t) elem_inc[(int64_t)inc[t] * npe + loc[t]] = (int32_t)t;
}

// bit 7 of inc_loc marks incidence entries of translate elements
__global__ void k_mark_translates(int64_t n_nodes, const int64_t *__restrict__ inc_ptr,
                                  const int32_t *__restrict__ inc, const uint8_t *__restrict__ tr, uint8_t *loc)
{
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= n_nodes) return;
    for (int64_t t = inc_ptr[n]; t < inc_ptr[n + 1]; ++t)
        if (tr[inc[t]]) loc[t] |= 0x80;
}

// map coefficients of the 20-node bricks (q1_wht's of the 8 vertices,
// scaled for q1_jac_at) as FP32 pairs: thread (e, S, i)
__global__ void k_q2s_map(int64_t n_el, const double *__restrict__ X, const int32_t *__restrict__ conn,
                          float2 *__restrict__ out)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 24 * n_el) return;
    const int64_t e = t / 24;
    const int r = (int)(t - 24 * e), S = r / 3, i = r - 3 * S;
    double v = 0.0;
    for (int a = 0; a < 8; ++a) {
        const double xa = X[3 * (int64_t)conn[20 * e + a] + i];
        v += (__popc(a & S) & 1) ? -xa : xa;
    }
    const double cv = v * ((__popc(S) & 1) ? -0.125 : 0.125);
    const float hi = __double2float_rn(cv);
    out[t] = make_float2(hi, __double2float_rn(cv - (double)hi));
}

// largest row of an adjacency
__global__ void k_max_deg(int64_t n_rows, const int64_t *__restrict__ ptr, int *out)
{
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r < n_rows) atomicMax(out, (int)(ptr[r + 1] - ptr[r]));
}

// slot map: position of conn[e][b] among the neighbours of conn[e][a],
// slot[(e * npe + a) * npe + b]
__global__ void k_slot_map(int64_t n_el, int npe, const int32_t *__restrict__ conn, const int64_t *__restrict__ ptr,
                           const int32_t *__restrict__ col, uint8_t *slot)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nn = (int64_t)npe * npe;
    if (t >= n_el * nn) return;
    const int64_t e = t / nn;
    const int r = (int)(t - e * nn);
    const int a = r / npe, b = r - a * npe;
    const int32_t n = conn[e * npe + a], m = conn[e * npe + b];
    slot[t] = (uint8_t)(find_pair(ptr, col, n, m) - ptr[n]);
}

// Q1 translates of element 0: equal edge vectors x_a - x_0 (FP64, exact
// comparison).  Counted per warp.
__global__ void k_translate_flags(int64_t n_el, const double *__restrict__ X, const int32_t *__restrict__ conn,
                                  uint8_t *__restrict__ tr, unsigned long long *count)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    bool t = false;
    if (e < n_el) {
        t = true;
        const int32_t *ce = conn + 8 * e;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const double r0 = X[3 * (int64_t)conn[0] + i], x0 = X[3 * (int64_t)ce[0] + i];
#pragma unroll
            for (int a = 1; a < 8; ++a)
                t = t && (X[3 * (int64_t)ce[a] + i] - x0 == X[3 * (int64_t)conn[a] + i] - r0);
        }
        tr[e] = t ? 1 : 0;
    }
    const unsigned bal = __ballot_sync(0xffffffffu, t);
    if ((threadIdx.x & 31) == 0 && bal) atomicAdd(count, (unsigned long long)__popc(bal));
}

// the reference entries as FP32 pairs
// lexicographic box check: element e = ex + nx (ey + ny ez) must have its
// local node a at node base(e) + off[a], base(e) = ex + nx1 (ey + ny1 ez)
__global__ void k_box_check(int64_t n_el, const int32_t *__restrict__ conn, int nx, int ny, int nx1, int ny1,
                            int4 off_lo, int4 off_hi, int *bad)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n_el) return;
    const int64_t ex = e % nx, ey = (e / nx) % ny, ez = e / ((int64_t)nx * ny);
    const int64_t base = ex + (int64_t)nx1 * (ey + (int64_t)ny1 * ez);
    const int off[8] = {off_lo.x, off_lo.y, off_lo.z, off_lo.w, off_hi.x, off_hi.y, off_hi.z, off_hi.w};
#pragma unroll
    for (int a = 0; a < 8; ++a)
        if ((int64_t)conn[8 * e + a] != base + off[a]) *bad = 1;
}

__global__ void k_kref_df(const double *__restrict__ kref, float2 *__restrict__ kref_df)
{
    const int t = threadIdx.x;
    if (t < 73 + 72) kref_df[t] = f64_to_df(kref[t]);
}

// kref = element 0's matrix and load vector with k = 1, f = 1 (kref[72] holds
// the 1), then its capacity matrix with C = 1 and a zero load at kref + 73
__global__ void k_kref(const double *__restrict__ X, const int32_t *__restrict__ conn, double *kref, int *status)
{
    kref[72] = 1.0;
    elem_thermal_q1(0, X, conn, kref + 72, 1.0, nullptr, kref, status);
    elem_capacity_q1(0, X, conn, kref + 72, nullptr, kref + 73, status);
}

// ---------------------------------------------------------------------------
// dof-level CSR of each form
// ---------------------------------------------------------------------------
__global__ void k_csr_thermal(int64_t n, const int64_t *__restrict__ ptr, int64_t *row_ptr)
{
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r <= n) row_ptr[r] = ptr[r];
}

__global__ void k_csr_elastic(int64_t n_nodes, const int64_t *__restrict__ ptr, const int32_t *__restrict__ col,
                              int64_t *row_ptr, int32_t *col_idx)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t > 3 * n_nodes) return;
    if (t == 3 * n_nodes) { row_ptr[t] = 9 * ptr[n_nodes]; return; }
    const int64_t n = t / 3;
    const int c = (int)(t % 3);
    const int64_t deg = ptr[n + 1] - ptr[n];
    const int64_t base = 9 * ptr[n] + 3 * c * deg;
    row_ptr[t] = base;
    for (int64_t k = 0; k < deg; ++k)
        for (int cp = 0; cp < 3; ++cp) col_idx[base + 3 * k + cp] = 3 * col[ptr[n] + k] + cp;
}

// flow: rows u_i(n) = [u_i cols over P2-P2 | p cols over P2-P1];
//       rows p(n)   = [u1 cols over P1-P2 | u2 cols over P1-P2 | p(n)]
__global__ void k_csr_oseen_len(int64_t n2, int64_t n1, const int64_t *__restrict__ pp, const int64_t *__restrict__ pq,
                                const int64_t *__restrict__ qp, int64_t *len)
{
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= 2 * n2 + n1) return;
    if (r < 2 * n2) {
        const int64_t n = r % n2;
        len[r] = (pp[n + 1] - pp[n]) + (pq[n + 1] - pq[n]);
    } else {
        const int64_t n = r - 2 * n2;
        len[r] = 2 * (qp[n + 1] - qp[n]) + 1;
    }
}

__global__ void k_csr_oseen_fill(int64_t n2, int64_t n1, const int64_t *__restrict__ pp, const int32_t *__restrict__ ppc,
                                 const int64_t *__restrict__ pq, const int32_t *__restrict__ pqc,
                                 const int64_t *__restrict__ qp, const int32_t *__restrict__ qpc,
                                 const int64_t *__restrict__ row_ptr, int32_t *col_idx)
{
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= 2 * n2 + n1) return;
    int32_t *out = col_idx + row_ptr[r];
    if (r < 2 * n2) {
        const int64_t i = r / n2, n = r % n2;
        int64_t o = 0;
        for (int64_t t = pp[n]; t < pp[n + 1]; ++t) out[o++] = (int32_t)(i * n2 + ppc[t]);
        for (int64_t t = pq[n]; t < pq[n + 1]; ++t) out[o++] = (int32_t)(2 * n2 + pqc[t]);
    } else {
        const int64_t n = r - 2 * n2;
        int64_t o = 0;
        for (int i = 0; i < 2; ++i)
            for (int64_t t = qp[n]; t < qp[n + 1]; ++t) out[o++] = (int32_t)(i * n2 + qpc[t]);
        out[o] = (int32_t)r;
    }
}

// Navier-Stokes rows: a velocity row of P2 node n has [u1: adj0 | u2: n2 +
// adj0 | p: 2 n2 + adj1], a pressure row of P1 node m [u1: adj2 | u2: n2 +
// adj2 | p: 2 n2 + adj3] (ascending, the diagonal present in both)
__global__ void k_csr_ns_len(int64_t n2, int64_t n1, const int64_t *__restrict__ pp, const int64_t *__restrict__ pq,
                             const int64_t *__restrict__ qp, const int64_t *__restrict__ qq, int64_t *len)
{
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= 2 * n2 + n1) return;
    if (r < 2 * n2) {
        const int64_t n = r % n2;
        len[r] = 2 * (pp[n + 1] - pp[n]) + (pq[n + 1] - pq[n]);
    } else {
        const int64_t n = r - 2 * n2;
        len[r] = 2 * (qp[n + 1] - qp[n]) + (qq[n + 1] - qq[n]);
    }
}

__global__ void k_csr_ns_fill(int64_t n2, int64_t n1, const int64_t *__restrict__ pp, const int32_t *__restrict__ ppc,
                              const int64_t *__restrict__ pq, const int32_t *__restrict__ pqc,
                              const int64_t *__restrict__ qp, const int32_t *__restrict__ qpc,
                              const int64_t *__restrict__ qq, const int32_t *__restrict__ qqc,
                              const int64_t *__restrict__ row_ptr, int32_t *col_idx)
{
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= 2 * n2 + n1) return;
    int32_t *out = col_idx + row_ptr[r];
    int64_t o = 0;
    if (r < 2 * n2) {
        const int64_t n = r % n2;
        for (int i = 0; i < 2; ++i)
            for (int64_t t = pp[n]; t < pp[n + 1]; ++t) out[o++] = (int32_t)(i * n2 + ppc[t]);
        for (int64_t t = pq[n]; t < pq[n + 1]; ++t) out[o++] = (int32_t)(2 * n2 + pqc[t]);
    } else {
        const int64_t n = r - 2 * n2;
        for (int i = 0; i < 2; ++i)
            for (int64_t t = qp[n]; t < qp[n + 1]; ++t) out[o++] = (int32_t)(i * n2 + qpc[t]);
        for (int64_t t = qq[n]; t < qq[n + 1]; ++t) out[o++] = (int32_t)(2 * n2 + qqc[t]);
    }
}

struct Incidence {
    int64_t *ptr = nullptr;
    int32_t *inc = nullptr;
    uint8_t *loc = nullptr;  // local index of the node in each incident element
};

mf_status build_incidence(int64_t n_nodes, int64_t n_el, int npe, const int32_t *conn, cudaStream_t st,
                          Incidence *out, int *status)
{
    int64_t *cursor = nullptr;
    MF_CUDA(cudaMallocAsync(&out->ptr, sizeof(int64_t) * (n_nodes + 1), st));
    MF_CUDA(cudaMallocAsync(&out->inc, sizeof(int32_t) * n_el * npe, st));
    MF_CUDA(cudaMallocAsync(&cursor, sizeof(int64_t) * n_nodes, st));
    MF_CUDA(cudaMemsetAsync(out->ptr, 0, sizeof(int64_t) * (n_nodes + 1), st));
    MF_CUDA(cudaMemsetAsync(cursor, 0, sizeof(int64_t) * n_nodes, st));
    k_inc_count<<<nblk(n_el * npe), TPB, 0, st>>>(n_el, npe, conn, out->ptr);
    MF_CUDA(mf_scan_i64(out->ptr, n_nodes + 1, nullptr, st));
    k_inc_fill<<<nblk(n_el * npe), TPB, 0, st>>>(n_el, npe, conn, out->ptr, cursor, out->inc);
    k_sort_segments_i32<<<nblk(n_nodes), TPB, 0, st>>>(n_nodes, out->ptr, out->inc, status);
    MF_CUDA(cudaMallocAsync(&out->loc, (size_t)n_el * npe, st));
    k_inc_local<<<nblk(n_nodes), TPB, 0, st>>>(n_nodes, npe, conn, out->ptr, out->inc, out->loc);
    MF_CUDA(cudaGetLastError());
    MF_CUDA(cudaFreeAsync(cursor, st));
    return MF_OK;
}

mf_status read_i64(const int64_t *d, int64_t *h, cudaStream_t st)
{
    MF_CUDA(cudaMemcpyAsync(h, d, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    MF_CUDA(cudaStreamSynchronize(st));
    return MF_OK;
}

// the largest row of an adjacency, to the host (sizes the shared memory of
// the kernels that stage whole rows)
mf_status read_max_deg(int64_t n_rows, mf_adj *a, cudaStream_t st)
{
    int *dmax = nullptr;
    MF_CUDA(cudaMallocAsync(&dmax, sizeof(int), st));
    MF_CUDA(cudaMemsetAsync(dmax, 0, sizeof(int), st));
    if (n_rows > 0) k_max_deg<<<nblk(n_rows), TPB, 0, st>>>(n_rows, a->ptr, dmax);
    int h = 0;
    MF_CUDA(cudaMemcpyAsync(&h, dmax, sizeof(int), cudaMemcpyDeviceToHost, st));
    MF_CUDA(cudaStreamSynchronize(st));
    MF_CUDA(cudaFreeAsync(dmax, st));
    a->max_deg = h;
    return MF_OK;
}

mf_status check_status(int *status, cudaStream_t st, const char *what)
{
    int h = 0;
    MF_CUDA(cudaMemcpyAsync(&h, status, sizeof(int), cudaMemcpyDeviceToHost, st));
    MF_CUDA(cudaStreamSynchronize(st));
    if (h) {
        const int zero = 0;
        MF_CUDA(cudaMemcpyAsync(status, &zero, sizeof(int), cudaMemcpyHostToDevice, st));
        MF_CUDA(cudaStreamSynchronize(st));
        if (h == MF_ERR_UNSUPPORTED)
            return mf_fail(MF_ERR_UNSUPPORTED, "%s: node valence above %d elements / %d neighbours", what,
                           MF_MAX_INC, MF_MAX_DEG);
        return mf_fail((mf_status)h, "%s: device status %d", what, h);
    }
    return MF_OK;
}

mf_status build_adj(int64_t n_rows, const Incidence &inc, const int32_t *conn_r, int npe_c, const int32_t *conn_c,
                    cudaStream_t st, mf_adj *A, int *status)
{
    A->n_rows = n_rows;
    MF_CUDA(cudaMallocAsync(&A->ptr, sizeof(int64_t) * (n_rows + 1), st));
    MF_CUDA(cudaMemsetAsync(A->ptr, 0, sizeof(int64_t) * (n_rows + 1), st));
    const bool self = conn_r == conn_c;
    // the 20-node brick (npe 20) has up to 81 neighbours per node on a grid
    const bool wide = npe_c > 8;
    if (wide)
        k_adj<false, MF_MAX_DEG_HO><<<nblk(n_rows, 128), 128, 0, st>>>(n_rows, inc.ptr, inc.inc, npe_c, conn_c, self,
                                                                      A->ptr, nullptr, nullptr, status);
    else
        k_adj<false, MF_MAX_DEG><<<nblk(n_rows, 128), 128, 0, st>>>(n_rows, inc.ptr, inc.inc, npe_c, conn_c, self,
                                                                   A->ptr, nullptr, nullptr, status);
    MF_CUDA(cudaGetLastError());
    mf_status s = check_status(status, st, "mf_pattern_build");
    if (s != MF_OK) return s;
    MF_CUDA(mf_scan_i64(A->ptr, n_rows + 1, nullptr, st));
    s = read_i64(A->ptr + n_rows, &A->n_pairs, st);
    if (s != MF_OK) return s;
    MF_CUDA(cudaMallocAsync(&A->col, sizeof(int32_t) * A->n_pairs, st));
    if (wide)
        k_adj<true, MF_MAX_DEG_HO><<<nblk(n_rows, 128), 128, 0, st>>>(n_rows, inc.ptr, inc.inc, npe_c, conn_c, self,
                                                                     nullptr, A->ptr, A->col, status);
    else
        k_adj<true, MF_MAX_DEG><<<nblk(n_rows, 128), 128, 0, st>>>(n_rows, inc.ptr, inc.inc, npe_c, conn_c, self,
                                                                  nullptr, A->ptr, A->col, status);
    return check_status(status, st, "mf_pattern_build");
}

// Element chunks of about 48 MB of scratch.  A node's rows are complete once
// its largest incident element is assembled; chunk c gathers the longest
// prefix of nodes whose prefix maximum of that value lies below the chunk's
// end, so node ranges stay contiguous for any numbering (badly ordered meshes
// just gather later).
mf_status plan_slabs(const mf_mesh *m, const Incidence &inc, int64_t stride, cudaStream_t st, mf_pattern *p)
{
    const int64_t nn = m->n_nodes, ne = m->n_elems;
    int32_t *d_ready = nullptr;
    MF_CUDA(cudaMallocAsync(&d_ready, sizeof(int32_t) * nn, st));
    k_node_ready<<<nblk(nn), TPB, 0, st>>>(nn, inc.ptr, inc.inc, d_ready);
    std::vector<int32_t> ready(nn);
    MF_CUDA(cudaMemcpyAsync(ready.data(), d_ready, sizeof(int32_t) * nn, cudaMemcpyDeviceToHost, st));
    MF_CUDA(cudaStreamSynchronize(st));
    MF_CUDA(cudaFreeAsync(d_ready, st));
    for (int64_t v = 1; v < nn; ++v) ready[v] = std::max(ready[v], ready[v - 1]);  // prefix maximum
    // MF_SLABS chunks of elements; with more than one, the finishing of the
    // nodes a chunk completes overlaps the element kernel of the next chunk on
    // a second stream.  Measured on the 64^3 elasticity workload, one chunk is
    // fastest: 8 overlapped chunks took 1.43 vs 1.32 ms (the element kernel,
    // bound by instruction issue, slows down next to the finishing pass), and
    // serial chunks lose to launch ramp-up and tail.
    (void)stride;
    const int64_t chunk = std::max<int64_t>(4096, (ne + MF_SLABS - 1) / MF_SLABS);
    p->slab_e.clear();
    p->slab_n.clear();
    p->slab_e.push_back(0);
    p->slab_n.push_back(0);
    int64_t v = 0;
    for (int64_t e1 = chunk;; e1 += chunk) {
        const int64_t eb = std::min(e1, ne);
        while (v < nn && ready[v] < eb) ++v;
        p->slab_e.push_back(eb);
        p->slab_n.push_back(eb == ne ? nn : v);
        if (eb == ne) break;
    }
    return MF_OK;
}

// A thermal Q1 mesh whose elements are all translates: is it a lexicographic
// box of one rectangular cell?  Element 0's node offsets give the line
// lengths and the corner -> local index table, a device pass checks every
// element, and the reference entries (computed in FP64 from element 0) must
// depend on the pair of corners only through the axes in which they differ,
// to 1e-14 of the largest entry (true of a rectangular cell; the class
// values are those of corner 0 with corner mask).  Otherwise box stays zero.
mf_status detect_box(const mf_mesh *m, mf_pattern *p, cudaStream_t st)
{
    p->box[0] = p->box[1] = p->box[2] = 0;
    int32_t c0[8];
    MF_CUDA(cudaMemcpyAsync(c0, m->conn, sizeof c0, cudaMemcpyDeviceToHost, st));
    double kr[73 + 72];
    MF_CUDA(cudaMemcpyAsync(kr, p->kref, sizeof kr, cudaMemcpyDeviceToHost, st));
    MF_CUDA(cudaStreamSynchronize(st));
    int32_t lo = c0[0];
    for (int a = 1; a < 8; ++a) lo = std::min(lo, c0[a]);
    if (lo != 0) return MF_OK;
    int32_t srt[8];
    for (int a = 0; a < 8; ++a) srt[a] = c0[a];
    std::sort(srt, srt + 8);
    const int64_t nx1 = srt[2], S = srt[4];
    if (nx1 < 2 || S % nx1 != 0) return MF_OK;
    const int64_t want[8] = {0, 1, nx1, nx1 + 1, S, S + 1, S + nx1, S + nx1 + 1};
    for (int a = 0; a < 8; ++a)
        if (srt[a] != want[a]) return MF_OK;
    const int64_t ny1 = S / nx1;
    if (ny1 < 2 || m->n_nodes % S != 0) return MF_OK;
    const int64_t nz1 = m->n_nodes / S;
    if (nz1 < 2 || (nx1 - 1) * (ny1 - 1) * (nz1 - 1) != m->n_elems || m->n_nodes > INT32_MAX) return MF_OK;
    int corner[8];  // corner bits (x | y << 1 | z << 2) of local node a
    for (int a = 0; a < 8; ++a) {
        const int64_t o = c0[a];
        corner[a] = (int)(o % nx1) | (int)((o / nx1) % ny1) << 1 | (int)(o / S) << 2;
    }
    int loc_of[8];
    for (int a = 0; a < 8; ++a) loc_of[corner[a]] = a;
    // class constants and their check
    double kmax = 0.0, mmax = 0.0;
    for (int i = 0; i < 64; ++i) {
        kmax = std::max(kmax, std::fabs(kr[i]));
        mmax = std::max(mmax, std::fabs(kr[73 + i]));
    }
    mf_box_classes C{};
    for (int cm = 0; cm < 8; ++cm) {
        C.k_cls[cm] = kr[loc_of[0] * 8 + loc_of[cm]];
        C.m_cls[cm] = kr[73 + loc_of[0] * 8 + loc_of[cm]];
    }
    C.dref = kr[64 + loc_of[0]];
    for (int a = 0; a < 8; ++a) {
        if (std::fabs(kr[64 + a] - C.dref) > 1e-14 * std::fabs(C.dref)) return MF_OK;
        for (int b = 0; b < 8; ++b) {
            const int cm = corner[a] ^ corner[b];
            if (std::fabs(kr[a * 8 + b] - C.k_cls[cm]) > 1e-14 * kmax) return MF_OK;
            if (std::fabs(kr[73 + a * 8 + b] - C.m_cls[cm]) > 1e-14 * mmax) return MF_OK;
        }
    }
    int *bad = nullptr;
    MF_CUDA(cudaMallocAsync(&bad, sizeof(int), st));
    MF_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), st));
    k_box_check<<<nblk(m->n_elems), TPB, 0, st>>>(m->n_elems, m->conn, (int)(nx1 - 1), (int)(ny1 - 1), (int)nx1,
                                                  (int)ny1, make_int4(c0[0], c0[1], c0[2], c0[3]),
                                                  make_int4(c0[4], c0[5], c0[6], c0[7]), bad);
    int hbad = 1;
    MF_CUDA(cudaMemcpyAsync(&hbad, bad, sizeof hbad, cudaMemcpyDeviceToHost, st));
    MF_CUDA(cudaStreamSynchronize(st));
    MF_CUDA(cudaFreeAsync(bad, st));
    if (hbad) return MF_OK;
    p->box[0] = (int32_t)nx1;
    p->box[1] = (int32_t)ny1;
    p->box[2] = (int32_t)nz1;
    p->box_cls = C;
    return MF_OK;
}

void free_inc(Incidence &I, cudaStream_t st)
{
    if (I.ptr) cudaFreeAsync(I.ptr, st);
    if (I.inc) cudaFreeAsync(I.inc, st);
    if (I.loc) cudaFreeAsync(I.loc, st);
    I = Incidence();
}

}  // namespace

mf_status mf_mesh_validate(const mf_mesh *m, cudaStream_t st)
{
    int *status = mf_status_word();
    if (!status) return mf_fail(MF_ERR_CUDA, "mf_mesh_create: status word unavailable");
    MF_CUDA(cudaMemsetAsync(status, 0, sizeof(int), st));
    k_validate<<<nblk(m->n_elems), TPB, 0, st>>>(m->elem, m->n_elems, m->n_nodes, m->coords, m->conn,
                                                 m->n_pnodes, m->pconn, status);
    MF_CUDA(cudaGetLastError());
    int h = 0;
    MF_CUDA(cudaMemcpyAsync(&h, status, sizeof(int), cudaMemcpyDeviceToHost, st));
    MF_CUDA(cudaStreamSynchronize(st));
    if (h) {
        const int zero = 0;
        MF_CUDA(cudaMemcpyAsync(status, &zero, sizeof(int), cudaMemcpyHostToDevice, st));
        MF_CUDA(cudaStreamSynchronize(st));
        return mf_fail((mf_status)h, h == MF_ERR_BAD_MESH
                                         ? "mf_mesh_create: index out of range or detJ <= 0"
                                         : "mf_mesh_create: non-finite coordinates");
    }
    return MF_OK;
}

void mf_pattern_free(mf_pattern *p)
{
    if (p->side) cudaStreamSynchronize(p->side);
    for (cudaEvent_t ev : p->slab_ev)
        if (ev) cudaEventDestroy(ev);
    p->slab_ev.clear();
    if (p->fork_ev) cudaEventDestroy(p->fork_ev);
    if (p->join_ev) cudaEventDestroy(p->join_ev);
    if (p->side) cudaStreamDestroy(p->side);
    p->fork_ev = p->join_ev = nullptr;
    p->side = nullptr;
    if (p->clr_fork) cudaEventDestroy(p->clr_fork);
    if (p->clr_join) cudaEventDestroy(p->clr_join);
    if (p->clr_side) cudaStreamDestroy(p->clr_side);
    p->clr_fork = p->clr_join = nullptr;
    p->clr_side = nullptr;
    cudaFree(p->row_ptr);
    cudaFree(p->col_idx);
    cudaFree(p->q2s_map);
    p->q2s_map = nullptr;
    for (int i = 0; i < 4; ++i) {
        cudaFree(p->adj[i].ptr);
        cudaFree(p->adj[i].col);
        p->adj[i] = mf_adj();
    }
    cudaFree(p->scratch);
    cudaFree(p->inc_ptr);
    cudaFree(p->inc);
    cudaFree(p->inc_loc);
    p->inc_loc = nullptr;
    cudaFree(p->pinc_ptr);
    cudaFree(p->pinc);
    cudaFree(p->slot);
    cudaFree(p->kacc);
    cudaFree(p->tpos);
    cudaFree(p->etgt);
    p->etgt = nullptr;
    cudaFree(p->cbase);
    p->cbase = nullptr;
    p->n_upper = 0;
    cudaFree(p->dacc);
    p->dacc = nullptr;
    p->kacc = nullptr;
    p->tpos = nullptr;
    cudaFree(p->inc_slot);
    p->inc_slot = nullptr;
    cudaFree(p->inc_slot_pq);
    cudaFree(p->pinc_slot);
    cudaFree(p->pinc_slot_pp);
    p->pinc_slot_pp = nullptr;
    cudaFree(p->pinc_loc);
    p->inc_slot_pq = p->pinc_slot = p->pinc_loc = nullptr;
    cudaFree(p->elem_inc);
    p->elem_inc = nullptr;
    cudaFree(p->mixed_state);
    cudaFree(p->tr);
    cudaFree(p->kref);
    cudaFree(p->kref_df);
    cudaFree(p->kc_df);
    cudaFree(p->bcrow);
    p->tr = nullptr;
    p->kref = nullptr;
    p->kref_df = p->kc_df = nullptr;
    p->bcrow = nullptr;
    p->n_translate = 0;
    p->box[0] = p->box[1] = p->box[2] = 0;
    p->slot = nullptr;
    p->mixed_state = nullptr;
    p->pinc_ptr = nullptr;
    p->pinc = nullptr;
    p->row_ptr = nullptr;
    p->col_idx = nullptr;
    p->scratch = nullptr;
    p->inc_ptr = nullptr;
    p->inc = nullptr;
}

mf_status mf_pattern_build_impl(const mf_mesh *m, int form, cudaStream_t st, mf_pattern *p)
{
    int *status = mf_status_word();
    if (!status) return mf_fail(MF_ERR_CUDA, "mf_pattern_build: status word unavailable");
    MF_CUDA(cudaMemsetAsync(status, 0, sizeof(int), st));
    const int npe = m->npe;
    Incidence incv;
    mf_status s = build_incidence(m->n_nodes, m->n_elems, npe, m->conn, st, &incv, status);
    if (s == MF_OK) s = check_status(status, st, "mf_pattern_build");
    if (s != MF_OK) { free_inc(incv, st); return s; }
    s = build_adj(m->n_nodes, incv, m->conn, npe, m->conn, st, &p->adj[0], status);
    p->n_adj = 1;
    if (s != MF_OK) { free_inc(incv, st); return s; }

    if (form == MF_FORM_THERMAL) {
        p->n_rows = m->n_nodes;
        p->nnz = p->adj[0].n_pairs;
        MF_CUDA(cudaMallocAsync(&p->row_ptr, sizeof(int64_t) * (p->n_rows + 1), st));
        MF_CUDA(cudaMallocAsync(&p->col_idx, sizeof(int32_t) * p->nnz, st));
        k_csr_thermal<<<nblk(p->n_rows + 1), TPB, 0, st>>>(p->n_rows, p->adj[0].ptr, p->row_ptr);
        MF_CUDA(cudaMemcpyAsync(p->col_idx, p->adj[0].col, sizeof(int32_t) * p->nnz, cudaMemcpyDeviceToDevice, st));
        if ((int64_t)npe * m->n_elems >= INT32_MAX) {
            free_inc(incv, st);
            return mf_fail(MF_ERR_UNSUPPORTED, "mf_pattern_build: more than 2^31 element-node incidences");
        }
        MF_CUDA(cudaMallocAsync(&p->elem_inc, sizeof(int32_t) * npe * m->n_elems, st));
        k_elem_inc<<<nblk(m->n_nodes), TPB, 0, st>>>(m->n_nodes, npe, incv.ptr, incv.inc, incv.loc, p->elem_inc);
        MF_CUDA(cudaMallocAsync(&p->inc_slot, (size_t)npe * npe * m->n_elems, st));
        k_inc_slot<<<nblk(m->n_nodes), TPB, 0, st>>>(m->n_nodes, npe, m->conn, incv.ptr, incv.inc, p->adj[0].ptr,
                                                     p->adj[0].col, p->inc_slot);
        p->scratch_stride = (int64_t)npe * mf_th_rs(npe);
        if (m->elem == MF_P2_TRI || m->elem == MF_Q2S_HEX || m->elem == MF_P2_TET) {
            // reference sums of the P2 stiffnesses, reference table of the 20-node brick
            s = mf_flow_consts_upload();
            if (s != MF_OK) { free_inc(incv, st); return s; }
        }
        if (m->elem == MF_Q2S_HEX && m->n_elems > 0) {
            MF_CUDA(cudaMallocAsync(&p->q2s_map, sizeof(float2) * 24 * m->n_elems, st));
            k_q2s_map<<<nblk(24 * m->n_elems), TPB, 0, st>>>(m->n_elems, m->coords, m->conn, p->q2s_map);
        }
        if (m->elem == MF_Q1_HEX && m->n_elems > 0) {
            unsigned long long *cnt = nullptr;
            MF_CUDA(cudaMallocAsync(&p->tr, (size_t)m->n_elems, st));
            MF_CUDA(cudaMallocAsync(&cnt, sizeof(unsigned long long), st));
            MF_CUDA(cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), st));
            k_translate_flags<<<nblk(m->n_elems), TPB, 0, st>>>(m->n_elems, m->coords, m->conn, p->tr, cnt);
            unsigned long long h = 0;
            MF_CUDA(cudaMemcpyAsync(&h, cnt, sizeof h, cudaMemcpyDeviceToHost, st));
            MF_CUDA(cudaStreamSynchronize(st));
            MF_CUDA(cudaFreeAsync(cnt, st));
            p->n_translate = (int64_t)h;
            if (h == 0) {
                MF_CUDA(cudaFreeAsync(p->tr, st));
                p->tr = nullptr;
            } else {
                MF_CUDA(cudaMallocAsync(&p->kref, sizeof(double) * (73 + 72), st));
                k_kref<<<1, 1, 0, st>>>(m->coords, m->conn, p->kref, status);
                k_mark_translates<<<nblk(m->n_nodes), TPB, 0, st>>>(m->n_nodes, incv.ptr, incv.inc, p->tr, incv.loc);
                MF_CUDA(cudaMallocAsync(&p->kref_df, sizeof(float2) * (73 + 72), st));
                k_kref_df<<<1, 160, 0, st>>>(p->kref, p->kref_df);
                MF_CUDA(cudaMallocAsync(&p->kc_df, sizeof(float2) * m->n_elems, st));
                MF_CUDA(cudaMallocAsync(&p->bcrow, (size_t)m->n_nodes, st));
                if ((int64_t)h == m->n_elems) {
                    s = detect_box(m, p, st);
                    if (s != MF_OK) { free_inc(incv, st); return s; }
                }
            }
        }
    } else if (form == MF_FORM_ELASTIC && m->elem == MF_Q2S_HEX) {
        // node-interleaved dofs 3 n + c; element rows in the incidence layout
        // (row a of element e at incidence entry elem_inc[e * 20 + a], 183
        // values: 20 blocks of 3 x 3, then the load)
        p->n_rows = 3 * m->n_nodes;
        p->nnz = 9 * p->adj[0].n_pairs;
        if (p->nnz >= INT32_MAX || (int64_t)npe * m->n_elems >= INT32_MAX) {
            free_inc(incv, st);
            return mf_fail(MF_ERR_UNSUPPORTED, "mf_pattern_build: nnz or element-node incidences above 2^31");
        }
        MF_CUDA(cudaMallocAsync(&p->row_ptr, sizeof(int64_t) * (p->n_rows + 1), st));
        MF_CUDA(cudaMallocAsync(&p->col_idx, sizeof(int32_t) * p->nnz, st));
        k_csr_elastic<<<nblk(p->n_rows + 1), TPB, 0, st>>>(m->n_nodes, p->adj[0].ptr, p->adj[0].col, p->row_ptr,
                                                           p->col_idx);
        MF_CUDA(cudaMallocAsync(&p->elem_inc, sizeof(int32_t) * npe * m->n_elems, st));
        k_elem_inc<<<nblk(m->n_nodes), TPB, 0, st>>>(m->n_nodes, npe, incv.ptr, incv.inc, incv.loc, p->elem_inc);
        MF_CUDA(cudaMallocAsync(&p->inc_slot, (size_t)npe * npe * m->n_elems, st));
        k_inc_slot<<<nblk(m->n_nodes), TPB, 0, st>>>(m->n_nodes, npe, m->conn, incv.ptr, incv.inc, p->adj[0].ptr,
                                                     p->adj[0].col, p->inc_slot);
        p->scratch_stride = (int64_t)npe * (9 * npe + 3);
        s = read_max_deg(m->n_nodes, &p->adj[0], st);
        if (s != MF_OK) { free_inc(incv, st); return s; }
        s = mf_flow_consts_upload();  // reference table of the 20-node brick
        if (s != MF_OK) { free_inc(incv, st); return s; }
        if (m->n_elems > 0) {
            MF_CUDA(cudaMallocAsync(&p->q2s_map, sizeof(float2) * 24 * m->n_elems, st));
            k_q2s_map<<<nblk(24 * m->n_elems), TPB, 0, st>>>(m->n_elems, m->coords, m->conn, p->q2s_map);
        }
    } else if (form == MF_FORM_ELASTIC) {
        p->n_rows = 3 * m->n_nodes;
        p->nnz = 9 * p->adj[0].n_pairs;
        if (p->nnz >= INT32_MAX) { free_inc(incv, st); return mf_fail(MF_ERR_UNSUPPORTED, "nnz above 2^31"); }
        MF_CUDA(cudaMallocAsync(&p->row_ptr, sizeof(int64_t) * (p->n_rows + 1), st));
        MF_CUDA(cudaMallocAsync(&p->col_idx, sizeof(int32_t) * p->nnz, st));
        k_csr_elastic<<<nblk(p->n_rows + 1), TPB, 0, st>>>(m->n_nodes, p->adj[0].ptr, p->adj[0].col, p->row_ptr,
                                                           p->col_idx);
        MF_CUDA(cudaMallocAsync(&p->slot, (size_t)64 * m->n_elems, st));
        k_slot_map<<<nblk(m->n_elems * 64), TPB, 0, st>>>(m->n_elems, 8, m->conn, p->adj[0].ptr, p->adj[0].col,
                                                           p->slot);
        MF_CUDA(cudaMallocAsync(&p->mixed_state, 64, st));
        {
            // compact numbering of the upper node pairs (the accumulator's blocks)
            const int64_t nn = m->n_nodes;
            int64_t *cnt = nullptr;
            MF_CUDA(cudaMallocAsync(&cnt, sizeof(int64_t) * (nn + 1), st));
            MF_CUDA(cudaMallocAsync(&p->cbase, sizeof(int64_t) * (nn + 1), st));
            MF_CUDA(cudaMemsetAsync(cnt + nn, 0, sizeof(int64_t), st));
            k_upper_count<<<nblk(nn), TPB, 0, st>>>(nn, p->adj[0].ptr, p->adj[0].col, cnt, p->cbase);
            MF_CUDA(mf_scan_i64(cnt, nn + 1, nullptr, st));
            k_upper_base<<<nblk(nn), TPB, 0, st>>>(nn, cnt, p->cbase);
            s = read_i64(cnt + nn, &p->n_upper, st);
            MF_CUDA(cudaFreeAsync(cnt, st));
            if (s != MF_OK) { free_inc(incv, st); return s; }
        }
        s = read_max_deg(m->n_nodes, &p->adj[0], st);
        if (s != MF_OK) { free_inc(incv, st); return s; }
        MF_CUDA(cudaMallocAsync(&p->tpos, sizeof(int32_t) * p->adj[0].n_pairs, st));
        k_tpos<<<nblk(m->n_nodes), TPB, 0, st>>>(m->n_nodes, p->adj[0].ptr, p->adj[0].col, p->cbase, p->tpos);
        MF_CUDA(cudaMallocAsync(&p->etgt, sizeof(int32_t) * 36 * m->n_elems, st));
        k_mixed_etgt<<<nblk(36 * m->n_elems), TPB, 0, st>>>(m->n_elems, m->conn, p->cbase, p->slot, p->etgt);
        MF_CUDA(cudaMallocAsync(&p->kacc, sizeof(long long) * 9 * p->n_upper, st));
        MF_CUDA(cudaMallocAsync(&p->dacc, sizeof(long long) * 3 * m->n_nodes, st));
        // per node a flag set per assembly when one of its dofs or a
        // neighbour's is constrained (the mixed finishing tests the mask there only)
        MF_CUDA(cudaMallocAsync(&p->bcrow, (size_t)m->n_nodes, st));
        MF_CUDA(cudaStreamCreateWithFlags(&p->clr_side, cudaStreamNonBlocking));
        MF_CUDA(cudaEventCreateWithFlags(&p->clr_fork, cudaEventDisableTiming));
        MF_CUDA(cudaEventCreateWithFlags(&p->clr_join, cudaEventDisableTiming));
        p->scratch_stride = 36 * 9 + 24;
        mf_status ss = plan_slabs(m, incv, p->scratch_stride, st, p);
        if (ss != MF_OK) { free_inc(incv, st); return ss; }
        if (p->slab_e.size() > 2) {
            MF_CUDA(cudaStreamCreateWithFlags(&p->side, cudaStreamNonBlocking));
            MF_CUDA(cudaEventCreateWithFlags(&p->fork_ev, cudaEventDisableTiming));
            MF_CUDA(cudaEventCreateWithFlags(&p->join_ev, cudaEventDisableTiming));
            p->slab_ev.resize(p->slab_e.size() - 1, nullptr);
            for (cudaEvent_t &ev : p->slab_ev) MF_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        }
    } else {
        Incidence incp;
        s = build_incidence(m->n_pnodes, m->n_elems, 3, m->pconn, st, &incp, status);
        if (s == MF_OK)
            s = build_adj(m->n_nodes, incv, m->conn, 3, m->pconn, st, &p->adj[1], status);
        if (s == MF_OK)
            s = build_adj(m->n_pnodes, incp, m->pconn, 6, m->conn, st, &p->adj[2], status);
        const bool ns = form == MF_FORM_NS;
        if (s == MF_OK && ns)  // P1 rows x P1 columns: the SUPG pressure block
            s = build_adj(m->n_pnodes, incp, m->pconn, 3, m->pconn, st, &p->adj[3], status);
        p->pinc_ptr = incp.ptr;
        p->pinc = incp.inc;
        p->pinc_loc = incp.loc;
        p->n_adj = ns ? 4 : 3;
        if (s == MF_OK) {
            // slots: P2 rows x P2 columns, P2 rows x P1 columns, P1 rows x P2 columns
            MF_CUDA(cudaMallocAsync(&p->inc_slot, (size_t)36 * m->n_elems, st));
            MF_CUDA(cudaMallocAsync(&p->inc_slot_pq, (size_t)18 * m->n_elems, st));
            MF_CUDA(cudaMallocAsync(&p->pinc_slot, (size_t)18 * m->n_elems, st));
            k_inc_slot<<<nblk(m->n_nodes), TPB, 0, st>>>(m->n_nodes, 6, m->conn, incv.ptr, incv.inc, p->adj[0].ptr,
                                                         p->adj[0].col, p->inc_slot);
            k_inc_slot<<<nblk(m->n_nodes), TPB, 0, st>>>(m->n_nodes, 3, m->pconn, incv.ptr, incv.inc, p->adj[1].ptr,
                                                         p->adj[1].col, p->inc_slot_pq);
            k_inc_slot<<<nblk(m->n_pnodes), TPB, 0, st>>>(m->n_pnodes, 6, m->conn, incp.ptr, incp.inc,
                                                          p->adj[2].ptr, p->adj[2].col, p->pinc_slot);
            if (ns) {
                MF_CUDA(cudaMallocAsync(&p->pinc_slot_pp, (size_t)9 * m->n_elems, st));
                k_inc_slot<<<nblk(m->n_pnodes), TPB, 0, st>>>(m->n_pnodes, 3, m->pconn, incp.ptr, incp.inc,
                                                              p->adj[3].ptr, p->adj[3].col, p->pinc_slot_pp);
            }
        }
        if (s != MF_OK) { free_inc(incv, st); return s; }
        const int64_t n2 = m->n_nodes, n1 = m->n_pnodes;
        p->n_rows = 2 * n2 + n1;
        MF_CUDA(cudaMallocAsync(&p->row_ptr, sizeof(int64_t) * (p->n_rows + 1), st));
        MF_CUDA(cudaMemsetAsync(p->row_ptr, 0, sizeof(int64_t) * (p->n_rows + 1), st));
        if (ns)
            k_csr_ns_len<<<nblk(p->n_rows), TPB, 0, st>>>(n2, n1, p->adj[0].ptr, p->adj[1].ptr, p->adj[2].ptr,
                                                         p->adj[3].ptr, p->row_ptr);
        else
            k_csr_oseen_len<<<nblk(p->n_rows), TPB, 0, st>>>(n2, n1, p->adj[0].ptr, p->adj[1].ptr, p->adj[2].ptr,
                                                            p->row_ptr);
        MF_CUDA(mf_scan_i64(p->row_ptr, p->n_rows + 1, nullptr, st));
        s = read_i64(p->row_ptr + p->n_rows, &p->nnz, st);
        if (s != MF_OK) { free_inc(incv, st); return s; }
        MF_CUDA(cudaMallocAsync(&p->col_idx, sizeof(int32_t) * p->nnz, st));
        if (ns)
            k_csr_ns_fill<<<nblk(p->n_rows), TPB, 0, st>>>(n2, n1, p->adj[0].ptr, p->adj[0].col, p->adj[1].ptr,
                                                          p->adj[1].col, p->adj[2].ptr, p->adj[2].col, p->adj[3].ptr,
                                                          p->adj[3].col, p->row_ptr, p->col_idx);
        else
            k_csr_oseen_fill<<<nblk(p->n_rows), TPB, 0, st>>>(n2, n1, p->adj[0].ptr, p->adj[0].col, p->adj[1].ptr,
                                                             p->adj[1].col, p->adj[2].ptr, p->adj[2].col, p->row_ptr,
                                                             p->col_idx);
        // flow forms: per row a flag set per assembly when the row or one of
        // its columns is constrained (the gathers skip the Dirichlet tests elsewhere)
        MF_CUDA(cudaMallocAsync(&p->bcrow, (size_t)p->n_rows, st));
        // Navier-Stokes: residual (15) and tangent (15 x 15) per element
        p->scratch_stride = ns ? 240 : 72;
        s = mf_flow_consts_upload();
        if (s != MF_OK) { free_inc(incv, st); return s; }
    }
    MF_CUDA(cudaGetLastError());
    p->inc_ptr = incv.ptr;
    p->inc = incv.inc;
    p->inc_loc = incv.loc;
    MF_CUDA(cudaMallocAsync(&p->scratch, sizeof(double) * p->scratch_stride * m->n_elems, st));
    MF_CUDA(cudaStreamSynchronize(st));
    return check_status(status, st, "mf_pattern_build");
}
