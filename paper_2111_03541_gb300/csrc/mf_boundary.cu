// Boundary (facet) terms: a boundary condition is the domain physics one
// dimension lower (Sec. 2.2).  Convection h(T, T_env - T) (Sec. 4.1) adds a
// facet mass matrix to K and a load to d; the loaded boundary
// (d_i, sigma^l_ij n_j) (Sec. 4.2) adds a load to d.
//
// Layout.  A facet set keeps, for every node on some facet (ascending), its
// incident facets in ascending order with the node's index in each, and for
// the thermal form the position of every facet node in the node's CSR row.
// The assembly is node-centric like the domain gather: one thread per
// boundary node walks its facets in order and updates only its own row, so
// no atomics are needed and the bits do not depend on the schedule.  The
// facet geometry of every incidence entry is computed once, when the facet
// set is made (FP64 runs at 1/58 of the FP32 rate here, and the mesh does not
// move), so an assembly reads per entry a few cached doubles and the
// coefficients.
//
// Geometry.  Edges are straight: |J| = L, and the edge mass matrix and load
// are L times the closed-form reference integrals (P1: [[1/3, 1/6],
// [1/6, 1/3]], [1/2, 1/2]; P2: [[4, -1, 2], [-1, 4, 2], [2, 2, 16]] / 30,
// [1/6, 1/6, 2/3]), which the 2- and 3-point Gauss-Legendre rules integrate
// exactly.  A hexahedron face x(u, v) = c0 + c1 u + c2 v + c3 uv has the area
// vector A = x_u x x_v = c1 x c2 + (c1 x c3) u + (c3 x c2) v, linear in
// (u, v): the convection matrix takes |A| at the 2 x 2 Gauss points, and the
// traction's integral of N_m A is exact in closed form,
// int N_m A du dv = c1 x c2 + (c1 x c3) s_u / 3 + (c3 x c2) s_v / 3 for the
// node at (s_u, s_v).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "mf_internal.h"

namespace {

constexpr int TPB = 256;
constexpr int BND_T = 128;     // threads per block of the boundary kernels
constexpr int MAX_FINC = 32;   // facets incident to one node

inline unsigned nblk(int64_t n, int t = TPB) { return (unsigned)((n + t - 1) / t); }

// ---------------------------------------------------------------------------
// facet set construction
// ---------------------------------------------------------------------------

// Local element nodes of facet `face`; returns the node count or 0 for a face
// the element does not have.
__device__ __forceinline__ int facet_local(int elem, int face, int (&loc)[8])
{
    if (elem == MF_P2_TET) {
        // face i opposite vertex i, vertices ordered outward, then the
        // midpoints of its edges (0,1), (1,2), (2,0)
        if (face < 0 || face > 3) return 0;
        const int fl[4][6] = {{1, 2, 3, 5, 9, 8}, {0, 3, 2, 7, 9, 6}, {0, 1, 3, 4, 8, 7}, {0, 2, 1, 6, 5, 4}};
        for (int m = 0; m < 6; ++m) loc[m] = fl[face][m];
        return 6;
    }
    if (elem == MF_Q2S_QUAD) {
        // edges counter-clockwise: the two ends, then the midpoint (a straight
        // 3-node edge, integrated as a P2 triangle's)
        if (face < 0 || face > 3) return 0;
        const int el[4][3] = {{0, 1, 4}, {1, 3, 7}, {3, 2, 5}, {2, 0, 6}};
        for (int m = 0; m < 3; ++m) loc[m] = el[face][m];
        return 3;
    }
    if (elem == MF_Q1_HEX || elem == MF_Q2S_HEX) {
        if (face < 0 || face > 5) return 0;
        const int d = face >> 1, s = face & 1;
        int m = 0;
        for (int a = 0; a < 8; ++a)
            if (((a >> d) & 1) == s) loc[m++] = a;
        if (elem == MF_Q1_HEX) return 4;
        // 20-node brick: the vertices as above (face node i + 2j, i and j the
        // bits of the face axes d1 < d2), then the edge midpoints in the
        // 8-node quadrilateral's order: the d1 edges at bit d2 = j (4 + j) and
        // the d2 edges at bit d1 = i (6 + i); the brick's edge along axis A at
        // bits b, c of its other two axes B < C is node 8 + 4 A + b + 2 c
        const int d1 = d == 0 ? 1 : 0, d2 = d == 2 ? 1 : 2;
        for (int k = 0; k < 4; ++k) {
            const int A = k < 2 ? d1 : d2, other = k < 2 ? d2 : d1;
            int bits[3] = {0, 0, 0};
            bits[d] = s;
            bits[other] = k & 1;
            const int B = A == 0 ? 1 : 0, C = A == 2 ? 1 : 2;
            loc[4 + k] = 8 + 4 * A + bits[B] + 2 * bits[C];
        }
        return 8;
    }
    if (face < 0 || face > 2) return 0;
    loc[0] = face;
    loc[1] = face == 2 ? 0 : face + 1;
    loc[2] = 3 + face;  // P2 midpoint (unused for P1)
    return elem == MF_P2_TRI ? 3 : 2;
}

// Validates the facets, writes their global nodes and counts the facets of
// every node.
__global__ void k_facet_nodes(int elem, int npe, int npf, int64_t n_el, const int32_t *__restrict__ conn,
                              int64_t n_facets, const int32_t *__restrict__ f_elem,
                              const uint8_t *__restrict__ f_face, int32_t *__restrict__ fnode,
                              uint8_t *__restrict__ fface, int64_t *__restrict__ cnt, int *status)
{
    const int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= n_facets) return;
    const int64_t e = f_elem[f];
    const int face = f_face[f];
    int loc[8];
    if (e < 0 || e >= n_el || facet_local(elem, face, loc) != npf) {
        mf_dev_fail(status, MF_ERR_BAD_MESH);
        for (int m = 0; m < npf; ++m) fnode[f * npf + m] = -1;
        return;
    }
    fface[f] = (uint8_t)face;
    for (int m = 0; m < npf; ++m) {
        const int32_t v = conn[e * npe + loc[m]];
        fnode[f * npf + m] = v;
        atomicAdd(reinterpret_cast<unsigned long long *>(&cnt[v]), 1ull);
    }
}

__global__ void k_flag_nonzero(int64_t n, const int64_t *__restrict__ cnt, int64_t *__restrict__ flag)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) flag[i] = cnt[i] > 0 ? 1 : 0;
}

// boundary node list (ascending, from the scanned flags) and its facet counts
__global__ void k_compact_nodes(int64_t n, const int64_t *__restrict__ cnt, const int64_t *__restrict__ pos,
                                int32_t *__restrict__ bnode, int64_t *__restrict__ bcnt, int *status)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || cnt[i] == 0) return;
    if (cnt[i] > MAX_FINC) mf_dev_fail(status, MF_ERR_UNSUPPORTED);
    bnode[pos[i]] = (int32_t)i;
    bcnt[pos[i]] = cnt[i];
}

// incidence entries (facet * 8 + local index) in arrival order
__global__ void k_facet_fill(int64_t n_entries, int npf, const int32_t *__restrict__ fnode,
                             const int64_t *__restrict__ pos, const int64_t *__restrict__ bptr,
                             int64_t *__restrict__ cursor, int64_t *__restrict__ key)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_entries) return;
    const int64_t b = pos[fnode[t]];
    const int64_t at = bptr[b] + (int64_t)atomicAdd(reinterpret_cast<unsigned long long *>(&cursor[b]), 1ull);
    key[at] = (t / npf) * 8 + (t % npf);
}

// sorts every node's entries by facet (then local index) and splits the keys;
// the thermal form also looks up each facet node's slot in the node's row
__global__ void k_facet_sort_slots(int64_t n_bnodes, int npf, const int64_t *__restrict__ bptr,
                                   int64_t *__restrict__ key, const int32_t *__restrict__ bnode,
                                   const int32_t *__restrict__ fnode, const int64_t *__restrict__ row_ptr,
                                   const int32_t *__restrict__ col, int32_t *__restrict__ binc,
                                   uint8_t *__restrict__ bloc, uint8_t *__restrict__ bslot,
                                   int64_t *__restrict__ brow, int *status)
{
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= n_bnodes) return;
    const int64_t lo = bptr[b], hi = bptr[b + 1];
    if (hi - lo > MAX_FINC) return;  // reported by k_compact_nodes
    for (int64_t i = lo + 1; i < hi; ++i) {  // insertion sort of a short segment
        const int64_t x = key[i];
        int64_t j = i - 1;
        while (j >= lo && key[j] > x) { key[j + 1] = key[j]; --j; }
        key[j + 1] = x;
    }
    const int32_t r = bnode[b];
    if (brow) brow[b] = row_ptr[r];
    for (int64_t t = lo; t < hi; ++t) {
        const int64_t f = key[t] >> 3;
        binc[t] = (int32_t)f;
        bloc[t] = (uint8_t)(key[t] & 7);
        if (!bslot) continue;
        const int64_t r0 = row_ptr[r], r1 = row_ptr[r + 1];
        for (int m = 0; m < npf; ++m) {
            const int32_t c = fnode[f * npf + m];
            int64_t a = r0, z = r1;  // lower bound of c in the ascending row
            while (a < z) {
                const int64_t mid = (a + z) >> 1;
                if (col[mid] < c) a = mid + 1; else z = mid;
            }
            if (a == r1 || col[a] != c || a - r0 > 255) {
                mf_dev_fail(status, MF_ERR_BAD_MESH);
                bslot[t * npf + m] = 0;
            } else {
                bslot[t * npf + m] = (uint8_t)(a - r0);
            }
        }
    }
}

mf_status check_status(int *status, cudaStream_t st)
{
    int h = 0;
    MF_CUDA(cudaMemcpyAsync(&h, status, sizeof(int), cudaMemcpyDeviceToHost, st));
    MF_CUDA(cudaStreamSynchronize(st));
    if (!h) return MF_OK;
    const int zero = 0;
    MF_CUDA(cudaMemcpyAsync(status, &zero, sizeof(int), cudaMemcpyHostToDevice, st));
    MF_CUDA(cudaStreamSynchronize(st));
    if (h == MF_ERR_UNSUPPORTED)
        return mf_fail(MF_ERR_UNSUPPORTED, "mf_facets_create: more than %d facets at one node", MAX_FINC);
    return mf_fail((mf_status)h, "mf_facets_create: facet element or face out of range");
}

// ---------------------------------------------------------------------------
// boundary assembly
// ---------------------------------------------------------------------------

__device__ __forceinline__ void cross3(const double *a, const double *b, double *c)
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

// bilinear face coefficients c1, c2, c3 (x = c0 + c1 u + c2 v + c3 uv) of the
// facet's four nodes, node m at (u, v) = (2(m & 1) - 1, 2(m >> 1) - 1)
__device__ __forceinline__ void face_coefs(const double *__restrict__ X, const int32_t *fn, double (&c1)[3],
                                           double (&c2)[3], double (&c3)[3])
{
    double x[4][3];
    for (int m = 0; m < 4; ++m)
        for (int i = 0; i < 3; ++i) x[m][i] = X[3 * (int64_t)fn[m] + i];
    for (int i = 0; i < 3; ++i) {
        c1[i] = 0.25 * ((x[1][i] - x[0][i]) + (x[3][i] - x[2][i]));
        c2[i] = 0.25 * ((x[2][i] - x[0][i]) + (x[3][i] - x[1][i]));
        c3[i] = 0.25 * ((x[0][i] - x[1][i]) - (x[2][i] - x[3][i]));
    }
}

// Row m of the facet's convection matrix for unit h (row[m']) and the facet
// load factor for unit h T_env (returned).
template <int ELEM>
constexpr int facet_npf()
{
    return ELEM == MF_P1_TRI ? 2 : (ELEM == MF_P2_TRI ? 3 : (ELEM == MF_Q1_HEX ? 4 : (ELEM == MF_Q2S_HEX ? 8 : 6)));
}

// 8-node serendipity face basis on [-1, 1]^2: vertex m = i + 2 j at
// (2i - 1, 2j - 1): (1 + su u)(1 + sv v)(su u + sv v - 1) / 4; the
// midpoint 4 + j of the edge v = 2j - 1: (1 - u^2)(1 + sv v) / 2; the
// midpoint 6 + i of the edge u = 2i - 1: (1 + su u)(1 - v^2) / 2
__device__ __forceinline__ double quad8_shape(int m, double u, double v)
{
    if (m < 4) {
        const double su = (m & 1) ? 1.0 : -1.0, sv = (m & 2) ? 1.0 : -1.0;
        return 0.25 * (1.0 + su * u) * (1.0 + sv * v) * (su * u + sv * v - 1.0);
    }
    if (m < 6) return 0.5 * (1.0 - u * u) * (1.0 + (m == 5 ? v : -v));
    return 0.5 * (1.0 + (m == 7 ? u : -u)) * (1.0 - v * v);
}

// 3 x 3 Gauss on [-1, 1]: points -sqrt(3/5), 0, sqrt(3/5), weights 5/9, 8/9, 5/9
__device__ __forceinline__ double g3_x(int i) { return i == 0 ? -0.77459666924148337704 : (i == 1 ? 0.0 : 0.77459666924148337704); }
__device__ __forceinline__ double g3_w(int i) { return i == 1 ? 8.0 / 9.0 : 5.0 / 9.0; }

// An 8-node brick face (straight edges: the vertices' bilinear map, area
// vector A(u, v) = P + Qu u + Qv v) on the 3 x 3 rule: the unit-h
// convection row m (row[k] = int N_m N_k |A|, returned: int N_m |A|), or
// the area moment int N_m A (mom).
__device__ __forceinline__ double q2s_face_row(const double *__restrict__ X, const int32_t *fn, int m,
                                               double (&row)[8], double (&mom)[3])
{
    double c1[3], c2[3], c3[3], P[3], Qu[3], Qv[3];
    face_coefs(X, fn, c1, c2, c3);
    cross3(c1, c2, P);
    cross3(c1, c3, Qu);
    cross3(c3, c2, Qv);
    for (int k = 0; k < 8; ++k) row[k] = 0.0;
    mom[0] = mom[1] = mom[2] = 0.0;
    double load = 0.0;
    for (int qi = 0; qi < 3; ++qi)
        for (int qj = 0; qj < 3; ++qj) {
            const double u = g3_x(qi), v = g3_x(qj), w = g3_w(qi) * g3_w(qj);
            const double a0 = P[0] + Qu[0] * u + Qv[0] * v;
            const double a1 = P[1] + Qu[1] * u + Qv[1] * v;
            const double a2 = P[2] + Qu[2] * u + Qv[2] * v;
            const double nm = w * quad8_shape(m, u, v);
            mom[0] += nm * a0;
            mom[1] += nm * a1;
            mom[2] += nm * a2;
            const double jn = nm * sqrt(a0 * a0 + a1 * a1 + a2 * a2);
            load += jn;
            for (int k = 0; k < 8; ++k) row[k] += jn * quad8_shape(k, u, v);
        }
    return load;
}

template <int ELEM>
__device__ __forceinline__ double conv_row(const double *__restrict__ X, const int32_t *fn, int m, double (&row)[8])
{
    if (ELEM == MF_P2_TET) {
        // flat 6-node face of area A: int N_m N_k = A / 180 [6 -1 -1 0 -4 0; ...]
        // (the P2 triangle's closed form), int N_m = 0 (vertex), A / 3 (edge)
        double e1[3], e2[3], c[3];
        for (int i = 0; i < 3; ++i) {
            e1[i] = X[3 * (int64_t)fn[1] + i] - X[3 * (int64_t)fn[0] + i];
            e2[i] = X[3 * (int64_t)fn[2] + i] - X[3 * (int64_t)fn[0] + i];
        }
        cross3(e1, e2, c);
        const double A = 0.5 * sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
        const double s = A / 180.0;
        if (m < 3) {
            for (int k = 0; k < 3; ++k) row[k] = s * (k == m ? 6.0 : -1.0);
            for (int k = 3; k < 6; ++k) row[k] = 0.0;
            row[3 + (m + 1) % 3] = -4.0 * s;  // the edge opposite vertex m
            return 0.0;
        }
        for (int k = 0; k < 3; ++k) row[k] = 0.0;
        row[(m - 3 + 2) % 3] = -4.0 * s;  // the vertex opposite edge m - 3
        for (int k = 3; k < 6; ++k) row[k] = s * (k == m ? 32.0 : 16.0);
        return A / 3.0;
    }
    if (ELEM == MF_P1_TRI || ELEM == MF_P2_TRI) {
        const double ex = X[2 * (int64_t)fn[1]] - X[2 * (int64_t)fn[0]];
        const double ey = X[2 * (int64_t)fn[1] + 1] - X[2 * (int64_t)fn[0] + 1];
        const double L = sqrt(ex * ex + ey * ey);
        if (ELEM == MF_P1_TRI) {
            row[0] = L * (m == 0 ? 1.0 / 3.0 : 1.0 / 6.0);
            row[1] = L * (m == 1 ? 1.0 / 3.0 : 1.0 / 6.0);
            return 0.5 * L;
        }
        // (1/30) [[4, -1, 2], [-1, 4, 2], [2, 2, 16]], load (1/6, 1/6, 2/3)
        if (m == 2) {
            row[0] = row[1] = L * (1.0 / 15.0);
            row[2] = L * (8.0 / 15.0);
            return L * (2.0 / 3.0);
        }
        row[0] = L * (m == 0 ? 2.0 / 15.0 : -1.0 / 30.0);
        row[1] = L * (m == 1 ? 2.0 / 15.0 : -1.0 / 30.0);
        row[2] = L * (1.0 / 15.0);
        return L * (1.0 / 6.0);
    } else {
        double c1[3], c2[3], c3[3], P[3], Qu[3], Qv[3];
        face_coefs(X, fn, c1, c2, c3);
        cross3(c1, c2, P);
        cross3(c1, c3, Qu);
        cross3(c3, c2, Qv);
        const double g = 0.57735026918962576451;   // 1 / sqrt(3)
        const double al = 0.5 * (1.0 + g), be = 0.5 * (1.0 - g);  // 1D shape values at +-g
        for (int k = 0; k < 4; ++k) row[k] = 0.0;
        double load = 0.0;
        for (int q = 0; q < 4; ++q) {
            const double u = (q & 1) ? g : -g, v = (q & 2) ? g : -g;
            const double a0 = P[0] + Qu[0] * u + Qv[0] * v;
            const double a1 = P[1] + Qu[1] * u + Qv[1] * v;
            const double a2 = P[2] + Qu[2] * u + Qv[2] * v;
            const double J = sqrt(a0 * a0 + a1 * a1 + a2 * a2);
            // N_k(q) = n1(k & 1 vs q & 1) n1(k >> 1 vs q >> 1), n1 = al on the
            // node's own side of the point, be on the other
            const double nm = ((m & 1) == (q & 1) ? al : be) * ((m >> 1) == (q >> 1) ? al : be);
            const double jn = J * nm;
            load += jn;
            for (int k = 0; k < 4; ++k)
                row[k] += jn * (((k & 1) == (q & 1) ? al : be) * ((k >> 1) == (q >> 1) ? al : be));
        }
        return load;
    }
}

// Facet quadrature (the rule of the convection terms): number of points,
// weight of point q times |J| at it, and the facet shape value N_b(q).
// Edges: Gauss-Legendre on t in [0, 1] (2 points for P1, 3 for P2), |J| = L;
// hexahedron faces: 2 x 2 Gauss on [-1, 1]^2, |J| = |x_u x x_v|.
template <int ELEM>
constexpr int facet_nq() { return ELEM == MF_P1_TRI ? 2 : (ELEM == MF_P2_TRI ? 3 : 4); }

template <int ELEM>
__device__ __forceinline__ double facet_shape(int q, int b)
{
    if (ELEM == MF_P1_TRI) {
        const double t = q == 0 ? 0.5 - 0.5 * 0.57735026918962576451 : 0.5 + 0.5 * 0.57735026918962576451;
        return b == 0 ? 1.0 - t : t;
    } else if (ELEM == MF_P2_TRI) {
        const double g = 0.5 * 0.77459666924148337704;  // sqrt(3/5) / 2
        const double t = q == 0 ? 0.5 - g : (q == 1 ? 0.5 : 0.5 + g);
        return b == 0 ? (1.0 - t) * (1.0 - 2.0 * t) : (b == 1 ? t * (2.0 * t - 1.0) : 4.0 * t * (1.0 - t));
    } else {
        const double al = 0.5 * (1.0 + 0.57735026918962576451), be = 0.5 * (1.0 - 0.57735026918962576451);
        return ((b & 1) == (q & 1) ? al : be) * ((b >> 1) == (q >> 1) ? al : be);
    }
}

template <int ELEM>
__device__ __forceinline__ void facet_wj(const double *__restrict__ X, const int32_t *fn, double (&wj)[4])
{
    if (ELEM == MF_P1_TRI || ELEM == MF_P2_TRI) {
        const double ex = X[2 * (int64_t)fn[1]] - X[2 * (int64_t)fn[0]];
        const double ey = X[2 * (int64_t)fn[1] + 1] - X[2 * (int64_t)fn[0] + 1];
        const double L = sqrt(ex * ex + ey * ey);
        if (ELEM == MF_P1_TRI) {
            wj[0] = wj[1] = 0.5 * L;
        } else {
            wj[0] = wj[2] = L * (5.0 / 18.0);
            wj[1] = L * (8.0 / 18.0);
        }
    } else {
        double c1[3], c2[3], c3[3], P[3], Qu[3], Qv[3];
        face_coefs(X, fn, c1, c2, c3);
        cross3(c1, c2, P);
        cross3(c1, c3, Qu);
        cross3(c3, c2, Qv);
        const double g = 0.57735026918962576451;
        for (int q = 0; q < 4; ++q) {
            const double u = (q & 1) ? g : -g, v = (q & 2) ? g : -g;
            const double a0 = P[0] + Qu[0] * u + Qv[0] * v;
            const double a1 = P[1] + Qu[1] * u + Qv[1] * v;
            const double a2 = P[2] + Qu[2] * u + Qv[2] * v;
            wj[q] = sqrt(a0 * a0 + a1 * a1 + a2 * a2);
        }
    }
}

// Facet geometry of every incidence entry, once per facet set (the mesh's
// coordinates do not change while it lives).  Thermal: the entry's row of the
// unit-h convection matrix and its unit-h T_env load factor, (npf + 1)
// doubles, and the facet's nodes as the row's columns.  Elasticity: the
// oriented area moment o int N_m A du dv (3 doubles).
template <int ELEM>
__global__ void k_facet_geometry(int64_t n_entries, const int32_t *__restrict__ binc,
                                 const uint8_t *__restrict__ bloc, const int32_t *__restrict__ fnode,
                                 const uint8_t *__restrict__ fface, const double *__restrict__ X, bool traction,
                                 double *__restrict__ bgeo, int32_t *__restrict__ bcol, double *__restrict__ bwq)
{
    constexpr int NPF = facet_npf<ELEM>();
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_entries) return;
    const int32_t f = binc[t];
    const int m = bloc[t];
    const int32_t *fn = fnode + (int64_t)f * NPF;
    if (ELEM == MF_Q2S_HEX) {
        double row[8], mom[3];
        const double lf = q2s_face_row(X, fn, m, row, mom);
        if (traction) {
            const int face = fface[f];
            const double o = ((face & 1) ? 1.0 : -1.0) * ((face >> 1) == 1 ? -1.0 : 1.0);
            for (int i = 0; i < 3; ++i) bgeo[3 * t + i] = o * mom[i];
        } else {
            for (int k = 0; k < 8; ++k) {
                bgeo[t * 9 + k] = row[k];
                bcol[t * 8 + k] = fn[k];
            }
            bgeo[t * 9 + 8] = lf;
        }
        return;  // no radiation terms on the 8-node faces
    }
    if (ELEM == MF_Q1_HEX && traction) {
        double c1[3], c2[3], c3[3], P[3], Qu[3], Qv[3];
        face_coefs(X, fn, c1, c2, c3);
        cross3(c1, c2, P);
        cross3(c1, c3, Qu);
        cross3(c3, c2, Qv);
        // outward orientation: (2s - 1), negated for d = 1 (left-handed frame)
        const int face = fface[f];
        const double o = ((face & 1) ? 1.0 : -1.0) * ((face >> 1) == 1 ? -1.0 : 1.0);
        const double su = (m & 1) ? 1.0 / 3.0 : -1.0 / 3.0, sv = (m & 2) ? 1.0 / 3.0 : -1.0 / 3.0;
        for (int i = 0; i < 3; ++i) bgeo[3 * t + i] = o * (P[i] + Qu[i] * su + Qv[i] * sv);
        return;
    }
    double row[8];
    const double lf = conv_row<ELEM>(X, fn, m, row);
    for (int k = 0; k < NPF; ++k) {
        bgeo[t * (NPF + 1) + k] = row[k];
        bcol[t * NPF + k] = fn[k];
    }
    bgeo[t * (NPF + 1) + NPF] = lf;
    if (ELEM == MF_P2_TET) return;  // no radiation terms on tetrahedron faces
    // per point: w |J| N_m, for the temperature-dependent (radiation) terms
    constexpr int NQ = facet_nq<ELEM>();
    double wj[4];
    facet_wj<ELEM>(X, fn, wj);
    for (int q = 0; q < NQ; ++q) bwq[t * NQ + q] = wj[q] * facet_shape<ELEM>(q, m);
}

// Convection: one thread per boundary node adds, in ascending facet order,
// each facet's cached row times h to its own CSR row (or, in a Dirichlet
// column, moves the term to the right-hand side) and the facet's load to its
// own d entry.  Each K entry and each d entry has one writer.

template <int NPF>
__global__ void __launch_bounds__(BND_T) k_bnd_thermal(int64_t n_bnodes, const int32_t *__restrict__ bnode,
                                                       const int64_t *__restrict__ brow,
                                                       const int64_t *__restrict__ bptr,
                                                       const int32_t *__restrict__ binc,
                                                       const uint8_t *__restrict__ bslot,
                                                       const double *__restrict__ bgeo,
                                                       const int32_t *__restrict__ bcol,
                                                       const double *__restrict__ h, const double *__restrict__ tenv,
                                                       const uint8_t *__restrict__ mask,
                                                       const double *__restrict__ bval, double *values, double *d,
                                                       int *status)
{
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= n_bnodes) return;
    const int32_t r = bnode[b];
    if (mask && mask[r]) return;  // a Dirichlet row stays the identity
    double *vrow = values + brow[b];
    double dr = 0.0;
    const int64_t lo = bptr[b], hi = bptr[b + 1];
    for (int64_t t = lo; t < hi; ++t) {
        const int32_t f = binc[t];
        const double hf = h[f], tf = tenv[f];
        if (!isfinite(hf) || !isfinite(tf)) mf_dev_fail(status, MF_ERR_NONFINITE);
        const double *g = bgeo + t * (NPF + 1);
        dr += hf * tf * g[NPF];
        for (int k = 0; k < NPF; ++k) {
            const double v = hf * g[k];
            const int32_t c = bcol[t * NPF + k];
            if (mask && mask[c]) dr -= v * bval[c];
            else vrow[bslot[t * NPF + k]] += v;
        }
    }
    d[r] += dr;
}

// facets whose loads a traction thread issues together
constexpr int BU = 4;

// Loaded boundary: one thread per (boundary node, component i) adds
// sum_j sigma^l_ij a_j of the node's facets, in ascending facet order.
__global__ void __launch_bounds__(BND_T) k_bnd_traction(int64_t n_bnodes, const int32_t *__restrict__ bnode,
                                                        const int64_t *__restrict__ bptr,
                                                        const int32_t *__restrict__ binc,
                                                        const double *__restrict__ bgeo,
                                                        const double *__restrict__ stress,
                                                        const uint8_t *__restrict__ mask, double *d, int *status)
{
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= 3 * n_bnodes) return;
    const int64_t b = g / 3;
    const int i = (int)(g - 3 * b);
    const int64_t dof = 3 * (int64_t)bnode[b] + i;
    if (mask && mask[dof]) return;
    double acc = 0.0;
    bool finite = true;
    const int64_t t1 = bptr[b + 1];
    for (int64_t t = bptr[b]; t < t1; t += BU) {
        int32_t f[BU];
        double a[BU][3], sg[BU][3];
#pragma unroll
        for (int u = 0; u < BU; ++u) {
            f[u] = t + u < t1 ? binc[t + u] : -1;
            for (int j = 0; j < 3; ++j) a[u][j] = t + u < t1 ? bgeo[3 * (t + u) + j] : 0.0;
        }
#pragma unroll
        for (int u = 0; u < BU; ++u)
            for (int j = 0; j < 3; ++j) sg[u][j] = f[u] >= 0 ? stress[9 * (int64_t)f[u] + 3 * i + j] : 0.0;
#pragma unroll
        for (int u = 0; u < BU; ++u) {
            finite = finite && isfinite(sg[u][0]) && isfinite(sg[u][1]) && isfinite(sg[u][2]);
            acc += sg[u][0] * a[u][0] + sg[u][1] * a[u][1] + sg[u][2] * a[u][2];
        }
    }
    if (!finite) mf_dev_fail(status, MF_ERR_NONFINITE);
    d[dof] += acc;
}

// Radiation (Sec. 4.1, e_m sigma^b (T, T_env^4 - T^4)) at nodal temperatures
// T, one thread per boundary node, its facets in ascending order:
//   load     R[r] = sum_f es_f sum_q (w |J| N_m)(q) (T_env^4 - T_q^4),
//   tangent  K_rad[r][c] = sum_f 4 es_f sum_q (w |J| N_m)(q) N_b(q) T_q^3,
// T_q = sum_b N_b(q) T_b.  The load goes to R[r] (Dirichlet rows untouched);
// scale times the tangent is added to the node's own CSR row, except in
// Dirichlet rows and columns.
template <int ELEM>
__device__ __forceinline__ void facet_tq(const int32_t *fn, const double *__restrict__ T, double (&tq)[4])
{
    constexpr int NPF = ELEM == MF_P1_TRI ? 2 : (ELEM == MF_P2_TRI ? 3 : 4);
    double tb[NPF];
#pragma unroll
    for (int b = 0; b < NPF; ++b) tb[b] = T[fn[b]];
#pragma unroll
    for (int q = 0; q < facet_nq<ELEM>(); ++q) {
        double v = 0.0;
#pragma unroll
        for (int b = 0; b < NPF; ++b) v += facet_shape<ELEM>(q, b) * tb[b];
        tq[q] = v;
    }
}

template <int ELEM>
__global__ void __launch_bounds__(BND_T) k_rad_load(int64_t n_bnodes, const int32_t *__restrict__ bnode,
                                                    const int64_t *__restrict__ bptr,
                                                    const int32_t *__restrict__ binc,
                                                    const double *__restrict__ bwq,
                                                    const int32_t *__restrict__ fnode,
                                                    const double *__restrict__ es, const double *__restrict__ tenv,
                                                    const double *__restrict__ T, const uint8_t *__restrict__ mask,
                                                    double *__restrict__ R, int *status)
{
    constexpr int NPF = ELEM == MF_P1_TRI ? 2 : (ELEM == MF_P2_TRI ? 3 : 4), NQ = facet_nq<ELEM>();
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= n_bnodes) return;
    const int32_t r = bnode[b];
    if (mask && mask[r]) return;
    double acc = 0.0;
    for (int64_t t = bptr[b]; t < bptr[b + 1]; ++t) {
        const int32_t f = binc[t];
        const double ef = es[f], te = tenv[f];
        if (!isfinite(ef) || !isfinite(te)) mf_dev_fail(status, MF_ERR_NONFINITE);
        const double te4 = (te * te) * (te * te);
        double tq[4];
        facet_tq<ELEM>(fnode + (int64_t)f * NPF, T, tq);
        double s = 0.0;
#pragma unroll
        for (int q = 0; q < NQ; ++q) s += bwq[t * NQ + q] * (te4 - (tq[q] * tq[q]) * (tq[q] * tq[q]));
        acc += ef * s;
    }
    R[r] = acc;
}

template <int ELEM>
__global__ void __launch_bounds__(BND_T) k_rad_tangent(int64_t n_bnodes, const int32_t *__restrict__ bnode,
                                                       const int64_t *__restrict__ brow,
                                                       const int64_t *__restrict__ bptr,
                                                       const int32_t *__restrict__ binc,
                                                       const uint8_t *__restrict__ bslot,
                                                       const int32_t *__restrict__ bcol,
                                                       const double *__restrict__ bwq,
                                                       const int32_t *__restrict__ fnode,
                                                       const double *__restrict__ es, const double *__restrict__ T,
                                                       const uint8_t *__restrict__ mask, double scale,
                                                       double *__restrict__ values)
{
    constexpr int NPF = ELEM == MF_P1_TRI ? 2 : (ELEM == MF_P2_TRI ? 3 : 4), NQ = facet_nq<ELEM>();
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= n_bnodes) return;
    const int32_t r = bnode[b];
    if (mask && mask[r]) return;
    double *vrow = values + brow[b];
    for (int64_t t = bptr[b]; t < bptr[b + 1]; ++t) {
        const int32_t f = binc[t];
        const double ef4 = 4.0 * es[f] * scale;
        double tq[4];
        facet_tq<ELEM>(fnode + (int64_t)f * NPF, T, tq);
        double wt[NQ];
#pragma unroll
        for (int q = 0; q < NQ; ++q) wt[q] = bwq[t * NQ + q] * (tq[q] * tq[q] * tq[q]);
#pragma unroll
        for (int k = 0; k < NPF; ++k) {
            const int32_t c = bcol[t * NPF + k];
            if (mask && mask[c]) continue;
            double v = 0.0;
#pragma unroll
            for (int q = 0; q < NQ; ++q) v += wt[q] * facet_shape<ELEM>(q, k);
            vrow[bslot[t * NPF + k]] += ef4 * v;
        }
    }
}

}  // namespace

mf_status mf_radiation_load(const mf_facets *f, const double *es, const double *tenv, const double *T,
                            const uint8_t *mask, double *R, cudaStream_t st)
{
    if (!f || f->n_bnodes == 0) return MF_OK;
    if (f->mesh->elem == MF_P2_TET || f->mesh->elem == MF_Q2S_HEX)
        return mf_fail(MF_ERR_UNSUPPORTED, "radiation: not provided on tetrahedron and 8-node brick faces");
    int *status = mf_status_word();
    if (!status) return mf_fail(MF_ERR_CUDA, "radiation: status word unavailable");
    const unsigned g = nblk(f->n_bnodes, BND_T);
#define RL_ARGS f->n_bnodes, f->bnode, f->bptr, f->binc, f->bwq, f->fnode, es, tenv, T, mask, R, status
    if (f->mesh->elem == MF_P1_TRI) k_rad_load<MF_P1_TRI><<<g, BND_T, 0, st>>>(RL_ARGS);
    else if (f->mesh->elem == MF_P2_TRI || f->mesh->elem == MF_Q2S_QUAD) k_rad_load<MF_P2_TRI><<<g, BND_T, 0, st>>>(RL_ARGS);
    else k_rad_load<MF_Q1_HEX><<<g, BND_T, 0, st>>>(RL_ARGS);
#undef RL_ARGS
    return mf_cuda_check(cudaGetLastError(), "radiation load");
}

mf_status mf_radiation_tangent(const mf_facets *f, const double *es, const double *T, const uint8_t *mask,
                               double scale, double *values, cudaStream_t st)
{
    if (!f || f->n_bnodes == 0) return MF_OK;
    if (f->mesh->elem == MF_P2_TET || f->mesh->elem == MF_Q2S_HEX)
        return mf_fail(MF_ERR_UNSUPPORTED, "radiation: not provided on tetrahedron and 8-node brick faces");
    const unsigned g = nblk(f->n_bnodes, BND_T);
#define RT_ARGS f->n_bnodes, f->bnode, f->brow, f->bptr, f->binc, f->bslot, f->bcol, f->bwq, f->fnode, es, T, mask, \
                scale, values
    if (f->mesh->elem == MF_P1_TRI) k_rad_tangent<MF_P1_TRI><<<g, BND_T, 0, st>>>(RT_ARGS);
    else if (f->mesh->elem == MF_P2_TRI || f->mesh->elem == MF_Q2S_QUAD)
        k_rad_tangent<MF_P2_TRI><<<g, BND_T, 0, st>>>(RT_ARGS);
    else k_rad_tangent<MF_Q1_HEX><<<g, BND_T, 0, st>>>(RT_ARGS);
#undef RT_ARGS
    return mf_cuda_check(cudaGetLastError(), "radiation tangent");
}

mf_status mf_facets_create_impl(const mf_mesh *m, const mf_pattern *p, int64_t n_facets, const int32_t *elem,
                                const uint8_t *face, cudaStream_t st, mf_facets *f)
{
    f->npf = m->elem == MF_P1_TRI ? 2
           : ((m->elem == MF_P2_TRI || m->elem == MF_Q2S_QUAD) ? 3
           : (m->elem == MF_Q1_HEX ? 4 : (m->elem == MF_Q2S_HEX ? 8 : 6)));
    f->n_facets = n_facets;
    if (n_facets == 0) return MF_OK;
    if (p->form == MF_FORM_ELASTIC && m->elem != MF_Q1_HEX && m->elem != MF_Q2S_HEX)
        return mf_fail(MF_ERR_UNSUPPORTED, "mf_facets_create: loaded boundaries are provided on brick faces");
    int *status = mf_status_word();
    if (!status) return mf_fail(MF_ERR_CUDA, "mf_facets_create: status word unavailable");
    const int npf = f->npf;
    const int64_t nn = m->n_nodes, ne = n_facets * npf;
    int64_t *cnt = nullptr, *pos = nullptr, *key = nullptr, *bcnt = nullptr;
    auto cleanup = [&]() {
        cudaFreeAsync(cnt, st);
        cudaFreeAsync(pos, st);
        cudaFreeAsync(key, st);
        cudaFreeAsync(bcnt, st);
    };
    auto fail = [&](cudaError_t e, const char *what) {
        cleanup();
        return mf_cuda_check(e, what);
    };
#define FC(call)                                   \
    do {                                           \
        cudaError_t e_ = (call);                   \
        if (e_ != cudaSuccess) return fail(e_, #call); \
    } while (0)
    FC(cudaMemsetAsync(status, 0, sizeof(int), st));
    FC(cudaMallocAsync(&f->fnode, sizeof(int32_t) * ne, st));
    FC(cudaMallocAsync(&f->fface, (size_t)n_facets, st));
    FC(cudaMallocAsync(&cnt, sizeof(int64_t) * (nn + 1), st));
    FC(cudaMallocAsync(&pos, sizeof(int64_t) * (nn + 1), st));
    FC(cudaMemsetAsync(cnt, 0, sizeof(int64_t) * (nn + 1), st));
    k_facet_nodes<<<nblk(n_facets), TPB, 0, st>>>(m->elem, m->npe, npf, m->n_elems, m->conn, n_facets, elem, face,
                                                 f->fnode, f->fface, cnt, status);
    FC(cudaGetLastError());
    {
        mf_status s = check_status(status, st);
        if (s != MF_OK) {
            cleanup();
            return s;
        }
    }
    k_flag_nonzero<<<nblk(nn + 1), TPB, 0, st>>>(nn + 1, cnt, pos);
    FC(cudaGetLastError());
    FC(mf_scan_i64(pos, nn + 1, nullptr, st));
    int64_t nb = 0;
    FC(cudaMemcpyAsync(&nb, pos + nn, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    FC(cudaStreamSynchronize(st));
    f->n_bnodes = nb;
    FC(cudaMallocAsync(&f->bnode, sizeof(int32_t) * nb, st));
    FC(cudaMallocAsync(&f->bptr, sizeof(int64_t) * (nb + 1), st));
    FC(cudaMallocAsync(&bcnt, sizeof(int64_t) * (nb + 1), st));
    FC(cudaMemsetAsync(bcnt, 0, sizeof(int64_t) * (nb + 1), st));
    k_compact_nodes<<<nblk(nn), TPB, 0, st>>>(nn, cnt, pos, f->bnode, bcnt, status);
    FC(cudaGetLastError());
    FC(mf_scan_i64(bcnt, nb + 1, nullptr, st));
    FC(cudaMemcpyAsync(f->bptr, bcnt, sizeof(int64_t) * (nb + 1), cudaMemcpyDeviceToDevice, st));
    FC(cudaMemsetAsync(bcnt, 0, sizeof(int64_t) * (nb + 1), st));  // now the fill cursors
    FC(cudaMallocAsync(&key, sizeof(int64_t) * ne, st));
    FC(cudaMallocAsync(&f->binc, sizeof(int32_t) * ne, st));
    FC(cudaMallocAsync(&f->bloc, (size_t)ne, st));
    const bool thermal = p->form == MF_FORM_THERMAL;
    if (thermal) {
        FC(cudaMallocAsync(&f->bslot, (size_t)ne * npf, st));
        FC(cudaMallocAsync(&f->bcol, sizeof(int32_t) * ne * npf, st));
        FC(cudaMallocAsync(&f->brow, sizeof(int64_t) * nb, st));
        FC(cudaMallocAsync(&f->bgeo, sizeof(double) * ne * (npf + 1), st));
        if (npf <= 4)  // radiation point weights (none on tetrahedron faces)
            FC(cudaMallocAsync(&f->bwq, sizeof(double) * ne * (npf == 3 ? 3 : (npf == 2 ? 2 : 4)), st));
    } else {
        FC(cudaMallocAsync(&f->bgeo, sizeof(double) * ne * 3, st));
    }
    k_facet_fill<<<nblk(ne), TPB, 0, st>>>(ne, npf, f->fnode, pos, f->bptr, bcnt, key);
    FC(cudaGetLastError());
    k_facet_sort_slots<<<nblk(nb), TPB, 0, st>>>(nb, npf, f->bptr, key, f->bnode, f->fnode, p->row_ptr,
                                                 p->col_idx, f->binc, f->bloc, f->bslot, f->brow, status);
    FC(cudaGetLastError());
    {
        // the incidence must be complete before anything follows it
        mf_status s = check_status(status, st);
        if (s != MF_OK) {
            cleanup();
            return s;
        }
    }
    if (m->elem == MF_P1_TRI)
        k_facet_geometry<MF_P1_TRI><<<nblk(ne), TPB, 0, st>>>(ne, f->binc, f->bloc, f->fnode, f->fface, m->coords,
                                                              false, f->bgeo, f->bcol, f->bwq);
    else if (m->elem == MF_P2_TRI || m->elem == MF_Q2S_QUAD)  // straight 3-node edges
        k_facet_geometry<MF_P2_TRI><<<nblk(ne), TPB, 0, st>>>(ne, f->binc, f->bloc, f->fnode, f->fface, m->coords,
                                                              false, f->bgeo, f->bcol, f->bwq);
    else if (m->elem == MF_P2_TET)
        k_facet_geometry<MF_P2_TET><<<nblk(ne), TPB, 0, st>>>(ne, f->binc, f->bloc, f->fnode, f->fface, m->coords,
                                                              false, f->bgeo, f->bcol, f->bwq);
    else if (m->elem == MF_Q2S_HEX)
        k_facet_geometry<MF_Q2S_HEX><<<nblk(ne), TPB, 0, st>>>(ne, f->binc, f->bloc, f->fnode, f->fface, m->coords,
                                                               !thermal, f->bgeo, f->bcol, f->bwq);
    else
        k_facet_geometry<MF_Q1_HEX><<<nblk(ne), TPB, 0, st>>>(ne, f->binc, f->bloc, f->fnode, f->fface, m->coords,
                                                              !thermal, f->bgeo, f->bcol, f->bwq);
    FC(cudaGetLastError());
#undef FC
    mf_status s = check_status(status, st);
    cleanup();
    if (s == MF_OK) s = mf_cuda_check(cudaStreamSynchronize(st), "mf_facets_create");
    return s;
}

void mf_facets_free(mf_facets *f)
{
    cudaFree(f->fnode);
    cudaFree(f->fface);
    cudaFree(f->bnode);
    cudaFree(f->bptr);
    cudaFree(f->binc);
    cudaFree(f->bloc);
    cudaFree(f->bslot);
    cudaFree(f->bcol);
    cudaFree(f->brow);
    cudaFree(f->bgeo);
    cudaFree(f->bwq);
    f->bwq = nullptr;
    f->fnode = f->bnode = f->binc = f->bcol = nullptr;
    f->fface = f->bloc = f->bslot = nullptr;
    f->bptr = f->brow = nullptr;
    f->bgeo = nullptr;
}

mf_status mf_assemble_boundary_impl(const mf_facets *f, const mf_facet_coeffs *c, double *values, double *d,
                                    cudaStream_t st)
{
    if (f->n_bnodes == 0) return MF_OK;
    int *status = mf_status_word();
    if (!status) return mf_fail(MF_ERR_CUDA, "mf_assemble_boundary: status word unavailable");
    const mf_mesh *m = f->mesh;
    const mf_pattern *p = f->pattern;
    if (p->form == MF_FORM_THERMAL) {
        mf_prof_begin("bnd_thermal", st);
        const unsigned g = nblk(f->n_bnodes, BND_T);
#define BND_ARGS f->n_bnodes, f->bnode, f->brow, f->bptr, f->binc, f->bslot, f->bgeo, f->bcol, c->h, c->t_env, \
                 c->bc_mask, c->bc_val, values, d, status
        if (m->elem == MF_P1_TRI) k_bnd_thermal<2><<<g, BND_T, 0, st>>>(BND_ARGS);
        else if (m->elem == MF_P2_TRI || m->elem == MF_Q2S_QUAD) k_bnd_thermal<3><<<g, BND_T, 0, st>>>(BND_ARGS);
        else if (m->elem == MF_P2_TET) k_bnd_thermal<6><<<g, BND_T, 0, st>>>(BND_ARGS);
        else if (m->elem == MF_Q2S_HEX) k_bnd_thermal<8><<<g, BND_T, 0, st>>>(BND_ARGS);
        else k_bnd_thermal<4><<<g, BND_T, 0, st>>>(BND_ARGS);
#undef BND_ARGS
        mf_prof_end(st);
    } else {
        mf_prof_begin("bnd_traction", st);
        k_bnd_traction<<<nblk(3 * f->n_bnodes, BND_T), BND_T, 0, st>>>(f->n_bnodes, f->bnode, f->bptr, f->binc,
                                                                        f->bgeo, c->stress, c->bc_mask, d, status);
        mf_prof_end(st);
    }
    return mf_cuda_check(cudaGetLastError(), "mf_assemble_boundary");
}
