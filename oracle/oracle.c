/*
 * CPU FP64 oracle for the FEM assembly + Krylov hot path of MetaFEM
 * (Xie, Ehmann, Cao, "MetaFEM: A Generic FEM Solver By Meta-expressions",
 * arXiv 2111.03541).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark load this file.  The product library never
 * links, calls or includes it, and it includes nothing of the product.
 *
 * Plain, slow, obviously correct: every routine is the definition written out
 * as nested loops in the order of the paper's sums, double precision
 * throughout, single threaded.  No blocking, no fusion, no reordering.
 *
 * Sign convention: the paper writes the residual of conduction and elasticity
 * with a minus on the stiffness term (Sec. 4.1, Sec. 4.2), so its tangent
 * dd/dphi (Eq. "stiffness", Sec. 2.1) is the negative of the positive matrix
 * returned here; the linear system K x = d is the same after multiplying both
 * sides by -1.  The flow form of Sec. 4.3 carries +mu(u_ij, u_ij) and is taken
 * with the paper's own signs.
 *
 * Pins: every routine here is checked by tests/test_oracle_pins.py against
 * closed forms, exact rational integration, invariants and dense solves.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* element kinds */
enum { OR_P1 = 0, OR_P2 = 1, OR_Q1 = 2, OR_Q2S = 3, OR_P2T = 4, OR_Q2Q = 5 };
/* quadrature kinds */
enum { OR_QTRI3 = 0, OR_QTRI6 = 1, OR_QHEX8 = 2, OR_QHEX27 = 3, OR_QTET64 = 4, OR_QQUAD9 = 5, OR_QTRI16 = 6, OR_QTET125 = 7 };
/* forms */
enum { OR_THERMAL = 0, OR_ELASTIC = 1, OR_OSEEN = 2, OR_CAPACITY = 3 };

/* ------------------------------------------------------------------------ */
/* Quadrature (Sec. 2.1: each bilinear form is approximated by a weighted     */
/* sum over integration points w_gamma, x_gamma).                            */
/* Triangle points are (xi, eta) = (lambda_1, lambda_2) on the reference     */
/* triangle (0,0),(1,0),(0,1) with weights summing to its area 1/2; hex      */
/* points live on [-1,1]^3 with weights summing to 8.                        */
/* ------------------------------------------------------------------------ */
int or_quad(int kind, double *pts, double *w)
{
    if (kind == OR_QTRI3) {
        /* interior 3-point rule, degree 2: barycentric (2/3,1/6,1/6) and permutations */
        const double bary[3][3] = {{2.0 / 3.0, 1.0 / 6.0, 1.0 / 6.0},
                                   {1.0 / 6.0, 2.0 / 3.0, 1.0 / 6.0},
                                   {1.0 / 6.0, 1.0 / 6.0, 2.0 / 3.0}};
        for (int q = 0; q < 3; ++q) {
            pts[2 * q + 0] = bary[q][1];
            pts[2 * q + 1] = bary[q][2];
            w[q] = 0.5 / 3.0;
        }
        return 3;
    }
    if (kind == OR_QTRI6) {
        /* symmetric 6-point rule, degree 4 (Strang-Fix / Dunavant): two orbits
         * (a, a, 1-2a) with the closed-form roots of its moment equations. */
        const double s10 = sqrt(10.0);
        const double r = sqrt(38.0 - 44.0 * sqrt(2.0 / 5.0));
        const double a1 = (8.0 - s10 + r) / 18.0;
        const double a2 = (8.0 - s10 - r) / 18.0;
        const double t = sqrt(213125.0 - 53320.0 * s10);
        const double w1 = (620.0 + t) / 3720.0; /* weights normalised to area 1 */
        const double w2 = (620.0 - t) / 3720.0;
        const double orb[2] = {a1, a2};
        const double wo[2] = {w1, w2};
        int q = 0;
        for (int o = 0; o < 2; ++o) {
            const double a = orb[o], b = 1.0 - 2.0 * a;
            const double bary[3][3] = {{b, a, a}, {a, b, a}, {a, a, b}};
            for (int p = 0; p < 3; ++p, ++q) {
                pts[2 * q + 0] = bary[p][1];
                pts[2 * q + 1] = bary[p][2];
                w[q] = 0.5 * wo[o];
            }
        }
        return 6;
    }
    if (kind == OR_QTET64) {
        /* reference tetrahedron x, y, z >= 0, x + y + z <= 1 (volume 1/6) as
         * the image of the unit cube under x = s, y = t (1 - s),
         * z = r (1 - s)(1 - t) (Jacobian (1 - s)^2 (1 - t)), with 4-point
         * Gauss-Legendre in s, t and r: a polynomial of total degree d becomes
         * one of degree d + 2, d + 1, d in s, t, r, so the rule is exact to
         * degree 5.  Point q = i + 4 j + 16 k. */
        const double a = sqrt(3.0 / 7.0 - 2.0 / 7.0 * sqrt(6.0 / 5.0));
        const double b = sqrt(3.0 / 7.0 + 2.0 / 7.0 * sqrt(6.0 / 5.0));
        const double wa = (18.0 + sqrt(30.0)) / 36.0, wb = (18.0 - sqrt(30.0)) / 36.0;
        const double x4[4] = {-b, -a, a, b}, w4[4] = {wb, wa, wa, wb};
        for (int q = 0; q < 64; ++q) {
            const int i = q % 4, j = (q / 4) % 4, k = q / 16;
            const double S = 0.5 * (x4[i] + 1.0), T = 0.5 * (x4[j] + 1.0), R = 0.5 * (x4[k] + 1.0);
            pts[3 * q + 0] = S;
            pts[3 * q + 1] = T * (1.0 - S);
            pts[3 * q + 2] = R * (1.0 - S) * (1.0 - T);
            w[q] = 0.125 * w4[i] * w4[j] * w4[k] * (1.0 - S) * (1.0 - S) * (1.0 - T);
        }
        return 64;
    }
    if (kind == OR_QTET125) {
        /* the collapsed map of OR_QTET64 with 5-point Gauss-Legendre (0,
         * +-sqrt(5 -+ 2 sqrt(10/7)) / 3): exact to total degree 7.
         * Point q = i + 5 j + 25 k. */
        const double a = sqrt(5.0 - 2.0 * sqrt(10.0 / 7.0)) / 3.0, b = sqrt(5.0 + 2.0 * sqrt(10.0 / 7.0)) / 3.0;
        const double wa = (322.0 + 13.0 * sqrt(70.0)) / 900.0, wb = (322.0 - 13.0 * sqrt(70.0)) / 900.0;
        const double x5[5] = {-b, -a, 0.0, a, b}, w5[5] = {wb, wa, 128.0 / 225.0, wa, wb};
        for (int q = 0; q < 125; ++q) {
            const int i = q % 5, j = (q / 5) % 5, k = q / 25;
            const double S = 0.5 * (x5[i] + 1.0), T = 0.5 * (x5[j] + 1.0), R = 0.5 * (x5[k] + 1.0);
            pts[3 * q + 0] = S;
            pts[3 * q + 1] = T * (1.0 - S);
            pts[3 * q + 2] = R * (1.0 - S) * (1.0 - T);
            w[q] = 0.125 * w5[i] * w5[j] * w5[k] * (1.0 - S) * (1.0 - S) * (1.0 - T);
        }
        return 125;
    }
    if (kind == OR_QTRI16) {
        /* reference triangle as the image of the unit square under x = s,
         * y = t (1 - s) (Jacobian 1 - s), 4-point Gauss-Legendre in s and t:
         * exact to total degree 6.  Point q = i + 4 j. */
        const double a = sqrt(3.0 / 7.0 - 2.0 / 7.0 * sqrt(6.0 / 5.0));
        const double b = sqrt(3.0 / 7.0 + 2.0 / 7.0 * sqrt(6.0 / 5.0));
        const double wa = (18.0 + sqrt(30.0)) / 36.0, wb = (18.0 - sqrt(30.0)) / 36.0;
        const double x4[4] = {-b, -a, a, b}, w4[4] = {wb, wa, wa, wb};
        for (int q = 0; q < 16; ++q) {
            const double S = 0.5 * (x4[q % 4] + 1.0), T = 0.5 * (x4[q / 4] + 1.0);
            pts[2 * q + 0] = S;
            pts[2 * q + 1] = T * (1.0 - S);
            w[q] = 0.25 * w4[q % 4] * w4[q / 4] * (1.0 - S);
        }
        return 16;
    }
    if (kind == OR_QQUAD9) {
        /* [-1, 1]^2, 3 x 3 Gauss-Legendre (0, +-sqrt(3/5); 8/9, 5/9), q = i + 3 j */
        const double g = sqrt(0.6);
        const double p1[3] = {-g, 0.0, g}, w1[3] = {5.0 / 9.0, 8.0 / 9.0, 5.0 / 9.0};
        for (int q = 0; q < 9; ++q) {
            pts[2 * q + 0] = p1[q % 3];
            pts[2 * q + 1] = p1[q / 3];
            w[q] = w1[q % 3] * w1[q / 3];
        }
        return 9;
    }
    if (kind == OR_QHEX27) {
        /* tensor Gauss-Legendre, 3 points per direction at 0, +-sqrt(3/5),
         * weights 8/9, 5/9; point q = i + 3 j + 9 k */
        const double g = sqrt(0.6);
        const double p1[3] = {-g, 0.0, g}, w1[3] = {5.0 / 9.0, 8.0 / 9.0, 5.0 / 9.0};
        for (int q = 0; q < 27; ++q) {
            const int i = q % 3, j = (q / 3) % 3, k = q / 9;
            pts[3 * q + 0] = p1[i];
            pts[3 * q + 1] = p1[j];
            pts[3 * q + 2] = p1[k];
            w[q] = w1[i] * w1[j] * w1[k];
        }
        return 27;
    }
    if (kind == OR_QHEX8) {
        /* tensor Gauss-Legendre, 2 points per direction at +-1/sqrt(3), weight 1 */
        const double g = 1.0 / sqrt(3.0);
        for (int q = 0; q < 8; ++q) {
            pts[3 * q + 0] = (q & 1) ? g : -g;
            pts[3 * q + 1] = (q & 2) ? g : -g;
            pts[3 * q + 2] = (q & 4) ? g : -g;
            w[q] = 1.0;
        }
        return 8;
    }
    return -1;
}

/* ------------------------------------------------------------------------ */
/* Shape functions N_alpha and reference derivatives dN/dxi (Sec. 2.1:      */
/* interpolation functions; Sec. 4: Lagrange simplex and cube elements).   */
/* dN[a*dim + j] = dN_a / dxi_j.                                             */
/* ------------------------------------------------------------------------ */
int or_shape(int elem, const double *xi, double *N, double *dN)
{
    if (elem == OR_P1) {
        const double l1 = xi[0], l2 = xi[1], l0 = 1.0 - l1 - l2;
        N[0] = l0; N[1] = l1; N[2] = l2;
        dN[0] = -1.0; dN[1] = -1.0;
        dN[2] = 1.0;  dN[3] = 0.0;
        dN[4] = 0.0;  dN[5] = 1.0;
        return 3;
    }
    if (elem == OR_P2) {
        const double l1 = xi[0], l2 = xi[1], l0 = 1.0 - l1 - l2;
        /* d lambda_k / d xi_j */
        const double dl[3][2] = {{-1.0, -1.0}, {1.0, 0.0}, {0.0, 1.0}};
        const double l[3] = {l0, l1, l2};
        /* vertices: lambda_i (2 lambda_i - 1) */
        for (int i = 0; i < 3; ++i) {
            N[i] = l[i] * (2.0 * l[i] - 1.0);
            for (int j = 0; j < 2; ++j) dN[2 * i + j] = (4.0 * l[i] - 1.0) * dl[i][j];
        }
        /* edge midpoints (0,1), (1,2), (2,0): 4 lambda_p lambda_q */
        const int ep[3][2] = {{0, 1}, {1, 2}, {2, 0}};
        for (int e = 0; e < 3; ++e) {
            const int p = ep[e][0], q = ep[e][1];
            N[3 + e] = 4.0 * l[p] * l[q];
            for (int j = 0; j < 2; ++j)
                dN[2 * (3 + e) + j] = 4.0 * (dl[p][j] * l[q] + l[p] * dl[q][j]);
        }
        return 6;
    }
    if (elem == OR_Q1) {
        /* trilinear: node a = i + 2j + 4k at (2i-1, 2j-1, 2k-1) */
        for (int a = 0; a < 8; ++a) {
            const double sa = (a & 1) ? 1.0 : -1.0;
            const double ta = (a & 2) ? 1.0 : -1.0;
            const double ua = (a & 4) ? 1.0 : -1.0;
            const double fx = 1.0 + sa * xi[0], fy = 1.0 + ta * xi[1], fz = 1.0 + ua * xi[2];
            N[a] = 0.125 * fx * fy * fz;
            dN[3 * a + 0] = 0.125 * sa * fy * fz;
            dN[3 * a + 1] = 0.125 * fx * ta * fz;
            dN[3 * a + 2] = 0.125 * fx * fy * ua;
        }
        return 8;
    }
    if (elem == OR_Q2Q) {
        /* 8-node serendipity quadrilateral on [-1, 1]^2.  Vertex a = i + 2j at
         * (xa, ya) = (2i-1, 2j-1): N = (1 + x xa)(1 + y ya)(x xa + y ya - 1) / 4;
         * x edges (at y = ya) 4 + j: N = (1 - x^2)(1 + y ya) / 2;
         * y edges (at x = xa) 6 + i: N = (1 - y^2)(1 + x xa) / 2. */
        const double x = xi[0], y = xi[1];
        for (int a = 0; a < 4; ++a) {
            const double xa = (a & 1) ? 1.0 : -1.0, ya = (a & 2) ? 1.0 : -1.0;
            const double A = 1.0 + x * xa, B = 1.0 + y * ya;
            N[a] = 0.25 * A * B * (x * xa + y * ya - 1.0);
            dN[2 * a + 0] = 0.25 * xa * B * (2.0 * x * xa + y * ya);
            dN[2 * a + 1] = 0.25 * ya * A * (x * xa + 2.0 * y * ya);
        }
        for (int j = 0; j < 2; ++j) {
            const double ya = j ? 1.0 : -1.0;
            N[4 + j] = 0.5 * (1.0 - x * x) * (1.0 + y * ya);
            dN[2 * (4 + j) + 0] = -x * (1.0 + y * ya);
            dN[2 * (4 + j) + 1] = 0.5 * ya * (1.0 - x * x);
        }
        for (int i = 0; i < 2; ++i) {
            const double xa = i ? 1.0 : -1.0;
            N[6 + i] = 0.5 * (1.0 - y * y) * (1.0 + x * xa);
            dN[2 * (6 + i) + 0] = 0.5 * xa * (1.0 - y * y);
            dN[2 * (6 + i) + 1] = -y * (1.0 + x * xa);
        }
        return 8;
    }
    if (elem == OR_P2T) {
        /* 10-node tetrahedron: lambda = (1 - x - y - z, x, y, z); vertices
         * lambda_i (2 lambda_i - 1), then the edges (0,1), (1,2), (2,0),
         * (0,3), (1,3), (2,3): 4 lambda_p lambda_q */
        const double l[4] = {1.0 - xi[0] - xi[1] - xi[2], xi[0], xi[1], xi[2]};
        const double dl[4][3] = {{-1.0, -1.0, -1.0}, {1.0, 0.0, 0.0}, {0.0, 1.0, 0.0}, {0.0, 0.0, 1.0}};
        for (int i = 0; i < 4; ++i) {
            N[i] = l[i] * (2.0 * l[i] - 1.0);
            for (int j = 0; j < 3; ++j) dN[3 * i + j] = (4.0 * l[i] - 1.0) * dl[i][j];
        }
        const int ep[6][2] = {{0, 1}, {1, 2}, {2, 0}, {0, 3}, {1, 3}, {2, 3}};
        for (int e = 0; e < 6; ++e) {
            const int p = ep[e][0], q = ep[e][1];
            N[4 + e] = 4.0 * l[p] * l[q];
            for (int j = 0; j < 3; ++j) dN[3 * (4 + e) + j] = 4.0 * (dl[p][j] * l[q] + l[p] * dl[q][j]);
        }
        return 10;
    }
    if (elem == OR_Q2S) {
        /* 20-node serendipity brick.  Vertex a = i + 2j + 4k at
         * (xa, ya, za) = (2i-1, 2j-1, 2k-1):
         *   N = (1 + x xa)(1 + y ya)(1 + z za)(x xa + y ya + z za - 2) / 8;
         * edge midpoints at a zero coordinate, e.g. an x edge at (0, ya, za):
         *   N = (1 - x^2)(1 + y ya)(1 + z za) / 4;
         * x edges 8 + j + 2k, y edges 12 + i + 2k, z edges 16 + i + 2j. */
        const double x = xi[0], y = xi[1], z = xi[2];
        for (int a = 0; a < 8; ++a) {
            const double xa = (a & 1) ? 1.0 : -1.0, ya = (a & 2) ? 1.0 : -1.0, za = (a & 4) ? 1.0 : -1.0;
            const double A = 1.0 + x * xa, B = 1.0 + y * ya, Cz = 1.0 + z * za;
            const double S = x * xa + y * ya + z * za - 2.0;
            N[a] = 0.125 * A * B * Cz * S;
            dN[3 * a + 0] = 0.125 * xa * B * Cz * (S + A);
            dN[3 * a + 1] = 0.125 * ya * A * Cz * (S + B);
            dN[3 * a + 2] = 0.125 * za * A * B * (S + Cz);
        }
        for (int axis = 0; axis < 3; ++axis)
            for (int t = 0; t < 4; ++t) {
                const int a = 8 + 4 * axis + t;
                /* the two other coordinates in increasing axis order */
                const int d1 = axis == 0 ? 1 : 0, d2 = axis == 2 ? 1 : 2;
                const double s1 = (t & 1) ? 1.0 : -1.0, s2 = (t & 2) ? 1.0 : -1.0;
                const double u = xi[axis], v1 = xi[d1], v2 = xi[d2];
                const double Q = 1.0 - u * u, P1 = 1.0 + v1 * s1, P2 = 1.0 + v2 * s2;
                N[a] = 0.25 * Q * P1 * P2;
                dN[3 * a + axis] = 0.25 * (-2.0 * u) * P1 * P2;
                dN[3 * a + d1] = 0.25 * Q * s1 * P2;
                dN[3 * a + d2] = 0.25 * Q * P1 * s2;
            }
        return 20;
    }
    return -1;
}

static int elem_dim(int elem) { return (elem == OR_Q1 || elem == OR_Q2S || elem == OR_P2T) ? 3 : 2; }
static int elem_npe(int elem)
{
    return elem == OR_P1 ? 3 : (elem == OR_P2 ? 6 : (elem == OR_Q1 || elem == OR_Q2Q ? 8 : (elem == OR_Q2S ? 20 : 10)));
}

/* Geometry at one point: J_ij = sum_a x_{a,i} dN_a/dxi_j, detJ, and the
 * physical gradients grad N_a = J^{-T} gradref N_a (Sec. 2.1: D_lambda N at
 * x_gamma).  Straight-sided P2 triangles and tetrahedra take the affine map
 * of their vertices (their isoparametric map is that same affine map).
 * Returns detJ. */
static double geometry(int elem, const double *X, const double *xi, double *N, double *gradN)
{
    const int dim = elem_dim(elem);
    const int npe = elem_npe(elem);
    double dN[20 * 3];
    or_shape(elem, xi, N, dN);
    double J[3][3] = {{0}};
    if (elem == OR_P2) {
        double Nv[3], dNv[6];
        or_shape(OR_P1, xi, Nv, dNv);
        for (int i = 0; i < 2; ++i)
            for (int j = 0; j < 2; ++j)
                for (int a = 0; a < 3; ++a) J[i][j] += X[2 * a + i] * dNv[2 * a + j];
    } else if (elem == OR_P2T) {
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) J[i][j] = X[3 * (j + 1) + i] - X[i];
    } else {
        for (int i = 0; i < dim; ++i)
            for (int j = 0; j < dim; ++j)
                for (int a = 0; a < npe; ++a) J[i][j] += X[dim * a + i] * dN[dim * a + j];
    }
    double det, Ji[3][3];
    if (dim == 2) {
        det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
        Ji[0][0] = J[1][1] / det;  Ji[0][1] = -J[0][1] / det;
        Ji[1][0] = -J[1][0] / det; Ji[1][1] = J[0][0] / det;
    } else {
        /* inverse = adjugate / det */
        const double c00 = J[1][1] * J[2][2] - J[1][2] * J[2][1];
        const double c01 = J[1][2] * J[2][0] - J[1][0] * J[2][2];
        const double c02 = J[1][0] * J[2][1] - J[1][1] * J[2][0];
        det = J[0][0] * c00 + J[0][1] * c01 + J[0][2] * c02;
        Ji[0][0] = c00 / det;
        Ji[1][0] = c01 / det;
        Ji[2][0] = c02 / det;
        Ji[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det;
        Ji[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det;
        Ji[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det;
        Ji[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det;
        Ji[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;
        Ji[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det;
    }
    /* dN/dx_i = sum_j dN/dxi_j * dxi_j/dx_i, with dxi/dx = J^{-1} */
    for (int a = 0; a < npe; ++a)
        for (int i = 0; i < dim; ++i) {
            double s = 0.0;
            for (int j = 0; j < dim; ++j) s += dN[dim * a + j] * Ji[j][i];
            gradN[dim * a + i] = s;
        }
    return det;
}

/* Exported for the geometry pins: sum_q w_q detJ_q (the element measure). */
double or_elem_measure(int elem, int quad, const double *X)
{
    double pts[64 * 3], w[64], N[20], g[60];
    const int nq = or_quad(quad, pts, w);
    const int dim = elem_dim(elem);
    double s = 0.0;
    for (int q = 0; q < nq; ++q) s += w[q] * geometry(elem, X, pts + dim * q, N, g);
    return s;
}

/* ------------------------------------------------------------------------ */
/* Thermal element (Sec. 4.1: -k(T_,i, T_,i) + (T, s), tangent negated).    */
/* Ke[a][b] = sum_q w detJ k gradN_a . gradN_b                               */
/* de[a]    = sum_q w detJ N_a f(x_q), f = fconst or, if fnodal != NULL, the  */
/* nodal interpolant sum_b fnodal[b] N_b(x_q).  Returns min detJ.            */
/* ------------------------------------------------------------------------ */
double or_elem_thermal(int elem, int quad, const double *X, double k, double fconst,
                       const double *fnodal, double *Ke, double *de)
{
    double pts[64 * 3], w[64], N[20], g[60];
    const int nq = or_quad(quad, pts, w);
    const int dim = elem_dim(elem), npe = elem_npe(elem);
    double mindet = 1e300;
    for (int a = 0; a < npe; ++a) {
        de[a] = 0.0;
        for (int b = 0; b < npe; ++b) Ke[a * npe + b] = 0.0;
    }
    for (int q = 0; q < nq; ++q) {
        const double det = geometry(elem, X, pts + dim * q, N, g);
        if (det < mindet) mindet = det;
        const double wd = w[q] * det;
        double f = fconst;
        if (fnodal) {
            f = 0.0;
            for (int b = 0; b < npe; ++b) f += fnodal[b] * N[b];
        }
        for (int a = 0; a < npe; ++a) {
            for (int b = 0; b < npe; ++b) {
                double dot = 0.0;
                for (int i = 0; i < dim; ++i) dot += g[dim * a + i] * g[dim * b + i];
                Ke[a * npe + b] += wd * k * dot;
            }
            de[a] += wd * f * N[a];
        }
    }
    return mindet;
}

/* ------------------------------------------------------------------------ */
/* Capacity element (Sec. 4.1: -C(T, T_t), the rate term; tangent negated):  */
/* Me[a][b] = sum_q w detJ C N_a N_b, with a rule exact for N_a N_b on an    */
/* affine element: the 3-point rule (P1, degree 2), the 6-point rule (P2,    */
/* degree 4), 2 x 2 x 2 Gauss (Q1), 3 x 3 x 3 Gauss (Q2S), 3 x 3 Gauss      */
/* (Q2Q), the 64-point collapsed rule (P2T, degree 5).  Returns min detJ.   */
/* ------------------------------------------------------------------------ */
double or_elem_capacity(int elem, const double *X, double C, double *Me)
{
    double pts[64 * 3], w[64], N[20], g[60];
    const int quad = elem == OR_P1 ? OR_QTRI3
                     : elem == OR_P2 ? OR_QTRI6
                     : elem == OR_Q1 ? OR_QHEX8
                     : elem == OR_Q2S ? OR_QHEX27
                     : elem == OR_Q2Q ? OR_QQUAD9 : OR_QTET64;
    const int nq = or_quad(quad, pts, w);
    const int dim = elem_dim(elem), npe = elem_npe(elem);
    double mindet = 1e300;
    for (int a = 0; a < npe * npe; ++a) Me[a] = 0.0;
    for (int q = 0; q < nq; ++q) {
        const double det = geometry(elem, X, pts + dim * q, N, g);
        if (det < mindet) mindet = det;
        for (int a = 0; a < npe; ++a)
            for (int b = 0; b < npe; ++b) Me[a * npe + b] += w[q] * det * C * N[a] * N[b];
    }
    return mindet;
}

/* ------------------------------------------------------------------------ */
/* Linear elasticity on Q1 or Q2S bricks or P2T tetrahedra (Sec. 4.2:      */
/* -(d_i,j, sigma_ij),                                                      */
/* sigma = lambda delta eps_mm + 2 mu eps, lambda = E nu / ((1+nu)(1-2nu)),  */
/* mu = E / (2(1+nu))).  With test w = N_a e_c and trial u = N_b e_c':        */
/* eps(w):sigma(u) = lambda d_c N_a d_c' N_b + mu d_c' N_a d_c N_b            */
/*                 + mu delta_cc' gradN_a . gradN_b.                         */
/* Rule: 2 x 2 x 2 Gauss (Q1), 3 x 3 x 3 Gauss (Q2S, the cantilever bricks   */
/* of Sec. 4.2), the 64-point collapsed rule (P2T, exact for the degree-2   */
/* integrands of an affine quadratic tetrahedron).                          */
/* With m = 3 npe: Ke[(3a+c)*m + 3b+c'],                                     */
/* de[3a+c] = sum_q w detJ body_c N_a.  Returns min detJ.                    */
/* ------------------------------------------------------------------------ */
double or_elem_elastic(int elem, const double *X, double E, double nu, const double *body,
                       double *Ke, double *de)
{
    double pts[64 * 3], w[64], N[20], g[60];
    const int nq = or_quad(elem == OR_Q2S ? OR_QHEX27 : (elem == OR_P2T ? OR_QTET64 : OR_QHEX8), pts, w);
    const int npe = elem_npe(elem), m = 3 * npe;
    const double lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
    const double mu = E / (2.0 * (1.0 + nu));
    double mindet = 1e300;
    memset(Ke, 0, sizeof(double) * m * m);
    memset(de, 0, sizeof(double) * m);
    for (int q = 0; q < nq; ++q) {
        const double det = geometry(elem, X, pts + 3 * q, N, g);
        if (det < mindet) mindet = det;
        const double wd = w[q] * det;
        for (int a = 0; a < npe; ++a)
            for (int c = 0; c < 3; ++c) {
                for (int b = 0; b < npe; ++b) {
                    double dot = 0.0;
                    for (int i = 0; i < 3; ++i) dot += g[3 * a + i] * g[3 * b + i];
                    for (int cp = 0; cp < 3; ++cp) {
                        double v = lam * g[3 * a + c] * g[3 * b + cp] + mu * g[3 * a + cp] * g[3 * b + c];
                        if (c == cp) v += mu * dot;
                        Ke[(3 * a + c) * m + 3 * b + cp] += wd * v;
                    }
                }
                de[3 * a + c] += wd * body[c] * N[a];
            }
    }
    return mindet;
}

/* The Q1 brick of or_elem_elastic: Ke [24][24], de [24]. */
double or_elem_elastic_q1(const double *X, double E, double nu, const double *body,
                          double *Ke, double *de)
{
    return or_elem_elastic(OR_Q1, X, E, nu, body, Ke, de);
}

/* ------------------------------------------------------------------------ */
/* Steady Navier-Stokes with SUPG on one Taylor-Hood P2-P1 triangle (Sec.    */
/* 4.3), the domain form as the paper writes it, with test functions v      */
/* (velocity) and q (pressure):                                             */
/*   -rho(v_i,j, u_i u_j) - (v_i,i, p) + (q, u_i,i) + mu(v_i,j, u_i,j)        */
/*   + tau_m rho(v_i,j, Rm_i u_j) + tau_m(q_,i, Rm_i) + tau_c(v_i,i, Rc),     */
/*   Rc = u_k,k,  Rm_i = rho u_k u_i,k + p_,i - mu u_i,kk.                    */
/* Element residual r[15]: velocity dof (a, i) at 2a + i (a < 6, i < 2),     */
/* pressure vertex b at 12 + b; u_i,kk is the constant Laplacian of the P2   */
/* basis on the affine triangle.  The 16-point rule (degree 6) integrates    */
/* every term exactly.  Complex arithmetic so that the tangent can be taken  */
/* by complex-step differentiation (exact to rounding: the residual is a     */
/* polynomial in the dofs).  Returns detJ.                                   */
/* ------------------------------------------------------------------------ */
static double ns_residual(const double *X, const double complex *U, const double complex *P, double mu,
                          double rho, double tm, double tc, double complex *r)
{
    double pts[32], w[16];
    const int nq = or_quad(OR_QTRI16, pts, w);
    /* affine map of the vertices: gradients of the barycentrics l0, l1, l2 */
    const double j00 = X[2] - X[0], j10 = X[3] - X[1], j01 = X[4] - X[0], j11 = X[5] - X[1];
    const double det = j00 * j11 - j01 * j10;
    const double gl[3][2] = {{(-j11 + j10) / det, (j01 - j00) / det}, {j11 / det, -j01 / det}, {-j10 / det, j00 / det}};
    /* P2 basis: vertices l_v (2 l_v - 1), edges (0,1), (1,2), (2,0): 4 l_p l_q;
     * constant Laplacians */
    const int ep[3][2] = {{0, 1}, {1, 2}, {2, 0}};
    double lap[6];
    for (int v = 0; v < 3; ++v) lap[v] = 4.0 * (gl[v][0] * gl[v][0] + gl[v][1] * gl[v][1]);
    for (int e = 0; e < 3; ++e) {
        const int pp = ep[e][0], qq = ep[e][1];
        lap[3 + e] = 8.0 * (gl[pp][0] * gl[qq][0] + gl[pp][1] * gl[qq][1]);
    }
    for (int k = 0; k < 15; ++k) r[k] = 0.0;
    for (int q = 0; q < nq; ++q) {
        const double l[3] = {1.0 - pts[2 * q] - pts[2 * q + 1], pts[2 * q], pts[2 * q + 1]};
        double N[6], g[6][2];
        for (int v = 0; v < 3; ++v) {
            N[v] = l[v] * (2.0 * l[v] - 1.0);
            for (int k = 0; k < 2; ++k) g[v][k] = (4.0 * l[v] - 1.0) * gl[v][k];
        }
        for (int e = 0; e < 3; ++e) {
            const int pp = ep[e][0], qq = ep[e][1];
            N[3 + e] = 4.0 * l[pp] * l[qq];
            for (int k = 0; k < 2; ++k) g[3 + e][k] = 4.0 * (gl[pp][k] * l[qq] + l[pp] * gl[qq][k]);
        }
        double complex u[2] = {0.0, 0.0}, du[2][2] = {{0.0, 0.0}, {0.0, 0.0}}, lu[2] = {0.0, 0.0};
        double complex ph = 0.0, dp[2] = {0.0, 0.0};
        for (int a = 0; a < 6; ++a)
            for (int i = 0; i < 2; ++i) {
                u[i] += N[a] * U[2 * a + i];
                for (int k = 0; k < 2; ++k) du[i][k] += g[a][k] * U[2 * a + i];
                lu[i] += lap[a] * U[2 * a + i];
            }
        for (int b = 0; b < 3; ++b) {
            ph += l[b] * P[b];
            for (int k = 0; k < 2; ++k) dp[k] += gl[b][k] * P[b];
        }
        const double complex Rc = du[0][0] + du[1][1];
        double complex Rm[2];
        for (int i = 0; i < 2; ++i) Rm[i] = rho * (u[0] * du[i][0] + u[1] * du[i][1]) + dp[i] - mu * lu[i];
        const double wd = w[q] * det;
        for (int a = 0; a < 6; ++a) {
            const double complex adv = g[a][0] * u[0] + g[a][1] * u[1]; /* v_i,j u_j for v = N_a e_i */
            for (int i = 0; i < 2; ++i) {
                double complex t = -rho * adv * u[i] - g[a][i] * ph + mu * (g[a][0] * du[i][0] + g[a][1] * du[i][1]);
                t += tm * rho * adv * Rm[i] + tc * g[a][i] * Rc;
                r[2 * a + i] += wd * t;
            }
        }
        for (int b = 0; b < 3; ++b)
            r[12 + b] += wd * (l[b] * Rc + tm * (gl[b][0] * Rm[0] + gl[b][1] * Rm[1]));
    }
    return det;
}

/* Residual r[15] and tangent Ke[15][15] = d r / d (u, p) at the element
 * state U [6][2] (velocity, node-major), P [3] (vertex pressures), the
 * tangent column c by a complex step of 1e-30 in dof c.  Returns detJ. */
double or_elem_ns(const double *X, const double *U, const double *P, double mu, double rho, double tm,
                  double tc, double *r, double *Ke)
{
    double complex Uc[12], Pc[3], rc[15];
    for (int k = 0; k < 12; ++k) Uc[k] = U[k];
    for (int k = 0; k < 3; ++k) Pc[k] = P[k];
    const double det = ns_residual(X, Uc, Pc, mu, rho, tm, tc, rc);
    for (int k = 0; k < 15; ++k) r[k] = creal(rc[k]);
    const double h = 1e-30;
    for (int c = 0; c < 15; ++c) {
        if (c < 12) Uc[c] += I * h; else Pc[c - 12] += I * h;
        ns_residual(X, Uc, Pc, mu, rho, tm, tc, rc);
        for (int k = 0; k < 15; ++k) Ke[15 * k + c] = cimag(rc[k]) / h;
        if (c < 12) Uc[c] = U[c]; else Pc[c - 12] = P[c - 12];
    }
    return det;
}

/* The same form on one Taylor-Hood P2-P1 tetrahedron (the 3D flow case of  */
/* Sec. 4.3): velocity dof (a, i) at 3a + i (a < 10, i < 3), pressure       */
/* vertex b at 30 + b; the 10-node basis (vertices, then edges (0,1), (1,2), */
/* (2,0), (0,3), (1,3), (2,3)) on the affine element, its constant          */
/* Laplacians, and the 125-point rule (exact: every term has degree <= 6).   */
static double ns3_residual(const double *X, const double complex *U, const double complex *P, double mu,
                           double rho, double tm, double tc, double complex *r)
{
    static double pts[375], w[125];
    const int nq = or_quad(OR_QTET125, pts, w);
    double J[3][3], Ji[3][3];
    for (int j = 0; j < 3; ++j)
        for (int i = 0; i < 3; ++i) J[i][j] = X[3 * (j + 1) + i] - X[i];
    const double c00 = J[1][1] * J[2][2] - J[1][2] * J[2][1];
    const double c01 = J[1][2] * J[2][0] - J[1][0] * J[2][2];
    const double c02 = J[1][0] * J[2][1] - J[1][1] * J[2][0];
    const double det = J[0][0] * c00 + J[0][1] * c01 + J[0][2] * c02;
    Ji[0][0] = c00 / det;
    Ji[1][0] = c01 / det;
    Ji[2][0] = c02 / det;
    Ji[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det;
    Ji[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det;
    Ji[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det;
    Ji[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det;
    Ji[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;
    Ji[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det;
    /* gradients of the barycentrics: l_{p+1} = xi_p, l_0 = 1 - sum */
    double gl[4][3];
    for (int k = 0; k < 3; ++k) {
        gl[1][k] = Ji[0][k];
        gl[2][k] = Ji[1][k];
        gl[3][k] = Ji[2][k];
        gl[0][k] = -(Ji[0][k] + Ji[1][k] + Ji[2][k]);
    }
    const int ep[6][2] = {{0, 1}, {1, 2}, {2, 0}, {0, 3}, {1, 3}, {2, 3}};
    double lap[10];
    for (int v = 0; v < 4; ++v) lap[v] = 4.0 * (gl[v][0] * gl[v][0] + gl[v][1] * gl[v][1] + gl[v][2] * gl[v][2]);
    for (int e = 0; e < 6; ++e) {
        const int pp = ep[e][0], qq = ep[e][1];
        lap[4 + e] = 8.0 * (gl[pp][0] * gl[qq][0] + gl[pp][1] * gl[qq][1] + gl[pp][2] * gl[qq][2]);
    }
    for (int k = 0; k < 34; ++k) r[k] = 0.0;
    for (int q = 0; q < nq; ++q) {
        const double l[4] = {1.0 - pts[3 * q] - pts[3 * q + 1] - pts[3 * q + 2], pts[3 * q], pts[3 * q + 1],
                             pts[3 * q + 2]};
        double N[10], g[10][3];
        for (int v = 0; v < 4; ++v) {
            N[v] = l[v] * (2.0 * l[v] - 1.0);
            for (int k = 0; k < 3; ++k) g[v][k] = (4.0 * l[v] - 1.0) * gl[v][k];
        }
        for (int e = 0; e < 6; ++e) {
            const int pp = ep[e][0], qq = ep[e][1];
            N[4 + e] = 4.0 * l[pp] * l[qq];
            for (int k = 0; k < 3; ++k) g[4 + e][k] = 4.0 * (gl[pp][k] * l[qq] + l[pp] * gl[qq][k]);
        }
        double complex u[3] = {0.0, 0.0, 0.0}, du[3][3] = {{0.0}}, lu[3] = {0.0, 0.0, 0.0};
        double complex ph = 0.0, dp[3] = {0.0, 0.0, 0.0};
        for (int a = 0; a < 10; ++a)
            for (int i = 0; i < 3; ++i) {
                u[i] += N[a] * U[3 * a + i];
                for (int k = 0; k < 3; ++k) du[i][k] += g[a][k] * U[3 * a + i];
                lu[i] += lap[a] * U[3 * a + i];
            }
        for (int b = 0; b < 4; ++b) {
            ph += l[b] * P[b];
            for (int k = 0; k < 3; ++k) dp[k] += gl[b][k] * P[b];
        }
        const double complex Rc = du[0][0] + du[1][1] + du[2][2];
        double complex Rm[3];
        for (int i = 0; i < 3; ++i)
            Rm[i] = rho * (u[0] * du[i][0] + u[1] * du[i][1] + u[2] * du[i][2]) + dp[i] - mu * lu[i];
        const double wd = w[q] * det;
        for (int a = 0; a < 10; ++a) {
            const double complex adv = g[a][0] * u[0] + g[a][1] * u[1] + g[a][2] * u[2];
            for (int i = 0; i < 3; ++i) {
                double complex t = -rho * adv * u[i] - g[a][i] * ph +
                                   mu * (g[a][0] * du[i][0] + g[a][1] * du[i][1] + g[a][2] * du[i][2]);
                t += tm * rho * adv * Rm[i] + tc * g[a][i] * Rc;
                r[3 * a + i] += wd * t;
            }
        }
        for (int b = 0; b < 4; ++b)
            r[30 + b] += wd * (l[b] * Rc + tm * (gl[b][0] * Rm[0] + gl[b][1] * Rm[1] + gl[b][2] * Rm[2]));
    }
    return det;
}

/* Residual r[34] and tangent Ke[34][34] (complex step) of ns3_residual at
 * U [10][3], P [4]; X holds the 4 vertices.  Returns detJ. */
double or_elem_ns3(const double *X, const double *U, const double *P, double mu, double rho, double tm,
                   double tc, double *r, double *Ke)
{
    double complex Uc[30], Pc[4], rc[34];
    for (int k = 0; k < 30; ++k) Uc[k] = U[k];
    for (int k = 0; k < 4; ++k) Pc[k] = P[k];
    const double det = ns3_residual(X, Uc, Pc, mu, rho, tm, tc, rc);
    for (int k = 0; k < 34; ++k) r[k] = creal(rc[k]);
    const double h = 1e-30;
    for (int c = 0; c < 34; ++c) {
        if (c < 30) Uc[c] += I * h; else Pc[c - 30] += I * h;
        ns3_residual(X, Uc, Pc, mu, rho, tm, tc, rc);
        for (int k = 0; k < 34; ++k) Ke[34 * k + c] = cimag(rc[k]) / h;
        if (c < 30) Uc[c] = U[c]; else Pc[c - 30] = P[c - 30];
    }
    return det;
}

/* The global system of the Navier-Stokes form: dofs [u1 (n2) | u2 (n2) |
 * p (n1)]; R [2 n2 + n1] accumulates the element residuals; the tangent goes
 * out as 225 triplets per element (rows, cols, vals [n_el * 225], duplicates
 * to be summed).  Returns the minimum detJ (<= 0: an inverted element). */
double or_ns_system(int64_t n2, int64_t n1, int64_t n_el, const double *coords, const int32_t *conn,
                    const int32_t *pconn, const double *u1, const double *u2, const double *p, double mu,
                    double rho, double tm, double tc, double *R, int64_t *rows, int32_t *cols, double *vals)
{
    double mindet = 1e300;
    for (int64_t k = 0; k < 2 * n2 + n1; ++k) R[k] = 0.0;
    for (int64_t e = 0; e < n_el; ++e) {
        const int32_t *cn = conn + 6 * e, *pn = pconn + 3 * e;
        double X[6], U[12], P[3], r[15], Ke[225];
        int64_t dof[15];
        for (int v = 0; v < 3; ++v)
            for (int i = 0; i < 2; ++i) X[2 * v + i] = coords[2 * (int64_t)cn[v] + i];
        for (int a = 0; a < 6; ++a) {
            U[2 * a] = u1[cn[a]];
            U[2 * a + 1] = u2[cn[a]];
            dof[2 * a] = cn[a];
            dof[2 * a + 1] = n2 + cn[a];
        }
        for (int b = 0; b < 3; ++b) {
            P[b] = p[pn[b]];
            dof[12 + b] = 2 * n2 + pn[b];
        }
        const double det = or_elem_ns(X, U, P, mu, rho, tm, tc, r, Ke);
        if (det < mindet) mindet = det;
        for (int k = 0; k < 15; ++k) {
            R[dof[k]] += r[k];
            for (int c = 0; c < 15; ++c) {
                rows[225 * e + 15 * k + c] = dof[k];
                cols[225 * e + 15 * k + c] = (int32_t)dof[c];
                vals[225 * e + 15 * k + c] = Ke[15 * k + c];
            }
        }
    }
    return mindet;
}

/* ------------------------------------------------------------------------ */
/* Picard-linearised flow on Taylor-Hood P2-P1 (Sec. 4.3, the NS part of the */
/* domain form with the advecting velocity a in place of u_j):              */
/*   mu(u_i,j, u_i,j) - rho(u_i,j, u_i a_j) - (u_i,i, p) + (p, u_i,i).        */
/* Per component i (the same matrix for i = 1, 2):                           */
/*   A[a][b]  = sum_q w detJ (mu gradN_a.gradN_b - rho (a_h . gradN_a) N_b)  */
/* velocity row a, pressure column b:  BT[i][a][b] = -sum_q w detJ d_iN_a M_b */
/* pressure row a, velocity column b:  B[i][a][b]  = +sum_q w detJ M_a d_iN_b */
/* pressure mass diagonal Mp[a] = sum_q w detJ M_a^2.                         */
/* aN is the nodal advecting field [6][2]; a_h = sum_b aN_b N_b.             */
/* ------------------------------------------------------------------------ */
double or_elem_oseen(const double *X, const double *aN, double mu, double rho,
                     double *A, double *BT, double *B, double *Mp)
{
    double pts[12], w[6], N[6], g[12], M[3], dM[6];
    const int nq = or_quad(OR_QTRI6, pts, w);
    double mindet = 1e300;
    memset(A, 0, sizeof(double) * 36);
    memset(BT, 0, sizeof(double) * 2 * 18);
    memset(B, 0, sizeof(double) * 2 * 18);
    memset(Mp, 0, sizeof(double) * 3);
    for (int q = 0; q < nq; ++q) {
        const double det = geometry(OR_P2, X, pts + 2 * q, N, g);
        if (det < mindet) mindet = det;
        or_shape(OR_P1, pts + 2 * q, M, dM);
        const double wd = w[q] * det;
        double ah[2] = {0.0, 0.0};
        for (int b = 0; b < 6; ++b)
            for (int j = 0; j < 2; ++j) ah[j] += aN[2 * b + j] * N[b];
        for (int a = 0; a < 6; ++a) {
            const double adv = ah[0] * g[2 * a] + ah[1] * g[2 * a + 1];
            for (int b = 0; b < 6; ++b) {
                const double dot = g[2 * a] * g[2 * b] + g[2 * a + 1] * g[2 * b + 1];
                A[6 * a + b] += wd * (mu * dot - rho * adv * N[b]);
            }
        }
        for (int i = 0; i < 2; ++i)
            for (int a = 0; a < 6; ++a)
                for (int b = 0; b < 3; ++b) BT[18 * i + 3 * a + b] += -wd * g[2 * a + i] * M[b];
        for (int i = 0; i < 2; ++i)
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 6; ++b) B[18 * i + 6 * a + b] += wd * M[a] * g[2 * b + i];
        for (int a = 0; a < 3; ++a) Mp[a] += wd * M[a] * M[a];
    }
    return mindet;
}

/* ------------------------------------------------------------------------ */
/* Boundary facets (Sec. 2.2: a boundary condition is the domain physics one */
/* dimension lower; Sec. 4.1 convection h(T, T_env - T); Sec. 4.2 loaded     */
/* boundary (d_i, sigma^l_ij n_j)).  A facet is local face `face` of an      */
/* element:                                                                  */
/*  - triangle face f is the edge from vertex f to vertex (f+1) % 3; P2 adds */
/*    the midpoint node 3 + f.  Edge parameter t in [0, 1] from vertex f;    */
/*    the edge is straight, x(t) = x_f + t (x_{f+1} - x_f).                  */
/*  - hexahedron face 2d + s is the face xi_d = 2s - 1: the element nodes a  */
/*    with bit d of a equal to s, ascending.  Its parameters (u, v) are the  */
/*    other two reference coordinates in increasing axis order, so facet     */
/*    node m sits at (u, v) = (2(m & 1) - 1, 2(m >> 1) - 1) and the face map */
/*    is the bilinear x(u, v) = sum_m N_m(u, v) x_m.                         */
/*  - tetrahedron face i (P2T) is opposite vertex i: 3 vertices, then the    */
/*    midpoints of its edges, the facet basis the P2 triangle's (or_shape    */
/*    OR_P2) on the reference triangle (xi, eta), the map affine.            */
/* Quadrature: Gauss-Legendre on the edge with 2 (P1) or 3 (P2) points,     */
/* exact for N_a N_b on a straight edge; 2 x 2 Gauss on a hexahedron face;   */
/* the 6-point degree-4 triangle rule on a tetrahedron face (exact for      */
/* N_a N_b on the flat face).                                               */
/* ------------------------------------------------------------------------ */
int or_facet_nodes(int elem, int face, int *loc)
{
    if (elem == OR_Q2S) {
        /* face 2d + s as on the Q1 brick: its 4 vertices (bit d of a equal to
         * s, ascending: face node i + 2j with i, j the bits of the face axes
         * d1 < d2), then, in the 8-node quadrilateral's order, the midpoints
         * of its d1 edges at bit d2 = j (4 + j) and of its d2 edges at bit
         * d1 = i (6 + i).  The brick's edge along axis A whose other two
         * coordinates B < C have bits b, c is node 8 + 4A + b + 2c. */
        if (face < 0 || face > 5) return -1;
        const int d = face / 2, s = face % 2;
        const int d1 = d == 0 ? 1 : 0, d2 = d == 2 ? 1 : 2;
        int m = 0;
        for (int a = 0; a < 8; ++a)
            if (((a >> d) & 1) == s) loc[m++] = a;
        for (int k = 0; k < 4; ++k) {
            const int A = k < 2 ? d1 : d2;            /* the edge's axis */
            const int other = k < 2 ? d2 : d1, ob = k & 1;
            int bits[3];
            bits[d] = s;
            bits[other] = ob;
            const int B = A == 0 ? 1 : 0, C = A == 2 ? 1 : 2;
            loc[4 + k] = 8 + 4 * A + bits[B] + 2 * bits[C];
        }
        return 8;
    }
    if (elem == OR_P2T) {
        /* face i is opposite vertex i: its vertices in the order that makes
         * (x1 - x0) x (x2 - x0) point outward for a positively oriented
         * tetrahedron, then the midpoints of its edges (0,1), (1,2), (2,0) */
        static const int fl[4][6] = {{1, 2, 3, 5, 9, 8}, {0, 3, 2, 7, 9, 6}, {0, 1, 3, 4, 8, 7}, {0, 2, 1, 6, 5, 4}};
        if (face < 0 || face > 3) return -1;
        for (int m = 0; m < 6; ++m) loc[m] = fl[face][m];
        return 6;
    }
    if (elem == OR_Q1) {
        if (face < 0 || face > 5) return -1;
        const int d = face / 2, s = face % 2;
        int m = 0;
        for (int a = 0; a < 8; ++a)
            if (((a >> d) & 1) == s) loc[m++] = a;
        return 4;
    }
    if (elem == OR_Q2Q) {
        /* edges counter-clockwise: (0,1 | 4), (1,3 | 7), (3,2 | 5), (2,0 | 6):
         * the two vertices, then the midpoint (a straight 3-node edge as P2's) */
        static const int el[4][3] = {{0, 1, 4}, {1, 3, 7}, {3, 2, 5}, {2, 0, 6}};
        if (face < 0 || face > 3) return -1;
        for (int m = 0; m < 3; ++m) loc[m] = el[face][m];
        return 3;
    }
    if (face < 0 || face > 2) return -1;
    loc[0] = face;
    loc[1] = (face + 1) % 3;
    if (elem == OR_P2) {
        loc[2] = 3 + face;
        return 3;
    }
    return 2;
}

/* Points and weights of the facet rule: t in [0, 1] (edges) or (u, v) in
 * [-1, 1]^2 (hexahedron faces). */
static int facet_quad(int elem, double *pts, double *w)
{
    if (elem == OR_Q2Q) elem = OR_P2;  /* straight 3-node edges */
    if (elem == OR_Q2S) return or_quad(OR_QQUAD9, pts, w);  /* 8-node faces: 3 x 3 Gauss */
    if (elem == OR_P2T) return or_quad(OR_QTRI6, pts, w);
    if (elem == OR_P1) {
        const double g = 0.5 / sqrt(3.0);
        pts[0] = 0.5 - g; pts[1] = 0.5 + g;
        w[0] = w[1] = 0.5;
        return 2;
    }
    if (elem == OR_P2) {
        const double g = 0.5 * sqrt(0.6);
        pts[0] = 0.5 - g; pts[1] = 0.5; pts[2] = 0.5 + g;
        w[0] = w[2] = 5.0 / 18.0;
        w[1] = 8.0 / 18.0;
        return 3;
    }
    const double g = 1.0 / sqrt(3.0);
    for (int q = 0; q < 4; ++q) {
        pts[2 * q + 0] = (q & 1) ? g : -g;
        pts[2 * q + 1] = (q & 2) ? g : -g;
        w[q] = 1.0;
    }
    return 4;
}

/* Facet shape functions at one point: the trace of the element's basis on
 * the facet (edge: 1 - t, t [, P2: (1-t)(1-2t), t(2t-1), 4t(1-t)]; face: the
 * bilinear N_m), and the facet's area vector A = dx/du x dx/dv (faces) or
 * its length element |dx/dt| (edges, returned in A[0]). */
static int facet_point(int elem, const double *Xf, const double *p, double *N, double *A)
{
    if (elem == OR_Q2Q) elem = OR_P2;  /* straight 3-node edges */
    if (elem == OR_P1 || elem == OR_P2) {
        const double t = p[0];
        int nf;
        if (elem == OR_P1) {
            N[0] = 1.0 - t; N[1] = t;
            nf = 2;
        } else {
            N[0] = (1.0 - t) * (1.0 - 2.0 * t);
            N[1] = t * (2.0 * t - 1.0);
            N[2] = 4.0 * t * (1.0 - t);
            nf = 3;
        }
        const double ex = Xf[2] - Xf[0], ey = Xf[3] - Xf[1];
        A[0] = sqrt(ex * ex + ey * ey);
        return nf;
    }
    if (elem == OR_P2T) {
        double dN[12];
        or_shape(OR_P2, p, N, dN);
        double e1[3], e2[3];
        for (int i = 0; i < 3; ++i) {
            e1[i] = Xf[3 + i] - Xf[i];
            e2[i] = Xf[6 + i] - Xf[i];
        }
        A[0] = e1[1] * e2[2] - e1[2] * e2[1];
        A[1] = e1[2] * e2[0] - e1[0] * e2[2];
        A[2] = e1[0] * e2[1] - e1[1] * e2[0];
        return 6;
    }
    const double u = p[0], v = p[1];
    double xu[3] = {0.0, 0.0, 0.0}, xv[3] = {0.0, 0.0, 0.0};
    double N8[8], dN8[16];
    if (elem == OR_Q2S) or_shape(OR_Q2Q, p, N8, dN8);  /* the 8-node face basis */
    for (int m = 0; m < 4; ++m) {
        const double su = (m & 1) ? 1.0 : -1.0, sv = (m & 2) ? 1.0 : -1.0;
        N[m] = 0.25 * (1.0 + su * u) * (1.0 + sv * v);
        const double dNu = 0.25 * su * (1.0 + sv * v), dNv = 0.25 * (1.0 + su * u) * sv;
        for (int i = 0; i < 3; ++i) {
            xu[i] += dNu * Xf[3 * m + i];
            xv[i] += dNv * Xf[3 * m + i];
        }
    }
    A[0] = xu[1] * xv[2] - xu[2] * xv[1];
    A[1] = xu[2] * xv[0] - xu[0] * xv[2];
    A[2] = xu[0] * xv[1] - xu[1] * xv[0];
    if (elem == OR_Q2S) {  /* the map stays the vertices' bilinear one (straight edges) */
        for (int m = 0; m < 8; ++m) N[m] = N8[m];
        return 8;
    }
    return 4;
}

/* Convection on one facet (Sec. 4.1, h(T, T_env - T), tangent negated):
 *   Kf[m][m'] = sum_q w_q |J_q| h N_m N_m',  df[m] = sum_q w_q |J_q| h T_env N_m,
 * |J| the length element (edges) or |A| (faces).  Xf holds the facet nodes'
 * coordinates in facet node order.  Returns the facet's measure sum_q w |J|. */
double or_facet_thermal(int elem, const double *Xf, double h, double tenv, double *Kf, double *df)
{
    double pts[18], w[9], N[8], A[3];
    const int nq = facet_quad(elem, pts, w);
    const int pdim = (elem == OR_Q1 || elem == OR_P2T || elem == OR_Q2S) ? 2 : 1;
    const int nf = elem == OR_P1 ? 2 : (elem == OR_P2 || elem == OR_Q2Q ? 3 : (elem == OR_Q1 ? 4 : (elem == OR_Q2S ? 8 : 6)));
    for (int a = 0; a < nf * nf; ++a) Kf[a] = 0.0;
    for (int a = 0; a < nf; ++a) df[a] = 0.0;
    double meas = 0.0;
    for (int q = 0; q < nq; ++q) {
        facet_point(elem, Xf, pts + pdim * q, N, A);
        const double J = (elem == OR_Q1 || elem == OR_P2T || elem == OR_Q2S) ? sqrt(A[0] * A[0] + A[1] * A[1] + A[2] * A[2]) : A[0];
        meas += w[q] * J;
        for (int a = 0; a < nf; ++a) {
            for (int b = 0; b < nf; ++b) Kf[a * nf + b] += w[q] * J * h * N[a] * N[b];
            df[a] += w[q] * J * h * tenv * N[a];
        }
    }
    return meas;
}

/* Loaded boundary on one hexahedron face (Sec. 4.2, (d_i, sigma^l_ij n_j)):
 *   df[3m + i] = sum_q w_q N_m sigma_ij n_j |A_q|,  n |A| = o A,
 * with o = +1 or -1 the orientation that makes n the outward normal.  The
 * reference frame (e_d, e_d1, e_d2), d1 < d2 the face's parameter axes, is
 * right-handed for d = 0, 2 and left-handed for d = 1, so e_d1 x e_d2 is
 * +e_d (d = 0, 2) or -e_d (d = 1); the outward reference normal of face
 * 2d + s is (2s - 1) e_d; a map with detJ > 0 keeps orientation.  sigma is
 * row-major 3 x 3. */
void or_facet_traction(int elem, int face, const double *Xf, const double *sigma, double *df)
{
    double pts[18], w[9], N[8], A[3];
    const int nq = facet_quad(elem, pts, w);
    const int nf = elem == OR_Q2S ? 8 : 4;
    const int d = face / 2, s = face % 2;
    const double o = (s ? 1.0 : -1.0) * (d == 1 ? -1.0 : 1.0);
    for (int a = 0; a < 3 * nf; ++a) df[a] = 0.0;
    for (int q = 0; q < nq; ++q) {
        facet_point(elem, Xf, pts + 2 * q, N, A);
        for (int m = 0; m < nf; ++m)
            for (int i = 0; i < 3; ++i) {
                double t = 0.0;
                for (int j = 0; j < 3; ++j) t += sigma[3 * i + j] * o * A[j];
                df[3 * m + i] += w[q] * N[m] * t;
            }
    }
}

/* The Q1 face of or_facet_traction: df [4][3]. */
void or_facet_traction_q1(int face, const double *Xf, const double *sigma, double *df)
{
    or_facet_traction(OR_Q1, face, Xf, sigma, df);
}

/* Radiation on one facet (Sec. 4.1, e_m sigma^b (T, T_env^4 - T^4)) at the
 * facet nodes' temperatures Tf, es = e_m sigma^b:
 *   rf[m]      = sum_q w_q |J_q| es N_m (T_env^4 - T_q^4),   T_q = sum_b N_b T_b,
 *   Kf[m][m'] = sum_q w_q |J_q| 4 es N_m N_m' T_q^3  (= -d rf[m] / d T_m').
 * Rule and |J| as or_facet_thermal. */
void or_facet_radiation(int elem, const double *Xf, double es, double tenv, const double *Tf, double *Kf,
                        double *rf)
{
    double pts[18], w[9], N[8], A[3];
    const int nq = facet_quad(elem, pts, w);
    const int pdim = (elem == OR_Q1 || elem == OR_P2T || elem == OR_Q2S) ? 2 : 1;
    const int nf = elem == OR_P1 ? 2 : (elem == OR_P2 || elem == OR_Q2Q ? 3 : (elem == OR_Q1 ? 4 : (elem == OR_Q2S ? 8 : 6)));
    for (int a = 0; a < nf * nf; ++a) Kf[a] = 0.0;
    for (int a = 0; a < nf; ++a) rf[a] = 0.0;
    const double te4 = tenv * tenv * tenv * tenv;
    for (int q = 0; q < nq; ++q) {
        facet_point(elem, Xf, pts + pdim * q, N, A);
        const double J = (elem == OR_Q1 || elem == OR_P2T || elem == OR_Q2S) ? sqrt(A[0] * A[0] + A[1] * A[1] + A[2] * A[2]) : A[0];
        double T = 0.0;
        for (int b = 0; b < nf; ++b) T += N[b] * Tf[b];
        for (int a = 0; a < nf; ++a) {
            rf[a] += w[q] * J * es * N[a] * (te4 - T * T * T * T);
            for (int b = 0; b < nf; ++b) Kf[a * nf + b] += w[q] * J * 4.0 * es * N[a] * N[b] * T * T * T;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Global assembly (Block B-3/B-4 numbering, Block D-2/D-3 accumulation).    */
/* Every element emits COO triplets (row, col, value) in element order, local */
/* row-major order; every dof also emits (g, g, 0) first, so that the        */
/* diagonal is always present.  A stable sort by (row, col) followed by the  */
/* sum of duplicates in emission order gives CSR K (ascending columns) and d. */
/* Boundary facets emit after all elements, in facet order.                  */
/* Dof numbering: thermal node; elasticity 3 node + c; flow [u1 | u2 | p].   */
/* ------------------------------------------------------------------------ */
typedef struct {
    int64_t *row;
    int32_t *col;
    double *val;
    int64_t n, cap;
} coo_t;

static int coo_push(coo_t *c, int64_t r, int64_t col, double v)
{
    if (c->n == c->cap) {
        int64_t nc = c->cap ? 2 * c->cap : 1 << 16;
        int64_t *nr = realloc(c->row, sizeof(int64_t) * nc);
        if (!nr) return -1;
        c->row = nr;
        int32_t *ncol = realloc(c->col, sizeof(int32_t) * nc);
        if (!ncol) return -1;
        c->col = ncol;
        double *nv = realloc(c->val, sizeof(double) * nc);
        if (!nv) return -1;
        c->val = nv;
        c->cap = nc;
    }
    c->row[c->n] = r;
    c->col[c->n] = (int32_t)col;
    c->val[c->n] = v;
    c->n++;
    return 0;
}

/* stable merge sort of an index permutation by (row, col) */
static const coo_t *g_sort_coo;
static int key_less(int64_t a, int64_t b)
{
    const coo_t *c = g_sort_coo;
    if (c->row[a] != c->row[b]) return c->row[a] < c->row[b];
    return c->col[a] < c->col[b];
}
static void merge_sort(int64_t *idx, int64_t *tmp, int64_t n)
{
    for (int64_t width = 1; width < n; width *= 2) {
        for (int64_t lo = 0; lo < n; lo += 2 * width) {
            int64_t mid = lo + width < n ? lo + width : n;
            int64_t hi = lo + 2 * width < n ? lo + 2 * width : n;
            int64_t i = lo, j = mid, k = lo;
            while (i < mid && j < hi) tmp[k++] = key_less(idx[j], idx[i]) ? idx[j++] : idx[i++];
            while (i < mid) tmp[k++] = idx[i++];
            while (j < hi) tmp[k++] = idx[j++];
        }
        memcpy(idx, tmp, sizeof(int64_t) * n);
    }
}

typedef struct {
    int form, elem, quad;
    int64_t n_nodes, n_el, n_pnodes;
    const double *coords;   /* [n_nodes][dim] */
    const int32_t *conn;    /* [n_el][npe] */
    const int32_t *pconn;   /* flow: [n_el][3] P1 vertex numbering */
    const double *coef;     /* [n_el]: k (thermal), E (elasticity) */
    double nu;              /* Poisson ratio (elasticity) */
    double mu, rho;         /* flow viscosity, density */
    const double *source;   /* thermal: source[0]; elasticity: body[3] */
    const double *fnodal;   /* thermal nodal source or NULL */
    const double *advect;   /* flow: [2][n_nodes] */
    /* boundary facets (thermal: convection; elasticity: loaded boundary) */
    int64_t n_facets;
    const int32_t *f_elem;  /* [n_facets] parent element */
    const uint8_t *f_face;  /* [n_facets] local face */
    const double *f_h;      /* thermal [n_facets]: h */
    const double *f_tenv;   /* thermal [n_facets]: T_env */
    const double *f_stress; /* elasticity [n_facets][3][3]: sigma^l */
} or_problem;

int64_t or_ndofs(const or_problem *p)
{
    if (p->form == OR_ELASTIC) return 3 * p->n_nodes;
    if (p->form == OR_CAPACITY) return p->n_nodes;
    if (p->form == OR_OSEEN) return 2 * p->n_nodes + p->n_pnodes;
    return p->n_nodes;
}

/* Emits all triplets of one problem; d accumulated in element order too.
 * With a node filter (keep != NULL), only elements with at least one node
 * marked in keep[] (or, for flow, one vertex marked in pkeep[]) are
 * evaluated; rows outside the filter are then incomplete and must be ignored.
 * Returns 0, or -2 if some element has detJ <= 0, -3 for a facet outside the
 * mesh, a form without boundary terms or an element the form does not take,
 * -1 on allocation failure. */
static int emit_filtered(const or_problem *p, coo_t *c, double *d, double *pmass, const uint8_t *keep,
                         const uint8_t *pkeep)
{
    const int64_t n = or_ndofs(p);
    const int dim = elem_dim(p->elem), npe = elem_npe(p->elem);
    for (int64_t g = 0; g < n; ++g)
        if (coo_push(c, g, g, 0.0)) return -1;
    double X[20 * 3], Ke[60 * 60], de[60], fn[20];
    for (int64_t e = 0; e < p->n_el; ++e) {
        const int32_t *cn = p->conn + e * npe;
        if (keep) {
            int hit = 0;
            for (int a = 0; a < npe; ++a) hit |= keep[cn[a]];
            if (pkeep && p->pconn)
                for (int a = 0; a < 3; ++a) hit |= pkeep[p->pconn[e * 3 + a]];
            if (!hit) continue;
        }
        for (int a = 0; a < npe; ++a)
            for (int i = 0; i < dim; ++i) X[dim * a + i] = p->coords[(int64_t)cn[a] * dim + i];
        if (p->form == OR_THERMAL) {
            if (p->fnodal)
                for (int a = 0; a < npe; ++a) fn[a] = p->fnodal[cn[a]];
            const double det = or_elem_thermal(p->elem, p->quad, X, p->coef[e], p->source[0],
                                               p->fnodal ? fn : NULL, Ke, de);
            if (!(det > 0.0)) return -2;
            for (int a = 0; a < npe; ++a) {
                for (int b = 0; b < npe; ++b)
                    if (coo_push(c, cn[a], cn[b], Ke[a * npe + b])) return -1;
                d[cn[a]] += de[a];
            }
        } else if (p->form == OR_CAPACITY) {
            const double det = or_elem_capacity(p->elem, X, p->coef[e], Ke);
            if (!(det > 0.0)) return -2;
            for (int a = 0; a < npe; ++a)
                for (int b = 0; b < npe; ++b)
                    if (coo_push(c, cn[a], cn[b], Ke[a * npe + b])) return -1;
        } else if (p->form == OR_ELASTIC) {
            if (p->elem != OR_Q1 && p->elem != OR_Q2S && p->elem != OR_P2T) return -3;
            const double det = or_elem_elastic(p->elem, X, p->coef[e], p->nu, p->source, Ke, de);
            if (!(det > 0.0)) return -2;
            const int m = 3 * npe;
            for (int a = 0; a < npe; ++a)
                for (int ci = 0; ci < 3; ++ci) {
                    for (int b = 0; b < npe; ++b)
                        for (int cj = 0; cj < 3; ++cj)
                            if (coo_push(c, 3 * (int64_t)cn[a] + ci, 3 * (int64_t)cn[b] + cj,
                                         Ke[(3 * a + ci) * m + 3 * b + cj]))
                                return -1;
                    d[3 * (int64_t)cn[a] + ci] += de[3 * a + ci];
                }
        } else {
            const int32_t *pn = p->pconn + e * 3;
            double aN[12], A[36], BT[36], B[36], Mp[3];
            for (int a = 0; a < 6; ++a)
                for (int j = 0; j < 2; ++j) aN[2 * a + j] = p->advect[j * p->n_nodes + cn[a]];
            const double det = or_elem_oseen(X, aN, p->mu, p->rho, A, BT, B, Mp);
            if (!(det > 0.0)) return -2;
            const int64_t n2 = p->n_nodes;
            for (int i = 0; i < 2; ++i) {
                for (int a = 0; a < 6; ++a) {
                    const int64_t r = i * n2 + cn[a];
                    for (int b = 0; b < 6; ++b)
                        if (coo_push(c, r, i * n2 + cn[b], A[6 * a + b])) return -1;
                    for (int b = 0; b < 3; ++b)
                        if (coo_push(c, r, 2 * n2 + pn[b], BT[18 * i + 3 * a + b])) return -1;
                }
                for (int a = 0; a < 3; ++a)
                    for (int b = 0; b < 6; ++b)
                        if (coo_push(c, 2 * n2 + pn[a], i * n2 + cn[b], B[18 * i + 6 * a + b])) return -1;
            }
            if (pmass)
                for (int a = 0; a < 3; ++a) pmass[pn[a]] += Mp[a];
        }
    }
    for (int64_t f = 0; f < p->n_facets; ++f) {
        const int64_t e = p->f_elem[f];
        int loc[8];
        if (e < 0 || e >= p->n_el) return -3;
        const int nf = or_facet_nodes(p->elem, p->f_face[f], loc);
        if (nf < 0 || p->form == OR_OSEEN || p->form == OR_CAPACITY) return -3;
        int64_t node[8];
        double Xf[24], Kf[64], df[24];
        int hit = keep == NULL;
        for (int m = 0; m < nf; ++m) {
            node[m] = p->conn[e * npe + loc[m]];
            if (keep) hit |= keep[node[m]];
            for (int i = 0; i < dim; ++i) Xf[dim * m + i] = p->coords[node[m] * dim + i];
        }
        if (!hit) continue;
        if (p->form == OR_THERMAL) {
            or_facet_thermal(p->elem, Xf, p->f_h[f], p->f_tenv[f], Kf, df);
            for (int a = 0; a < nf; ++a) {
                for (int b = 0; b < nf; ++b)
                    if (coo_push(c, node[a], node[b], Kf[a * nf + b])) return -1;
                d[node[a]] += df[a];
            }
        } else {
            if (p->elem != OR_Q1 && p->elem != OR_Q2S) return -3;
            or_facet_traction(p->elem, p->f_face[f], Xf, p->f_stress + 9 * f, df);
            for (int a = 0; a < nf; ++a)
                for (int i = 0; i < 3; ++i) d[3 * node[a] + i] += df[3 * a + i];
        }
    }
    return 0;
}

/* Assembles CSR K and d.  Output arrays are malloc'd here; free with or_free.
 * pmass_out (flow only, may be NULL) receives a malloc'd [n_pnodes] pressure
 * mass diagonal.  Returns 0, -1 (allocation), -2 (detJ <= 0) or -3 (bad facet). */
int or_assemble_filtered(const or_problem *p, const uint8_t *keep, const uint8_t *pkeep, int64_t *n_rows,
                         int64_t *nnz, int64_t **row_ptr, int32_t **col, double **val, double **d,
                         double **pmass_out)
{
    const int64_t n = or_ndofs(p);
    coo_t c = {0};
    double *dv = calloc((size_t)n, sizeof(double));
    double *pm = (p->form == OR_OSEEN) ? calloc((size_t)p->n_pnodes, sizeof(double)) : NULL;
    if (!dv) return -1;
    int rc = emit_filtered(p, &c, dv, pm, keep, pkeep);
    if (rc) {
        free(c.row); free(c.col); free(c.val); free(dv); free(pm);
        return rc;
    }
    int64_t *idx = malloc(sizeof(int64_t) * c.n), *tmp = malloc(sizeof(int64_t) * c.n);
    for (int64_t t = 0; t < c.n; ++t) idx[t] = t;
    g_sort_coo = &c;
    merge_sort(idx, tmp, c.n);
    /* count unique (row, col) */
    int64_t u = 0;
    for (int64_t t = 0; t < c.n; ++t)
        if (t == 0 || c.row[idx[t]] != c.row[idx[t - 1]] || c.col[idx[t]] != c.col[idx[t - 1]]) ++u;
    int64_t *rp = calloc((size_t)n + 1, sizeof(int64_t));
    int32_t *ci = malloc(sizeof(int32_t) * u);
    double *vv = malloc(sizeof(double) * u);
    int64_t k = -1;
    for (int64_t t = 0; t < c.n; ++t) {
        const int64_t s = idx[t];
        if (t == 0 || c.row[s] != c.row[idx[t - 1]] || c.col[s] != c.col[idx[t - 1]]) {
            ++k;
            ci[k] = c.col[s];
            vv[k] = 0.0;
            rp[c.row[s] + 1]++;
        }
        vv[k] += c.val[s]; /* duplicates summed in emission order */
    }
    for (int64_t r = 0; r < n; ++r) rp[r + 1] += rp[r];
    free(idx); free(tmp); free(c.row); free(c.col); free(c.val);
    *n_rows = n;
    *nnz = u;
    *row_ptr = rp;
    *col = ci;
    *val = vv;
    *d = dv;
    if (pmass_out) *pmass_out = pm; else free(pm);
    return 0;
}

/* The whole system: every element evaluated. */
int or_assemble(const or_problem *p, int64_t *n_rows, int64_t *nnz, int64_t **row_ptr, int32_t **col,
                double **val, double **d, double **pmass_out)
{
    return or_assemble_filtered(p, NULL, NULL, n_rows, nnz, row_ptr, col, val, d, pmass_out);
}

/* ------------------------------------------------------------------------ */
/* The same assembly on several host threads (the all-core CPU baseline).    */
/* Compiled with -fopenmp into a second library; without it the pragmas are */
/* ignored and it runs on one thread.  Element matrices are the same calls   */
/* as above, each element's triplets land at the position the serial         */
/* emission gives them, and the stable order by (row, col) is built by a     */
/* stable counting sort on rows (per-thread counts, chunks in emission       */
/* order) followed by a stable merge sort of each row by column; duplicates  */
/* are summed in emission order.  The result equals or_assemble bit for bit. */
/* Domain forms (thermal, capacity, elasticity) without facets; -3 otherwise.*/
/* ------------------------------------------------------------------------ */
static void merge_sort_cols(int64_t *idx, int64_t *tmp, int64_t n, const int32_t *col)
{
    for (int64_t width = 1; width < n; width *= 2) {
        for (int64_t lo = 0; lo < n; lo += 2 * width) {
            int64_t mid = lo + width < n ? lo + width : n;
            int64_t hi = lo + 2 * width < n ? lo + 2 * width : n;
            int64_t i = lo, j = mid, k = lo;
            while (i < mid && j < hi) tmp[k++] = col[idx[j]] < col[idx[i]] ? idx[j++] : idx[i++];
            while (i < mid) tmp[k++] = idx[i++];
            while (j < hi) tmp[k++] = idx[j++];
        }
        memcpy(idx, tmp, sizeof(int64_t) * n);
    }
}

int or_assemble_threads(const or_problem *p, int threads, int64_t *n_rows, int64_t *nnz, int64_t **row_ptr,
                        int32_t **col, double **val, double **d)
{
    if (p->n_facets > 0 || p->form == OR_OSEEN) return -3;
    if (p->form == OR_ELASTIC && p->elem != OR_Q1 && p->elem != OR_Q2S && p->elem != OR_P2T) return -3;
    const int64_t n = or_ndofs(p), ne = p->n_el;
    const int dim = elem_dim(p->elem), npe = elem_npe(p->elem);
    const int m = p->form == OR_ELASTIC ? 3 * npe : npe, mm = m * m;
    const int64_t nt = n + ne * mm; /* triplets: the diagonal, then every element */
    int64_t *trow = malloc(sizeof(int64_t) * nt);
    int32_t *tcol = malloc(sizeof(int32_t) * nt);
    double *tval = malloc(sizeof(double) * nt);
    double *de_all = malloc(sizeof(double) * (ne * m + 1));
    double *dv = calloc((size_t)n, sizeof(double));
    if (!trow || !tcol || !tval || !de_all || !dv) {
        free(trow); free(tcol); free(tval); free(de_all); free(dv);
        return -1;
    }
    int bad = 0;
#pragma omp parallel for num_threads(threads) schedule(static)
    for (int64_t g = 0; g < n; ++g) {
        trow[g] = g;
        tcol[g] = (int32_t)g;
        tval[g] = 0.0;
    }
#pragma omp parallel for num_threads(threads) schedule(dynamic, 256)
    for (int64_t e = 0; e < ne; ++e) {
        double X[20 * 3], Ke[60 * 60], de[60];
        const int32_t *cn = p->conn + e * npe;
        for (int a = 0; a < npe; ++a)
            for (int i = 0; i < dim; ++i) X[dim * a + i] = p->coords[(int64_t)cn[a] * dim + i];
        double det;
        if (p->form == OR_THERMAL) det = or_elem_thermal(p->elem, p->quad, X, p->coef[e], p->source[0], NULL, Ke, de);
        else if (p->form == OR_CAPACITY) { det = or_elem_capacity(p->elem, X, p->coef[e], Ke); memset(de, 0, sizeof de); }
        else det = or_elem_elastic(p->elem, X, p->coef[e], p->nu, p->source, Ke, de);
        if (!(det > 0.0)) {
#pragma omp atomic write
            bad = 1;
        }
        int64_t t = n + e * mm;
        for (int a = 0; a < npe; ++a)
            for (int ci = 0; ci < m / npe; ++ci)
                for (int b = 0; b < npe; ++b)
                    for (int cj = 0; cj < m / npe; ++cj) {
                        const int k = m / npe;
                        trow[t] = k * (int64_t)cn[a] + ci;
                        tcol[t] = (int32_t)(k * (int64_t)cn[b] + cj);
                        tval[t] = Ke[(k * a + ci) * m + k * b + cj];
                        ++t;
                    }
        for (int r = 0; r < m; ++r) de_all[e * m + r] = de[r];
    }
    if (bad) {
        free(trow); free(tcol); free(tval); free(de_all); free(dv);
        return -2;
    }
    /* the load vector in element order, as the serial emission adds it */
    if (p->form != OR_CAPACITY)
        for (int64_t e = 0; e < ne; ++e) {
            const int32_t *cn = p->conn + e * npe;
            const int k = m / npe;
            for (int a = 0; a < npe; ++a)
                for (int ci = 0; ci < k; ++ci) dv[k * (int64_t)cn[a] + ci] += de_all[e * m + k * a + ci];
        }
    free(de_all);
    /* stable counting sort by row: per-thread counts over contiguous chunks */
    int T = threads > 0 ? threads : 1;
    int64_t *cnt = calloc((size_t)T * (size_t)(n + 1), sizeof(int64_t));
    int64_t *rs = calloc((size_t)n + 1, sizeof(int64_t));
    int64_t *perm = malloc(sizeof(int64_t) * nt);
    if (!cnt || !rs || !perm) {
        free(cnt); free(rs); free(perm); free(trow); free(tcol); free(tval); free(dv);
        return -1;
    }
    const int64_t chunk = (nt + T - 1) / T;
#pragma omp parallel for num_threads(T) schedule(static, 1)
    for (int th = 0; th < T; ++th) {
        const int64_t lo = th * chunk, hi = lo + chunk < nt ? lo + chunk : nt;
        int64_t *c = cnt + (size_t)th * (n + 1);
        for (int64_t t = lo; t < hi; ++t) c[trow[t]]++;
    }
    for (int64_t r = 0; r < n; ++r) {
        int64_t s = rs[r];
        for (int th = 0; th < T; ++th) {
            int64_t *c = cnt + (size_t)th * (n + 1);
            const int64_t v = c[r];
            c[r] = s;
            s += v;
        }
        rs[r + 1] = s;
    }
#pragma omp parallel for num_threads(T) schedule(static, 1)
    for (int th = 0; th < T; ++th) {
        const int64_t lo = th * chunk, hi = lo + chunk < nt ? lo + chunk : nt;
        int64_t *c = cnt + (size_t)th * (n + 1);
        for (int64_t t = lo; t < hi; ++t) perm[c[trow[t]]++] = t;
    }
    free(cnt);
    /* per row: stable sort by column, then unique columns with sums in
       emission order */
    int64_t *ucnt = calloc((size_t)n + 1, sizeof(int64_t));
#pragma omp parallel num_threads(T)
    {
        int64_t cap = 1024;
        int64_t *tmp = malloc(sizeof(int64_t) * cap);
#pragma omp for schedule(dynamic, 512)
        for (int64_t r = 0; r < n; ++r) {
            const int64_t lo = rs[r], len = rs[r + 1] - lo;
            if (len > cap) {
                free(tmp);
                cap = len;
                tmp = malloc(sizeof(int64_t) * cap);
            }
            merge_sort_cols(perm + lo, tmp, len, tcol);
            int64_t u = 0;
            for (int64_t t = 0; t < len; ++t)
                if (t == 0 || tcol[perm[lo + t]] != tcol[perm[lo + t - 1]]) ++u;
            ucnt[r + 1] = u;
        }
        free(tmp);
    }
    for (int64_t r = 0; r < n; ++r) ucnt[r + 1] += ucnt[r];
    const int64_t u = ucnt[n];
    int32_t *ci = malloc(sizeof(int32_t) * (u > 0 ? u : 1));
    double *vv = malloc(sizeof(double) * (u > 0 ? u : 1));
#pragma omp parallel for num_threads(T) schedule(dynamic, 512)
    for (int64_t r = 0; r < n; ++r) {
        const int64_t lo = rs[r], len = rs[r + 1] - lo;
        int64_t k = ucnt[r] - 1;
        for (int64_t t = 0; t < len; ++t) {
            const int64_t s = perm[lo + t];
            if (t == 0 || tcol[s] != tcol[perm[lo + t - 1]]) {
                ++k;
                ci[k] = tcol[s];
                vv[k] = 0.0;
            }
            vv[k] += tval[s];
        }
    }
    free(perm); free(rs); free(trow); free(tcol); free(tval);
    *n_rows = n;
    *nnz = u;
    *row_ptr = ucnt;
    *col = ci;
    *val = vv;
    *d = dv;
    return 0;
}

void or_free(void *ptr) { free(ptr); }

/* ------------------------------------------------------------------------ */
/* Strong symmetric Dirichlet elimination (replaces the paper's penalty      */
/* terms h_penalty, tau, tau^b of Sec. 4.1-4.3).  For a constrained dof g:   */
/* row g -> identity, d[g] = value; for every other row i: d[i] -= K[i][g]   */
/* value and K[i][g] = 0.  The pattern is left unchanged (explicit zeros).   */
/* ------------------------------------------------------------------------ */
void or_dirichlet(int64_t n, const int64_t *rp, const int32_t *ci, double *val, double *d,
                  const uint8_t *mask, const double *bval)
{
    for (int64_t i = 0; i < n; ++i) {
        if (mask[i]) continue;
        for (int64_t t = rp[i]; t < rp[i + 1]; ++t) {
            const int32_t j = ci[t];
            if (mask[j]) {
                d[i] -= val[t] * bval[j];
                val[t] = 0.0;
            }
        }
    }
    for (int64_t g = 0; g < n; ++g) {
        if (!mask[g]) continue;
        for (int64_t t = rp[g]; t < rp[g + 1]; ++t) val[t] = (ci[t] == g) ? 1.0 : 0.0;
        d[g] = bval[g];
    }
}

/* ------------------------------------------------------------------------ */
/* Krylov solvers for Block D-4 (the paper leaves the solver open).          */
/* ------------------------------------------------------------------------ */
void or_spmv(int64_t n, const int64_t *rp, const int32_t *ci, const double *val,
             const double *x, double *y)
{
    for (int64_t i = 0; i < n; ++i) {
        double s = 0.0;
        for (int64_t t = rp[i]; t < rp[i + 1]; ++t) s += val[t] * x[ci[t]];
        y[i] = s;
    }
}

static double dotp(int64_t n, const double *a, const double *b)
{
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) s += a[i] * b[i];
    return s;
}

/* Jacobi-preconditioned conjugate gradients from x0 = x (in/out); stops when
 * ||d - K x|| <= tol ||d|| (recursive residual), then reports the true
 * relative residual.  Returns the iteration count, or -1 if maxit is hit. */
int64_t or_pcg(int64_t n, const int64_t *rp, const int32_t *ci, const double *val,
               const double *d, double *x, double tol, int64_t maxit, double *relres)
{
    double *r = malloc(sizeof(double) * n), *z = malloc(sizeof(double) * n);
    double *p = malloc(sizeof(double) * n), *q = malloc(sizeof(double) * n);
    double *dinv = malloc(sizeof(double) * n);
    for (int64_t i = 0; i < n; ++i) {
        double di = 0.0;
        for (int64_t t = rp[i]; t < rp[i + 1]; ++t)
            if (ci[t] == i) di = val[t];
        dinv[i] = 1.0 / di;
    }
    or_spmv(n, rp, ci, val, x, q);
    for (int64_t i = 0; i < n; ++i) r[i] = d[i] - q[i];
    const double dn = sqrt(dotp(n, d, d));
    for (int64_t i = 0; i < n; ++i) z[i] = dinv[i] * r[i];
    memcpy(p, z, sizeof(double) * n);
    double rz = dotp(n, r, z);
    int64_t it = 0, ok = 0;
    if (sqrt(dotp(n, r, r)) <= tol * dn) ok = 1;
    while (!ok && it < maxit) {
        or_spmv(n, rp, ci, val, p, q);
        const double alpha = rz / dotp(n, p, q);
        for (int64_t i = 0; i < n; ++i) {
            x[i] += alpha * p[i];
            r[i] -= alpha * q[i];
        }
        ++it;
        if (sqrt(dotp(n, r, r)) <= tol * dn) { ok = 1; break; }
        for (int64_t i = 0; i < n; ++i) z[i] = dinv[i] * r[i];
        const double rz1 = dotp(n, r, z);
        const double beta = rz1 / rz;
        rz = rz1;
        for (int64_t i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];
    }
    or_spmv(n, rp, ci, val, x, q);
    for (int64_t i = 0; i < n; ++i) r[i] = d[i] - q[i];
    *relres = sqrt(dotp(n, r, r)) / dn;
    free(r); free(z); free(p); free(q); free(dinv);
    return ok ? it : -1;
}

/* Restarted GMRES(m), right preconditioned by the diagonal pdiag
 * (K P^{-1} y = d, x = P^{-1} y), modified Gram-Schmidt Arnoldi, Givens
 * rotations on the Hessenberg matrix.  x in/out; stops when the true
 * relative residual ||d - K x|| / ||d|| (equal to the Arnoldi estimate)
 * drops to tol.  Returns the total inner iteration count or -1. */
int64_t or_gmres(int64_t n, const int64_t *rp, const int32_t *ci, const double *val,
                 const double *d, double *x, const double *pdiag, int m, double tol,
                 int64_t maxit, double *relres)
{
    double *V = malloc(sizeof(double) * n * (m + 1));
    double *H = calloc((size_t)(m + 1) * m, sizeof(double));
    double *cs = malloc(sizeof(double) * m), *sn = malloc(sizeof(double) * m);
    double *s = malloc(sizeof(double) * (m + 1)), *y = malloc(sizeof(double) * m);
    double *w = malloc(sizeof(double) * n), *z = malloc(sizeof(double) * n);
    const double dn = sqrt(dotp(n, d, d));
    int64_t it = 0;
    int ok = 0;
    while (!ok && it < maxit) {
        or_spmv(n, rp, ci, val, x, w);
        for (int64_t i = 0; i < n; ++i) V[i] = d[i] - w[i];
        double beta = sqrt(dotp(n, V, V));
        if (beta <= tol * dn) { ok = 1; break; }
        for (int64_t i = 0; i < n; ++i) V[i] /= beta;
        memset(s, 0, sizeof(double) * (m + 1));
        s[0] = beta;
        int j = 0;
        for (; j < m && it < maxit; ++j) {
            double *vj = V + (int64_t)j * n, *vn = V + (int64_t)(j + 1) * n;
            for (int64_t i = 0; i < n; ++i) z[i] = vj[i] / pdiag[i];
            or_spmv(n, rp, ci, val, z, vn);
            for (int k = 0; k <= j; ++k) {
                const double h = dotp(n, vn, V + (int64_t)k * n);
                H[k * m + j] = h;
                for (int64_t i = 0; i < n; ++i) vn[i] -= h * V[(int64_t)k * n + i];
            }
            const double hn = sqrt(dotp(n, vn, vn));
            H[(j + 1) * m + j] = hn;
            if (hn > 0.0)
                for (int64_t i = 0; i < n; ++i) vn[i] /= hn;
            for (int k = 0; k < j; ++k) {
                const double a = H[k * m + j], b = H[(k + 1) * m + j];
                H[k * m + j] = cs[k] * a + sn[k] * b;
                H[(k + 1) * m + j] = -sn[k] * a + cs[k] * b;
            }
            const double a = H[j * m + j], b = H[(j + 1) * m + j];
            const double rr = sqrt(a * a + b * b);
            cs[j] = a / rr;
            sn[j] = b / rr;
            H[j * m + j] = rr;
            H[(j + 1) * m + j] = 0.0;
            s[j + 1] = -sn[j] * s[j];
            s[j] = cs[j] * s[j];
            ++it;
            if (fabs(s[j + 1]) <= tol * dn) { ++j; ok = 1; break; }
        }
        /* back substitution H y = s, then x += P^{-1} V y */
        for (int k = j - 1; k >= 0; --k) {
            double t = s[k];
            for (int l = k + 1; l < j; ++l) t -= H[k * m + l] * y[l];
            y[k] = t / H[k * m + k];
        }
        for (int64_t i = 0; i < n; ++i) {
            double t = 0.0;
            for (int k = 0; k < j; ++k) t += V[(int64_t)k * n + i] * y[k];
            x[i] += t / pdiag[i];
        }
        if (ok) {
            /* confirm with the true residual */
            or_spmv(n, rp, ci, val, x, w);
            for (int64_t i = 0; i < n; ++i) w[i] = d[i] - w[i];
            if (sqrt(dotp(n, w, w)) > tol * dn) ok = 0;
        }
    }
    or_spmv(n, rp, ci, val, x, w);
    for (int64_t i = 0; i < n; ++i) w[i] = d[i] - w[i];
    *relres = sqrt(dotp(n, w, w)) / dn;
    free(V); free(H); free(cs); free(sn); free(s); free(y); free(w); free(z);
    return ok ? it : -1;
}

/* ------------------------------------------------------------------------ */
/* 3x3x3 convolution layers of the learned preconditioner correction       */
/* (growth line of the hot path; not in the paper).  Channels-last grids    */
/* [nz][ny][nx][c], zero padding outside the grid, weights [co][ci][27]     */
/* with offset index o = (dz+1)*9 + (dy+1)*3 + (dx+1):                      */
/*   out[v][co] = b[co] + sum_ci sum_o w[co][ci][o] in[v + off(o)][ci].     */
/* ------------------------------------------------------------------------ */
static int in_grid(int64_t z, int64_t y, int64_t x, int64_t nz, int64_t ny, int64_t nx)
{
    return z >= 0 && z < nz && y >= 0 && y < ny && x >= 0 && x < nx;
}

void or_conv3d_fwd(int64_t nz, int64_t ny, int64_t nx, int ci_n, int co_n, const double *in, const double *w,
                   const double *b, int relu, double *out)
{
    for (int64_t z = 0; z < nz; ++z)
        for (int64_t y = 0; y < ny; ++y)
            for (int64_t x = 0; x < nx; ++x) {
                const int64_t v = (z * ny + y) * nx + x;
                for (int co = 0; co < co_n; ++co) {
                    double s = b ? b[co] : 0.0;
                    for (int ci = 0; ci < ci_n; ++ci)
                        for (int o = 0; o < 27; ++o) {
                            const int dz = o / 9 - 1, dy = (o / 3) % 3 - 1, dx = o % 3 - 1;
                            if (!in_grid(z + dz, y + dy, x + dx, nz, ny, nx)) continue;
                            const int64_t u = ((z + dz) * ny + (y + dy)) * nx + (x + dx);
                            s += w[((int64_t)co * ci_n + ci) * 27 + o] * in[u * ci_n + ci];
                        }
                    out[v * co_n + co] = (relu && s < 0.0) ? 0.0 : s;
                }
            }
}

/* gin[u][ci] = sum over (v, o) with u = v + off(o) of w[co][ci][o] gout[v][co] */
void or_conv3d_bwd_data(int64_t nz, int64_t ny, int64_t nx, int ci_n, int co_n, const double *gout,
                        const double *w, double *gin)
{
    const int64_t nv = nz * ny * nx;
    for (int64_t i = 0; i < nv * ci_n; ++i) gin[i] = 0.0;
    for (int64_t z = 0; z < nz; ++z)
        for (int64_t y = 0; y < ny; ++y)
            for (int64_t x = 0; x < nx; ++x) {
                const int64_t v = (z * ny + y) * nx + x;
                for (int co = 0; co < co_n; ++co)
                    for (int ci = 0; ci < ci_n; ++ci)
                        for (int o = 0; o < 27; ++o) {
                            const int dz = o / 9 - 1, dy = (o / 3) % 3 - 1, dx = o % 3 - 1;
                            if (!in_grid(z + dz, y + dy, x + dx, nz, ny, nx)) continue;
                            const int64_t u = ((z + dz) * ny + (y + dy)) * nx + (x + dx);
                            gin[u * ci_n + ci] += w[((int64_t)co * ci_n + ci) * 27 + o] * gout[v * co_n + co];
                        }
            }
}

/* gw[co][ci][o] = sum_v gout[v][co] in[v + off(o)][ci];  gb[co] = sum_v gout[v][co] */
void or_conv3d_bwd_weight(int64_t nz, int64_t ny, int64_t nx, int ci_n, int co_n, const double *in,
                          const double *gout, double *gw, double *gb)
{
    for (int64_t i = 0; i < (int64_t)co_n * ci_n * 27; ++i) gw[i] = 0.0;
    for (int co = 0; co < co_n; ++co) gb[co] = 0.0;
    for (int64_t z = 0; z < nz; ++z)
        for (int64_t y = 0; y < ny; ++y)
            for (int64_t x = 0; x < nx; ++x) {
                const int64_t v = (z * ny + y) * nx + x;
                for (int co = 0; co < co_n; ++co) {
                    gb[co] += gout[v * co_n + co];
                    for (int ci = 0; ci < ci_n; ++ci)
                        for (int o = 0; o < 27; ++o) {
                            const int dz = o / 9 - 1, dy = (o / 3) % 3 - 1, dx = o % 3 - 1;
                            if (!in_grid(z + dz, y + dy, x + dx, nz, ny, nx)) continue;
                            const int64_t u = ((z + dz) * ny + (y + dy)) * nx + (x + dx);
                            gw[((int64_t)co * ci_n + ci) * 27 + o] += gout[v * co_n + co] * in[u * ci_n + ci];
                        }
                }
            }
}

/* ------------------------------------------------------------------------ */
/* Generalised-alpha time stepping (Sec. 2.1, Eq. time_constraints and       */
/* time_effective; Blocks C and D of Sec. 2.2) of the linear conduction      */
/* system, maximum derivative order 2: per dof the basic value phi, its rate */
/* u and its second rate a.  The residual of the form (tangent negated, as   */
/* K and M here are the positive matrices) at the effective values is        */
/*   d = F - K phi~ - M u~        (zero on Dirichlet rows),                  */
/* and the tangent of Block D-3 is T = c1 K + c2 / (b1 dt) M.  K and M share */
/* the CSR pattern (rp, ci).  Dirichlet dofs keep phi = bval, u = a = 0.     */
/* Per time step:                                                            */
/*  C-1  phi += dphi, u += du, a += da (last step's increments);             */
/*  C-2  da = 0;                                                             */
/*  C-3  the increments that satisfy the constraints with da = 0:            */
/*       du = dt (a + b2 da), dphi = dt (u + b1 du);                         */
/*  D-1  phi~ = phi + c1 dphi, u~ = u + c2 du, a~ = a + c3 da;               */
/*  D-2  d; stop when ||d|| <= newton_tol ||d_0|| (d_0: the step's first),  */
/*       or ||d|| <= 1e-13 (||F|| + ||K phi~|| + ||M u~||), the level below  */
/*       which rounding decides d;                                           */
/* With radiation facets (rad != NULL, Sec. 4.1 e_m sigma^b (T, T_env^4 -   */
/* T^4)), F becomes F + R(phi~) (in the rounding floor too) and the tangent  */
/* gains c1 times the radiation tangent 4 e_m sigma^b int N_a N_b T~^3.      */
/*  D-3/4  T x = d by Jacobi-PCG, dphi += x, and du, da from the             */
/*       constraints: du = (dphi / dt - u) / b1, da = (du / dt - a) / b2.    */
/* After the last step the increments are applied (C-1), so phi, u, a hold   */
/* the values at t = steps dt.  newton_its[m] (may be NULL) counts the       */
/* solves of step m.  Returns 0, or -1 if a step hit max_newton without      */
/* converging, -4 on allocation failure.                                     */
/* ------------------------------------------------------------------------ */
/* Radiation facets of a thermal mesh for or_genalpha (may be absent). */
typedef struct {
    int elem, dim, npe;
    const double *coords;
    const int32_t *conn;
    int64_t n_facets;
    const int32_t *f_elem;
    const uint8_t *f_face;
    const double *es;    /* [n_facets] e_m sigma^b */
    const double *tenv;  /* [n_facets] */
} or_radiation;

/* Adds the radiation loads at temperatures T to Fe (all rows) and, with
 * Tv != NULL, scale times the radiation tangent into the CSR values Tv. */
static void radiation_terms(const or_radiation *rd, const int64_t *rp, const int32_t *ci, const double *T,
                            double *Fe, double *Tv, double scale)
{
    for (int64_t f = 0; f < rd->n_facets; ++f) {
        int loc[8];
        const int nf = or_facet_nodes(rd->elem, rd->f_face[f], loc);
        int64_t node[8];
        double Xf[24], Tf[8], Kf[64], rf[8];
        for (int m = 0; m < nf; ++m) {
            node[m] = rd->conn[(int64_t)rd->f_elem[f] * rd->npe + loc[m]];
            Tf[m] = T[node[m]];
            for (int i = 0; i < rd->dim; ++i) Xf[rd->dim * m + i] = rd->coords[node[m] * rd->dim + i];
        }
        or_facet_radiation(rd->elem, Xf, rd->es[f], rd->tenv[f], Tf, Kf, rf);
        for (int a = 0; a < nf; ++a) {
            Fe[node[a]] += rf[a];
            if (!Tv) continue;
            for (int b = 0; b < nf; ++b)
                for (int64_t t = rp[node[a]]; t < rp[node[a] + 1]; ++t)
                    if (ci[t] == node[b]) Tv[t] += scale * Kf[a * nf + b];
        }
    }
}

int or_genalpha(int64_t n, const int64_t *rp, const int32_t *ci, const double *Kv, const double *Mv,
                const double *F, const uint8_t *mask, const double *bval, double *phi, double *u, double *a,
                double b1, double b2, double c1, double c2, double c3, double dt, int64_t steps,
                double newton_tol, int max_newton, double pcg_tol, int64_t *newton_its, const or_radiation *rad)
{
    const int64_t nnz = rp[n];
    double *dphi = calloc((size_t)n, sizeof(double)), *du = calloc((size_t)n, sizeof(double));
    double *da = calloc((size_t)n, sizeof(double)), *pt = malloc(sizeof(double) * n);
    double *ut = malloc(sizeof(double) * n), *d = malloc(sizeof(double) * n), *x = malloc(sizeof(double) * n);
    double *Tv = malloc(sizeof(double) * nnz), *zero = calloc((size_t)n, sizeof(double));
    double *y = malloc(sizeof(double) * n), *Fe = malloc(sizeof(double) * n);
    if (!dphi || !du || !da || !pt || !ut || !d || !x || !Tv || !zero || !y || !Fe) {
        free(dphi); free(du); free(da); free(pt); free(ut); free(d); free(x); free(Tv); free(zero); free(y);
        free(Fe);
        return -4;
    }
    int rc = 0;
    for (int64_t i = 0; i < n; ++i)
        if (mask[i]) { phi[i] = bval[i]; u[i] = 0.0; a[i] = 0.0; }
    for (int64_t m = 0; m < steps; ++m) {
        for (int64_t i = 0; i < n; ++i) {          /* C-1 */
            phi[i] += dphi[i];
            u[i] += du[i];
            a[i] += da[i];
        }
        for (int64_t i = 0; i < n; ++i) {          /* C-2, C-3 */
            da[i] = 0.0;
            du[i] = mask[i] ? 0.0 : dt * (a[i] + b2 * da[i]);
            dphi[i] = mask[i] ? 0.0 : dt * (u[i] + b1 * du[i]);
        }
        double d0 = -1.0;
        int it = 0;
        for (;;) {
            for (int64_t i = 0; i < n; ++i) {      /* D-1 */
                pt[i] = phi[i] + c1 * dphi[i];
                ut[i] = u[i] + c2 * du[i];
            }
            for (int64_t i = 0; i < n; ++i) Fe[i] = F[i];  /* D-2: loads incl. radiation at phi~ */
            if (rad) radiation_terms(rad, rp, ci, pt, Fe, NULL, 0.0);
            or_spmv(n, rp, ci, Kv, pt, d);
            or_spmv(n, rp, ci, Mv, ut, y);
            double r2 = 0.0, f2 = 0.0, k2 = 0.0, m2 = 0.0;
            for (int64_t i = 0; i < n; ++i) {
                if (!mask[i]) {
                    f2 += Fe[i] * Fe[i];
                    k2 += d[i] * d[i];
                    m2 += y[i] * y[i];
                }
                d[i] = mask[i] ? 0.0 : Fe[i] - d[i] - y[i];
                r2 += d[i] * d[i];
            }
            const double r = sqrt(r2);
            if (d0 < 0.0) d0 = r;
            /* converged: reduced by newton_tol, or at the rounding floor of
             * its three terms */
            if (r <= newton_tol * d0 || r <= 1e-13 * (sqrt(f2) + sqrt(k2) + sqrt(m2))) break;
            if (it == max_newton) { rc = -1; break; }
            const double s = c2 / (b1 * dt);       /* D-3 */
            for (int64_t t = 0; t < nnz; ++t) Tv[t] = c1 * Kv[t] + s * Mv[t];
            if (rad) radiation_terms(rad, rp, ci, pt, y, Tv, c1);  /* y: scratch */
            or_dirichlet(n, rp, ci, Tv, d, mask, zero);
            for (int64_t i = 0; i < n; ++i) x[i] = 0.0;
            double rr;
            or_pcg(n, rp, ci, Tv, d, x, pcg_tol, 100000, &rr);
            for (int64_t i = 0; i < n; ++i) {      /* increments from the constraints */
                if (mask[i]) continue;
                dphi[i] += x[i];
                du[i] = (dphi[i] / dt - u[i]) / b1;
                da[i] = (du[i] / dt - a[i]) / b2;
            }
            ++it;
        }
        if (newton_its) newton_its[m] = it;
        if (rc) break;
    }
    for (int64_t i = 0; i < n; ++i) {              /* C-1 of the next step */
        phi[i] += dphi[i];
        u[i] += du[i];
        a[i] += da[i];
    }
    free(dphi); free(du); free(da); free(pt); free(ut); free(d); free(x); free(Tv); free(zero); free(y);
    free(Fe);
    return rc;
}
