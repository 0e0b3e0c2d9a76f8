// Host check of the kernels' double-float arithmetic (mf_fem.cuh) against FP64:
// prints the largest errors; the test asserts the bounds.
#include <cstdio>
#include <cmath>
#include <random>
#include "mf_fem.cuh"
static double jac_fp64(const double (&c)[8][3], double xs, double ys, double zs, double (&Ji)[3][3]) {
    double J[3][3];
    for (int i = 0; i < 3; ++i) {
        J[i][0] = zs * (ys * c[7][i] + c[5][i]) + (ys * c[3][i] + c[1][i]);
        J[i][1] = zs * (xs * c[7][i] + c[6][i]) + (xs * c[3][i] + c[2][i]);
        J[i][2] = ys * (xs * c[7][i] + c[6][i]) + (xs * c[5][i] + c[4][i]);
    }
    double c00 = J[1][1]*J[2][2]-J[1][2]*J[2][1], c01 = J[1][2]*J[2][0]-J[1][0]*J[2][2], c02 = J[1][0]*J[2][1]-J[1][1]*J[2][0];
    double det = J[0][0]*c00 + J[0][1]*c01 + J[0][2]*c02, r = 1.0/det;
    Ji[0][0]=c00*r; Ji[1][0]=c01*r; Ji[2][0]=c02*r;
    Ji[0][1]=(J[0][2]*J[2][1]-J[0][1]*J[2][2])*r; Ji[1][1]=(J[0][0]*J[2][2]-J[0][2]*J[2][0])*r; Ji[2][1]=(J[0][1]*J[2][0]-J[0][0]*J[2][1])*r;
    Ji[0][2]=(J[0][1]*J[1][2]-J[0][2]*J[1][1])*r; Ji[1][2]=(J[0][2]*J[1][0]-J[0][0]*J[1][2])*r; Ji[2][2]=(J[0][0]*J[1][1]-J[0][1]*J[1][0])*r;
    return det;
}
int main() {
    std::mt19937_64 rng(7);
    std::uniform_real_distribution<double> U(-1, 1);
    double emax_M = 0, emax_w = 0;
    for (int trial = 0; trial < 2000; ++trial) {
        const double h = (trial % 3 == 0) ? 1.0 / 48 : (trial % 3 == 1 ? 1.0 : 1.0 / 512);
        double x[8][3];
        for (int a = 0; a < 8; ++a) for (int i = 0; i < 3; ++i)
            x[a][i] = h * (((a >> i) & 1) + 0.15 * U(rng)) + 0.37 + 3.0 * (trial % 7);
        double c[8][3]; float2 cf[8][3];
        for (int S = 0; S < 8; ++S) for (int i = 0; i < 3; ++i) {
            double v = 0; for (int a = 0; a < 8; ++a) v += (__builtin_popcount(a & S) & 1) ? -x[a][i] : x[a][i];
            c[S][i] = v * ((__builtin_popcount(S) & 1) ? -0.125 : 0.125);
            float hi = (float)c[S][i]; cf[S][i] = make_float2(hi, (float)(c[S][i] - (double)hi));
        }
        for (int q = 0; q < 27; ++q) {
            const double g3 = 0.77459666924148337704;
            int qi = q % 3, qj = (q / 3) % 3, qk = q / 9;
            double Ji[3][3];
            double det = jac_fp64(c, (qi - 1) * g3, (qj - 1) * g3, (qk - 1) * g3, Ji);
            double w = (qi == 1 ? 8.0/9 : 5.0/9) * (qj == 1 ? 8.0/9 : 5.0/9) * (qk == 1 ? 8.0/9 : 5.0/9);
            double wd = w * det, sw = sqrt(wd);
            float2 M9[9];
            float2 wdf = q2s_point_df(cf, q, M9);
            emax_w = fmax(emax_w, fabs(df_to_double(wdf) - wd) / wd);
            double mmax = 0; for (int i = 0; i < 3; ++i) for (int j = 0; j < 3; ++j) mmax = fmax(mmax, fabs(sw * Ji[j][i]));
            for (int i = 0; i < 3; ++i) for (int j = 0; j < 3; ++j)
                emax_M = fmax(emax_M, fabs(df_to_double(M9[3*i+j]) - sw * Ji[j][i]) / mmax);
        }
    }
    printf("geometry: max rel err w detJ %.3e, sqrt(w detJ) J^-T (row of 9 scaled) %.3e\n", emax_w, emax_M);
    double er = 0, es = 0, ec = 0;
    for (int t = 0; t < 100000; ++t) {
        double v = exp(40 * U(rng)) * (U(rng) > 0 ? 1 : -1);
        float hi = (float)v; float2 a = make_float2(hi, (float)(v - hi));
        double av = (double)a.x + (double)a.y;
        er = fmax(er, fabs(df_to_double(df_recip(a)) * av - 1.0));
        double p = fabs(av); float2 ap = make_float2(fabs(a.x), a.x < 0 ? -a.y : a.y);
        es = fmax(es, fabs(df_to_double(df_sqrt(ap)) / sqrt(p) - 1.0));
        float f = (float)v; if (f32_to_f64_exact(f) != (double)f) ec += 1;
    }
    float specials[] = {0.0f, -0.0f, INFINITY, -INFINITY, 1e-30f, -3.5e37f, 1.17549435e-38f};
    for (float f : specials) if (f32_to_f64_exact(f) != (double)f) { printf("special mismatch %g\n", f); ec += 1; }
    printf("recip max rel err %.3e, sqrt %.3e, exact conversion mismatches %.0f\n", er, es, ec);
    return 0;
}
