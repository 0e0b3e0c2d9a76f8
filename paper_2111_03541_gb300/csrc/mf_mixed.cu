// Mixed-precision element contraction of Q1 elasticity (tensor cores).
#include "mf_internal.h"

mf_status mf_assemble_mixed(int form, const mf_mesh *m, const mf_pattern *p, const mf_coeffs *c, double *values,
                            double *d, cudaStream_t st)
{
    (void)form; (void)m; (void)p; (void)c; (void)values; (void)d; (void)st;
    return mf_fail(MF_ERR_UNSUPPORTED, "mf_assemble: mixed path not built");
}
