// Internal declarations of the mf library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/mf.h"
#include "mf_device.cuh"

#define MF_MAX_DEG 64   // neighbours of one node in one adjacency
#define MF_MAX_DEG_HO 128  // the same for the 20-node serendipity brick
#define MF_SLABS 1      // element chunks of the mixed elasticity assembly (see plan_slabs)
#define MF_MAX_INC 32   // elements incident to one node

// Adjacency between a row node space and a column node space (Block B-1: the
// unique control-point pairs).
struct mf_adj {
    int64_t n_rows = 0;      // row nodes
    int64_t n_pairs = 0;     // unique (row node, col node) pairs
    int64_t *ptr = nullptr;  // [n_rows + 1]
    int32_t *col = nullptr;  // [n_pairs] ascending per row
    int32_t max_deg = 0;     // largest row (set where a kernel sizes shared memory by it)
};

struct mf_mesh {
    int dim, elem, npe;
    int64_t n_nodes, n_elems, n_pnodes;
    const double *coords;
    const int32_t *conn;
    const int32_t *pconn;
    int device;
};

// reference entries of a rectangular Q1 cell by corner class (see
// mf_pattern::box): conduction k_cls, capacity m_cls, load per corner dref
struct mf_box_classes {
    double k_cls[8];
    double m_cls[8];
    double dref;
};

struct mf_pattern {
    int form;
    const mf_mesh *mesh;
    int64_t n_rows = 0, nnz = 0;
    int64_t *row_ptr = nullptr;
    int32_t *col_idx = nullptr;
    // adjacencies: [0] row space x row space; flow adds [1] P2 rows x P1
    // cols and [2] P1 rows x P2 cols
    mf_adj adj[4];
    int n_adj = 0;
    // element-matrix scratch of the FP64 path (doubles per element x n_elems)
    double *scratch = nullptr;
    int64_t scratch_stride = 0;
    // incident elements per row node (ascending), for the mixed path
    int64_t *inc_ptr = nullptr;
    int32_t *inc = nullptr;
    uint8_t *inc_loc = nullptr;  // position of the node in each incident element (thermal
                                 // Q1: bit 7 set when the element is a translate)
    // flow: elements incident to each P1 pressure node, ascending, with the
    // node's local index (0..2) in each
    int64_t *pinc_ptr = nullptr;
    int32_t *pinc = nullptr;
    uint8_t *pinc_loc = nullptr;
    // flow slot maps per incidence entry: P2 row x the element's P2 nodes
    // (inc_slot, 6 per entry), P2 row x its P1 nodes (inc_slot_pq, 3), P1 row
    // x its P2 nodes (pinc_slot, 6)
    uint8_t *inc_slot_pq = nullptr, *pinc_slot = nullptr;
    // Navier-Stokes: P1 row x the element's P1 nodes (pinc_slot_pp, 3 per
    // entry) in adj[3] (P1 rows x P1 columns)
    uint8_t *pinc_slot_pp = nullptr;
    // elasticity: slot[e][a][b] = position of node conn[e][b] among the sorted
    // neighbours of node conn[e][a] (u8, n_elems x 64)
    uint8_t *slot = nullptr;
    // thermal: inc_slot[t][b] = the same position for incidence entry t of a
    // node (element inc[t], local index inc_loc[t]) (u8, n_elems x npe x npe);
    // elem_inc[e][a] = the incidence entry of (e, a): the scratch holds row a
    // of K_e and d_e[a] there ((npe + 1) doubles per entry)
    uint8_t *inc_slot = nullptr;
    int32_t *elem_inc = nullptr;
    // thermal Q1: tr[e] = 1 when element e is an exact translate of element 0
    // (equal edge vectors x_a - x_0 in FP64), so K_e = k_e Kref and
    // d_e = f dref with kref = [Kref (8 x 8), dref (8)] element 0's unit-k,
    // unit-f matrices, then [1.0], then [Mref (8 x 8), 0 (8)] its unit-C
    // capacity matrix at kref + 73; null when no element is a translate
    uint8_t *tr = nullptr;
    double *kref = nullptr;
    int64_t n_translate = 0;
    // the same reference entries as FP32 pairs (hi, lo), the translates'
    // coefficients as pairs (written per assembly), and per node a flag set
    // per assembly when the node or a neighbour is constrained (thermal Q1
    // with translates; for the flow forms bcrow is the same flag per CSR
    // row: the row or one of its columns constrained; for Q1 elasticity per
    // node: one of its dofs or a neighbour's constrained)
    float2 *kref_df = nullptr;
    float2 *kc_df = nullptr;
    uint8_t *bcrow = nullptr;
    // thermal Q1 whose elements are all translates of one rectangular cell,
    // numbered as a lexicographic box (node (x, y, z) = x + nx1 (y + ny1 z),
    // the element whose lowest node that is, x fastest): box = {nx1, ny1,
    // nz1} (else zeros) and the reference entries by class, i.e. by the axes
    // in which two corners differ (mask dx | dy << 1 | dz << 2)
    int32_t box[3] = {0, 0, 0};
    mf_box_classes box_cls{};
    // 20-node bricks: the vertices' trilinear-map coefficients of q1_jac_at
    // per element as FP32 pairs (hi, lo), [n_elems][8][3]
    float2 *q2s_map = nullptr;
    // elasticity, mixed path: int64 3x3 block accumulator per upper node pair
    // (n, m >= n; a diagonal block as its upper triangle), numbered compactly:
    // upper pair (n, slot k) is block cbase[n] + k; tpos gives, for a lower
    // pair (n, m < n), the number of the upper pair (m, n), and for an upper
    // pair its own number: the block every CSR block of n reads
    long long *kacc = nullptr;
    int32_t *tpos = nullptr;
    // the accumulator block of each upper block pair (a <= b) of every element
    // (bit 31: the pair is stored transposed), [n_elems][36]
    int32_t *etgt = nullptr;
    int64_t *cbase = nullptr;
    int64_t n_upper = 0;
    long long *dacc = nullptr;  // int64 load vector accumulator (3 per node)
    // mixed path: device scalars of the fixed-point scale (see mf_mixed.cu)
    void *mixed_state = nullptr;
    // elasticity slabs: element chunk c = [slab_e[c], slab_e[c+1]) completes the
    // rows of nodes [slab_n[c], slab_n[c+1]); assembling chunk by chunk keeps the
    // element scratch of the gather in L2
    std::vector<int64_t> slab_e, slab_n;
    // with more than one chunk, the gather of chunk k runs on `side` while
    // chunk k + 1 is computed on the caller's stream (forked and joined by
    // events, so the pair can be captured in a CUDA graph)
    cudaStream_t side = nullptr;
    cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
    std::vector<cudaEvent_t> slab_ev;
    // mixed path: the accumulator clears run on clr_side beside the bound
    // pass (forked and joined by events, capturable in a CUDA graph)
    cudaStream_t clr_side = nullptr;
    cudaEvent_t clr_fork = nullptr, clr_join = nullptr;
};

// Boundary facets of a mesh for one pattern (thermal or elasticity form): the
// facets incident to every boundary node, ascending, as a CSR over the
// boundary nodes.
struct mf_facets {
    const mf_mesh *mesh = nullptr;
    const mf_pattern *pattern = nullptr;
    int npf = 0;                 // nodes per facet: 2 (P1 edge), 3 (P2 edge), 4 (Q1 face)
    int64_t n_facets = 0;
    int32_t *fnode = nullptr;    // [n_facets][npf] global nodes in facet node order
    uint8_t *fface = nullptr;    // [n_facets] local face of the parent element
    int64_t n_bnodes = 0;
    int32_t *bnode = nullptr;    // [n_bnodes] nodes on some facet, ascending
    int64_t *bptr = nullptr;     // [n_bnodes + 1] offsets into binc / bloc
    int32_t *binc = nullptr;     // incident facets of each boundary node, ascending
    uint8_t *bloc = nullptr;     // the node's index within each incident facet
    uint8_t *bslot = nullptr;    // thermal: [entry][npf] position of facet node m' in the node's row
    int32_t *bcol = nullptr;     // thermal: [entry][npf] facet node m' (the column)
    int64_t *brow = nullptr;     // thermal: [n_bnodes] start of the node's CSR row
    double *bgeo = nullptr;      // facet geometry per entry: thermal [entry][npf + 1] unit-h convection
                                 // row and load factor; elasticity [entry][3] oriented area moment
    double *bwq = nullptr;       // thermal: [entry][nq] w_q |J_q| N_m(q) at the facet rule's points
};

// status word (device) of the current device
int *mf_status_word();
mf_status mf_fail(mf_status s, const char *fmt, ...);
mf_status mf_cuda_check(cudaError_t e, const char *what);
// clears the calling thread's error message (entry points start with it)
void mf_clear_error();
// a CSR system with rows, entries and all three arrays
bool mf_csr_ok(const mf_csr *K);

// exclusive scan of n int64 counts in place; total written to *d_total (device)
cudaError_t mf_scan_i64(int64_t *d_data, int64_t n, int64_t *d_total, cudaStream_t st);

static inline int mf_npe(int elem)
{
    return elem == MF_P1_TRI ? 3
         : elem == MF_P2_TRI ? 6
         : (elem == MF_Q1_HEX || elem == MF_Q2S_QUAD) ? 8
         : elem == MF_Q2S_HEX ? 20 : 10;
}
static inline int mf_ndim(int elem) { return (elem == MF_Q1_HEX || elem == MF_Q2S_HEX || elem == MF_P2_TET) ? 3 : 2; }
// 8-byte words per incidence row of the thermal scratch: row a of K_e, then
// d_e[a]; the 10-node tetrahedron's rows are padded to 12 words (96 bytes,
// three whole 32-byte sectors), so that no sector holds parts of rows that
// different elements write at different times
__host__ __device__ constexpr int mf_th_rs(int npe) { return npe == 10 ? 12 : npe + 1; }

// pattern / assembly entry points implemented in the .cu files
mf_status mf_pattern_build_impl(const mf_mesh *m, int form, cudaStream_t st, mf_pattern *p);
void mf_pattern_free(mf_pattern *p);
mf_status mf_mesh_validate(const mf_mesh *m, cudaStream_t st);
mf_status mf_assemble_fp64(int form, const mf_mesh *m, const mf_pattern *p, const mf_coeffs *c,
                           double *values, double *d, cudaStream_t st);
mf_status mf_assemble_mixed(int form, const mf_mesh *m, const mf_pattern *p, const mf_coeffs *c,
                            double *values, double *d, cudaStream_t st);
// Navier-Stokes with SUPG (mf_ns.cu): tangent and d = -r at the state c->advect
mf_status mf_assemble_ns(const mf_mesh *m, const mf_pattern *p, const mf_coeffs *c, double *values, double *d,
                         cudaStream_t st);
mf_status mf_ns_newton_impl(const mf_mesh *m, const mf_pattern *p, const mf_coeffs *coeffs, double *x,
                            double newton_tol, int32_t max_newton, const mf_solver_opts *lin, double *hist,
                            int32_t *n_steps, cudaStream_t st);
mf_status mf_flow_precond_impl(const mf_mesh *m, const mf_pattern *p, const mf_csr *K, const uint8_t *mask,
                               double p_scale, double *out, cudaStream_t st);
// elasticity gather: FP64 sums of element blocks, or (fixed_point) exact int64
// sums of the mixed path's A'' blocks finished as K = fp A + fq (A^T + I tr A)
// reference sums of the P2 integrands (flow form, P2 thermal) and the 20-node
// brick's reference table, in the current device's copies of mf_assemble.cu
// (once per such pattern build)
mf_status mf_flow_consts_upload();
void mf_launch_gather_elastic(bool fixed_point, int fp, int fq, int64_t n0, int64_t n1, const mf_mesh *m,
                              const mf_pattern *p, const mf_coeffs *c, double *values, double *d, cudaStream_t st);
mf_status mf_facets_create_impl(const mf_mesh *m, const mf_pattern *p, int64_t n_facets, const int32_t *elem,
                                const uint8_t *face, cudaStream_t st, mf_facets *f);
void mf_facets_free(mf_facets *f);
// radiation terms of a thermal facet set at nodal temperatures T (mf_boundary.cu)
mf_status mf_radiation_load(const mf_facets *f, const double *es, const double *tenv, const double *T,
                            const uint8_t *mask, double *R, cudaStream_t st);
mf_status mf_radiation_tangent(const mf_facets *f, const double *es, const double *T, const uint8_t *mask,
                               double scale, double *values, cudaStream_t st);
mf_status mf_assemble_boundary_impl(const mf_facets *f, const mf_facet_coeffs *c, double *values, double *d,
                                    cudaStream_t st);
mf_status mf_genalpha_params_from_rho_impl(double rho, mf_genalpha_params *out);
mf_status mf_genalpha_run_impl(const mf_csr *K, const double *Mv, const double *F, const uint8_t *mask,
                               const double *bval, const mf_facets *rad, const double *rad_es,
                               const double *rad_tenv, double *phi, double *u, double *a, const mf_genalpha_params *prm,
                               double dt, int64_t steps, double newton_tol, int32_t max_newton, double pcg_tol,
                               int64_t pcg_max_iter, int64_t *newton_its, int64_t *pcg_its, cudaStream_t st);
mf_status mf_genalpha_initial_rate_impl(const mf_csr *K, const double *Mv, const double *F, const uint8_t *mask,
                                        const mf_facets *rad, const double *rad_es, const double *rad_tenv,
                                        const double *phi, double *u, double pcg_tol, int64_t pcg_max_iter,
                                        cudaStream_t st);
mf_status mf_pmass_impl(const mf_mesh *m, const mf_pattern *p, double *out, cudaStream_t st);
mf_status mf_solve_impl(const mf_csr *K, const double *d, double *x, const mf_solver_opts *o,
                        mf_solve_info *info, cudaStream_t st);
mf_status mf_spmv_impl(const mf_csr *K, const double *x, double *y, cudaStream_t st);
mf_status mf_flow_mg_create_impl(int levels, const mf_csr *const *K, const int64_t *cells,
                                 const uint8_t *const *bc_mask, const double *pmass, double visc, cudaStream_t st,
                                 mf_flow_mg **out);
void mf_flow_mg_destroy_impl(mf_flow_mg *G);

// kernel timing (tracing): bracket a launch on stream st with events when enabled
void mf_prof_begin(const char *name, cudaStream_t st);
void mf_prof_end(cudaStream_t st);

#define MF_CUDA(call)                                                      \
    do {                                                                   \
        cudaError_t e_ = (call);                                           \
        if (e_ != cudaSuccess) return mf_cuda_check(e_, #call);            \
    } while (0)

// Element chunks and their gathers, overlapped across the caller's stream and
// the pattern's side stream: elem(k, st) is launched for every chunk k in
// turn, gather(k, s) on the stream s it is given.
template <typename Elem, typename Gather>
mf_status mf_slab_pipeline(const mf_pattern *p, cudaStream_t st, Elem elem, Gather gather)
{
    const size_t nsl = p->slab_e.size() - 1;
    const bool two = nsl > 1 && p->side;
    auto fail = [](const char *what) { return mf_cuda_check(cudaGetLastError(), what); };
    if (two) {
        if (cudaEventRecord(p->fork_ev, st) != cudaSuccess) return fail("mf_assemble");
        if (cudaStreamWaitEvent(p->side, p->fork_ev, 0) != cudaSuccess) return fail("mf_assemble");
    }
    for (size_t k = 0; k < nsl; ++k) {
        mf_status s = elem(k, st);
        if (s != MF_OK) return s;
        if (two) {
            if (cudaEventRecord(p->slab_ev[k], st) != cudaSuccess) return fail("mf_assemble");
            if (cudaStreamWaitEvent(p->side, p->slab_ev[k], 0) != cudaSuccess) return fail("mf_assemble");
        }
        s = gather(k, two ? p->side : st);
        if (s != MF_OK) return s;
    }
    if (two) {
        if (cudaEventRecord(p->join_ev, p->side) != cudaSuccess) return fail("mf_assemble");
        if (cudaStreamWaitEvent(st, p->join_ev, 0) != cudaSuccess) return fail("mf_assemble");
    }
    return MF_OK;
}
