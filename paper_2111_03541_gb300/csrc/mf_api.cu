// C ABI entry points: argument checks, handles, status word, error messages.
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "mf_internal.h"

static thread_local char g_msg[512] = "";

mf_status mf_fail(mf_status s, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_msg, sizeof g_msg, fmt, ap);
    va_end(ap);
    return s;
}

mf_status mf_cuda_check(cudaError_t e, const char *what)
{
    if (e == cudaSuccess) return MF_OK;
    cudaGetLastError();  // clear a non-sticky error
    if (e == cudaErrorMemoryAllocation) return mf_fail(MF_ERR_OOM, "%s: %s", what, cudaGetErrorString(e));
    return mf_fail(MF_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

extern "C" const char *mf_last_error(void) { return g_msg; }

void mf_clear_error() { g_msg[0] = 0; }

bool mf_csr_ok(const mf_csr *K)
{
    return K && K->n_rows > 0 && K->nnz > 0 && K->row_ptr && K->col_idx && K->values;
}

// ---------------------------------------------------------------------------
// device status word: one int per device in a __device__ variable; kernels get
// its address as an argument (set-up once per device with that device current)
// ---------------------------------------------------------------------------
static __device__ int g_status_word;
static std::mutex g_status_mu;
static int *g_status_ptr[64];

int *mf_status_word()
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> lk(g_status_mu);
    if (!g_status_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_status_word) != cudaSuccess) return nullptr;
        g_status_ptr[dev] = static_cast<int *>(p);
    }
    return g_status_ptr[dev];
}

extern "C" mf_status mf_sync_status(void *stream)
{
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int *w = mf_status_word();
    if (!w) return mf_fail(MF_ERR_CUDA, "no device status word");
    int h = 0;
    MF_CUDA(cudaMemcpyAsync(&h, w, sizeof(int), cudaMemcpyDeviceToHost, st));
    MF_CUDA(cudaStreamSynchronize(st));
    if (h != 0) {
        const int zero = 0;
        MF_CUDA(cudaMemcpyAsync(w, &zero, sizeof(int), cudaMemcpyHostToDevice, st));
        MF_CUDA(cudaStreamSynchronize(st));
        return mf_fail(static_cast<mf_status>(h), "device reported status %d", h);
    }
    return MF_OK;
}

// ---------------------------------------------------------------------------
// kernel timing: pairs of events per launch, reduced when read
// ---------------------------------------------------------------------------
namespace {
struct ProfRec {
    std::string name;
    cudaEvent_t a, b;
};
std::mutex g_prof_mu;
bool g_prof_on = false;
std::vector<ProfRec> g_prof_pending;
std::vector<cudaEvent_t> g_prof_pool;
std::map<std::string, std::pair<long long, double>> g_prof_acc;
std::vector<size_t> g_prof_open;  // open records (indices), innermost last

cudaEvent_t prof_event()
{
    if (!g_prof_pool.empty()) {
        cudaEvent_t e = g_prof_pool.back();
        g_prof_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}
}  // namespace

void mf_prof_begin(const char *name, cudaStream_t st)
{
    std::lock_guard<std::mutex> lk(g_prof_mu);
    if (!g_prof_on) return;
    g_prof_pending.push_back(ProfRec{name, prof_event(), prof_event()});
    g_prof_open.push_back(g_prof_pending.size() - 1);
    cudaEventRecord(g_prof_pending.back().a, st);
}

void mf_prof_end(cudaStream_t st)
{
    std::lock_guard<std::mutex> lk(g_prof_mu);
    if (!g_prof_on || g_prof_open.empty()) return;
    cudaEventRecord(g_prof_pending[g_prof_open.back()].b, st);
    g_prof_open.pop_back();
}

extern "C" mf_status mf_set_kernel_timing(int32_t enable)
{
    std::lock_guard<std::mutex> lk(g_prof_mu);
    g_prof_on = enable != 0;
    return MF_OK;
}

extern "C" mf_status mf_kernel_times(char *buf, size_t len)
{
    if (!buf || len == 0) return mf_fail(MF_ERR_INVALID_ARG, "mf_kernel_times: empty buffer");
    std::lock_guard<std::mutex> lk(g_prof_mu);
    for (ProfRec &r : g_prof_pending) {
        if (cudaEventSynchronize(r.b) != cudaSuccess) return mf_cuda_check(cudaGetLastError(), "mf_kernel_times");
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, r.a, r.b) != cudaSuccess) {
            cudaGetLastError();  // a record closed after mf_kernel_times: dropped
            ms = 0.f;
        }
        auto &acc = g_prof_acc[r.name];
        acc.first += 1;
        acc.second += ms;
        g_prof_pool.push_back(r.a);
        g_prof_pool.push_back(r.b);
    }
    g_prof_pending.clear();
    g_prof_open.clear();
    std::string out;
    char line[256];
    for (auto &kv : g_prof_acc) {
        snprintf(line, sizeof line, "%s %lld %.6f\n", kv.first.c_str(), kv.second.first, kv.second.second);
        out += line;
    }
    g_prof_acc.clear();
    snprintf(buf, len, "%s", out.c_str());
    return MF_OK;
}

// ---------------------------------------------------------------------------
// exclusive scan of int64 counts (three passes: block scan, scan of block
// totals, add block offsets)
// ---------------------------------------------------------------------------
static constexpr int SCAN_T = 512, SCAN_V = 8, SCAN_TILE = SCAN_T * SCAN_V;

__device__ int64_t block_exclusive_scan(int64_t v, int64_t *sh, int64_t *total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int64_t x = v;
    for (int o = 1; o < 32; o <<= 1) {
        int64_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int64_t s = (lane < (int)(blockDim.x >> 5)) ? sh[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            int64_t y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        sh[lane] = s;  // inclusive warp totals
    }
    __syncthreads();
    const int64_t before = (warp > 0 ? sh[warp - 1] : 0) + x - v;
    if (total) *total = sh[(blockDim.x >> 5) - 1];
    __syncthreads();
    return before;
}

__global__ void k_scan_tiles(int64_t *data, int64_t n, int64_t *tile_sums)
{
    __shared__ int64_t sh[32];
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_V;
    int64_t v[SCAN_V], s = 0;
    for (int i = 0; i < SCAN_V; ++i) {
        v[i] = (base + i < n) ? data[base + i] : 0;
        s += v[i];
    }
    int64_t tot;
    int64_t run = block_exclusive_scan(s, sh, &tot);
    for (int i = 0; i < SCAN_V; ++i) {
        if (base + i < n) data[base + i] = run;
        run += v[i];
    }
    if (threadIdx.x == 0) tile_sums[blockIdx.x] = tot;
}

__global__ void k_scan_single(int64_t *data, int64_t n, int64_t *total)
{
    __shared__ int64_t sh[32];
    int64_t carry = 0;
    for (int64_t start = 0; start < n; start += blockDim.x) {
        const int64_t i = start + threadIdx.x;
        const int64_t v = i < n ? data[i] : 0;
        int64_t tot;
        const int64_t ex = block_exclusive_scan(v, sh, &tot);
        if (i < n) data[i] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0 && total) *total = carry;
}

__global__ void k_scan_add(int64_t *data, int64_t n, const int64_t *tile_off)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) data[i] += tile_off[i / SCAN_TILE];
}

cudaError_t mf_scan_i64(int64_t *d_data, int64_t n, int64_t *d_total, cudaStream_t st)
{
    if (n <= SCAN_TILE) {
        k_scan_single<<<1, 1024, 0, st>>>(d_data, n, d_total);
        return cudaGetLastError();
    }
    const int64_t tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
    int64_t *sums = nullptr;
    cudaError_t e = cudaMallocAsync(&sums, sizeof(int64_t) * tiles, st);
    if (e != cudaSuccess) return e;
    k_scan_tiles<<<(unsigned)tiles, SCAN_T, 0, st>>>(d_data, n, sums);
    e = mf_scan_i64(sums, tiles, d_total, st);
    if (e == cudaSuccess) {
        k_scan_add<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(d_data, n, sums);
        e = cudaGetLastError();
    }
    cudaFreeAsync(sums, st);
    return e;
}

// ---------------------------------------------------------------------------
// mesh
// ---------------------------------------------------------------------------
extern "C" mf_status mf_mesh_create(const mf_mesh_desc *desc, void *stream, mf_mesh **out)
{
    g_msg[0] = 0;
    if (!desc || !out) return mf_fail(MF_ERR_INVALID_ARG, "mf_mesh_create: NULL argument");
    *out = nullptr;
    if (desc->elem < MF_P1_TRI || desc->elem > MF_Q2S_QUAD)
        return mf_fail(MF_ERR_INVALID_ARG, "mf_mesh_create: unknown element %d", desc->elem);
    if (desc->dim != mf_ndim(desc->elem))
        return mf_fail(MF_ERR_INVALID_ARG, "mf_mesh_create: dim %d does not match element", desc->dim);
    if (desc->n_nodes <= 0 || desc->n_elems <= 0 || !desc->coords || !desc->conn)
        return mf_fail(MF_ERR_INVALID_ARG, "mf_mesh_create: empty mesh or NULL arrays");
    if (desc->n_nodes > INT32_MAX || desc->n_elems >= (int64_t(1) << 25))
        return mf_fail(MF_ERR_UNSUPPORTED, "mf_mesh_create: at most 2^31-1 nodes and 2^25 elements");
    if ((desc->pconn == nullptr) != (desc->n_pnodes == 0) || (desc->pconn && desc->elem != MF_P2_TRI))
        return mf_fail(MF_ERR_INVALID_ARG, "mf_mesh_create: pconn/n_pnodes are for P2 flow meshes");
    mf_mesh *m = new (std::nothrow) mf_mesh();
    if (!m) return mf_fail(MF_ERR_OOM, "mf_mesh_create: host allocation");
    m->dim = desc->dim;
    m->elem = desc->elem;
    m->npe = mf_npe(desc->elem);
    m->n_nodes = desc->n_nodes;
    m->n_elems = desc->n_elems;
    m->n_pnodes = desc->n_pnodes;
    m->coords = desc->coords;
    m->conn = desc->conn;
    m->pconn = desc->pconn;
    cudaGetDevice(&m->device);
    mf_status s = mf_mesh_validate(m, static_cast<cudaStream_t>(stream));
    if (s != MF_OK) {
        delete m;
        return s;
    }
    *out = m;
    return MF_OK;
}

extern "C" mf_status mf_mesh_destroy(mf_mesh *mesh)
{
    delete mesh;
    return MF_OK;
}

// ---------------------------------------------------------------------------
// pattern
// ---------------------------------------------------------------------------
extern "C" mf_status mf_pattern_build(const mf_mesh *mesh, int32_t form, void *stream, mf_pattern **out)
{
    g_msg[0] = 0;
    if (!mesh || !out) return mf_fail(MF_ERR_INVALID_ARG, "mf_pattern_build: NULL argument");
    *out = nullptr;
    if (form == MF_FORM_ELASTIC && mesh->elem != MF_Q1_HEX && mesh->elem != MF_Q2S_HEX)
        return mf_fail(MF_ERR_UNSUPPORTED, "mf_pattern_build: elasticity is provided on Q1 and Q2S bricks");
    if ((form == MF_FORM_OSEEN || form == MF_FORM_NS) && (mesh->elem != MF_P2_TRI || !mesh->pconn))
        return mf_fail(MF_ERR_UNSUPPORTED, "mf_pattern_build: flow needs a P2 mesh with pconn");
    if (form < MF_FORM_THERMAL || form > MF_FORM_NS || form == MF_FORM_CAPACITY)
        return mf_fail(MF_ERR_INVALID_ARG, "mf_pattern_build: unknown form %d", form);
    mf_pattern *p = new (std::nothrow) mf_pattern();
    if (!p) return mf_fail(MF_ERR_OOM, "mf_pattern_build: host allocation");
    p->form = form;
    p->mesh = mesh;
    mf_status s = mf_pattern_build_impl(mesh, form, static_cast<cudaStream_t>(stream), p);
    if (s != MF_OK) {
        mf_pattern_free(p);
        delete p;
        return s;
    }
    *out = p;
    return MF_OK;
}

extern "C" mf_status mf_pattern_csr(const mf_pattern *pattern, mf_csr *out)
{
    if (!pattern || !out) return mf_fail(MF_ERR_INVALID_ARG, "mf_pattern_csr: NULL argument");
    out->n_rows = pattern->n_rows;
    out->nnz = pattern->nnz;
    out->row_ptr = pattern->row_ptr;
    out->col_idx = pattern->col_idx;
    out->values = nullptr;
    return MF_OK;
}

extern "C" mf_status mf_pattern_copy_csr(const mf_pattern *pattern, int64_t *row_ptr, int32_t *col_idx, void *stream)
{
    if (!pattern || !row_ptr || !col_idx) return mf_fail(MF_ERR_INVALID_ARG, "mf_pattern_copy_csr: NULL argument");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    MF_CUDA(cudaMemcpyAsync(row_ptr, pattern->row_ptr, sizeof(int64_t) * (pattern->n_rows + 1),
                            cudaMemcpyDeviceToDevice, st));
    MF_CUDA(cudaMemcpyAsync(col_idx, pattern->col_idx, sizeof(int32_t) * pattern->nnz, cudaMemcpyDeviceToDevice, st));
    return MF_OK;
}

extern "C" mf_status mf_pattern_destroy(mf_pattern *pattern)
{
    if (!pattern) return MF_OK;
    mf_pattern_free(pattern);
    delete pattern;
    return MF_OK;
}

// ---------------------------------------------------------------------------
// assembly and solve
// ---------------------------------------------------------------------------
static bool csr_ok(const mf_csr *K) { return mf_csr_ok(K); }

extern "C" mf_status mf_assemble(int32_t form, const mf_mesh *mesh, const mf_pattern *pattern,
                                 const mf_coeffs *coeffs, int32_t prec, mf_csr *K, double *d,
                                 void *stream)
{
    g_msg[0] = 0;
    if (!mesh || !pattern || !coeffs || !K || !d || !K->values)
        return mf_fail(MF_ERR_INVALID_ARG, "mf_assemble: NULL argument");
    const int pform = form == MF_FORM_CAPACITY ? MF_FORM_THERMAL : form;  // capacity: on a thermal pattern
    if (pattern->form != pform || pattern->mesh != mesh)
        return mf_fail(MF_ERR_INVALID_ARG, "mf_assemble: pattern was built for another form or mesh");
    if (form == MF_FORM_CAPACITY && prec != MF_PREC_FP64)
        return mf_fail(MF_ERR_UNSUPPORTED, "mf_assemble: the capacity form is assembled in FP64");
    if (mesh->elem == MF_Q2S_HEX && ((form != MF_FORM_THERMAL && form != MF_FORM_ELASTIC) || prec != MF_PREC_FP64))
        return mf_fail(MF_ERR_UNSUPPORTED,
                       "mf_assemble: serendipity bricks carry the thermal and elasticity forms in FP64");
    if ((mesh->elem == MF_P2_TET || mesh->elem == MF_Q2S_QUAD) &&
        ((form != MF_FORM_THERMAL && form != MF_FORM_CAPACITY) || prec != MF_PREC_FP64))
        return mf_fail(MF_ERR_UNSUPPORTED,
                       "mf_assemble: tetrahedra and serendipity quadrilaterals carry the thermal and capacity forms in FP64");
    if (K->n_rows != pattern->n_rows || K->nnz != pattern->nnz || K->row_ptr != pattern->row_ptr ||
        K->col_idx != pattern->col_idx)
        return mf_fail(MF_ERR_INVALID_ARG, "mf_assemble: K does not carry the pattern's CSR arrays");
    const bool flow = form == MF_FORM_OSEEN || form == MF_FORM_NS;
    if (!flow && !coeffs->elem_coef)
        return mf_fail(MF_ERR_INVALID_ARG, "mf_assemble: elem_coef is NULL");
    if (flow && !coeffs->advect)
        return mf_fail(MF_ERR_INVALID_ARG, "mf_assemble: advect (the advecting field or the state) is NULL");
    if (form == MF_FORM_NS && prec != MF_PREC_FP64)
        return mf_fail(MF_ERR_UNSUPPORTED, "mf_assemble: the Navier-Stokes form is assembled in FP64");
    if ((coeffs->bc_mask == nullptr) != (coeffs->bc_val == nullptr))
        return mf_fail(MF_ERR_INVALID_ARG, "mf_assemble: bc_mask and bc_val go together");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (form == MF_FORM_NS) return mf_assemble_ns(mesh, pattern, coeffs, K->values, d, st);
    if (prec == MF_PREC_FP64) return mf_assemble_fp64(form, mesh, pattern, coeffs, K->values, d, st);
    if (prec == MF_PREC_MIXED) {
        if (form != MF_FORM_ELASTIC)
            return mf_fail(MF_ERR_UNSUPPORTED, "mf_assemble: the mixed path covers Q1 elasticity");
        return mf_assemble_mixed(form, mesh, pattern, coeffs, K->values, d, st);
    }
    return mf_fail(MF_ERR_INVALID_ARG, "mf_assemble: unknown precision %d", prec);
}

extern "C" mf_status mf_ns_newton(const mf_mesh *mesh, const mf_pattern *pattern, const mf_coeffs *coeffs,
                                  double *x, double newton_tol, int32_t max_newton, const mf_solver_opts *lin,
                                  double *resid_hist, int32_t *n_steps, void *stream)
{
    g_msg[0] = 0;
    if (!mesh || !pattern || !coeffs || !x || !lin) return mf_fail(MF_ERR_INVALID_ARG, "mf_ns_newton: NULL argument");
    if (pattern->form != MF_FORM_NS || pattern->mesh != mesh)
        return mf_fail(MF_ERR_INVALID_ARG, "mf_ns_newton: the pattern was not built for MF_FORM_NS on this mesh");
    if ((coeffs->bc_mask == nullptr) != (coeffs->bc_val == nullptr))
        return mf_fail(MF_ERR_INVALID_ARG, "mf_ns_newton: bc_mask and bc_val go together");
    if (max_newton < 0 || !(newton_tol >= 0.0))
        return mf_fail(MF_ERR_INVALID_ARG, "mf_ns_newton: negative step count or tolerance");
    if (lin->solver != MF_SOLVER_GMRES && lin->solver != MF_SOLVER_GMRES_FLOW_MG)
        return mf_fail(MF_ERR_INVALID_ARG, "mf_ns_newton: the linear solver is GMRES or GMRES with the flow hierarchy");
    if (lin->solver == MF_SOLVER_GMRES_FLOW_MG && !lin->flow_mg)
        return mf_fail(MF_ERR_INVALID_ARG, "mf_ns_newton: MF_SOLVER_GMRES_FLOW_MG needs lin->flow_mg");
    return mf_ns_newton_impl(mesh, pattern, coeffs, x, newton_tol, max_newton, lin, resid_hist, n_steps,
                             static_cast<cudaStream_t>(stream));
}

extern "C" mf_status mf_facets_create(const mf_mesh *mesh, const mf_pattern *pattern, int64_t n_facets,
                                      const int32_t *elem, const uint8_t *face, void *stream, mf_facets **out)
{
    g_msg[0] = 0;
    if (!mesh || !pattern || !out) return mf_fail(MF_ERR_INVALID_ARG, "mf_facets_create: NULL argument");
    *out = nullptr;
    if (pattern->mesh != mesh)
        return mf_fail(MF_ERR_INVALID_ARG, "mf_facets_create: the pattern was built on another mesh");
    if (pattern->form != MF_FORM_THERMAL && pattern->form != MF_FORM_ELASTIC)
        return mf_fail(MF_ERR_INVALID_ARG, "mf_facets_create: boundary terms exist for the thermal and elasticity forms");
    if (n_facets < 0 || (n_facets > 0 && (!elem || !face)))
        return mf_fail(MF_ERR_INVALID_ARG, "mf_facets_create: negative count or NULL facet arrays");
    if (n_facets >= (int64_t(1) << 28))
        return mf_fail(MF_ERR_UNSUPPORTED, "mf_facets_create: at most 2^28 facets");
    mf_facets *f = new (std::nothrow) mf_facets();
    if (!f) return mf_fail(MF_ERR_OOM, "mf_facets_create: host allocation");
    f->mesh = mesh;
    f->pattern = pattern;
    mf_status s = mf_facets_create_impl(mesh, pattern, n_facets, elem, face, static_cast<cudaStream_t>(stream), f);
    if (s != MF_OK) {
        mf_facets_free(f);
        delete f;
        return s;
    }
    *out = f;
    return MF_OK;
}

extern "C" mf_status mf_facets_destroy(mf_facets *facets)
{
    if (!facets) return MF_OK;
    mf_facets_free(facets);
    delete facets;
    return MF_OK;
}

extern "C" mf_status mf_assemble_boundary(const mf_facets *facets, const mf_facet_coeffs *coeffs, mf_csr *K,
                                          double *d, void *stream)
{
    g_msg[0] = 0;
    if (!facets || !coeffs || !K || !d || !K->values)
        return mf_fail(MF_ERR_INVALID_ARG, "mf_assemble_boundary: NULL argument");
    const mf_pattern *p = facets->pattern;
    if (K->n_rows != p->n_rows || K->nnz != p->nnz || K->row_ptr != p->row_ptr || K->col_idx != p->col_idx)
        return mf_fail(MF_ERR_INVALID_ARG, "mf_assemble_boundary: K does not carry the facets' pattern");
    if ((coeffs->bc_mask == nullptr) != (coeffs->bc_val == nullptr))
        return mf_fail(MF_ERR_INVALID_ARG, "mf_assemble_boundary: bc_mask and bc_val go together");
    if (facets->n_facets == 0) return MF_OK;
    if (p->form == MF_FORM_THERMAL ? (!coeffs->h || !coeffs->t_env) : !coeffs->stress)
        return mf_fail(MF_ERR_INVALID_ARG, "mf_assemble_boundary: the form's facet coefficients are NULL");
    return mf_assemble_boundary_impl(facets, coeffs, K->values, d, static_cast<cudaStream_t>(stream));
}

extern "C" mf_status mf_genalpha_params_from_rho(double rho_inf, mf_genalpha_params *out)
{
    g_msg[0] = 0;
    if (!out) return mf_fail(MF_ERR_INVALID_ARG, "mf_genalpha_params_from_rho: NULL argument");
    if (!(rho_inf >= 0.0 && rho_inf <= 1.0))
        return mf_fail(MF_ERR_INVALID_ARG, "mf_genalpha_params_from_rho: rho_inf must lie in [0, 1]");
    return mf_genalpha_params_from_rho_impl(rho_inf, out);
}

extern "C" mf_status mf_genalpha_run(const mf_csr *K, const double *M_values, const double *F, const uint8_t *bc_mask,
                                     const double *bc_val, const mf_facets *rad, const double *rad_es,
                                     const double *rad_tenv, double *phi, double *u, double *a,
                                     const mf_genalpha_params *prm, double dt, int64_t steps, double newton_tol,
                                     int32_t max_newton, double pcg_tol, int64_t pcg_max_iter, int64_t *newton_its,
                                     int64_t *pcg_its, void *stream)
{
    g_msg[0] = 0;
    if (!csr_ok(K) || !M_values || !F || !phi || !u || !a || !prm)
        return mf_fail(MF_ERR_INVALID_ARG, "mf_genalpha_run: NULL argument");
    if ((bc_mask == nullptr) != (bc_val == nullptr))
        return mf_fail(MF_ERR_INVALID_ARG, "mf_genalpha_run: bc_mask and bc_val go together");
    if (rad && (rad->pattern->row_ptr != K->row_ptr || rad->pattern->form != MF_FORM_THERMAL ||
                (rad->n_facets > 0 && (!rad_es || !rad_tenv))))
        return mf_fail(MF_ERR_INVALID_ARG, "mf_genalpha_run: radiation facets need K's thermal pattern, es, t_env");
    if (rad && rad->n_facets > 0 && rad->mesh->elem == MF_P2_TET)
        return mf_fail(MF_ERR_UNSUPPORTED, "mf_genalpha_run: no radiation on tetrahedron faces");
    if (!(dt > 0.0) || steps < 0 || !(prm->b1 != 0.0) || !(prm->b2 != 0.0) || !(newton_tol > 0.0) ||
        max_newton < 1 || !(pcg_tol > 0.0) || pcg_max_iter < 1)
        return mf_fail(MF_ERR_INVALID_ARG,
                       "mf_genalpha_run: dt > 0, steps >= 0, b1, b2 != 0, tolerances > 0, iteration caps >= 1");
    return mf_genalpha_run_impl(K, M_values, F, bc_mask, bc_val, rad, rad_es, rad_tenv, phi, u, a, prm, dt, steps,
                                newton_tol, max_newton, pcg_tol, pcg_max_iter, newton_its, pcg_its,
                                static_cast<cudaStream_t>(stream));
}

extern "C" mf_status mf_genalpha_initial_rate(const mf_csr *K, const double *M_values, const double *F,
                                              const uint8_t *bc_mask, const mf_facets *rad, const double *rad_es,
                                              const double *rad_tenv, const double *phi, double *u, double pcg_tol,
                                              int64_t pcg_max_iter, void *stream)
{
    g_msg[0] = 0;
    if (!csr_ok(K) || !M_values || !F || !phi || !u)
        return mf_fail(MF_ERR_INVALID_ARG, "mf_genalpha_initial_rate: NULL argument");
    if (rad && (rad->pattern->row_ptr != K->row_ptr || rad->pattern->form != MF_FORM_THERMAL ||
                (rad->n_facets > 0 && (!rad_es || !rad_tenv))))
        return mf_fail(MF_ERR_INVALID_ARG, "mf_genalpha_initial_rate: radiation facets need K's thermal pattern");
    if (rad && rad->n_facets > 0 && rad->mesh->elem == MF_P2_TET)
        return mf_fail(MF_ERR_UNSUPPORTED, "mf_genalpha_initial_rate: no radiation on tetrahedron faces");
    if (!(pcg_tol > 0.0) || pcg_max_iter < 1)
        return mf_fail(MF_ERR_INVALID_ARG, "mf_genalpha_initial_rate: pcg_tol > 0 and pcg_max_iter >= 1");
    return mf_genalpha_initial_rate_impl(K, M_values, F, bc_mask, rad, rad_es, rad_tenv, phi, u, pcg_tol,
                                         pcg_max_iter, static_cast<cudaStream_t>(stream));
}

extern "C" mf_status mf_pressure_mass_diag(const mf_mesh *mesh, const mf_pattern *pattern, double *out,
                                           void *stream)
{
    g_msg[0] = 0;
    if (!mesh || !pattern || !out) return mf_fail(MF_ERR_INVALID_ARG, "mf_pressure_mass_diag: NULL argument");
    if (pattern->form != MF_FORM_OSEEN || pattern->mesh != mesh)
        return mf_fail(MF_ERR_INVALID_ARG, "mf_pressure_mass_diag: needs the flow pattern of this mesh");
    return mf_pmass_impl(mesh, pattern, out, static_cast<cudaStream_t>(stream));
}

extern "C" mf_status mf_flow_precond(const mf_mesh *mesh, const mf_pattern *pattern, const mf_csr *K,
                                     const uint8_t *bc_mask, double p_scale, double *out, void *stream)
{
    g_msg[0] = 0;
    if (!mesh || !pattern || !csr_ok(K) || !out)
        return mf_fail(MF_ERR_INVALID_ARG, "mf_flow_precond: NULL argument");
    if (pattern->form != MF_FORM_OSEEN || pattern->mesh != mesh || K->row_ptr != pattern->row_ptr)
        return mf_fail(MF_ERR_INVALID_ARG, "mf_flow_precond: needs the flow pattern of this mesh");
    return mf_flow_precond_impl(mesh, pattern, K, bc_mask, p_scale, out, static_cast<cudaStream_t>(stream));
}

extern "C" mf_status mf_solve(const mf_csr *K, const double *d, double *x, const mf_solver_opts *opts,
                              mf_solve_info *info, void *stream)
{
    g_msg[0] = 0;
    if (!csr_ok(K) || !d || !x || !opts) return mf_fail(MF_ERR_INVALID_ARG, "mf_solve: NULL argument");
    if (opts->solver < MF_SOLVER_PCG || opts->solver > MF_SOLVER_GMRES_FLOW_MG)
        return mf_fail(MF_ERR_INVALID_ARG, "mf_solve: unknown solver %d", opts->solver);
    if (opts->solver == MF_SOLVER_GMRES_FLOW_MG && !opts->flow_mg)
        return mf_fail(MF_ERR_INVALID_ARG, "mf_solve: MF_SOLVER_GMRES_FLOW_MG needs opts->flow_mg");
    const bool gm = opts->solver == MF_SOLVER_GMRES || opts->solver == MF_SOLVER_GMRES_FLOW_MG;
    if (!(opts->tol > 0.0) || opts->max_iter < 0 || (gm && opts->restart < 1))
        return mf_fail(MF_ERR_INVALID_ARG, "mf_solve: tol > 0, max_iter >= 0, restart >= 1 required");
    return mf_solve_impl(K, d, x, opts, info, static_cast<cudaStream_t>(stream));
}

extern "C" mf_status mf_flow_mg_create(int32_t levels, const mf_csr *const *K, const int64_t *cells,
                                       const uint8_t *const *bc_mask, const double *pmass, double visc,
                                       void *stream, mf_flow_mg **out)
{
    g_msg[0] = 0;
    if (!K || !cells || !bc_mask || !pmass || !out || levels < 1 || levels > 12 || !(visc > 0.0))
        return mf_fail(MF_ERR_INVALID_ARG, "mf_flow_mg_create: NULL argument, levels outside [1, 12] or visc <= 0");
    for (int l = 0; l < levels; ++l)
        if (!csr_ok(K[l]) || !bc_mask[l]) return mf_fail(MF_ERR_INVALID_ARG, "mf_flow_mg_create: level %d", l);
    *out = nullptr;
    return mf_flow_mg_create_impl(levels, K, cells, bc_mask, pmass, visc, static_cast<cudaStream_t>(stream), out);
}

extern "C" mf_status mf_flow_mg_destroy(mf_flow_mg *mg)
{
    g_msg[0] = 0;
    mf_flow_mg_destroy_impl(mg);
    return MF_OK;
}

extern "C" mf_status mf_spmv(const mf_csr *K, const double *x, double *y, void *stream)
{
    g_msg[0] = 0;
    if (!csr_ok(K) || !x || !y) return mf_fail(MF_ERR_INVALID_ARG, "mf_spmv: NULL argument");
    return mf_spmv_impl(K, x, y, static_cast<cudaStream_t>(stream));
}
