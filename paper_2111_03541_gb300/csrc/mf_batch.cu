// Batched assembly: many thermal problems of uneven size and mixed element
// order (P1, P2 triangles, Q1 hexahedra) assembled by one persistent launch
// over (problem, tile) work items, replayed from a CUDA graph, with tile
// shapes picked by a measuring autotuner (results cached in a small JSON
// file).  Blocks take items from a queue: element tiles (scratch rows) and
// node tiles (CSR rows gathered from the scratch rows); a problem's node
// tiles sit about two waves of blocks after its last element tile, so the
// latency-bound gathers of finished problems overlap the FP64-bound element
// work of later ones.
//
// Every element and every CSR row is computed by the same device routines as
// the single-problem path (mf_fem.cuh), in the same order, so each problem's
// K and d are bitwise equal to mf_assemble's.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "mf_fem.cuh"

struct BatchProblem {
    int elem, npe;
    int64_t n_el, n_nodes;
    const double *X;
    const int32_t *conn;
    const double *kc;
    double f;
    double *scratch;
    int64_t stride;
    const int64_t *ptr;
    const int32_t *col;
    const int64_t *inc_ptr;
    const int32_t *inc;
    const uint8_t *inc_loc;
    const uint8_t *inc_slot;
    const int32_t *elem_inc;
    const uint8_t *tr;
    const double *kref;
    const uint8_t *mask;
    const double *bval;
    const int64_t *row_ptr;
    double *values;
    double *d;
    // a Q1 mesh of translates: reference entries and coefficients as FP32
    // pairs (the double-float gather of the single-problem path); else null
    const float2 *kref_df;
    float2 *kc_df;
    // a lexicographic box of a rectangular cell (every element a translate):
    // nodes per line (box[0] > 0) and the reference entries by corner class
    int32_t box[3];
    mf_box_classes box_cls;
};

struct BatchTile {
    int32_t prob;
    int32_t type;
    int64_t first;
    int64_t count;
};

struct mf_batch {
    int n = 0;
    std::vector<BatchProblem> host;
    BatchProblem *dev = nullptr;
    mf_batch_tiling tiling{};
    BatchTile *etiles = nullptr, *ntiles = nullptr;
    int n_etiles = 0, n_ntiles = 0;
    int32_t *items = nullptr;  // queue order: element tile k as k, node tile k as -(k + 1)
    int32_t *need = nullptr;   // element tiles per problem
    int *ctr = nullptr;        // finished element tiles per problem, then the queue head
    int n_items = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int sm_count = 0;
    std::string signature;
};

namespace {

constexpr int BG_WARPS = 8;        // most warps per block (shared row accumulators)
constexpr int BQ_POLLS = 1 << 22;  // bounded wait of a node tile (about a second of 256 ns naps)

__device__ __forceinline__ void batch_elem_tile(const BatchProblem &p, const BatchTile &T, int *status)
{
    for (int64_t i = threadIdx.x; i < T.count; i += blockDim.x) {
        const int64_t e = T.first + i;
        if (T.type == MF_P1_TRI) elem_thermal_p1(e, p.X, p.conn, p.kc, p.f, p.elem_inc, p.scratch, status);
        else if (T.type == MF_P2_TRI) elem_thermal_p2(e, p.X, p.conn, p.kc, p.f, p.elem_inc, p.scratch, status);
        else if (p.kc_df) {
            const double k = p.kc[e];
            if (!isfinite(k)) mf_dev_fail(status, MF_ERR_NONFINITE);
            p.kc_df[e] = f64_to_df(k);
        } else if (!q1_translate(e, p.tr, p.kc, status))
            elem_thermal_q1(e, p.X, p.conn, p.kc, p.f, p.elem_inc, p.scratch, status);
    }
}

template <int NPE>
__device__ __forceinline__ void batch_gather_tile(const BatchProblem &p, const BatchTile &T, int warp, int lane,
                                                  int nwarps, double (*acc_all)[MF_MAX_DEG])
{
    constexpr int L = th_lanes<NPE>(), G = 32 / L;
    const int grp = warp * G + lane / L;
    const unsigned gmask = (L == 32 ? 0xffffffffu : ((1u << L) - 1u)) << (lane & ~(L - 1));
    if (NPE == 8 && p.box[0] > 0) {  // box of translates: the single-problem path's row routine, one thread
                                     // per node (every row checks the mask: the same values)
        for (int64_t i = threadIdx.x; i < T.count; i += blockDim.x) {
            const int n = (int)(T.first + i);
            double *row = p.values + p.row_ptr[n];
            p.d[n] = box_row_q1(n, p.box[0], p.box[1], p.box[2], p.box_cls.k_cls, p.f * p.box_cls.dref, p.kc,
                                p.mask != nullptr, p.mask, p.bval, [row](int k, double v) { row[k] = v; });
        }
        return;
    }
    if (NPE == 8 && p.kc_df) {  // translates: the single-problem path's double-float row (every row
                                // takes the Dirichlet branch when there is a mask: the same values)
        const float2 f_df = f64_to_df(p.f);
        for (int64_t i = grp; i < T.count; i += nwarps * G)
            gather_row_th_q1df<true>(T.first + i, lane & (L - 1), gmask, reinterpret_cast<float2 *>(acc_all[grp]),
                                     p.mask != nullptr, p.ptr, p.col, p.inc_ptr, p.inc, p.inc_loc, p.inc_slot,
                                     p.kref_df, p.kc_df, f_df, p.mask, p.bval, p.row_ptr, p.values, p.d);
        return;
    }
    for (int64_t i = grp; i < T.count; i += nwarps * G)  // group-uniform
        gather_row_th<NPE, true>(T.first + i, lane & (L - 1), gmask, acc_all[grp], p.ptr, p.col, p.inc_ptr, p.inc,
                                 p.inc_loc, p.inc_slot, p.scratch, p.kref, p.kc, p.f, p.mask, p.bval, p.row_ptr,
                                 p.values, p.d);
}

// The whole batch in one persistent launch.  A block takes the next queue
// item (one atomic per item), computes an element tile (then every thread
// fences its stores and one thread counts the tile for its problem) or a node
// tile (one thread first waits until all of the problem's element tiles are
// counted, fences, and the block reads the scratch rows through L2).  Every
// element tile of a problem comes before its node tiles in the queue, and a
// block only waits while holding a node tile, so the tiles waited for are
// held by running blocks that do not wait: no deadlock, whatever the number
// of resident blocks.  The wait is bounded: after BQ_POLLS polls the launch
// records MF_ERR_TIMEOUT and goes on.  Registers are capped at 80 per thread
// (three blocks of 256 per SM): the element routines spill, but the
// latency-bound gathers keep their occupancy (measured with the 512-problem
// batch: 254 registers 30.2 ms, 128 23.2 ms, 80 22.3 ms, 64 22.3 ms).
__global__ void __launch_bounds__(BG_WARPS * 32, 3) k_batch(const BatchProblem *__restrict__ P,
                                                        const BatchTile *__restrict__ etiles,
                                                        const BatchTile *__restrict__ ntiles,
                                                        const int32_t *__restrict__ items, int n_items,
                                                        const int32_t *__restrict__ need, int *ctr, int n_prob,
                                                        int *status)
{
    __shared__ double acc_all[BG_WARPS * 8][MF_MAX_DEG];
    __shared__ int s_item;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    int *done = ctr, *head = ctr + n_prob;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(head, 1);
        __syncthreads();
        const int it = s_item;
        __syncthreads();  // every thread has read s_item before it is rewritten
        if (it >= n_items) break;
        const int code = items[it];
        if (code >= 0) {
            const BatchTile T = etiles[code];
            batch_elem_tile(P[T.prob], T, status);
            __threadfence();
            __syncthreads();
            if (threadIdx.x == 0) atomicAdd(&done[T.prob], 1);
        } else {
            const BatchTile T = ntiles[-code - 1];
            if (threadIdx.x == 0) {
                const int want = need[T.prob];
                const volatile int *dp = done + T.prob;
                for (int polls = 0; *dp < want; ++polls) {
                    if (polls >= BQ_POLLS) {
                        mf_dev_fail(status, MF_ERR_TIMEOUT);
                        break;
                    }
                    __nanosleep(256);
                }
                __threadfence();
            }
            __syncthreads();
            const BatchProblem &p = P[T.prob];
            if (T.type == MF_P1_TRI) batch_gather_tile<3>(p, T, warp, lane, nwarps, acc_all);
            else if (T.type == MF_P2_TRI) batch_gather_tile<6>(p, T, warp, lane, nwarps, acc_all);
            else batch_gather_tile<8>(p, T, warp, lane, nwarps, acc_all);
            __syncthreads();  // the next item may give a group another node type
        }
    }
}

void free_tiles(mf_batch *b)
{
    cudaFree(b->etiles);
    cudaFree(b->ntiles);
    cudaFree(b->items);
    cudaFree(b->need);
    cudaFree(b->ctr);
    b->etiles = b->ntiles = nullptr;
    b->items = b->need = nullptr;
    b->ctr = nullptr;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
}

// Work items.  Element tiles sorted by element type (P1, P2, Q1), problems in
// order within a type; a problem's node tiles go into the queue after the
// element tile that comes two grids of blocks after its last element tile (so
// its element tiles are most likely finished when they are taken; one grid
// and half a grid measured 1% and 2% slower), the rest at the end in the same
// problem order.
mf_status make_tiles(mf_batch *b, const mf_batch_tiling &t)
{
    std::vector<BatchTile> et, nt;
    std::vector<int> last(b->n, -1), order;
    std::vector<int32_t> need(b->n, 0);
    for (int type = MF_P1_TRI; type <= MF_Q1_HEX; ++type)
        for (int i = 0; i < b->n; ++i) {
            const BatchProblem &p = b->host[i];
            if (p.elem != type) continue;
            for (int64_t s = 0; s < p.n_el; s += t.elem_tile) {
                et.push_back(BatchTile{i, type, s, std::min<int64_t>(t.elem_tile, p.n_el - s)});
                ++need[i];
            }
            last[i] = (int)et.size() - 1;
            order.push_back(i);
        }
    std::vector<int> first_nt(b->n, 0), cnt_nt(b->n, 0);
    for (int i : order) {
        const BatchProblem &p = b->host[i];
        first_nt[i] = (int)nt.size();
        for (int64_t s = 0; s < p.n_nodes; s += t.node_tile)
            nt.push_back(BatchTile{i, p.elem, s, std::min<int64_t>(t.node_tile, p.n_nodes - s)});
        cnt_nt[i] = (int)nt.size() - first_nt[i];
    }
    const int lag = std::max(1, 2 * b->sm_count * t.grid_per_sm);
    std::vector<int32_t> items;
    items.reserve(et.size() + nt.size());
    size_t next = 0;  // next problem (in `order`) whose node tiles are not queued yet
    auto emit_nodes = [&](int i) {
        for (int k = 0; k < cnt_nt[i]; ++k) items.push_back(-(first_nt[i] + k) - 1);
    };
    for (int k = 0; k < (int)et.size(); ++k) {
        items.push_back(k);
        while (next < order.size() && last[order[next]] + lag <= k) emit_nodes(order[next++]);
    }
    while (next < order.size()) emit_nodes(order[next++]);
    free_tiles(b);
    MF_CUDA(cudaMalloc(&b->etiles, sizeof(BatchTile) * std::max<size_t>(1, et.size())));
    MF_CUDA(cudaMalloc(&b->ntiles, sizeof(BatchTile) * std::max<size_t>(1, nt.size())));
    MF_CUDA(cudaMalloc(&b->items, sizeof(int32_t) * std::max<size_t>(1, items.size())));
    MF_CUDA(cudaMalloc(&b->need, sizeof(int32_t) * b->n));
    MF_CUDA(cudaMalloc(&b->ctr, sizeof(int) * (b->n + 1)));
    MF_CUDA(cudaMemcpy(b->etiles, et.data(), sizeof(BatchTile) * et.size(), cudaMemcpyHostToDevice));
    MF_CUDA(cudaMemcpy(b->ntiles, nt.data(), sizeof(BatchTile) * nt.size(), cudaMemcpyHostToDevice));
    MF_CUDA(cudaMemcpy(b->items, items.data(), sizeof(int32_t) * items.size(), cudaMemcpyHostToDevice));
    MF_CUDA(cudaMemcpy(b->need, need.data(), sizeof(int32_t) * b->n, cudaMemcpyHostToDevice));
    b->n_etiles = (int)et.size();
    b->n_ntiles = (int)nt.size();
    b->n_items = (int)items.size();
    b->tiling = t;
    return MF_OK;
}

void launch_batch(mf_batch *b, cudaStream_t st, int *status)
{
    const mf_batch_tiling &t = b->tiling;
    const int grid = std::max(1, std::min(b->n_items, b->sm_count * t.grid_per_sm));
    cudaMemsetAsync(b->ctr, 0, sizeof(int) * (b->n + 1), st);
    k_batch<<<grid, t.elem_block, 0, st>>>(b->dev, b->etiles, b->ntiles, b->items, b->n_items, b->need, b->ctr, b->n,
                                           status);
}

mf_status capture(mf_batch *b, int *status)
{
    cudaStream_t cs;
    MF_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        launch_batch(b, cs, status);
        e = cudaStreamEndCapture(cs, &b->graph);
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
    cudaStreamDestroy(cs);
    if (e != cudaSuccess) return mf_cuda_check(e, "mf_batch: graph capture");
    return MF_OK;
}

// tiny flat JSON cache: {"<signature>": [elem_tile, elem_block, node_tile, grid_per_sm], ...}
bool cache_lookup(const char *path, const std::string &sig, mf_batch_tiling *t)
{
    if (!path) return false;
    FILE *f = fopen(path, "r");
    if (!f) return false;
    std::string s;
    char buf[4096];
    size_t k;
    while ((k = fread(buf, 1, sizeof buf, f)) > 0) s.append(buf, k);
    fclose(f);
    const std::string key = "\"" + sig + "\"";
    const size_t pos = s.find(key);
    if (pos == std::string::npos) return false;
    const size_t br = s.find('[', pos);
    if (br == std::string::npos) return false;
    int v[4];
    if (sscanf(s.c_str() + br, "[%d, %d, %d, %d]", &v[0], &v[1], &v[2], &v[3]) != 4) return false;
    if (v[0] <= 0 || v[1] <= 0 || v[1] % 32 || v[1] > 1024 || v[2] <= 0 || v[3] <= 0) return false;
    *t = mf_batch_tiling{v[0], v[1], v[2], v[3]};
    return true;
}

void cache_store(const char *path, const std::string &sig, const mf_batch_tiling &t)
{
    if (!path) return;
    std::string s;
    if (FILE *f = fopen(path, "r")) {
        char buf[4096];
        size_t k;
        while ((k = fread(buf, 1, sizeof buf, f)) > 0) s.append(buf, k);
        fclose(f);
    }
    char entry[512];
    snprintf(entry, sizeof entry, "\"%s\": [%d, %d, %d, %d]", sig.c_str(), t.elem_tile, t.elem_block, t.node_tile,
             t.grid_per_sm);
    const size_t a = s.find('{'), z = s.rfind('}');
    std::string body = (a != std::string::npos && z != std::string::npos && z > a) ? s.substr(a + 1, z - a - 1) : "";
    // drop an older entry of the same signature
    const std::string key = "\"" + sig + "\"";
    size_t p = body.find(key);
    if (p != std::string::npos) {
        size_t e = body.find(']', p);
        size_t from = p;
        while (from > 0 && (body[from - 1] == ' ' || body[from - 1] == ',' || body[from - 1] == '\n')) --from;
        body.erase(from, e + 1 - from);
    }
    while (!body.empty() && (body[0] == ',' || body[0] == '\n' || body[0] == ' ')) body.erase(0, 1);
    std::string out = "{\n";
    if (!body.empty()) out += body + ",\n";
    out += entry;
    out += "\n}\n";
    if (FILE *f = fopen(path, "w")) {
        fputs(out.c_str(), f);
        fclose(f);
    }
}

}  // namespace

extern "C" mf_status mf_batch_create(int32_t n, const mf_mesh *const *meshes, const mf_pattern *const *patterns,
                                     const mf_coeffs *coeffs, double *const *values, double *const *d, mf_batch **out)
{
    if (!out || n <= 0 || !meshes || !patterns || !coeffs || !values || !d)
        return mf_fail(MF_ERR_INVALID_ARG, "mf_batch_create: NULL argument or empty batch");
    *out = nullptr;
    mf_batch *b = new (std::nothrow) mf_batch();
    if (!b) return mf_fail(MF_ERR_OOM, "mf_batch_create: host allocation");
    b->n = n;
    long long cnt[3] = {0, 0, 0}, nodes = 0;
    for (int i = 0; i < n; ++i) {
        const mf_mesh *m = meshes[i];
        const mf_pattern *p = patterns[i];
        const mf_coeffs &c = coeffs[i];
        if (!m || !p || p->mesh != m || p->form != MF_FORM_THERMAL || !c.elem_coef || !values[i] || !d[i] ||
            (c.bc_mask == nullptr) != (c.bc_val == nullptr)) {
            delete b;
            return mf_fail(MF_ERR_INVALID_ARG, "mf_batch_create: problem %d is not a thermal mesh/pattern/coeffs", i);
        }
        if (m->elem == MF_Q2S_HEX || m->elem == MF_P2_TET || m->elem == MF_Q2S_QUAD) {
            delete b;
            return mf_fail(MF_ERR_UNSUPPORTED,
                           "mf_batch_create: problem %d: serendipity elements and tetrahedra are not batched", i);
        }
        const mf_adj &A = p->adj[0];
        b->host.push_back(BatchProblem{m->elem, m->npe, m->n_elems, m->n_nodes, m->coords, m->conn, c.elem_coef,
                                       c.source[0], p->scratch, p->scratch_stride, A.ptr, A.col, p->inc_ptr, p->inc,
                                       p->inc_loc, p->inc_slot, p->elem_inc, p->tr, p->kref, c.bc_mask, c.bc_val,
                                       p->row_ptr, values[i], d[i],
                                       (m->elem == MF_Q1_HEX && p->kc_df && p->n_translate == m->n_elems)
                                           ? p->kref_df : nullptr,
                                       (m->elem == MF_Q1_HEX && p->kref_df && p->n_translate == m->n_elems)
                                           ? p->kc_df : nullptr,
                                       {p->box[0], p->box[1], p->box[2]}, p->box_cls});
        cnt[m->elem] += m->n_elems;
        nodes += m->n_nodes;
    }
    if (cnt[MF_P2_TRI] > 0) {
        mf_status su = fem_consts_upload();  // this file's copy of the P2 reference sums
        if (su != MF_OK) {
            delete b;
            return su;
        }
    }
    char sig[256];
    snprintf(sig, sizeof sig, "n%d_p1_%lld_p2_%lld_q1_%lld_nodes_%lld", n, cnt[0], cnt[1], cnt[2], nodes);
    b->signature = sig;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&b->sm_count, cudaDevAttrMultiProcessorCount, dev);
    cudaError_t e = cudaMalloc(&b->dev, sizeof(BatchProblem) * n);
    if (e == cudaSuccess) e = cudaMemcpy(b->dev, b->host.data(), sizeof(BatchProblem) * n, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(b->dev);
        delete b;
        return mf_cuda_check(e, "mf_batch_create");
    }
    mf_status s = make_tiles(b, mf_batch_tiling{1024, 128, 256, 8});
    if (s != MF_OK) {
        mf_batch_destroy(b);
        return s;
    }
    *out = b;
    return MF_OK;
}

extern "C" mf_status mf_batch_set_tiling(mf_batch *b, const mf_batch_tiling *t)
{
    if (!b || !t || t->elem_tile <= 0 || t->elem_block <= 0 || t->elem_block % 32 || t->elem_block > 256 ||
        t->node_tile <= 0 || t->grid_per_sm <= 0)
        return mf_fail(MF_ERR_INVALID_ARG, "mf_batch_set_tiling: bad tiling");
    return make_tiles(b, *t);
}

extern "C" mf_status mf_batch_get_tiling(const mf_batch *b, mf_batch_tiling *t)
{
    if (!b || !t) return mf_fail(MF_ERR_INVALID_ARG, "mf_batch_get_tiling: NULL argument");
    *t = b->tiling;
    return MF_OK;
}

extern "C" mf_status mf_batch_assemble(mf_batch *b, void *stream)
{
    if (!b) return mf_fail(MF_ERR_INVALID_ARG, "mf_batch_assemble: NULL batch");
    int *status = mf_status_word();
    if (!status) return mf_fail(MF_ERR_CUDA, "mf_batch_assemble: status word unavailable");
    if (!b->exec) {
        mf_status s = capture(b, status);
        if (s != MF_OK) return s;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    mf_prof_begin("batch_graph", st);
    MF_CUDA(cudaGraphLaunch(b->exec, st));
    mf_prof_end(st);
    return MF_OK;
}

extern "C" mf_status mf_batch_autotune(mf_batch *b, const char *cache_path, void *stream, mf_batch_tiling *chosen)
{
    if (!b) return mf_fail(MF_ERR_INVALID_ARG, "mf_batch_autotune: NULL batch");
    mf_batch_tiling best{};
    if (cache_lookup(cache_path, b->signature, &best)) {
        mf_status s = make_tiles(b, best);
        if (s == MF_OK && chosen) *chosen = best;
        return s;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaEvent_t e0, e1;
    MF_CUDA(cudaEventCreate(&e0));
    MF_CUDA(cudaEventCreate(&e1));
    float best_ms = 1e30f;
    const int etile[] = {256, 1024, 4096};
    const int eblock[] = {128, 256};
    const int ntile[] = {64, 512};
    const int gps[] = {4, 16};
    for (int a : etile)
        for (int bb : eblock)
            for (int c : ntile)
                for (int g : gps) {
                    mf_status s = make_tiles(b, mf_batch_tiling{a, bb, c, g});
                    if (s == MF_OK) s = mf_batch_assemble(b, stream);  // warm-up, captures the graph
                    if (s != MF_OK) {
                        cudaEventDestroy(e0);
                        cudaEventDestroy(e1);
                        return s;
                    }
                    MF_CUDA(cudaEventRecord(e0, st));
                    for (int r = 0; r < 3; ++r) MF_CUDA(cudaGraphLaunch(b->exec, st));
                    MF_CUDA(cudaEventRecord(e1, st));
                    MF_CUDA(cudaEventSynchronize(e1));
                    float ms = 0.f;
                    cudaEventElapsedTime(&ms, e0, e1);
                    if (ms < best_ms) {
                        best_ms = ms;
                        best = b->tiling;
                    }
                }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    mf_status s = make_tiles(b, best);
    if (s != MF_OK) return s;
    cache_store(cache_path, b->signature, best);
    if (chosen) *chosen = best;
    return MF_OK;
}

extern "C" mf_status mf_batch_destroy(mf_batch *b)
{
    if (!b) return MF_OK;
    free_tiles(b);
    cudaFree(b->dev);
    delete b;
    return MF_OK;
}
