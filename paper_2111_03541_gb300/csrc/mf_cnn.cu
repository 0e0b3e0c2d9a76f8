// Learned preconditioner correction: a small 3D CNN on the node grid of a
// structured Q1 thermal problem, trained on the GPU by these kernels and used
// inside flexible CG (growth line of the hot path; the paper has none).
//
// Network: 4 layers of 3x3x3 convolutions, 2 -> 16 -> 16 -> 16 -> 1 channels,
// ReLU after the first three, zero padding at the grid boundary.  Weights and
// activations are BF16, every sum accumulates in FP32; the trainer keeps FP32
// master weights and AdamW moments.  Layout: channels last, node v of a batch
// grid b at (b * nv + v) * C + c, v = (z * ny + y) * nx + x.
//
// Preconditioner (per FCG iteration):
//   z = D^-1 r + s (1 - mask) CNN(r / s, log k_nodal),  s = max |r|,
// with the Jacobi step z = D^-1 r whenever z . r <= 0 or z is not finite.
// Training loss over a batch of residuals r_b of systems K_b:
//   L = (1/B) sum_b || K_b z_b - r_b ||^2 / || r_b ||^2.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include <cuda_bf16.h>

#include "mf_internal.h"

namespace {

constexpr int NL = 4;
constexpr int CIN[NL] = {2, 16, 16, 16};
constexpr int COUT[NL] = {16, 16, 16, 1};

int w_count(int l) { return COUT[l] * CIN[l] * 27; }
int p_offset_w(int l)
{
    int o = 0;
    for (int i = 0; i < l; ++i) o += w_count(i) + COUT[i];
    return o;
}
int p_offset_b(int l) { return p_offset_w(l) + w_count(l); }
int p_total() { return p_offset_b(NL - 1) + COUT[NL - 1]; }

inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

// Forward kernels are persistent (grid-stride over nodes or runs, a few
// blocks per SM), so each block stages its layer's weights in shared memory
// once.  Activations are channels-last BF16: a node's 16 channels are 32 bytes,
// moved as two 16-byte vectors.

// D += A B on one m16n8k16 tile (BF16 operands, FP32 accumulators)
__device__ __forceinline__ void mma16816(float (&c)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// Shared tiles of 16-channel BF16 rows (32 bytes per node or channel row) hold
// row k's two 16-byte halves at k * 32 + ((h ^ (k >> 2 & 1)) * 16): the 8
// rows of every ldmatrix phase over consecutive rows then hit distinct banks.
__device__ __forceinline__ uint32_t wg_swz(int k, int h) { return (uint32_t)(k * 32 + ((h ^ ((k >> 2) & 1)) << 4)); }

__device__ __forceinline__ void ldsm_x4(uint32_t addr, uint32_t &r0, uint32_t &r1, uint32_t &r2, uint32_t &r3)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(addr));
}

__device__ __forceinline__ void ldsm_x4_trans(uint32_t addr, uint32_t &r0, uint32_t &r1, uint32_t &r2, uint32_t &r3)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(addr));
}

// 16-byte global -> shared copy, zero-filled (nothing read) when !valid
__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src, bool valid)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src), "r"(valid ? 16 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// 16 -> 16 channel layer on tensor cores, forward and input gradient.
// Implicit GEMM, one warp per x-run of 16 nodes: M = 16 nodes, N = 2 x 8
// channels, K = 27 offsets x 16 channels (one mma.sync m16n8k16 per offset and
// n-tile).  The run's 9 neighbour rows (18 nodes each, zero outside the grid)
// are staged in shared memory by cp.async, the next run's rows in flight while
// this one computes; A fragments come from them by ldmatrix (row = node, the
// shift dx is a row offset), B fragments by ldmatrix from the weights, kept
// per offset as [n][k] rows.
//   Forward (BWD = false): out[v][co] = ReLU(b[co] + sum_o sum_ci
//     w[co][ci][o] in[v + off(o)][ci]), n = co, k = ci.
//   Input gradient (BWD = true): with the stencil symmetric (v - off(o) =
//     v + off(26 - o)), gin[v][ci] = sum_o sum_co w[co][ci][26 - o]
//     g[v + off(o)][co] is the same GEMM with n = ci, k = co and the offsets
//     flipped; g is the output gradient already masked by its ReLU and rounded
//     to BF16, and the result is written the same way for the layer below:
//     out[v][ci] = bf16(gin[v][ci]) where act[v][ci] > 0 (its ReLU output), else 0.
//   Last layer (MODE CV_LAST, 16 -> 1): y[v] = b + sum_o sum_ci w[ci][o]
//     in[v + off(o)][ci] in FP32 to yout; one n-tile whose column 0 holds the
//     weights (the other seven are zero).
constexpr int CV_WARPS = 8;
constexpr int CV_ROW = 18 * 32;     // one staged neighbour row
constexpr int CV_RUN = 9 * CV_ROW;  // the 9 (dz, dy) rows of one run
constexpr int CV_SMEM = 27 * 512 + CV_WARPS * 2 * CV_RUN;

// position of x-run `run` (B * nz * ny * ceil(nx / 16) runs, fewer than 2^31)
struct RunPos {
    int b, z, y, xb;
};
__device__ __forceinline__ RunPos run_pos(int run, int xt, int ny, int nz)
{
    RunPos p;
    const int row = run / xt;
    p.xb = (run - row * xt) * 16;
    const int plane = row / ny;
    p.y = row - plane * ny;
    p.b = plane / nz;
    p.z = plane - p.b * nz;
    return p;
}

// stage the 9 neighbour rows of the run at p: nodes xb - 1 .. xb + 16 of rows
// (z + dz, y + dy), 36 16-byte chunks per row; lane l copies chunk l and,
// for l < 4, chunk 32 + l
__device__ __forceinline__ void cv_stage(const RunPos &p, int nz, int ny, int nx, const __nv_bfloat16 *in,
                                         uint32_t dst, int lane)
{
    const int64_t bo = (int64_t)p.b * nz * ny * nx;
    const int k1 = lane >> 1, k2 = 16 + (lane >> 1), h = lane & 1;
    const uint32_t s1 = wg_swz(k1, h), s2 = wg_swz(k2, h);
    const int x1 = p.xb - 1 + k1, x2 = p.xb - 1 + k2;
    const bool v1 = x1 >= 0 && x1 < nx, v2 = lane < 4 && x2 < nx;
#pragma unroll
    for (int r = 0; r < 9; ++r) {
        const int zz = p.z + r / 3 - 1, yy = p.y + r % 3 - 1;
        const bool rv = zz >= 0 && zz < nz && yy >= 0 && yy < ny;
        const __nv_bfloat16 *row = in + (bo + ((int64_t)zz * ny + yy) * nx) * 16 + h * 8;
        cp_async16(dst + r * CV_ROW + s1, rv && v1 ? row + x1 * 16 : in, rv && v1);
        if (lane < 4) cp_async16(dst + r * CV_ROW + s2, rv && v2 ? row + x2 * 16 : in, rv && v2);
    }
}

enum { CV_FWD = 0, CV_BWD = 1, CV_LAST = 2 };

template <int MODE>
__global__ void __launch_bounds__(CV_WARPS * 32, 2) k_conv16_tc(int B, int nz, int ny, int nx,
                                                               const __nv_bfloat16 *__restrict__ in,
                                                               const __nv_bfloat16 *__restrict__ w,
                                                               const float *__restrict__ bias,
                                                               const __nv_bfloat16 *__restrict__ act,
                                                               __nv_bfloat16 *__restrict__ out, float *__restrict__ yout)
{
    constexpr bool BWD = MODE == CV_BWD, LAST = MODE == CV_LAST;
    extern __shared__ __align__(128) unsigned char cv_smem[];
    for (int i = threadIdx.x; i < 16 * 16 * 27; i += blockDim.x) {
        if (LAST) {  // B rows n = 0..15 of offset o: w[0][k][o] in row 0, zero elsewhere
            const int o = i / 256, n = (i / 16) % 16, k = i % 16;
            *reinterpret_cast<__nv_bfloat16 *>(cv_smem + o * 512 + wg_swz(n, k >> 3) + (k & 7) * 2) =
                n == 0 ? w[k * 27 + o] : __float2bfloat16_rn(0.f);
        } else {
            const int co = i / (16 * 27), ci = (i / 27) % 16, o = i % 27;  // source layout [co][ci][o]
            const int n = BWD ? ci : co, k = BWD ? co : ci, oo = BWD ? 26 - o : o;
            *reinterpret_cast<__nv_bfloat16 *>(cv_smem + oo * 512 + wg_swz(n, k >> 3) + (k & 7) * 2) = w[i];
        }
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const uint32_t sw_a = (uint32_t)__cvta_generic_to_shared(cv_smem);
    const uint32_t buf_a = sw_a + 27 * 512 + warp * 2 * CV_RUN;
    const int xt = (nx + 15) / 16;
    const int runs = B * nz * ny * xt;
    const int nv = nz * ny * nx;
    const int stride = gridDim.x * CV_WARPS;
    // ldmatrix rows of this lane.  A: (node, channel half) = (lane & 15, lane >> 4)
    // gives a0..a3; B: matrices (n 0-7, k 0-7), (n 0-7, k 8-15), (n 8-15, k 0-7),
    // (n 8-15, k 8-15) give b0, b1 of n-tile 0, then of n-tile 1.
    const int a_node = lane & 15, a_half = lane >> 4;
    const int b_n = (lane & 7) + ((lane >> 4) << 3), b_half = (lane >> 3) & 1;
    int run = blockIdx.x * CV_WARPS + warp;
    RunPos p = run_pos(run < runs ? run : 0, xt, ny, nz);
    if (run < runs) cv_stage(p, nz, ny, nx, in, buf_a, lane);
    cp_async_commit();
    int cur = 0;
    for (; run < runs; run += stride) {  // warp-uniform
        const RunPos pc = p;
        if (run + stride < runs) {
            p = run_pos(run + stride, xt, ny, nz);
            cv_stage(p, nz, ny, nx, in, buf_a + (cur ^ 1) * CV_RUN, lane);
        }
        cp_async_commit();
        cp_async_wait<1>();
        __syncwarp();
        const uint32_t rb = buf_a + cur * CV_RUN;
        float acc[2][4] = {};
#pragma unroll 3
        for (int r9 = 0; r9 < 9; ++r9) {
#pragma unroll
            for (int dx = 0; dx < 3; ++dx) {
                uint32_t a0, a1, a2, a3, b0, b1, b2, b3;
                ldsm_x4(rb + r9 * CV_ROW + wg_swz(a_node + dx, a_half), a0, a1, a2, a3);
                ldsm_x4(sw_a + (3 * r9 + dx) * 512 + wg_swz(b_n, b_half), b0, b1, b2, b3);
                mma16816(acc[0], a0, a1, a2, a3, b0, b1);
                if (!LAST) mma16816(acc[1], a0, a1, a2, a3, b2, b3);
            }
        }
        // C fragment: rows g, g + 8 (nodes xb + g, xb + g + 8), columns 2t, 2t + 1 of each n-tile
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int xx = pc.xb + g + 8 * h;
            if (xx >= nx) continue;
            const int64_t v = (int64_t)pc.b * nv + ((int64_t)pc.z * ny + pc.y) * nx + xx;
            if (LAST) {  // column 0 sits in c0 (node g) and c2 (node g + 8) of the lanes with t = 0
                if (t == 0) yout[v] = acc[0][2 * h] + bias[0];
            }
#pragma unroll
            for (int nt = 0; nt < (LAST ? 0 : 2); ++nt) {
                const int n = nt * 8 + 2 * t;
                float v0 = acc[nt][2 * h], v1 = acc[nt][2 * h + 1];
                if (BWD) {
                    const __nv_bfloat162 m = *reinterpret_cast<const __nv_bfloat162 *>(act + v * 16 + n);
                    v0 = __bfloat162float(m.x) > 0.f ? v0 : 0.f;
                    v1 = __bfloat162float(m.y) > 0.f ? v1 : 0.f;
                } else {
                    v0 = fmaxf(v0 + bias[n], 0.f);
                    v1 = fmaxf(v1 + bias[n + 1], 0.f);
                }
                __nv_bfloat162 pr;
                pr.x = __float2bfloat16_rn(v0);
                pr.y = __float2bfloat16_rn(v1);
                *reinterpret_cast<__nv_bfloat162 *>(out + v * 16 + n) = pr;
            }
        }
        __syncwarp();  // every lane done with this buffer before it is refilled
        cur ^= 1;
    }
    cp_async_wait<0>();
}

// Weight gradient of a 16 -> 16 layer on the tensor cores:
//   dW[co][ci][o] = sum_v g[v][co] in[v + off(o)][ci],   db[co] = sum_v g[v][co],
// with g the ReLU-masked output gradient in BF16.  For each offset this is a
// 16 x 16 GEMM whose K dimension runs over nodes: M = co, N = ci, K = the 16
// nodes of an x-run.  Both operands have the node index as their K index, the
// strided one of the channels-last layout, so each warp stages the run's g
// tile (16 nodes x 16 channels) and its input row (the 18 nodes x - 1 .. x + 16
// of one (dz, dy) neighbour row) in shared memory (swizzled as wg_swz) and
// transposes them into fragments with ldmatrix.trans.  Block = 9 warps, warp
// r9 = 3 (dz + 1) + (dy + 1) owns the three offsets (dz, dy, -1..1) and 24
// accumulators; the warp with dz = dy = 0 also forms db (one more MMA against
// a ones operand).  Each block walks a contiguous chunk of runs, every warp
// keeping WG_DEPTH - 1 runs in flight (cp.async), and writes its partial
// gradient; k_reduce_part sums the partials in block order (deterministic).

// two floats rounded to BF16 in one 32-bit fragment register (lo in bits 0..15)
__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi)
{
    return (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(lo)) |
           ((uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(hi)) << 16);
}

constexpr int WG_WARPS = 9;
constexpr int WG_DEPTH = 4;
constexpr int WG_STAGE = 512 + 18 * 32;  // g tile + input row

__global__ void __launch_bounds__(WG_WARPS * 32) k_conv16_mma_wgrad(int B, int nz, int ny, int nx, int chunk,
                                                                   const __nv_bfloat16 *__restrict__ in,
                                                                   const __nv_bfloat16 *__restrict__ g16,
                                                                   float *__restrict__ part)
{
    __shared__ __align__(128) unsigned char smem[WG_WARPS][WG_DEPTH][WG_STAGE];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const int dz = warp / 3 - 1, dy = warp % 3 - 1;
    const uint32_t base_a = (uint32_t)__cvta_generic_to_shared(smem[warp][0]);
    const int xt = (nx + 15) / 16;
    const int runs = B * nz * ny * xt;
    const int r0 = blockIdx.x * chunk, r1 = min(runs, r0 + chunk);
    // this lane's copies: g tile chunk (node lane / 2, half lane % 2); input
    // row chunks lane and (lane < 4) 32 + lane
    const int kg = lane >> 1, h = lane & 1, k1 = lane >> 1, k2 = 16 + (lane >> 1);
    const uint32_t sg = wg_swz(kg, h), s1 = 512 + wg_swz(k1, h), s2 = 512 + wg_swz(k2, h);
    // runs are staged in order, so their positions advance incrementally
    RunPos p = run_pos(r0 < runs ? r0 : 0, xt, ny, nz);
    auto stage = [&](uint32_t dst) {
        const int64_t bo = (int64_t)p.b * nz * ny * nx;
        const int xg = p.xb + kg;
        cp_async16(dst + sg, xg < nx ? g16 + (bo + ((int64_t)p.z * ny + p.y) * nx + xg) * 16 + h * 8 : g16, xg < nx);
        const int zz = p.z + dz, yy = p.y + dy;
        const bool rv = zz >= 0 && zz < nz && yy >= 0 && yy < ny;
        const __nv_bfloat16 *row = in + (bo + ((int64_t)zz * ny + yy) * nx) * 16 + h * 8;
        const int x1 = p.xb - 1 + k1, x2 = p.xb - 1 + k2;
        const bool v1 = rv && x1 >= 0 && x1 < nx, v2 = rv && x2 < nx;
        cp_async16(dst + s1, v1 ? row + x1 * 16 : in, v1);
        if (lane < 4) cp_async16(dst + s2, v2 ? row + x2 * 16 : in, v2);
        p.xb += 16;  // next run
        if (p.xb >= xt * 16) {
            p.xb = 0;
            if (++p.y == ny) {
                p.y = 0;
                if (++p.z == nz) {
                    p.z = 0;
                    ++p.b;
                }
            }
        }
    };
    float acc[3][2][4] = {};
    float accb[4] = {};
    const uint32_t ones = 0x3f803f80u;  // two BF16 1.0
    // this lane's ldmatrix row addresses (offset dx added per MMA group)
    const int a_node = (lane & 7) + ((lane >> 4) << 3), a_half = (lane >> 3) & 1;
    const int b_node = (lane & 7) + (((lane >> 3) & 1) << 3), b_half = lane >> 4;
#pragma unroll
    for (int i = 0; i < WG_DEPTH - 1; ++i) {
        if (r0 + i < r1) stage(base_a + i * WG_STAGE);
        cp_async_commit();
    }
    int slot = 0;
#pragma unroll 1
    for (int run = r0; run < r1; ++run) {
        const int nr = run + WG_DEPTH - 1;
        if (nr < r1) stage(base_a + ((slot + WG_DEPTH - 1) % WG_DEPTH) * WG_STAGE);
        cp_async_commit();
        cp_async_wait<WG_DEPTH - 1>();
        __syncwarp();
        const uint32_t gt_a = base_a + slot * WG_STAGE, xt_a = gt_a + 512;
        uint32_t a0, a1, a2, a3;
        ldsm_x4_trans(gt_a + wg_swz(a_node, a_half), a0, a1, a2, a3);
#pragma unroll
        for (int dx = 0; dx < 3; ++dx) {
            uint32_t b00, b01, b10, b11;
            ldsm_x4_trans(xt_a + wg_swz(b_node + dx, b_half), b00, b01, b10, b11);
            mma16816(acc[dx][0], a0, a1, a2, a3, b00, b01);
            mma16816(acc[dx][1], a0, a1, a2, a3, b10, b11);
        }
        if (warp == 4) mma16816(accb, a0, a1, a2, a3, ones, ones);
        __syncwarp();  // every lane done with this slot before it is refilled
        slot = (slot + 1) % WG_DEPTH;
    }
    cp_async_wait<0>();
    const int nw = 16 * 16 * 27;
    float *pb = part + (int64_t)blockIdx.x * (nw + 16);
#pragma unroll
    for (int dx = 0; dx < 3; ++dx) {
        const int o = 3 * warp + dx;
#pragma unroll
        for (int nt = 0; nt < 2; ++nt) {
            const int ci = nt * 8 + 2 * t;
            pb[(g * 16 + ci) * 27 + o] = acc[dx][nt][0];
            pb[(g * 16 + ci + 1) * 27 + o] = acc[dx][nt][1];
            pb[((g + 8) * 16 + ci) * 27 + o] = acc[dx][nt][2];
            pb[((g + 8) * 16 + ci + 1) * 27 + o] = acc[dx][nt][3];
        }
    }
    if (warp == 4 && t == 0) {
        pb[nw + g] = accb[0];
        pb[nw + g + 8] = accb[2];
    }
}

// Weight gradients of the first (2 -> 16) and last (16 -> 1) layers on the
// tensor cores.  One warp per x-run of 16 nodes takes all nine (dz, dy) rows
// (one MMA each, 36 accumulators); the offsets along x and the narrow channel
// side share the MMA's N = 8 columns.  Each warp keeps WF_DEPTH - 1 runs in
// flight (cp.async into its own stages: the 16-channel tile of the run and
// the nine 18-node rows of the narrow operand, one 32-bit word per node).
// The 8 warps of a block add their accumulators in warp order through shared
// memory (reusing the stages) and write one partial per block, summed by
// k_reduce_part.
//
// First layer: dW[co][ci][o] = sum_v g[v][co] x[v + off(o)][ci], ci < 2, with
// g the ReLU-masked BF16 gradient: M = co, K = nodes (the g tile transposed by
// ldmatrix.trans), N = 2 dx + ci (6 used); db[co] by an MMA against ones.
// Last layer: dW[0][ci][o] = sum_u a[u][ci] gy[u - off(o)] (the sum over
// output nodes v = u - off(o) moved onto the input node u), db = sum_v gy[v]:
// M = ci, K = nodes (the run's own activation tile, transposed), N = dx (3
// used), the B column of row (dz, dy) read from gy at (z - dz, y - dy) and
// rounded to BF16; the bias sum stays in FP32.
constexpr int WF_WARPS = 8;
constexpr int WF_DEPTH = 3;
constexpr int WF_STAGE = 1280;  // 512-byte tile + 648 bytes of rows, padded to 128 bytes

__device__ __forceinline__ void cp_async4(uint32_t dst, const void *src, bool valid)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(dst), "l"(src), "r"(valid ? 4 : 0)
                 : "memory");
}

template <bool LAST>
__global__ void __launch_bounds__(WF_WARPS * 32) k_wgrad_edge(int B, int nz, int ny, int nx, int chunk,
                                                             const __nv_bfloat16 *__restrict__ tile16,
                                                             const void *__restrict__ narrow,
                                                             float *__restrict__ part)
{
    // tile16: first layer g (masked gradient), last layer a (activations);
    // narrow: first layer x (BF16 pairs), last layer gy (FP32)
    constexpr int NW = LAST ? 16 * 27 : 16 * 2 * 27, NP = NW + (LAST ? 1 : 16);
    constexpr int BUF = WF_WARPS * WF_DEPTH * WF_STAGE > WF_WARPS * NP * 4 ? WF_WARPS * WF_DEPTH * WF_STAGE
                                                                           : WF_WARPS * NP * 4;
    __shared__ __align__(128) unsigned char smem[BUF];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const uint32_t base_a = (uint32_t)__cvta_generic_to_shared(smem) + warp * WF_DEPTH * WF_STAGE;
    const unsigned char *base_p = smem + warp * WF_DEPTH * WF_STAGE;
    const int xt = (nx + 15) / 16;
    const int runs = B * nz * ny * xt;
    const int r0 = blockIdx.x * chunk, r1 = min(runs, r0 + chunk);
    const uint32_t *nw32 = static_cast<const uint32_t *>(narrow);
    const int kg = lane >> 1, h = lane & 1;
    const uint32_t sg = wg_swz(kg, h);
    auto stage = [&](int run, uint32_t dst) {
        const RunPos p = run_pos(run, xt, ny, nz);
        const int64_t bo = (int64_t)p.b * nz * ny * nx;
        const int xg = p.xb + kg;
        cp_async16(dst + sg, xg < nx ? tile16 + (bo + ((int64_t)p.z * ny + p.y) * nx + xg) * 16 + h * 8 : tile16,
                   xg < nx);
        for (int c = lane; c < 9 * 18; c += 32) {
            const int r = c / 18, k = c - r * 18;
            // first layer: row (z + dz, y + dy); last layer: row (z - dz, y - dy)
            const int zz = LAST ? p.z - (r / 3 - 1) : p.z + r / 3 - 1;
            const int yy = LAST ? p.y - (r % 3 - 1) : p.y + r % 3 - 1;
            const int x = p.xb - 1 + k;
            const bool v = zz >= 0 && zz < nz && yy >= 0 && yy < ny && x >= 0 && x < nx;
            cp_async4(dst + 512 + c * 4, v ? nw32 + bo + ((int64_t)zz * ny + yy) * nx + x : nw32, v);
        }
    };
    float acc[9][4] = {};
    float accb[4] = {};
    float accs = 0.f;
    const uint32_t ones = 0x3f803f80u;
    const int a_node = (lane & 7) + ((lane >> 4) << 3), a_half = (lane >> 3) & 1;
    // first-layer runs go to warps round-robin; a warp's runs: r0 + warp + WF_WARPS i
#pragma unroll
    for (int i = 0; i < WF_DEPTH - 1; ++i) {
        const int run = r0 + warp + i * WF_WARPS;
        if (run < r1) stage(run, base_a + i * WF_STAGE);
        cp_async_commit();
    }
    int slot = 0;
#pragma unroll 1
    for (int run = r0 + warp; run < r1; run += WF_WARPS) {
        const int nr = run + (WF_DEPTH - 1) * WF_WARPS;
        if (nr < r1) stage(nr, base_a + ((slot + WF_DEPTH - 1) % WF_DEPTH) * WF_STAGE);
        cp_async_commit();
        cp_async_wait<WF_DEPTH - 1>();
        __syncwarp();
        const uint32_t ta = base_a + slot * WF_STAGE;
        const unsigned char *rows = base_p + slot * WF_STAGE + 512;
        uint32_t a0, a1, a2, a3;
        ldsm_x4_trans(ta + wg_swz(a_node, a_half), a0, a1, a2, a3);
        if (!LAST) {
            mma16816(accb, a0, a1, a2, a3, ones, ones);
            const int dx = g >> 1, ci = g & 1;  // this lane's B column n = g
            const uint32_t sel = ci ? 0x7632u : 0x5410u;
#pragma unroll
            for (int r = 0; r < 9; ++r) {
                // B[k][n] = x[xb + k + dx - 1][ci] of row r: stage index k + dx
                uint32_t b0 = 0u, b1 = 0u;
                if (g < 6) {
                    const uint32_t *row = reinterpret_cast<const uint32_t *>(rows) + r * 18;
                    b0 = __byte_perm(row[2 * t + dx], row[2 * t + 1 + dx], sel);
                    b1 = __byte_perm(row[2 * t + 8 + dx], row[2 * t + 9 + dx], sel);
                }
                mma16816(acc[r], a0, a1, a2, a3, b0, b1);
            }
        } else {
            if (lane < 16) accs += reinterpret_cast<const float *>(rows)[4 * 18 + 1 + lane];  // own nodes
#pragma unroll
            for (int r = 0; r < 9; ++r) {
                // B[k][dx] = gy[xb + k - dx + 1] of row r: stage index k - dx + 2
                uint32_t b0 = 0u, b1 = 0u;
                if (g < 3) {
                    const float *row = reinterpret_cast<const float *>(rows) + r * 18;
                    const int k0 = 2 * t - g + 2;
                    b0 = pack_bf16(row[k0], row[k0 + 1]);
                    b1 = pack_bf16(row[k0 + 8], row[k0 + 9]);
                }
                mma16816(acc[r], a0, a1, a2, a3, b0, b1);
            }
        }
        __syncwarp();  // every lane done with this slot before it is refilled
        slot = (slot + 1) % WF_DEPTH;
    }
    cp_async_wait<0>();
    __syncthreads();  // the stages become the reduction buffer
    float *rw = reinterpret_cast<float *>(smem) + warp * NP;
    if (!LAST) {
        // C[co][n]: c0 = (g, 2t), c1 = (g, 2t + 1), c2 / c3 the same for co = g + 8;
        // column n = 2 dx + ci, so lanes t < 3 hold dx = t, ci = 0 and 1
        if (t < 3) {
#pragma unroll
            for (int r = 0; r < 9; ++r) {
                const int o = 3 * r + t;
                rw[(g * 2 + 0) * 27 + o] = acc[r][0];
                rw[(g * 2 + 1) * 27 + o] = acc[r][1];
                rw[((g + 8) * 2 + 0) * 27 + o] = acc[r][2];
                rw[((g + 8) * 2 + 1) * 27 + o] = acc[r][3];
            }
        }
        if (t == 0) {
            rw[NW + g] = accb[0];
            rw[NW + g + 8] = accb[2];
        }
    } else {
        // C[ci][dx]: c0 = (g, 2t), c1 = (g, 2t + 1), c2 / c3 the same for ci = g + 8
#pragma unroll
        for (int r = 0; r < 9; ++r) {
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const int d = 2 * t + j;
                if (d < 3) {
                    rw[g * 27 + 3 * r + d] = acc[r][j];
                    rw[(g + 8) * 27 + 3 * r + d] = acc[r][2 + j];
                }
            }
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) accs += __shfl_xor_sync(0xffffffffu, accs, off);
        if (lane == 0) rw[NW] = accs;
    }
    __syncthreads();
    const float *red = reinterpret_cast<const float *>(smem);
    float *pb = part + (int64_t)blockIdx.x * NP;
    for (int i = threadIdx.x; i < NP; i += blockDim.x) {
        float sum = 0.f;
#pragma unroll
        for (int w = 0; w < WF_WARPS; ++w) sum += red[w * NP + i];
        pb[i] = sum;
    }
}

// Sum of per-block partials part[b][i], b < nblocks, in two fixed-order
// levels: slice s (blockIdx.y) adds blocks [s per, (s + 1) per) into
// tmp[s][i]; k_reduce_part then adds the slices.
__global__ void k_reduce_split(int nblocks, int n, int per, const float *__restrict__ part, float *__restrict__ tmp)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x, sl = blockIdx.y;
    if (i >= n) return;
    const int b0 = sl * per, b1 = min(nblocks, b0 + per);
    float s = 0.f;
    for (int b = b0; b < b1; ++b) s += part[(int64_t)b * n + i];
    tmp[(int64_t)sl * n + i] = s;
}

__global__ void k_reduce_part(int nblocks, int n, const float *__restrict__ part, float *__restrict__ out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float s = 0.f;
    for (int b = 0; b < nblocks; ++b) s += part[(int64_t)b * n + i];
    out[i] = s;
}

__global__ void k_adamw(int n, float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                        float *__restrict__ v, float lr, float b1, float b2, float eps, float wd, float c1, float c2,
                        const int *__restrict__ is_weight, __nv_bfloat16 *__restrict__ pbf)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    float pi = p[i];
    if (is_weight[i]) pi -= lr * wd * pi;
    pi -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    p[i] = pi;
    pbf[i] = __float2bfloat16_rn(pi);
}

__global__ void k_to_bf16(int n, const float *__restrict__ a, __nv_bfloat16 *__restrict__ b)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = __float2bfloat16_rn(a[i]);
}

// ---- preconditioner pieces (FP64 vectors of the Krylov solve) ----

// log k at the nodes: mean of log k over the cells touching each node; the
// cells form an (nz-1) x (ny-1) x (nx-1) grid
__global__ void k_node_logk(int nz, int ny, int nx, const double *__restrict__ kcell, float *__restrict__ out)
{
    const int nv = nz * ny * nx;
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nv) return;
    const int x = v % nx, y = (v / nx) % ny, z = v / (nx * ny);
    double s = 0.0;
    int c = 0;
    for (int dz = -1; dz <= 0; ++dz)
        for (int dy = -1; dy <= 0; ++dy)
            for (int dx = -1; dx <= 0; ++dx) {
                const int cz = z + dz, cy = y + dy, cx = x + dx;
                if (cz < 0 || cz >= nz - 1 || cy < 0 || cy >= ny - 1 || cx < 0 || cx >= nx - 1) continue;
                s += log(kcell[((int64_t)cz * (ny - 1) + cy) * (nx - 1) + cx]);
                ++c;
            }
    out[v] = c ? (float)(s / c) : 0.f;
}

// network input [nv][2] = (r / s, log k / 2) in BF16
__global__ void k_cnn_input(int64_t n, const double *__restrict__ r, const double *__restrict__ s_inv,
                            const float *__restrict__ logk, __nv_bfloat16 *__restrict__ x)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    x[2 * i] = __float2bfloat16_rn((float)(r[i] * *s_inv));
    x[2 * i + 1] = __float2bfloat16_rn(0.5f * logk[i]);
}

constexpr int RB = 256, RG = 512;  // reduction block and fixed grid

__device__ double block_sum_d(double v, double *sh)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[w] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += sh[i];
    return s;
}

// partial dot products (a.b) of up to 3 pairs, per block
__global__ void __launch_bounds__(RB) k_dots(int64_t n, const double *a0, const double *b0, const double *a1,
                                             const double *b1, const double *a2, const double *b2,
                                             double *__restrict__ part)
{
    __shared__ double sh[RB / 32];
    double s0 = 0, s1 = 0, s2 = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        if (a0) s0 = fma(a0[i], b0[i], s0);
        if (a1) s1 = fma(a1[i], b1[i], s1);
        if (a2) s2 = fma(a2[i], b2[i], s2);
    }
    s0 = block_sum_d(s0, sh);
    s1 = block_sum_d(s1, sh);
    s2 = block_sum_d(s2, sh);
    if (threadIdx.x == 0) {
        part[3 * blockIdx.x] = s0;
        part[3 * blockIdx.x + 1] = s1;
        part[3 * blockIdx.x + 2] = s2;
    }
}

__global__ void __launch_bounds__(RB) k_absmax(int64_t n, const double *__restrict__ a, double *__restrict__ part)
{
    __shared__ double sh[RB / 32];
    double m = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        m = fmax(m, fabs(a[i]));
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) sh[w] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s = fmax(s, sh[i]);
        part[blockIdx.x] = s;
    }
}

// host helpers: finish reductions on the host (few hundred doubles)
struct Reducer {
    double *part = nullptr;
    std::vector<double> h;
    cudaStream_t st;
    cudaError_t init(cudaStream_t s)
    {
        st = s;
        h.resize(3 * RG);
        return cudaMallocAsync(&part, sizeof(double) * 3 * RG, s);
    }
    ~Reducer()
    {
        if (part) cudaFreeAsync(part, st);
    }
    cudaError_t dots(int64_t n, const double *a0, const double *b0, const double *a1, const double *b1,
                     const double *a2, const double *b2, double out[3])
    {
        k_dots<<<RG, RB, 0, st>>>(n, a0, b0, a1, b1, a2, b2, part);
        cudaError_t e = cudaMemcpyAsync(h.data(), part, sizeof(double) * 3 * RG, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        out[0] = out[1] = out[2] = 0.0;
        for (int b = 0; b < RG; ++b)
            for (int k = 0; k < 3; ++k) out[k] += h[3 * b + k];
        return e;
    }
    cudaError_t absmax(int64_t n, const double *a, double *out)
    {
        k_absmax<<<RG, RB, 0, st>>>(n, a, part);
        cudaError_t e = cudaMemcpyAsync(h.data(), part, sizeof(double) * RG, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        *out = 0.0;
        for (int b = 0; b < RG; ++b) *out = fmax(*out, h[b]);
        return e;
    }
};

// Flexible CG orthogonalisation on the device: dots of z with the stored
// K-directions Q[k] (per-block partials, 8 at a time), the coefficients
// beta_k = -(z . Q[k]) / (P[k] . Q[k]) (one block per k, fixed order), and
// p = z + sum_k beta_k P[k] (k ascending).
constexpr int FCG_MAXD = 256;

__global__ void __launch_bounds__(RB) k_fcg_dots(int64_t n, const double *__restrict__ z,
                                                 const double *__restrict__ Q, int nd, double *__restrict__ part)
{
    __shared__ double sh[RB / 32];
    for (int k0 = 0; k0 < nd; k0 += 8) {
        double acc[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
            const double zi = z[i];
#pragma unroll
            for (int u = 0; u < 8; ++u)
                if (k0 + u < nd) acc[u] = fma(zi, Q[(int64_t)(k0 + u) * n + i], acc[u]);
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            if (k0 + u >= nd) break;
            double v = acc[u];
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            __syncthreads();
            if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
            __syncthreads();
            if (threadIdx.x == 0) {
                double t = 0.0;
                for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
                part[(int64_t)blockIdx.x * FCG_MAXD + k0 + u] = t;
            }
        }
    }
}

__global__ void __launch_bounds__(RB) k_fcg_beta(int nb, const double *__restrict__ part,
                                                 const double *__restrict__ pq, double *__restrict__ beta)
{
    __shared__ double sh[RB / 32];
    const int k = blockIdx.x;
    double acc = 0.0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) acc += part[(int64_t)b * FCG_MAXD + k];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
        beta[k] = -t / pq[k];
    }
}

__global__ void k_fcg_dir(int64_t n, const double *__restrict__ z, const double *__restrict__ P, int nd,
                          const double *__restrict__ beta, double *__restrict__ p)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double v = z[i];
    for (int k = 0; k < nd; ++k) v = fma(beta[k], P[(int64_t)k * n + i], v);
    p[i] = v;
}

// z = dinv r + s (1 - mask) y    (y: network output, FP32)
__global__ void k_compose_z(int64_t n, const double *__restrict__ dinv, const double *__restrict__ r,
                            const float *__restrict__ y, const uint8_t *__restrict__ mask, double s,
                            double *__restrict__ z)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double corr = (mask && mask[i]) ? 0.0 : s * (double)y[i];
    z[i] = fma(dinv[i], r[i], corr);
}

__global__ void k_jacobi(int64_t n, const double *__restrict__ dinv, const double *__restrict__ r,
                         double *__restrict__ z)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) z[i] = dinv[i] * r[i];
}

__global__ void k_axpby(int64_t n, double a, const double *__restrict__ x, double b, double *__restrict__ y)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] = fma(a, x[i], b * y[i]);
}

__global__ void k_diag_inv2(int64_t n, const int64_t *__restrict__ rp, const int32_t *__restrict__ ci,
                            const double *__restrict__ v, double *__restrict__ dinv)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double di = 0.0;
    for (int64_t t = rp[i]; t < rp[i + 1]; ++t)
        if (ci[t] == i) di = v[t];
    dinv[i] = 1.0 / di;
}

// training: e = K z - r (q holds K z), partial sums of e.e and r.r per sample
__global__ void k_train_err(int64_t n, const double *__restrict__ q, const double *__restrict__ r,
                            double *__restrict__ e)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) e[i] = q[i] - r[i];
}

// gy = coef s (1 - mask) (K e)   (FP32 gradient of the network output)
__global__ void k_train_gy(int64_t n, const double *__restrict__ ke, const uint8_t *__restrict__ mask, double coef,
                           float *__restrict__ gy)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    gy[i] = (mask && mask[i]) ? 0.f : (float)(coef * ke[i]);
}

}  // namespace

// ---------------------------------------------------------------------------
// network object
// ---------------------------------------------------------------------------
struct mf_cnn {
    int np = 0;
    float *p = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;  // FP32 master, grad, AdamW moments
    __nv_bfloat16 *pb = nullptr;                                    // BF16 copy used by the kernels
    int *is_w = nullptr;
    long long step = 0;
    // activation workspace (grown on demand)
    size_t ws_bytes = 0;
    void *ws = nullptr;
};

namespace {

// persistent grid: at most 8 blocks per SM
int num_sms()
{
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    return sms;
}

// blocks for items / per_block work units, at most blocks_per_sm per SM
unsigned conv_grid(int64_t items, int per_block, int blocks_per_sm = 8)
{
    return (unsigned)std::max<int64_t>(
        1, std::min<int64_t>((items + per_block - 1) / per_block, (int64_t)num_sms() * blocks_per_sm));
}

struct Acts {
    __nv_bfloat16 *a1, *a2, *a3;  // outputs of layers 1..3 (ReLU), BF16
    float *y;                      // layer 4 output, FP32
    __nv_bfloat16 *gA, *gB;        // ReLU-masked gradients in BF16, 16 channels (tensor-core operands)
    float *part;                   // weight-gradient partials
    int wparts;
};

mf_status ensure_ws(mf_cnn *c, int B, int nv, bool train, Acts *A, cudaStream_t st)
{
    // every region starts on a 256-byte boundary: the tensor-core kernels move
    // 16-byte vectors (uint4) and FP32 pairs, whatever B * nv is
    auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
    const size_t act = up((size_t)B * nv * 16 * sizeof(__nv_bfloat16));
    const size_t yb = up((size_t)B * nv * sizeof(float));
    const size_t gb = train ? act : 0;
    const int wparts = 1024;
    const size_t pb = train ? up((size_t)wparts * (16 * 16 * 27 + 16) * sizeof(float)) : 0;
    const size_t need = 3 * act + yb + 2 * gb + pb + 4096;
    if (need > c->ws_bytes) {
        if (c->ws) cudaFreeAsync(c->ws, st);
        c->ws = nullptr;
        MF_CUDA(cudaMallocAsync(&c->ws, need, st));
        c->ws_bytes = need;
    }
    char *q = static_cast<char *>(c->ws);
    A->a1 = reinterpret_cast<__nv_bfloat16 *>(q);
    A->a2 = reinterpret_cast<__nv_bfloat16 *>(q + act);
    A->a3 = reinterpret_cast<__nv_bfloat16 *>(q + 2 * act);
    A->y = reinterpret_cast<float *>(q + 3 * act);
    A->gA = train ? reinterpret_cast<__nv_bfloat16 *>(q + 3 * act + yb) : nullptr;
    A->gB = train ? reinterpret_cast<__nv_bfloat16 *>(q + 3 * act + yb + gb) : nullptr;
    A->part = train ? reinterpret_cast<float *>(q + 3 * act + yb + 2 * gb) : nullptr;
    A->wparts = wparts;
    return MF_OK;
}

// First layer, 2 -> 16 channels, ReLU, BF16 out, on the tensor cores.  One
// warp per x-run of 16 nodes, M = 16 nodes, N = 2 x 8 output channels; K packs
// two (dz, dy) rows of 8 values each (dx = 0..3 x 2 channels, dx = 3 with zero
// weight), so 9 rows take 5 m16n8k16 steps per n-tile.  A node's two input
// channels are one 32-bit word, so every A fragment register is one shared
// load from the staged rows (18 words per row, nodes xb - 1 .. xb + 16);
// the B fragments (weights) stay in registers.  Each warp keeps WF_DEPTH - 1
// runs in flight (cp.async).
constexpr int C1_ROWW = 18;                // words per staged row
constexpr int C1_STAGE = 9 * C1_ROWW * 4;  // bytes per run

__global__ void __launch_bounds__(CV_WARPS * 32) k_conv_first_tc(int B, int nz, int ny, int nx,
                                                                const __nv_bfloat16 *__restrict__ xin,
                                                                const __nv_bfloat16 *__restrict__ w,
                                                                const float *__restrict__ bias,
                                                                __nv_bfloat16 *__restrict__ out)
{
    __shared__ __align__(16) uint32_t stg[CV_WARPS][WF_DEPTH][9 * C1_ROWW];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    // B[k][n]: k = 8 (row parity) + 2 dx + ci, n = co (n-tile nt)
    uint32_t bw[5][2][2];
#pragma unroll
    for (int j = 0; j < 5; ++j)
#pragma unroll
        for (int nt = 0; nt < 2; ++nt)
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const int r = 2 * j + q, co = nt * 8 + g;
                uint32_t v = 0u;
                if (r < 9 && t < 3) {
                    const int o = 3 * r + t;  // source layout [co][ci][o]
                    v = (uint32_t)__bfloat16_as_ushort(w[(co * 2 + 0) * 27 + o]) |
                        ((uint32_t)__bfloat16_as_ushort(w[(co * 2 + 1) * 27 + o]) << 16);
                }
                bw[j][nt][q] = v;
            }
    float bs[2][2];
#pragma unroll
    for (int nt = 0; nt < 2; ++nt) {
        bs[nt][0] = bias[nt * 8 + 2 * t];
        bs[nt][1] = bias[nt * 8 + 2 * t + 1];
    }
    const uint32_t base_a = (uint32_t)__cvta_generic_to_shared(stg[warp][0]);
    const uint32_t *xw = reinterpret_cast<const uint32_t *>(xin);
    const int xt = (nx + 15) / 16;
    const int runs = B * nz * ny * xt;
    const int nv = nz * ny * nx;
    const int stride = gridDim.x * CV_WARPS;
    auto stage = [&](const RunPos &p, uint32_t dst) {
        const int64_t bo = (int64_t)p.b * nv;
        for (int c = lane; c < 9 * C1_ROWW; c += 32) {
            const int r = c / C1_ROWW, k = c - r * C1_ROWW;
            const int zz = p.z + r / 3 - 1, yy = p.y + r % 3 - 1, x = p.xb - 1 + k;
            const bool v = zz >= 0 && zz < nz && yy >= 0 && yy < ny && x >= 0 && x < nx;
            cp_async4(dst + c * 4, v ? xw + bo + ((int64_t)zz * ny + yy) * nx + x : xw, v);
        }
    };
    static_assert(WF_DEPTH == 3, "two runs in flight: q0 (computing), q1 (staged)");
    int run = blockIdx.x * CV_WARPS + warp;
    RunPos q0 = run_pos(run < runs ? run : 0, xt, ny, nz);
    if (run < runs) stage(q0, base_a);
    cp_async_commit();
    RunPos q1 = run_pos(run + stride < runs ? run + stride : 0, xt, ny, nz);
    if (run + stride < runs) stage(q1, base_a + C1_STAGE);
    cp_async_commit();
    int slot = 0;
    for (; run < runs; run += stride) {  // warp-uniform
        const int nr = run + 2 * stride;
        const int ns = (slot + 2) % 3;
        RunPos q2 = q1;
        if (nr < runs) {
            q2 = run_pos(nr, xt, ny, nz);
            stage(q2, base_a + ns * C1_STAGE);
        }
        cp_async_commit();
        cp_async_wait<WF_DEPTH - 1>();
        __syncwarp();
        const uint32_t *rw = stg[warp][slot];
        float acc[2][4] = {};
#pragma unroll
        for (int j = 0; j < 5; ++j) {
            // A[m][k]: node m, row 2j (k < 8) or 2j + 1, dx = t, both channels: staged word m + t
            const uint32_t *r0 = rw + (2 * j) * C1_ROWW, *r1 = rw + (2 * j + 1) * C1_ROWW;
            const uint32_t a0 = t < 3 ? r0[g + t] : 0u, a1 = t < 3 ? r0[g + 8 + t] : 0u;
            const uint32_t a2 = (t < 3 && j < 4) ? r1[g + t] : 0u, a3 = (t < 3 && j < 4) ? r1[g + 8 + t] : 0u;
            mma16816(acc[0], a0, a1, a2, a3, bw[j][0][0], bw[j][0][1]);
            mma16816(acc[1], a0, a1, a2, a3, bw[j][1][0], bw[j][1][1]);
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int xx = q0.xb + g + 8 * h;
            if (xx >= nx) continue;
            const int64_t v = (int64_t)q0.b * nv + ((int64_t)q0.z * ny + q0.y) * nx + xx;
#pragma unroll
            for (int nt = 0; nt < 2; ++nt) {
                __nv_bfloat162 pr;
                pr.x = __float2bfloat16_rn(fmaxf(acc[nt][2 * h] + bs[nt][0], 0.f));
                pr.y = __float2bfloat16_rn(fmaxf(acc[nt][2 * h + 1] + bs[nt][1], 0.f));
                *reinterpret_cast<__nv_bfloat162 *>(out + v * 16 + nt * 8 + 2 * t) = pr;
            }
        }
        __syncwarp();  // every lane done with this slot before it is refilled
        q0 = q1;
        q1 = q2;
        slot = (slot + 1) % 3;
    }
    cp_async_wait<0>();
}

// Gradient wrt the input of the last layer (16 -> 1, no ReLU on its output),
// on the tensor cores: with v - off(o) = v + off(26 - o),
//   gin[v][ci] = sum_o w[0][ci][o] gy[v - off(o)] = sum_o' w[0][ci][26 - o'] gy[v + off(o')],
// written masked by the ReLU of the layer below (act > 0) and rounded to BF16.
// One warp per x-run: M = 16 nodes, N = 2 x 8 channels, K = the 27 offsets o'
// = 3 r + dx, 15 per m16n8k16 step (5 rows x 3 dx, the 16th column zero), so
// 2 steps per n-tile; A[m][k] = gy (rounded to BF16) at staged row r, node m +
// dx; the B fragments stay in registers.  Staging as k_conv_first_tc (FP32
// words instead of channel pairs).
__global__ void __launch_bounds__(CV_WARPS * 32) k_conv_bwd_last_tc(int B, int nz, int ny, int nx,
                                                                   const float *__restrict__ gy,
                                                                   const __nv_bfloat16 *__restrict__ w,
                                                                   const __nv_bfloat16 *__restrict__ act,
                                                                   __nv_bfloat16 *__restrict__ out)
{
    __shared__ __align__(16) float stg[CV_WARPS][3][9 * C1_ROWW];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    // this lane's four K positions per step: 2t, 2t + 1 (registers a0 / a1, b0)
    // and 2t + 8, 2t + 9 (a2 / a3, b1); position k of step s is o' = 15 s + k
    // (k < 15), staged at row o' / 3, node offset o' % 3
    int aoff[2][4];
    bool aval[2][4];
    uint32_t bw[2][2][2];
#pragma unroll
    for (int st = 0; st < 2; ++st) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int k = 2 * t + (q & 1) + 8 * (q >> 1), op = 15 * st + k;
            aval[st][q] = k < 15 && op < 27;
            aoff[st][q] = aval[st][q] ? (op / 3) * C1_ROWW + op % 3 : 0;
        }
#pragma unroll
        for (int nt = 0; nt < 2; ++nt)
#pragma unroll
            for (int hh = 0; hh < 2; ++hh) {  // b0 (positions 2t, 2t + 1) and b1 (2t + 8, 2t + 9)
                const int ci = nt * 8 + g;
                uint32_t v = 0u;
#pragma unroll
                for (int j = 0; j < 2; ++j)
                    if (aval[st][2 * hh + j]) {
                        const int op = 15 * st + 2 * t + j + 8 * hh;
                        v |= (uint32_t)__bfloat16_as_ushort(w[ci * 27 + 26 - op]) << (16 * j);
                    }
                bw[st][nt][hh] = v;
            }
    }
    const uint32_t base_a = (uint32_t)__cvta_generic_to_shared(stg[warp][0]);
    const int xt = (nx + 15) / 16;
    const int runs = B * nz * ny * xt;
    const int nv = nz * ny * nx;
    const int stride = gridDim.x * CV_WARPS;
    auto stage = [&](const RunPos &p, uint32_t dst) {
        const int64_t bo = (int64_t)p.b * nv;
        for (int c = lane; c < 9 * C1_ROWW; c += 32) {
            const int r = c / C1_ROWW, k = c - r * C1_ROWW;
            const int zz = p.z + r / 3 - 1, yy = p.y + r % 3 - 1, x = p.xb - 1 + k;
            const bool v = zz >= 0 && zz < nz && yy >= 0 && yy < ny && x >= 0 && x < nx;
            cp_async4(dst + c * 4, v ? gy + bo + ((int64_t)zz * ny + yy) * nx + x : gy, v);
        }
    };
    int run = blockIdx.x * CV_WARPS + warp;
    RunPos q0 = run_pos(run < runs ? run : 0, xt, ny, nz);
    if (run < runs) stage(q0, base_a);
    cp_async_commit();
    RunPos q1 = run_pos(run + stride < runs ? run + stride : 0, xt, ny, nz);
    if (run + stride < runs) stage(q1, base_a + C1_STAGE);
    cp_async_commit();
    int slot = 0;
    for (; run < runs; run += stride) {  // warp-uniform
        const int nr = run + 2 * stride;
        RunPos q2 = q1;
        if (nr < runs) {
            q2 = run_pos(nr, xt, ny, nz);
            stage(q2, base_a + ((slot + 2) % 3) * C1_STAGE);
        }
        cp_async_commit();
        cp_async_wait<2>();
        __syncwarp();
        const float *rw = stg[warp][slot];
        float acc[2][4] = {};
#pragma unroll
        for (int st = 0; st < 2; ++st) {
            uint32_t a[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                // a0 / a2: node g; a1 / a3: node g + 8 (positions from aoff pairs)
                const int m = (q & 1) ? g + 8 : g;
                const int p0 = (q >> 1) * 2;  // first position of the pair
                const float lo = aval[st][p0] ? rw[aoff[st][p0] + m] : 0.f;
                const float hi = aval[st][p0 + 1] ? rw[aoff[st][p0 + 1] + m] : 0.f;
                a[q] = pack_bf16(lo, hi);
            }
            mma16816(acc[0], a[0], a[1], a[2], a[3], bw[st][0][0], bw[st][0][1]);
            mma16816(acc[1], a[0], a[1], a[2], a[3], bw[st][1][0], bw[st][1][1]);
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int xx = q0.xb + g + 8 * h;
            if (xx >= nx) continue;
            const int64_t v = (int64_t)q0.b * nv + ((int64_t)q0.z * ny + q0.y) * nx + xx;
#pragma unroll
            for (int nt = 0; nt < 2; ++nt) {
                const int n = nt * 8 + 2 * t;
                const __nv_bfloat162 m = *reinterpret_cast<const __nv_bfloat162 *>(act + v * 16 + n);
                __nv_bfloat162 pr;
                pr.x = __float2bfloat16_rn(__bfloat162float(m.x) > 0.f ? acc[nt][2 * h] : 0.f);
                pr.y = __float2bfloat16_rn(__bfloat162float(m.y) > 0.f ? acc[nt][2 * h + 1] : 0.f);
                *reinterpret_cast<__nv_bfloat162 *>(out + v * 16 + n) = pr;
            }
        }
        __syncwarp();  // every lane done with this slot before it is refilled
        q0 = q1;
        q1 = q2;
        slot = (slot + 1) % 3;
    }
    cp_async_wait<0>();
}

// One layer with 16 input channels on the tensor cores (mode: a 16 -> 16
// forward, a 16 -> 16 input gradient, or the 16 -> 1 last layer into yout):
// persistent, two blocks of CV_WARPS warps per SM.
void conv16(int mode, int B, int nz, int ny, int nx, const __nv_bfloat16 *in, const __nv_bfloat16 *w,
            const float *bias, const __nv_bfloat16 *act, __nv_bfloat16 *out, float *yout, cudaStream_t st)
{
    // the attribute is per device: set on every call (a host-side call of a
    // few microseconds; a failure surfaces as the launch's error)
    if (mode == CV_BWD)
        cudaFuncSetAttribute(k_conv16_tc<CV_BWD>, cudaFuncAttributeMaxDynamicSharedMemorySize, CV_SMEM);
    else if (mode == CV_LAST)
        cudaFuncSetAttribute(k_conv16_tc<CV_LAST>, cudaFuncAttributeMaxDynamicSharedMemorySize, CV_SMEM);
    else
        cudaFuncSetAttribute(k_conv16_tc<CV_FWD>, cudaFuncAttributeMaxDynamicSharedMemorySize, CV_SMEM);
    const int64_t runs = (int64_t)B * nz * ny * ((nx + 15) / 16);
    const unsigned grid = conv_grid(runs, CV_WARPS, 2);
    if (mode == CV_BWD)
        k_conv16_tc<CV_BWD><<<grid, CV_WARPS * 32, CV_SMEM, st>>>(B, nz, ny, nx, in, w, bias, act, out, yout);
    else if (mode == CV_LAST)
        k_conv16_tc<CV_LAST><<<grid, CV_WARPS * 32, CV_SMEM, st>>>(B, nz, ny, nx, in, w, bias, act, out, yout);
    else
        k_conv16_tc<CV_FWD><<<grid, CV_WARPS * 32, CV_SMEM, st>>>(B, nz, ny, nx, in, w, bias, act, out, yout);
}

void forward(mf_cnn *c, int B, int nz, int ny, int nx, const __nv_bfloat16 *x, Acts &A, cudaStream_t st)
{
    const __nv_bfloat16 *W = c->pb;
    const float *P = c->p;
    mf_prof_begin("cnn_conv1", st);
    k_conv_first_tc<<<conv_grid(B * nz * ny * ((nx + 15) / 16), CV_WARPS, 3), CV_WARPS * 32, 0, st>>>(
        B, nz, ny, nx, x, W + p_offset_w(0), P + p_offset_b(0), A.a1);
    mf_prof_end(st);
    mf_prof_begin("cnn_conv2", st);
    conv16(CV_FWD, B, nz, ny, nx, A.a1, W + p_offset_w(1), P + p_offset_b(1), nullptr, A.a2, nullptr, st);
    mf_prof_end(st);
    mf_prof_begin("cnn_conv3", st);
    conv16(CV_FWD, B, nz, ny, nx, A.a2, W + p_offset_w(2), P + p_offset_b(2), nullptr, A.a3, nullptr, st);
    mf_prof_end(st);
    mf_prof_begin("cnn_conv4", st);
    conv16(CV_LAST, B, nz, ny, nx, A.a3, W + p_offset_w(3), P + p_offset_b(3), nullptr, nullptr, A.y, st);
    mf_prof_end(st);
}

// Blocks for a weight-gradient kernel: one wave at its occupancy, leaving
// RED_SLICES rows of the partial buffer for the first reduction level.
constexpr int RED_SLICES = 16;

template <typename K>
int wgrad_blocks(K kernel, int threads, int runs, const Acts &A)
{
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, threads, 0) != cudaSuccess || occ < 1) occ = 1;
    return std::max(1, std::min({runs, occ * num_sms(), A.wparts - RED_SLICES}));
}

// out[i] = sum_b part[b][i] over nblocks partials of n values (deterministic)
void reduce_parts(int nblocks, int n, float *part, float *out, cudaStream_t st)
{
    const int per = (nblocks + RED_SLICES - 1) / RED_SLICES;
    float *tmp = part + (int64_t)nblocks * n;
    k_reduce_split<<<dim3(nblk(n, 128), RED_SLICES), 128, 0, st>>>(nblocks, n, per, part, tmp);
    k_reduce_part<<<nblk(n, 128), 128, 0, st>>>(RED_SLICES, n, tmp, out);
}

// Weight gradient of a 16 -> 16 layer (index l) from its input activations
// and its ReLU-masked BF16 output gradient, on the tensor cores.
void bwd_weight16(mf_cnn *c, int l, int B, int nz, int ny, int nx, const __nv_bfloat16 *in,
                  const __nv_bfloat16 *g16, Acts &A, cudaStream_t st)
{
    const int runs = B * nz * ny * ((nx + 15) / 16);
    const int nb = wgrad_blocks(k_conv16_mma_wgrad, WG_WARPS * 32, runs, A);
    const int chunk = (runs + nb - 1) / nb;
    const int nblocks = (runs + chunk - 1) / chunk;
    static const char *names[4] = {"cnn_bwd_weight1", "cnn_bwd_weight2", "cnn_bwd_weight3", "cnn_bwd_weight4"};
    mf_prof_begin(names[l], st);
    k_conv16_mma_wgrad<<<nblocks, WG_WARPS * 32, 0, st>>>(B, nz, ny, nx, chunk, in, g16, A.part);
    reduce_parts(nblocks, 16 * 16 * 27 + 16, A.part, c->g + p_offset_w(l), st);
    mf_prof_end(st);
}

// Weight gradient of the first (2 -> 16, l = 0) or last (16 -> 1, l = 3)
// layer on the tensor cores.
void bwd_weight_edge(mf_cnn *c, int l, int B, int nz, int ny, int nx, const __nv_bfloat16 *in,
                     const __nv_bfloat16 *g16, const float *gy, Acts &A, cudaStream_t st)
{
    const int runs = B * nz * ny * ((nx + 15) / 16);
    const int nb = l == 0 ? wgrad_blocks(k_wgrad_edge<false>, WF_WARPS * 32, runs, A)
                          : wgrad_blocks(k_wgrad_edge<true>, WF_WARPS * 32, runs, A);
    const int chunk = (runs + nb - 1) / nb;
    const int nblocks = (runs + chunk - 1) / chunk;
    static const char *names[4] = {"cnn_bwd_weight1", "cnn_bwd_weight2", "cnn_bwd_weight3", "cnn_bwd_weight4"};
    mf_prof_begin(names[l], st);
    int n;
    if (l == 0) {
        k_wgrad_edge<false><<<nblocks, WF_WARPS * 32, 0, st>>>(B, nz, ny, nx, chunk, g16, in, A.part);
        n = 16 * 2 * 27 + 16;
    } else {
        k_wgrad_edge<true><<<nblocks, WF_WARPS * 32, 0, st>>>(B, nz, ny, nx, chunk, in, gy, A.part);
        n = 16 * 27 + 1;
    }
    reduce_parts(nblocks, n, A.part, c->g + p_offset_w(l), st);
    mf_prof_end(st);
}

void backward(mf_cnn *c, int B, int nz, int ny, int nx, const __nv_bfloat16 *x, const float *gy, Acts &A,
              cudaStream_t st)
{
    const __nv_bfloat16 *W = c->pb;
    __nv_bfloat16 *gA = A.gA, *gB = A.gB;
    // layer 4 (no ReLU): dL/dy = gy; gradient wrt a3, masked by a3 > 0 -> gA
    bwd_weight_edge(c, 3, B, nz, ny, nx, A.a3, nullptr, gy, A, st);
    mf_prof_begin("cnn_bwd_data4", st);
    k_conv_bwd_last_tc<<<conv_grid(B * nz * ny * ((nx + 15) / 16), CV_WARPS, 3), CV_WARPS * 32, 0, st>>>(
        B, nz, ny, nx, gy, W + p_offset_w(3), A.a3, gA);
    mf_prof_end(st);
    // layer 3: input a2; gradient wrt a2, masked by a2 > 0 -> gB
    bwd_weight16(c, 2, B, nz, ny, nx, A.a2, gA, A, st);
    mf_prof_begin("cnn_bwd_data3", st);
    conv16(CV_BWD, B, nz, ny, nx, gA, W + p_offset_w(2), nullptr, A.a2, gB, nullptr, st);
    mf_prof_end(st);
    // layer 2: input a1; gradient wrt a1, masked by a1 > 0 -> gA
    bwd_weight16(c, 1, B, nz, ny, nx, A.a1, gB, A, st);
    mf_prof_begin("cnn_bwd_data2", st);
    conv16(CV_BWD, B, nz, ny, nx, gB, W + p_offset_w(1), nullptr, A.a1, gA, nullptr, st);
    mf_prof_end(st);
    // layer 1 (input gradient not needed)
    bwd_weight_edge(c, 0, B, nz, ny, nx, x, gA, nullptr, A, st);
}

}  // namespace

extern "C" int64_t mf_cnn_num_params(void) { return p_total(); }

extern "C" mf_status mf_cnn_create(const float *init, mf_cnn **out)
{
    if (!init || !out) return mf_fail(MF_ERR_INVALID_ARG, "mf_cnn_create: NULL argument");
    *out = nullptr;
    mf_cnn *c = new (std::nothrow) mf_cnn();
    if (!c) return mf_fail(MF_ERR_OOM, "mf_cnn_create: host allocation");
    c->np = p_total();
    const size_t n = c->np;
    cudaError_t e = cudaMalloc(&c->p, 4 * n * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&c->pb, n * sizeof(__nv_bfloat16));
    if (e == cudaSuccess) e = cudaMalloc(&c->is_w, n * sizeof(int));
    if (e != cudaSuccess) {
        mf_cnn_destroy(c);
        return mf_cuda_check(e, "mf_cnn_create");
    }
    c->g = c->p + n;
    c->m = c->p + 2 * n;
    c->v = c->p + 3 * n;
    std::vector<int> isw(n, 0);
    for (int l = 0; l < NL; ++l)
        for (int i = 0; i < w_count(l); ++i) isw[p_offset_w(l) + i] = 1;
    cudaMemcpy(c->p, init, n * sizeof(float), cudaMemcpyHostToDevice);
    cudaMemset(c->m, 0, 2 * n * sizeof(float));
    cudaMemcpy(c->is_w, isw.data(), n * sizeof(int), cudaMemcpyHostToDevice);
    k_to_bf16<<<nblk(n, 256), 256>>>((int)n, c->p, c->pb);
    e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        mf_cnn_destroy(c);
        return mf_cuda_check(e, "mf_cnn_create");
    }
    *out = c;
    return MF_OK;
}

extern "C" mf_status mf_cnn_destroy(mf_cnn *c)
{
    if (!c) return MF_OK;
    cudaFree(c->p);
    cudaFree(c->pb);
    cudaFree(c->is_w);
    cudaFree(c->ws);
    delete c;
    return MF_OK;
}

extern "C" mf_status mf_cnn_get_params(const mf_cnn *c, float *host, int64_t n)
{
    if (!c || !host || n != c->np) return mf_fail(MF_ERR_INVALID_ARG, "mf_cnn_get_params: bad argument");
    MF_CUDA(cudaMemcpy(host, c->p, n * sizeof(float), cudaMemcpyDeviceToHost));
    return MF_OK;
}

extern "C" mf_status mf_cnn_get_grads(const mf_cnn *c, float *host, int64_t n)
{
    if (!c || !host || n != c->np) return mf_fail(MF_ERR_INVALID_ARG, "mf_cnn_get_grads: bad argument");
    MF_CUDA(cudaMemcpy(host, c->g, n * sizeof(float), cudaMemcpyDeviceToHost));
    return MF_OK;
}

extern "C" mf_status mf_cnn_forward(mf_cnn *c, int32_t B, int32_t nz, int32_t ny, int32_t nx, const void *x,
                                    float *y, void *stream)
{
    if (!c || !x || !y || B <= 0 || nz <= 0 || ny <= 0 || nx <= 0 || (int64_t)B * nz * ny * nx > INT32_MAX / 16 ||
        (reinterpret_cast<uintptr_t>(x) & 3))
        return mf_fail(MF_ERR_INVALID_ARG, "mf_cnn_forward: bad argument");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    Acts A;
    mf_status s = ensure_ws(c, B, nz * ny * nx, false, &A, st);
    if (s != MF_OK) return s;
    mf_prof_begin("cnn_forward", st);
    forward(c, B, nz, ny, nx, static_cast<const __nv_bfloat16 *>(x), A, st);
    mf_prof_end(st);
    MF_CUDA(cudaMemcpyAsync(y, A.y, sizeof(float) * (size_t)B * nz * ny * nx, cudaMemcpyDeviceToDevice, st));
    MF_CUDA(cudaGetLastError());
    return MF_OK;
}

extern "C" mf_status mf_cnn_backward(mf_cnn *c, int32_t B, int32_t nz, int32_t ny, int32_t nx, const void *x,
                                     const float *gy, void *stream)
{
    if (!c || !x || !gy || B <= 0 || nz <= 0 || ny <= 0 || nx <= 0 || (int64_t)B * nz * ny * nx > INT32_MAX / 16 ||
        (reinterpret_cast<uintptr_t>(x) & 3))
        return mf_fail(MF_ERR_INVALID_ARG, "mf_cnn_backward: bad argument");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    Acts A;
    mf_status s = ensure_ws(c, B, nz * ny * nx, true, &A, st);
    if (s != MF_OK) return s;
    forward(c, B, nz, ny, nx, static_cast<const __nv_bfloat16 *>(x), A, st);
    backward(c, B, nz, ny, nx, static_cast<const __nv_bfloat16 *>(x), gy, A, st);
    MF_CUDA(cudaGetLastError());
    return MF_OK;
}

extern "C" mf_status mf_cnn_train_step(mf_cnn *c, int32_t B, int32_t nz, int32_t ny, int32_t nx,
                                       const mf_csr *K, const double *const *kvals, const double *const *r,
                                       const double *const *err, const void *const *x, const uint8_t *mask,
                                       float lr, float weight_decay, double *loss, void *stream)
{
    if (!c || !K || !kvals || !r || !x || B <= 0 || K->n_rows != (int64_t)nz * ny * nx ||
        (int64_t)B * nz * ny * nx > INT32_MAX / 16)
        return mf_fail(MF_ERR_INVALID_ARG, "mf_cnn_train_step: bad argument");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int nv = nz * ny * nx;
    // the batch input: B node grids of 2 channels, gathered into one buffer
    __nv_bfloat16 *xb = nullptr;
    double *z = nullptr, *q = nullptr, *e = nullptr, *dinv = nullptr;
    float *gy = nullptr;
    MF_CUDA(cudaMallocAsync(&xb, sizeof(__nv_bfloat16) * 2 * (size_t)B * nv, st));
    MF_CUDA(cudaMallocAsync(&z, sizeof(double) * nv * 4, st));
    MF_CUDA(cudaMallocAsync(&gy, sizeof(float) * (size_t)B * nv, st));
    q = z + nv;
    e = z + 2 * nv;
    dinv = z + 3 * nv;
    for (int b = 0; b < B; ++b)
        MF_CUDA(cudaMemcpyAsync(xb + (size_t)2 * b * nv, x[b], sizeof(__nv_bfloat16) * 2 * nv,
                                cudaMemcpyDeviceToDevice, st));
    Acts A;
    mf_status s = ensure_ws(c, B, nv, true, &A, st);
    if (s != MF_OK) return s;
    forward(c, B, nz, ny, nx, xb, A, st);
    Reducer red;
    MF_CUDA(red.init(st));
    double Ltot = 0.0;
    for (int b = 0; b < B; ++b) {
        // s_b = max |r_b|; z = D^-1 r + s (1 - mask) y; e = K z - r
        double smax = 0.0, dd[3];
        MF_CUDA(red.absmax(nv, r[b], &smax));
        k_diag_inv2<<<nblk(nv, 256), 256, 0, st>>>(nv, K->row_ptr, K->col_idx, kvals[b], dinv);
        k_compose_z<<<nblk(nv, 256), 256, 0, st>>>(nv, dinv, r[b], A.y + (size_t)b * nv, mask, smax, z);
        mf_csr Kb = *K;
        Kb.values = const_cast<double *>(kvals[b]);
        if (err && err[b]) {
            // energy left after one optimally scaled step along z (CG picks the
            // step length, so the loss ignores the scale of z):
            //   L = ||e - a z||_K^2 / ||e||_K^2 = 1 - (z.Ke)^2 / ((z.Kz)(e.Ke)),  a = z.Ke / z.Kz
            //   dL/dz = -2 (z.Ke) / ((z.Kz)(e.Ke)) (Ke - (z.Ke / z.Kz) K z)
            // (Ke, not the stored residual, keeps L in [0, 1] by Cauchy-Schwarz)
            mf_spmv_impl(&Kb, z, q, st);
            mf_spmv_impl(&Kb, err[b], e, st);  // e <- K err
            MF_CUDA(red.dots(nv, z, e, z, q, err[b], e, dd));
            const double zr = dd[0], zq = dd[1] > 0 ? dd[1] : 1.0, er = dd[2] > 0 ? dd[2] : 1.0;
            Ltot += (1.0 - zr * zr / (zq * er)) / B;
            // e <- K err - (z.Ke / z.Kz) K z ; gy = -2 (z.Ke) / ((z.Kz)(e.Ke)) s e / B
            k_axpby<<<nblk(nv, 256), 256, 0, st>>>(nv, -zr / zq, q, 1.0, e);
            k_train_gy<<<nblk(nv, 256), 256, 0, st>>>(nv, e, mask, -2.0 * zr * smax / (zq * er * B),
                                                      gy + (size_t)b * nv);
        } else {
            mf_spmv_impl(&Kb, z, q, st);
            k_train_err<<<nblk(nv, 256), 256, 0, st>>>(nv, q, r[b], e);
            MF_CUDA(red.dots(nv, e, e, r[b], r[b], nullptr, nullptr, dd));
            const double rr = dd[1] > 0 ? dd[1] : 1.0;
            Ltot += dd[0] / rr / B;
            // dL/dz = (2 / (B rr)) K e (K symmetric);  dL/dy = s (1 - mask) dL/dz
            mf_spmv_impl(&Kb, e, q, st);
            k_train_gy<<<nblk(nv, 256), 256, 0, st>>>(nv, q, mask, 2.0 * smax / (B * rr), gy + (size_t)b * nv);
        }
    }
    backward(c, B, nz, ny, nx, xb, gy, A, st);
    if (lr > 0.f) {
        c->step += 1;
        const float b1 = 0.9f, b2 = 0.999f;
        const float c1 = 1.f - powf(b1, (float)c->step), c2 = 1.f - powf(b2, (float)c->step);
        k_adamw<<<nblk(c->np, 256), 256, 0, st>>>(c->np, c->p, c->g, c->m, c->v, lr, b1, b2, 1e-8f, weight_decay, c1,
                                                  c2, c->is_w, c->pb);
    }
    MF_CUDA(cudaGetLastError());
    cudaFreeAsync(xb, st);
    cudaFreeAsync(z, st);
    cudaFreeAsync(gy, st);
    if (loss) *loss = Ltot;
    return MF_OK;
}

extern "C" mf_status mf_cnn_node_logk(int32_t nz, int32_t ny, int32_t nx, const double *kcell, float *out,
                                      void *stream)
{
    if (!kcell || !out || nz < 2 || ny < 2 || nx < 2) return mf_fail(MF_ERR_INVALID_ARG, "mf_cnn_node_logk");
    k_node_logk<<<nblk((int64_t)nz * ny * nx, 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(nz, ny, nx, kcell,
                                                                                                  out);
    MF_CUDA(cudaGetLastError());
    return MF_OK;
}

extern "C" mf_status mf_cnn_input(int64_t n, const double *r, const float *logk, void *x_bf16, void *stream)
{
    if (!r || !logk || !x_bf16 || n <= 0) return mf_fail(MF_ERR_INVALID_ARG, "mf_cnn_input");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    Reducer red;
    MF_CUDA(red.init(st));
    double smax = 0.0;
    MF_CUDA(red.absmax(n, r, &smax));
    const double sinv = smax > 0 ? 1.0 / smax : 0.0;
    double *d_sinv = nullptr;
    MF_CUDA(cudaMallocAsync(&d_sinv, sizeof(double), st));
    MF_CUDA(cudaMemcpyAsync(d_sinv, &sinv, sizeof(double), cudaMemcpyHostToDevice, st));
    k_cnn_input<<<nblk(n, 256), 256, 0, st>>>(n, r, d_sinv, logk, static_cast<__nv_bfloat16 *>(x_bf16));
    cudaFreeAsync(d_sinv, st);
    MF_CUDA(cudaGetLastError());
    return MF_OK;
}

// y = a x + b y (helper for residual bookkeeping of the training data)
extern "C" mf_status mf_axpby(int64_t n, double a, const double *x, double b, double *y, void *stream)
{
    if (!x || !y || n <= 0) return mf_fail(MF_ERR_INVALID_ARG, "mf_axpby");
    k_axpby<<<nblk(n, 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(n, a, x, b, y);
    MF_CUDA(cudaGetLastError());
    return MF_OK;
}

// Flexible CG (Notay 2000, one stored direction) with the CNN correction.
extern "C" mf_status mf_solve_fcg_cnn(const mf_csr *K, const double *d, double *x, mf_cnn *c, int32_t nz,
                                      int32_t ny, int32_t nx, const float *logk, const uint8_t *mask, double tol,
                                      int64_t max_iter, int32_t m_dirs, mf_solve_info *info, int64_t *fallbacks,
                                      void *stream)
{
    if (!K || !d || !x || !c || !logk || K->n_rows != (int64_t)nz * ny * nx || !(tol > 0) || m_dirs < 1 ||
        m_dirs > FCG_MAXD || (int64_t)nz * ny * nx > INT32_MAX / 16)
        return mf_fail(MF_ERR_INVALID_ARG, "mf_solve_fcg_cnn: bad argument");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int64_t n = K->n_rows;
    const int M = m_dirs;
    double *buf = nullptr;
    MF_CUDA(cudaMallocAsync(&buf, sizeof(double) * (4 + 2 * (size_t)M) * n, st));
    // P[i], Q[i] = K P[i]: the stored directions, ring buffer of M slots
    double *r = buf, *zv = buf + n, *dinv = buf + 2 * n, *tmp = buf + 3 * n;
    double *P = buf + 4 * n, *Q = P + (size_t)M * n;
    double *small = nullptr;  // [RG * FCG_MAXD] partials, [FCG_MAXD] p.q, [FCG_MAXD] beta
    MF_CUDA(cudaMallocAsync(&small, sizeof(double) * (RG + 2) * FCG_MAXD, st));
    double *opart = small, *pq_d = small + (size_t)RG * FCG_MAXD, *beta_d = pq_d + FCG_MAXD;
    __nv_bfloat16 *xin = nullptr;
    MF_CUDA(cudaMallocAsync(&xin, sizeof(__nv_bfloat16) * 2 * n, st));
    Acts A;
    mf_status s = ensure_ws(c, 1, (int)n, false, &A, st);
    if (s != MF_OK) return s;
    Reducer red;
    MF_CUDA(red.init(st));
    k_diag_inv2<<<nblk(n, 256), 256, 0, st>>>(n, K->row_ptr, K->col_idx, K->values, dinv);
    // r = d - K x
    mf_spmv_impl(K, x, tmp, st);
    MF_CUDA(cudaMemcpyAsync(r, d, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
    k_axpby<<<nblk(n, 256), 256, 0, st>>>(n, -1.0, tmp, 1.0, r);
    double dd3[3];
    MF_CUDA(red.dots(n, d, d, r, r, nullptr, nullptr, dd3));
    const double dn2 = dd3[0];
    double rr = dd3[1];
    int64_t it = 0, fb = 0;
    int done = rr <= tol * tol * dn2 ? 1 : 0;
    while (!done && it < max_iter) {
        // z = M(r): Jacobi plus the network correction
        double smax = 0.0;
        MF_CUDA(red.absmax(n, r, &smax));
        const double sinv = smax > 0 ? 1.0 / smax : 0.0;
        MF_CUDA(cudaMemcpyAsync(tmp, &sinv, sizeof(double), cudaMemcpyHostToDevice, st));  // tmp[0] as a scalar slot
        k_cnn_input<<<nblk(n, 256), 256, 0, st>>>(n, r, tmp, logk, xin);
        forward(c, 1, nz, ny, nx, xin, A, st);
        k_compose_z<<<nblk(n, 256), 256, 0, st>>>(n, dinv, r, A.y, mask, smax, zv);
        double zr[3];
        MF_CUDA(red.dots(n, zv, r, zv, zv, nullptr, nullptr, zr));
        if (!(zr[0] > 0.0) || !std::isfinite(zr[0]) || !std::isfinite(zr[1])) {  // descent test failed: Jacobi
            k_jacobi<<<nblk(n, 256), 256, 0, st>>>(n, dinv, r, zv);
            ++fb;
        }
        // p = z - sum_k (z . q_k / p_k . q_k) p_k over the stored directions
        // (classical Gram-Schmidt: every coefficient from z), on the device
        const int slot = (int)(it % M);
        double *p = P + (size_t)slot * n, *q = Q + (size_t)slot * n;
        const int nst = (int)std::min<int64_t>(it, M);
        if (nst > 0) {
            k_fcg_dots<<<RG, RB, 0, st>>>(n, zv, Q, nst, opart);
            k_fcg_beta<<<nst, RB, 0, st>>>(RG, opart, pq_d, beta_d);
            k_fcg_dir<<<nblk(n, 256), 256, 0, st>>>(n, zv, P, nst, beta_d, tmp);
            // the new direction takes the oldest slot only after all coefficients are known
            MF_CUDA(cudaMemcpyAsync(p, tmp, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
        } else {
            MF_CUDA(cudaMemcpyAsync(p, zv, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
        }
        mf_spmv_impl(K, p, q, st);
        double pr[3];
        MF_CUDA(red.dots(n, p, r, p, q, nullptr, nullptr, pr));
        if (!(pr[1] > 0.0) || !std::isfinite(pr[1])) {
            done = 3;
            break;
        }
        const double alpha = pr[0] / pr[1];
        MF_CUDA(cudaMemcpyAsync(pq_d + slot, &pr[1], sizeof(double), cudaMemcpyHostToDevice, st));
        MF_CUDA(cudaStreamSynchronize(st));  // pr lives on this stack frame
        k_axpby<<<nblk(n, 256), 256, 0, st>>>(n, alpha, p, 1.0, x);
        k_axpby<<<nblk(n, 256), 256, 0, st>>>(n, -alpha, q, 1.0, r);
        double rn[3];
        MF_CUDA(red.dots(n, r, r, nullptr, nullptr, nullptr, nullptr, rn));
        rr = rn[0];
        ++it;
        if (!std::isfinite(rr)) { done = 3; break; }
        if (rr <= tol * tol * dn2) done = 1;
    }
    // true residual
    mf_spmv_impl(K, x, tmp, st);
    MF_CUDA(cudaMemcpyAsync(r, d, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
    k_axpby<<<nblk(n, 256), 256, 0, st>>>(n, -1.0, tmp, 1.0, r);
    double tr[3];
    MF_CUDA(red.dots(n, r, r, nullptr, nullptr, nullptr, nullptr, tr));
    cudaFreeAsync(buf, st);
    cudaFreeAsync(xin, st);
    cudaFreeAsync(small, st);
    if (info) {
        info->iterations = it;
        info->rel_residual = dn2 > 0 ? sqrt(tr[0] / dn2) : sqrt(tr[0]);
        info->converged = done == 1;
        info->refinements = 0;
    }
    if (fallbacks) *fallbacks = fb;
    if (done == 3) return mf_fail(MF_ERR_NONFINITE, "mf_solve_fcg_cnn: breakdown");
    if (done != 1) return mf_fail(MF_ERR_NOT_CONVERGED, "mf_solve_fcg_cnn: %lld iterations", (long long)it);
    return MF_OK;
}
