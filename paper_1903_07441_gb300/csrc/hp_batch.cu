// Batched relaxation: many planners with uneven grids solved together.
//
// Every instance gets its own colour-split planes, free-cell bits and
// convergence state (RelaxCtl: omega, residual history, sweeps).  One CUDA
// graph with a conditional while-node runs the check intervals for the whole
// batch:
//   * batch_tb_kernel: a persistent, grid-stride kernel (one wave of CTAs,
//     sized from the occupancy calculator) that walks a device-side list of
//     the tiles of every still-active instance and applies the T-fused
//     red-black SOR tile update (the same tile code as the single-field
//     kernel) with that instance's omega;
//   * batch_residual_kernel: per-instance FP32 residual max over the same list;
//   * batch_control_kernel: one thread per instance applies relax_control,
//     retires converged (or capped) instances with their completion time
//     (%globaltimer, for the per-instance latency), compacts the tile list of
//     the remaining ones and sets the loop condition.
// The tile configuration (blocking depth T and tile shape) and the check
// interval K are chosen per batch shape by a small autotuner that times the
// candidates on the batch itself (Gauss-Seidel sweeps that count towards the
// solve) and caches the choice.
#include <float.h>
#include <string.h>

#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "common.cuh"
#include "hp_internal.cuh"
#include "hp_tile.cuh"

namespace tw {

constexpr int kMaxBatch = 1024;

// Tile configurations, chosen by the autotuner independently of the blocking
// depth T: small tiles, 8 rows x 8 warps (two CTAs per SM), or deep tiles,
// 14 rows x 12 warps (one CTA per SM; the single field's T = 5..7 shape).  A
// configuration code c = T + 8 * deep names both.
template <int T, int DEEP>
struct BCfg {
    static constexpr int RB = DEEP ? 14 : 8;
    static constexpr int WARPS = DEEP ? 12 : 8;
};
constexpr int cfg_code(int T, int deep) { return T + 8 * deep; }
constexpr int cfg_T(int c) { return c & 7; }
constexpr int cfg_deep(int c) { return c >> 3; }
// the candidates: T = 2 and 4 on small tiles, T = 4, 6 and 7 on deep tiles
constexpr int kCfgCands[5] = {cfg_code(2, 0), cfg_code(4, 0), cfg_code(4, 1), cfg_code(6, 1), cfg_code(7, 1)};

struct BatchInst {
    int nx, ny, gx, gy;
    int W2, W4, S, MW;
    int tx, ty, pad0, pad1;           // tiles per row / column for the chosen T
    float *P[2][2];                   // [buffer][colour] planes
    uint32_t *MR, *MB;
    const uint8_t *occ;
    float *field;
    float *P3[2];                     // snapshot planes [colour] (error tolerance only, else null)
    float *l2p;                       // per-tile sums of squared residuals of this instance (etol only)
    unsigned int rmax;                // FP32 residual max (bits) of the current interval
    unsigned int dmax;                // FP32 max change of a free cell since the snapshot (bits)
    int active;                       // 1 while the instance is being relaxed
    int error;                        // TW_EGOAL_BLOCKED if the goal cell is occupied
    unsigned long long t_done;        // %globaltimer at retirement
    unsigned long long max64;         // final FP64 residual max (bits) and sum of squares
    double sum64;
    RelaxCtl ctl;
};

struct BatchHdr {
    int n, n_active, rounds, T;
    unsigned long long t_start;
};

__device__ __forceinline__ unsigned long long globaltimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

template <int T, int DEEP>
struct BShape {
    static constexpr int HK4 = (T + 1 + 3) / 4, HY = 2 * T;
    static constexpr int KI4 = 32 - 2 * HK4, YI = BCfg<T, DEEP>::WARPS * BCfg<T, DEEP>::RB - 2 * HY;
};

// Tiles per row and column of an instance for configuration code c.
static void tiles_for(int c, int W4, int ny, int *tx, int *ty) {
    const int T = cfg_T(c);
    const int rows = cfg_deep(c) ? BCfg<7, 1>::WARPS * BCfg<7, 1>::RB : BCfg<4, 0>::WARPS * BCfg<4, 0>::RB;
    int KI4 = 32 - 2 * ((T + 4) / 4), YI = rows - 4 * T;
    *tx = (W4 + KI4 - 1) / KI4;
    *ty = (ny + YI - 1) / YI;
}

// ---- kernels ---------------------------------------------------------------------

// Zero both ping-pong pairs of every instance, pad columns included (one
// launch for the whole batch).
__global__ void batch_zero_kernel(const BatchInst *I) {
    const BatchInst &b = I[blockIdx.y];
    const size_t n = (size_t)b.ny * b.S;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        b.P[0][0][i] = 0.0f;
        b.P[0][1][i] = 0.0f;
        b.P[1][0][i] = 0.0f;
        b.P[1][1][i] = 0.0f;
    }
}

// Instance and row of block `r` of a launch with one block per row of every
// instance (row_off: prefix sums of the instances' ny, n + 1 entries).
__device__ __forceinline__ int batch_row(const int *row_off, int n, int r, int *y) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (row_off[mid] <= r) lo = mid;
        else hi = mid - 1;
    }
    *y = r - row_off[lo];
    return lo;
}

// One block per row of every instance (the grid holds exactly the rows).
__global__ void batch_pack_kernel(BatchInst *I, const int *row_off, int n, int warm) {
    int y;
    BatchInst &b = I[batch_row(row_off, n, (int)blockIdx.x, &y)];
    const int lane = threadIdx.x & 31;
    const int kend = (b.W2 + 31) & ~31;   // whole warps: the ballot below needs every lane
    for (int k = threadIdx.x; k < kend; k += blockDim.x) {
#pragma unroll
        for (int color = 0; color < 2; color++) {
            const int x = 2 * k + ((y + color) & 1);
            float v = 0.0f;
            bool free_cell = false;
            if (k < b.W2 && x < b.nx) {
                const size_t c = (size_t)y * b.nx + x;
                const bool goal = (x == b.gx && y == b.gy);
                if (goal && b.occ[c] != 0) b.error = TW_EGOAL_BLOCKED;
                const bool fixed = goal || x == 0 || y == 0 || x == b.nx - 1 || y == b.ny - 1 || b.occ[c] != 0;
                free_cell = !fixed;
                v = goal ? 1.0f : (fixed ? 0.0f : (warm ? b.field[c] : 0.5f));
            }
            const unsigned bits = __ballot_sync(0xffffffffu, free_cell);
            if (k < b.W2) b.P[0][color][(size_t)y * b.S + 4 + k] = v;
            if (lane == 0 && (k >> 5) < b.MW) (color ? b.MB : b.MR)[(size_t)y * b.MW + (k >> 5)] = bits;
        }
    }
}

template <int T, int DEEP>
__global__ void __launch_bounds__(BCfg<T, DEEP>::WARPS * 32, DEEP ? 1 : 2)
batch_tb_kernel(BatchInst *__restrict__ I, const int2 *__restrict__ list, const BatchHdr *__restrict__ H,
                int parity) {
    constexpr int RB = BCfg<T, DEEP>::RB, WARPS = BCfg<T, DEEP>::WARPS;
    __shared__ TBShared<WARPS> sh;
    const int n_active = H->n_active;
    for (int t = blockIdx.x; t < n_active; t += gridDim.x) {
        __syncthreads();   // the previous tile's exchange buffers are free again
        const int2 it = list[t];
        const BatchInst &b = I[it.x];
        const int bx = it.y % b.tx, by = it.y / b.tx;
        tb_tile<T, RB, WARPS>(b.P[parity][0], b.P[parity][1], b.P[1 - parity][0], b.P[1 - parity][1], b.MR, b.MB,
                              b.ny, b.W4, b.S, b.MW, b.ctl.omega_f, bx, by, sh);
    }
}

// FP32 residual max of each active tile's interior, one atomic per CTA and tile.
// With an error tolerance (the instance has snapshot planes) also the tile's
// sum of squared residuals, into its own slot (added in tile order by the
// control kernel: deterministic), and the snapshot work of the single-field
// residual pass (snap 1: copy the planes; 2: also the largest change of a
// free cell since the copy, atomicMax into dmax).
template <int T, int DEEP>
__global__ void __launch_bounds__(256)
batch_residual_kernel(BatchInst *__restrict__ I, const int2 *__restrict__ list, const BatchHdr *__restrict__ H) {
    using Sh = BShape<T, DEEP>;
    __shared__ float s_q[8];
    const int n_active = H->n_active;
    for (int t = blockIdx.x; t < n_active; t += gridDim.x) {
        const int2 it = list[t];
        BatchInst &b = I[it.x];
        const int bx = it.y % b.tx, by = it.y / b.tx;
        const int snap = b.P3[0] ? b.ctl.snap : 0;
        float r = 0.0f, q = 0.0f, dm = 0.0f;
        for (int idx = threadIdx.x; idx < Sh::KI4 * Sh::YI; idx += blockDim.x) {
            const int k4 = bx * Sh::KI4 + idx % Sh::KI4;
            const int y = by * Sh::YI + idx / Sh::KI4;
            if (k4 >= b.W4 || y < 1 || y >= b.ny - 1) continue;
            const int k = 4 * k4;
#pragma unroll
            for (int color = 0; color < 2; color++) {
                const float *U = b.P[0][color], *V = b.P[0][1 - color];
                const uint32_t bits = ((color ? b.MB : b.MR)[(size_t)y * b.MW + (k >> 5)] >> (k & 31)) & 0xFu;
                if (!bits) continue;
                float4 nb[4];
                rb_load_neighbours(V, b.S, y, k, (y + color) & 1, nb);
                const float4 c = *reinterpret_cast<const float4 *>(U + (size_t)y * b.S + 4 + k);
                const float t0 = rb_step(c.x, nb[0].x, nb[1].x, nb[2].x, nb[3].x);
                const float t1 = rb_step(c.y, nb[0].y, nb[1].y, nb[2].y, nb[3].y);
                const float t2 = rb_step(c.z, nb[0].z, nb[1].z, nb[2].z, nb[3].z);
                const float t3 = rb_step(c.w, nb[0].w, nb[1].w, nb[2].w, nb[3].w);
                if (bits & 1u) { r = fmaxf(r, fabsf(t0)); q = fmaf(t0, t0, q); }
                if (bits & 2u) { r = fmaxf(r, fabsf(t1)); q = fmaf(t1, t1, q); }
                if (bits & 4u) { r = fmaxf(r, fabsf(t2)); q = fmaf(t2, t2, q); }
                if (bits & 8u) { r = fmaxf(r, fabsf(t3)); q = fmaf(t3, t3, q); }
                if (snap) {
                    float4 *Pp = reinterpret_cast<float4 *>(b.P3[color] + (size_t)y * b.S + 4 + k);
                    if (snap == 2) {
                        const float4 o = *Pp;
                        if (bits & 1u) dm = fmaxf(dm, fabsf(c.x - o.x));
                        if (bits & 2u) dm = fmaxf(dm, fabsf(c.y - o.y));
                        if (bits & 4u) dm = fmaxf(dm, fabsf(c.z - o.z));
                        if (bits & 8u) dm = fmaxf(dm, fabsf(c.w - o.w));
                    }
                    *Pp = c;
                }
            }
        }
        if (b.l2p) {   // the tile's sum of squares, reduced in a fixed order
            for (int o = 16; o > 0; o >>= 1) q += __shfl_xor_sync(0xffffffffu, q, o);
            if ((threadIdx.x & 31) == 0) s_q[threadIdx.x >> 5] = q;
            __syncthreads();
            if (threadIdx.x == 0) {
                float v = 0.0f;
                for (int w = 0; w < 8; w++) v += s_q[w];
                b.l2p[it.y] = v;
            }
        }
        block_max2_atomic(r, &b.rmax, dm, snap == 2 ? &b.dmax : nullptr);
        __syncthreads();
    }
}

// Per-instance control and tile-list compaction (one block, one thread per instance).
__global__ void __launch_bounds__(kMaxBatch)
batch_control_kernel(BatchInst *__restrict__ I, BatchHdr *__restrict__ H, int2 *__restrict__ list, int max_rounds,
                     int final_check, cudaGraphConditionalHandle handle, int use_handle) {
    __shared__ int s_scan[kMaxBatch];
    const int i = threadIdx.x;
    const int n = H->n;
    int my_tiles = 0;
    if (i < n) {
        BatchInst &b = I[i];
        if (b.active) {
            RelaxCtl c = b.ctl;
            const float rf = __uint_as_float(b.rmax);
            b.rmax = 0u;
            double e = -1.0, d = -1.0;
            if (b.l2p) {   // error tolerance: the 2-norm (tile order) and the change since the snapshot
                double sum = 0.0;
                for (int t = 0; t < b.tx * b.ty; t++) sum += (double)b.l2p[t];
                e = sqrt(sum);
                if (c.snap == 2) d = (double)__uint_as_float(b.dmax);
                b.dmax = 0u;
            }
            c.sweeps += c.K;
            int go = relax_control(c, (double)rf, e, c.K, d);
            if (c.sweeps + c.K > c.max_sweeps || final_check) go = 0;
            if (b.error) go = 0;
            c.omega_f = (float)c.omega;
            b.ctl = c;
            if (!go) {
                b.active = 0;
                b.t_done = globaltimer();
            } else {
                my_tiles = b.tx * b.ty;
            }
        }
    }
    // exclusive scan of the active instances' tile counts
    s_scan[i] = my_tiles;
    __syncthreads();
    for (int off = 1; off < kMaxBatch; off <<= 1) {
        const int v = i >= off ? s_scan[i - off] : 0;
        __syncthreads();
        s_scan[i] += v;
        __syncthreads();
    }
    const int end = s_scan[i], start = end - my_tiles;
    for (int t = 0; t < my_tiles; t++) list[start + t] = make_int2(i, t);
    if (i == kMaxBatch - 1) {
        H->n_active = end;
        H->rounds += 1;
        const int go = end > 0 && H->rounds < max_rounds;
        if (use_handle) cudaGraphSetConditional(handle, go ? 1u : 0u);
    }
}

__global__ void batch_unpack_kernel(BatchInst *I, const int *row_off, int n, int to_phi) {
    int y;
    const BatchInst &b = I[batch_row(row_off, n, (int)blockIdx.x, &y)];
    for (int x = threadIdx.x; x < b.nx; x += blockDim.x) {
        const float v = b.P[0][(x + y) & 1][(size_t)y * b.S + 4 + (x >> 1)];
        b.field[(size_t)y * b.nx + x] = to_phi ? 1.0f - v : v;
    }
}

__global__ void __launch_bounds__(256) batch_final_residual_kernel(BatchInst *I, const int *row_off, int n) {
    int y;
    BatchInst &b = I[batch_row(row_off, n, (int)blockIdx.x, &y)];
    float hi = 0.0f, lo = 0.0f, q = 0.0f;
    if (y > 0 && y < b.ny - 1) {
        for (int x = 1 + threadIdx.x; x < b.nx - 1; x += blockDim.x) {
            const size_t c = (size_t)y * b.nx + x;
            const bool fixed = b.occ[c] != 0 || (x == b.gx && y == b.gy);
            if (!fixed) {
                const float *u = b.field;
                float h, l;
                resid_pair(u[c + 1], u[c - 1], u[c + b.nx], u[c - b.nx], u[c], h, l);
                pair_max(hi, lo, h, l);
                q = fmaf(h, h, q);
            }
        }
    }
    block_max_sum_pair(hi, lo, q, &b.max64, &b.sum64);
}

__global__ void batch_start_kernel(BatchHdr *H) { H->t_start = globaltimer(); }

// ---- host side ------------------------------------------------------------------------

struct BatchLayout {
    BatchHdr *hdr;
    BatchInst *inst;
    int *row_off;     // prefix sums of the instances' ny (n + 1 entries)
    int2 *list;
    float *l2p;       // per-tile sums of squares (error tolerance only), max_tiles entries
    size_t max_tiles;
};

// est: carve the error estimate's snapshot planes and per-tile partial sums
static size_t carve_batch(Carver &cv, int n, const hp_instance *in, std::vector<BatchInst> *host,
                          BatchLayout *L, bool est) {
    BatchLayout l;
    l.hdr = cv.take<BatchHdr>(1);
    l.inst = cv.take<BatchInst>(n > 0 ? n : 1);
    l.row_off = cv.take<int>((size_t)(n > 0 ? n : 1) + 1);
    size_t max_tiles = 0;
    for (int i = 0; i < n; i++) {
        RBLayout g = rb_layout(in[i].nx, in[i].ny);
        int tx2, ty2;
        tiles_for(cfg_code(4, 0), g.W4, in[i].ny, &tx2, &ty2);   // the candidate with the most tiles
        max_tiles += (size_t)tx2 * ty2;
    }
    l.list = cv.take<int2>(max_tiles > 0 ? max_tiles : 1);
    l.l2p = est ? cv.take<float>(max_tiles > 0 ? max_tiles : 1) : nullptr;
    l.max_tiles = max_tiles;
    for (int i = 0; i < n; i++) {
        RBLayout g = rb_layout(in[i].nx, in[i].ny);
        const size_t plane = (size_t)in[i].ny * g.S;
        BatchInst b;
        memset(&b, 0, sizeof(b));
        b.nx = in[i].nx; b.ny = in[i].ny; b.gx = in[i].gx; b.gy = in[i].gy;
        b.W2 = g.W2; b.W4 = g.W4; b.S = g.S; b.MW = g.MW;
        b.P[0][0] = cv.take<float>(plane); b.P[0][1] = cv.take<float>(plane);
        b.P[1][0] = cv.take<float>(plane); b.P[1][1] = cv.take<float>(plane);
        b.MR = cv.take<uint32_t>((size_t)in[i].ny * g.MW);
        b.MB = cv.take<uint32_t>((size_t)in[i].ny * g.MW);
        if (est) {   // written before they are read (the first check takes the snapshot)
            b.P3[0] = cv.take<float>(plane);
            b.P3[1] = cv.take<float>(plane);
        }
        b.occ = in[i].occ_dev;
        b.field = in[i].field_dev;
        if (host) host->push_back(b);
    }
    if (L) *L = l;
    return cv.need;
}

static std::mutex g_batch_mutex;
// per batch shape (dev, ws, n, cells): the tuned configuration code and check interval, and the
// slowest instance's sweeps at the last call (the autotuner's estimate of S)
typedef std::tuple<int, const void *, int, size_t> BatchKey;
static std::map<BatchKey, std::pair<int, int>> g_tuned;
static std::map<BatchKey, int> g_last_sweeps;

struct BatchGraph {
    int dev, T, K, rounds;   // T: the configuration code
    const void *ws;
    int n;
    cudaGraph_t graph;
    cudaGraphExec_t exec;
};
static std::vector<BatchGraph> g_batch_graphs;

static int persistent_grid(const void *func, int threads, size_t smem) {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, func, threads, smem);
    if (per < 1) per = 1;
    return sms * per;
}

template <int T, int DEEP>
static void launch_batch_sweep(BatchLayout &L, int parity, cudaStream_t s) {
    constexpr int threads = BCfg<T, DEEP>::WARPS * 32;
    const int grid = persistent_grid((const void *)batch_tb_kernel<T, DEEP>, threads, 0);
    TW_LAUNCH((batch_tb_kernel<T, DEEP>), grid, threads, 0, s, L.inst, L.list, L.hdr, parity);
}

// c: configuration code (cfg_code)
static void launch_batch_sweep_T(int c, BatchLayout &L, int parity, cudaStream_t s) {
    switch (c) {
        case cfg_code(7, 1): launch_batch_sweep<7, 1>(L, parity, s); break;
        case cfg_code(6, 1): launch_batch_sweep<6, 1>(L, parity, s); break;
        case cfg_code(4, 1): launch_batch_sweep<4, 1>(L, parity, s); break;
        case cfg_code(4, 0): launch_batch_sweep<4, 0>(L, parity, s); break;
        default: launch_batch_sweep<2, 0>(L, parity, s); break;
    }
}

static void launch_batch_residual_T(int c, BatchLayout &L, cudaStream_t s) {
    int sms = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    switch (c) {
        case cfg_code(7, 1): TW_LAUNCH((batch_residual_kernel<7, 1>), sms * 4, 256, 0, s, L.inst, L.list, L.hdr); break;
        case cfg_code(6, 1): TW_LAUNCH((batch_residual_kernel<6, 1>), sms * 4, 256, 0, s, L.inst, L.list, L.hdr); break;
        case cfg_code(4, 1): TW_LAUNCH((batch_residual_kernel<4, 1>), sms * 4, 256, 0, s, L.inst, L.list, L.hdr); break;
        case cfg_code(4, 0): TW_LAUNCH((batch_residual_kernel<4, 0>), sms * 4, 256, 0, s, L.inst, L.list, L.hdr); break;
        default: TW_LAUNCH((batch_residual_kernel<2, 0>), sms * 4, 256, 0, s, L.inst, L.list, L.hdr); break;
    }
}

// c: configuration code (cfg_code); K: sweeps per check interval (an even number of launches)
static int build_batch_graph(BatchLayout L, int c, int K, int max_rounds, BatchGraph *out) {
    const int T = cfg_T(c);
    cudaGraph_t g;
    TW_CUDA(cudaGraphCreate(&g, 0));
    cudaGraphConditionalHandle h;
    cudaError_t e = cudaGraphConditionalHandleCreate(&h, g, 1u, cudaGraphCondAssignDefault);
    if (e != cudaSuccess) { cudaGraphDestroy(g); set_cuda_error(e); return 1; }
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t cnode;
    e = cudaGraphAddNode(&cnode, g, nullptr, nullptr, 0, &cp);
    if (e != cudaSuccess) { cudaGraphDestroy(g); set_cuda_error(e); return 1; }
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    // capture the body from a private stream (the launch helpers are stream-based)
    cudaStream_t cs;
    TW_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    e = cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) { cudaStreamDestroy(cs); cudaGraphDestroy(g); set_cuda_error(e); return 1; }
    for (int i = 0; i < K / T; i++) launch_batch_sweep_T(c, L, i & 1, cs);
    launch_batch_residual_T(c, L, cs);
    TW_LAUNCH(batch_control_kernel, 1, kMaxBatch, 0, cs, L.inst, L.hdr, L.list, max_rounds, 0, h, 1);
    cudaGraph_t captured = nullptr;
    e = cudaStreamEndCapture(cs, &captured);
    cudaStreamDestroy(cs);
    if (e != cudaSuccess) { cudaGraphDestroy(g); set_cuda_error(e); return TW_ECUDA; }
    cudaGraphExec_t exec;
    e = cudaGraphInstantiate(&exec, g, 0);
    if (e != cudaSuccess) { cudaGraphDestroy(g); set_cuda_error(e); return 1; }
    out->graph = g;
    out->exec = exec;
    return TW_OK;
}

// Autotuner: time each tile configuration (blocking depth and tile shape,
// kCfgCands) with two launches of Gauss-Seidel sweeps (omega = 1) on the batch
// (the sweeps count towards the solve), and the residual check once.  The
// fastest configuration per sweep wins.  The check interval K then follows
// from the measured costs: an instance that needs S sweeps pays about
// S / K checks of cost c_chk and overshoots by K / 2 sweeps of cost c_sw, so
// K* = sqrt(2 S c_chk / c_sw), rounded to an even number of launches (S: the
// slowest instance's sweeps at the previous call of this batch shape, else
// 256).
static int autotune(BatchLayout &L, std::vector<BatchInst> &hb, int n, cudaStream_t s, int S_est, int *c_out,
                    int *K_out, int *gs_sweeps) {
    float best = FLT_MAX, best_chk = 0.0f;
    int bestc = cfg_code(4, 0);
    cudaEvent_t a, b, m;
    TW_CUDA(cudaEventCreate(&a));
    TW_CUDA(cudaEventCreate(&b));
    TW_CUDA(cudaEventCreate(&m));
    *gs_sweeps = 0;
    for (int ci = 0; ci < 5; ci++) {
        const int c = kCfgCands[ci], T = cfg_T(c);
        std::vector<int2> lst;
        for (int i = 0; i < n; i++) {
            tiles_for(c, hb[i].W4, hb[i].ny, &hb[i].tx, &hb[i].ty);
            for (int t = 0; t < hb[i].tx * hb[i].ty; t++) lst.push_back(make_int2(i, t));
        }
        BatchHdr h = {n, (int)lst.size(), 0, T, 0ull};
        TW_CUDA(cudaMemcpyAsync(L.inst, hb.data(), sizeof(BatchInst) * n, cudaMemcpyHostToDevice, s));
        TW_CUDA(cudaMemcpyAsync(L.list, lst.data(), sizeof(int2) * lst.size(), cudaMemcpyHostToDevice, s));
        TW_CUDA(cudaMemcpyAsync(L.hdr, &h, sizeof(h), cudaMemcpyHostToDevice, s));
        TW_CUDA(cudaEventRecord(a, s));
        launch_batch_sweep_T(c, L, 0, s);
        launch_batch_sweep_T(c, L, 1, s);
        TW_CUDA(cudaEventRecord(m, s));
        launch_batch_residual_T(c, L, s);   // only its time is used (the interval maxima are reset below)
        TW_CUDA(cudaEventRecord(b, s));
        TW_CUDA(cudaEventSynchronize(b));
        float ms = 0.0f, chk = 0.0f;
        TW_CUDA(cudaEventElapsedTime(&ms, a, m));
        TW_CUDA(cudaEventElapsedTime(&chk, m, b));
        *gs_sweeps += 2 * T;
        const float per_sweep = ms / (2 * T);
        if (per_sweep < best) {
            best = per_sweep;
            bestc = c;
            best_chk = chk;
        }
    }
    for (int i = 0; i < n; i++) hb[i].rmax = 0u;
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaEventDestroy(m);
    // the check also runs the control kernel (about as long as a small launch)
    const double c_chk = (double)best_chk + 0.005, c_sw = (double)best;
    const double kstar = sqrt(2.0 * (double)S_est * c_chk / (c_sw > 1e-6 ? c_sw : 1e-6));
    const int T = cfg_T(bestc);
    int mm = (int)floor(kstar / (2.0 * T) + 0.5);
    if (mm < 1) mm = 1;
    if (mm > 8) mm = 8;
    *c_out = bestc;
    *K_out = 2 * T * mm;
    return TW_OK;
}

}  // namespace tw

using namespace tw;

extern "C" size_t hp_relax_batched_workspace_size(int n, const hp_instance *inst, const hp_params *p) {
    if (n < 1 || n > kMaxBatch || !inst) return 0;
    Carver cv;
    return carve_batch(cv, n, inst, nullptr, nullptr, p && p->etol > 0.0);
}

extern "C" int hp_relax_batched(int n, const hp_instance *inst, const hp_params *p, hp_stats *stats,
                                double *latency_ms, void *workspace, size_t workspace_bytes, void *stream) {
    if (n < 1 || n > kMaxBatch || !inst || !p || !stats) return TW_EINVAL;
    if (p->method != HP_RBSOR || !(p->tol >= 0.0) || p->max_sweeps < 1 ||
        ((p->flags & HP_WARM_START) && (p->flags & HP_OUT_PHI)) ||
        !(p->omega == 0.0 || (p->omega > 0.0 && p->omega < 2.0)) || !isfinite(p->etol) || p->etol < 0.0)
        return TW_EINVAL;
    const bool est = p->etol > 0.0;
    size_t cells = 0;
    for (int i = 0; i < n; i++) {
        const hp_instance &q = inst[i];
        if (q.nx < 3 || q.ny < 3 || q.nx > 65535 || q.ny > 65535 || !q.occ_dev || !q.field_dev) return TW_EINVAL;
        if (q.gx < 1 || q.gy < 1 || q.gx > q.nx - 2 || q.gy > q.ny - 2) return TW_EGOAL_BLOCKED;
        cells += (size_t)q.nx * q.ny;
    }
    if (!workspace || !ws_aligned(workspace)) return TW_EWORKSPACE;
    Carver cv(workspace, workspace_bytes);
    std::vector<BatchInst> hb;
    BatchLayout L;
    carve_batch(cv, n, inst, &hb, &L, est);
    if (!cv.ok()) return TW_EWORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    for (int i = 0; i < n; i++) {
        hb[i].active = 1;
        hb[i].ctl.omega = 1.0;
        hb[i].ctl.omega_f = 1.0f;
    }
    std::vector<int> row_off(n + 1, 0);
    for (int i = 0; i < n; i++) row_off[i + 1] = row_off[i] + hb[i].ny;
    const int rows = row_off[n];
    TW_CUDA(cudaMemcpyAsync(L.inst, hb.data(), sizeof(BatchInst) * n, cudaMemcpyHostToDevice, s));
    TW_CUDA(cudaMemcpyAsync(L.row_off, row_off.data(), sizeof(int) * (n + 1), cudaMemcpyHostToDevice, s));
    TW_LAUNCH(batch_zero_kernel, dim3(64, n), 256, 0, s, L.inst);
    TW_LAUNCH(batch_pack_kernel, rows, 128, 0, s, L.inst, L.row_off, n, (p->flags & HP_WARM_START) ? 1 : 0);
    TW_CHECK_LAUNCH();
    {   // goal checks made by the pack kernel
        std::vector<BatchInst> dev_copy(n);
        TW_CUDA(cudaMemcpyAsync(dev_copy.data(), L.inst, sizeof(BatchInst) * n, cudaMemcpyDeviceToHost, s));
        TW_CUDA(cudaStreamSynchronize(s));
        for (int i = 0; i < n; i++) hb[i].error = dev_copy[i].error;
    }

    std::lock_guard<std::mutex> lock(g_batch_mutex);
    int dev = 0;
    TW_CUDA(cudaGetDevice(&dev));
    // pick the tile configuration and check interval (tuned once per batch shape)
    const BatchKey key = std::make_tuple(dev, (const void *)workspace, n, cells);
    int C;
    int Kt = 0;
    int gs_sweeps = 0;
    if (p->tblock == 2 || p->tblock == 4) {
        C = cfg_code(p->tblock, 0);
    } else if (p->tblock == 6 || p->tblock == 7) {
        C = cfg_code(p->tblock, 1);
    } else {
        auto f = g_tuned.find(key);
        if (f != g_tuned.end()) {
            C = f->second.first;
            Kt = f->second.second;
        } else {
            auto ls = g_last_sweeps.find(key);
            int e = autotune(L, hb, n, s, ls != g_last_sweeps.end() ? ls->second : 256, &C, &Kt, &gs_sweeps);
            if (e) return e;
            g_tuned[key] = std::make_pair(C, Kt);
        }
    }
    const int T = cfg_T(C);
    int K;
    if (p->check_every > 0)
        K = p->check_every / (2 * T) > 0 ? p->check_every / (2 * T) * (2 * T) : 2 * T;   // an even number of launches
    else
        K = Kt > 0 ? Kt : (32 / (2 * T) > 0 ? 32 / (2 * T) * (2 * T) : 2 * T);
    // control state and the initial tile list for the configuration
    std::vector<int2> lst;
    size_t l2off = 0;
    for (int i = 0; i < n; i++) {
        tiles_for(C, hb[i].W4, hb[i].ny, &hb[i].tx, &hb[i].ty);
        RelaxCtl &c = hb[i].ctl;
        memset(&c, 0, sizeof(c));
        c.adapt = p->omega == 0.0;
        c.omega = c.adapt ? sor_initial_omega(hb[i].nx, hb[i].ny) : p->omega;
        c.omega_max = sor_omega_cap(hb[i].nx, hb[i].ny);
        c.omega_f = (float)c.omega;
        c.r_prev = -1.0;
        c.tol = p->tol;
        c.K = K;
        c.max_sweeps = p->max_sweeps;
        c.sweeps = gs_sweeps;
        c.status = TW_NOT_CONVERGED;
        if (est) {   // the error estimate of the single-field solve; omega still adapts on the max norm
            c.etol = p->etol;
            c.Tl = K;
            c.err_raw = DBL_MAX;
            c.maxnorm_adapt = 1;
            hb[i].l2p = L.l2p + l2off;
            l2off += (size_t)hb[i].tx * hb[i].ty;
        }
        hb[i].active = hb[i].error ? 0 : 1;
        hb[i].rmax = 0;
        if (hb[i].active)
            for (int t = 0; t < hb[i].tx * hb[i].ty; t++) lst.push_back(make_int2(i, t));
    }
    BatchHdr h = {n, (int)lst.size(), 0, T, 0ull};
    TW_CUDA(cudaMemcpyAsync(L.inst, hb.data(), sizeof(BatchInst) * n, cudaMemcpyHostToDevice, s));
    if (!lst.empty())
        TW_CUDA(cudaMemcpyAsync(L.list, lst.data(), sizeof(int2) * lst.size(), cudaMemcpyHostToDevice, s));
    TW_CUDA(cudaMemcpyAsync(L.hdr, &h, sizeof(h), cudaMemcpyHostToDevice, s));
    TW_LAUNCH(batch_start_kernel, 1, 1, 0, s, L.hdr);

    const int max_rounds = (p->max_sweeps - gs_sweeps) / K > 0 ? (p->max_sweeps - gs_sweeps) / K : 1;
    BatchGraph *gr = nullptr;
    for (auto &g : g_batch_graphs)
        if (g.dev == dev && g.ws == workspace && g.n == n && g.T == C && g.K == K && g.rounds == max_rounds) gr = &g;
    if (!gr) {
        if (g_batch_graphs.size() >= 8) {
            cudaGraphExecDestroy(g_batch_graphs.front().exec);
            cudaGraphDestroy(g_batch_graphs.front().graph);
            g_batch_graphs.erase(g_batch_graphs.begin());
        }
        BatchGraph ng;
        ng.dev = dev; ng.T = C; ng.K = K; ng.rounds = max_rounds; ng.ws = workspace; ng.n = n;
        int e = build_batch_graph(L, C, K, max_rounds, &ng);
        if (e < 0) return e;
        if (e == 0) { g_batch_graphs.push_back(ng); gr = &g_batch_graphs.back(); }
    }
    if (lst.empty()) {
        // every instance failed its checks: nothing to relax
    } else if (gr) {
        TW_CUDA(cudaGraphLaunch(gr->exec, s));
    } else {   // no graph support: the same intervals driven from the host
        for (int r = 0; r < max_rounds; r++) {
            for (int i = 0; i < K / T; i++) launch_batch_sweep_T(C, L, i & 1, s);
            launch_batch_residual_T(C, L, s);
            TW_LAUNCH(batch_control_kernel, 1, kMaxBatch, 0, s, L.inst, L.hdr, L.list, max_rounds, 0,
                      (cudaGraphConditionalHandle)0, 0);
            BatchHdr hh;
            TW_CUDA(cudaMemcpyAsync(&hh, L.hdr, sizeof(hh), cudaMemcpyDeviceToHost, s));
            TW_CUDA(cudaStreamSynchronize(s));
            if (hh.n_active == 0) break;
        }
    }
    TW_LAUNCH(batch_unpack_kernel, rows, 256, 0, s, L.inst, L.row_off, n, (p->flags & HP_OUT_PHI) ? 1 : 0);
    TW_LAUNCH(batch_final_residual_kernel, rows, 256, 0, s, L.inst, L.row_off, n);
    TW_CHECK_LAUNCH();
    BatchHdr hh;
    TW_CUDA(cudaMemcpyAsync(hb.data(), L.inst, sizeof(BatchInst) * n, cudaMemcpyDeviceToHost, s));
    TW_CUDA(cudaMemcpyAsync(&hh, L.hdr, sizeof(hh), cudaMemcpyDeviceToHost, s));
    TW_CUDA(cudaStreamSynchronize(s));
    // launches run inside the graph: rounds x (K/T sweeps + residual + control)
    count_launches((unsigned long long)hh.rounds * (K / T + 2));
    int worst = TW_OK, slowest = 0;
    for (int i = 0; i < n; i++) {
        if (!hb[i].error && hb[i].ctl.sweeps > slowest) slowest = hb[i].ctl.sweeps;
        const BatchInst &b = hb[i];
        hp_stats &st = stats[i];
        memset(&st, 0, sizeof(st));
        double rinf;
        memcpy(&rinf, &b.max64, sizeof(double));
        st.resid_inf = rinf;
        st.resid_l2 = sqrt(b.sum64);
        st.sweeps = b.ctl.sweeps;
        st.checks = b.ctl.checks;
        st.omega = b.ctl.omega;
        st.tblock = T;
        st.loop = HP_LOOP_GRAPH;
        // with an error tolerance also the estimate (the control's own verdict, TW_OK only once both met)
        const bool err_ok = !est || b.ctl.status == TW_OK;
        st.status = b.error ? b.error : ((p->tol > 0.0 && rinf <= p->tol && err_ok) ? TW_OK : TW_NOT_CONVERGED);
        st.err_est = est ? b.ctl.err_est : 0.0;
        if (latency_ms) latency_ms[i] = b.t_done > hh.t_start ? (double)(b.t_done - hh.t_start) * 1e-6 : 0.0;
        if (st.status < 0) worst = st.status;
        else if (st.status > 0 && worst == TW_OK) worst = st.status;
    }
    if (slowest > 0) g_last_sweeps[key] = slowest;
    return worst;
}
