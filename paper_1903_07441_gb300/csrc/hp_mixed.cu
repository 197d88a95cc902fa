// Mixed-precision defect correction (HP_MIXED).
//
// The field is kept as an FP64 master x (full layout).  Each outer step
//   1. r = (1/4) sum_nbr x - x on free cells, in FP64 (the Eq. 1 residual);
//      s = max |r|; stop when s <= tol;
//   2. q = r / s stored in low precision (FP16 or BF16, colour-split planes);
//   3. the correction equation e = (1/4) sum_nbr e + q (e = 0 on Dirichlet
//      cells) is relaxed by red-black SOR with e stored in FP16/BF16 and every
//      update computed in FP32, T sweeps fused per launch, until its own
//      residual drops by a fixed factor (the storage precision bounds what one
//      inner solve can reach);
//   4. x += s * e in FP64.
// Since A x_true = b, A e_exact = r, so x + s e converges to the solution
// while every low-precision rounding only enters through the correction;
// the final residual is that of the FP64 master, far below the FP32 floor.
// The inner sweeps move 2 + 2 + 2 bytes per cell (e read, e write, q read)
// plus the mask bit instead of 4 + 4 for FP32 storage.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <math.h>
#include <string.h>

#include <mutex>
#include <type_traits>
#include <vector>

#include "common.cuh"
#include "hp_internal.cuh"

namespace tw {

// ---- storage conversions ---------------------------------------------------
template <class S> struct Store;
template <> struct Store<float> {
    static __device__ __forceinline__ float4 load4(const float *p) { return *reinterpret_cast<const float4 *>(p); }
    static __device__ __forceinline__ void store4(float *p, float4 v) { *reinterpret_cast<float4 *>(p) = v; }
    static __device__ __forceinline__ float from(float v) { return v; }
};
template <> struct Store<__half> {
    static __device__ __forceinline__ float4 load4(const __half *p) {
        uint2 u = *reinterpret_cast<const uint2 *>(p);
        float2 a = __half22float2(*reinterpret_cast<__half2 *>(&u.x));
        float2 b = __half22float2(*reinterpret_cast<__half2 *>(&u.y));
        return make_float4(a.x, a.y, b.x, b.y);
    }
    static __device__ __forceinline__ void store4(__half *p, float4 v) {
        __half2 a = __floats2half2_rn(v.x, v.y), b = __floats2half2_rn(v.z, v.w);
        uint2 u;
        u.x = *reinterpret_cast<unsigned *>(&a);
        u.y = *reinterpret_cast<unsigned *>(&b);
        *reinterpret_cast<uint2 *>(p) = u;
    }
};
template <> struct Store<__nv_bfloat16> {
    static __device__ __forceinline__ float4 load4(const __nv_bfloat16 *p) {
        uint2 u = *reinterpret_cast<const uint2 *>(p);
        float2 a = __bfloat1622float2(*reinterpret_cast<__nv_bfloat162 *>(&u.x));
        float2 b = __bfloat1622float2(*reinterpret_cast<__nv_bfloat162 *>(&u.y));
        return make_float4(a.x, a.y, b.x, b.y);
    }
    static __device__ __forceinline__ void store4(__nv_bfloat16 *p, float4 v) {
        __nv_bfloat162 a = __floats2bfloat162_rn(v.x, v.y), b = __floats2bfloat162_rn(v.z, v.w);
        uint2 u;
        u.x = *reinterpret_cast<unsigned *>(&a);
        u.y = *reinterpret_cast<unsigned *>(&b);
        *reinterpret_cast<uint2 *>(p) = u;
    }
};

// ---- layout ------------------------------------------------------------------
struct MxLayout {
    RBLayout g;          // geometry (W2, W4, S, MW) and the free-cell bits MR/MB
    double *x;           // FP64 master, [ny][nx]
    void *e[2][2];       // [buffer][colour] correction planes, ny x S entries
    void *q[2];          // [colour] scaled right-hand side planes
    int esize;           // bytes per stored entry
};

static int storage_bytes(int storage) { return storage == HP_STORE_F32 ? 4 : 2; }

size_t carve_mixed(Carver &cv, int nx, int ny, int storage, RelaxLayout *R) {
    RBLayout g = rb_layout(nx, ny);
    const size_t plane = (size_t)ny * g.S * storage_bytes(storage);
    double *x = cv.take<double>((size_t)nx * ny);
    g.MR = cv.take<uint32_t>((size_t)ny * g.MW);
    g.MB = cv.take<uint32_t>((size_t)ny * g.MW);
    void *e00 = cv.take<char>(plane), *e01 = cv.take<char>(plane);
    void *e10 = cv.take<char>(plane), *e11 = cv.take<char>(plane);
    void *q0 = cv.take<char>(plane), *q1 = cv.take<char>(plane);
    if (R) {
        R->rb = g;
        R->mx.x = x;
        R->mx.e_r = e00; R->mx.e_b = e01; R->mx.e_r2 = e10; R->mx.e_b2 = e11;
        R->mx.q_r = q0; R->mx.q_b = q1;
    }
    return cv.need;
}

// ---- kernels -------------------------------------------------------------------

// Free-cell bits and the FP64 master's initial value.
// mode 0: planner (occ + goal; cold 0.5 unless warm); mode 1: general Dirichlet.
__global__ void mx_init_kernel(const uint8_t *__restrict__ occ, const float *__restrict__ u_in, int nx, int ny,
                               int gx, int gy, int mode, int warm, RBLayout g, double *__restrict__ x) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    int y = blockIdx.y;
    int lane = threadIdx.x & 31;
#pragma unroll
    for (int color = 0; color < 2; color++) {
        int xx = 2 * k + ((y + color) & 1);
        bool free_cell = false;
        if (k < g.W2 && xx < nx) {
            size_t c = (size_t)y * nx + xx;
            bool border = xx == 0 || y == 0 || xx == nx - 1 || y == ny - 1;
            double v;
            if (mode == 0) {
                bool goal = (xx == gx && y == gy);
                bool fixed = goal || border || occ[c] != 0;
                free_cell = !fixed;
                v = goal ? 1.0 : (fixed ? 0.0 : (warm ? (double)u_in[c] : 0.5));
            } else {
                free_cell = !(border || occ[c] != 0);
                v = (double)u_in[c];
            }
            x[c] = v;
        }
        unsigned bits = __ballot_sync(0xffffffffu, free_cell);
        if (lane == 0) {
            uint32_t *M = color ? g.MB : g.MR;
            int w = k >> 5;
            if (w < g.MW) M[(size_t)y * g.MW + w] = bits;
        }
    }
}

__device__ __forceinline__ bool mx_free(const RBLayout &g, int x, int y) {
    const int color = (x + y) & 1, k = x >> 1;
    const uint32_t *M = color ? g.MB : g.MR;
    return (M[(size_t)y * g.MW + (k >> 5)] >> (k & 31)) & 1u;
}

// FP64 residual of the master: max |r| (pass 0) or q = r / s into the planes (pass 1).
template <class S>
__global__ void __launch_bounds__(256) mx_residual_kernel(RBLayout g, const double *__restrict__ x, int nx, int ny,
                                                          int pass, const double *__restrict__ scale,
                                                          S *__restrict__ qr, S *__restrict__ qb,
                                                          unsigned long long *__restrict__ out_max) {
    // one thread per 4 entries of one colour row; both colours
    const int k4 = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    double rmax = 0.0;
    if (k4 < g.W4) {
#pragma unroll
        for (int color = 0; color < 2; color++) {
            float4 qv;
            float *qa = &qv.x;
#pragma unroll
            for (int e = 0; e < 4; e++) {
                const int k = 4 * k4 + e;
                const int xx = 2 * k + ((y + color) & 1);
                double r = 0.0;
                if (xx > 0 && xx < nx - 1 && y > 0 && y < ny - 1 && mx_free(g, xx, y)) {
                    const size_t c = (size_t)y * nx + xx;
                    r = 0.25 * (((x[c + 1] + x[c - 1]) + x[c + nx]) + x[c - nx]) - x[c];
                }
                rmax = fmax(rmax, fabs(r));
                qa[e] = pass ? (float)(r / *scale) : 0.0f;
            }
            if (pass) {
                S *q = color ? qb : qr;
                Store<S>::store4(q + (size_t)y * g.S + 4 + 4 * k4, qv);
            }
        }
    }
    if (pass == 0) block_max_sum_f64(rmax, out_max, reinterpret_cast<double *>(out_max + 1));
}

// x += s * e (FP64), e read from the colour-split planes; the largest |s e|
// of the update goes to *dmax (bits of a non-negative double, atomicMax).
template <class S>
__global__ void __launch_bounds__(256) mx_update_kernel(RBLayout g, double *__restrict__ x, int nx, int ny,
                                                        const double *__restrict__ scale, const S *__restrict__ er,
                                                        const S *__restrict__ eb,
                                                        unsigned long long *__restrict__ dmax) {
    const int xx = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    double d = 0.0;
    if (xx < nx && y < ny) {
        const int color = (xx + y) & 1, k = xx >> 1;
        const S *e = color ? eb : er;
        float4 q4 = Store<S>::load4(e + (size_t)y * g.S + 4 + (k & ~3));
        const float ev = (&q4.x)[k & 3];
        if (mx_free(g, xx, y)) {
            d = *scale * (double)ev;
            x[(size_t)y * nx + xx] += d;
        }
    }
    d = fabs(d);
    for (int o = 16; o > 0; o >>= 1) d = fmax(d, __shfl_xor_sync(0xffffffffu, d, o));
    __shared__ double sm[8];
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = d;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); w++) d = fmax(d, sm[w]);
        if (d > 0.0) atomicMax(dmax, (unsigned long long)__double_as_longlong(d));
    }
}

__global__ void mx_output_kernel(const double *__restrict__ x, float *__restrict__ out, size_t n) {
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (float)x[i];
}

// Inner residual max |(1/4) sum e_n + q - e| over free cells (FP32 from storage).
template <class S>
__global__ void __launch_bounds__(256) mx_inner_residual_kernel(RBLayout g, int ny, const S *__restrict__ er,
                                                                const S *__restrict__ eb, const S *__restrict__ qr,
                                                                const S *__restrict__ qb,
                                                                unsigned int *__restrict__ out_max) {
    const int k4 = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y + 1;
    float r = 0.0f;
    if (k4 < g.W4 && y < ny - 1) {
        const int k = 4 * k4;
#pragma unroll
        for (int color = 0; color < 2; color++) {
            const S *U = color ? eb : er;
            const S *V = color ? er : eb;
            const S *Q = color ? qb : qr;
            const uint32_t *M = color ? g.MB : g.MR;
            const uint32_t bits = (M[(size_t)y * g.MW + (k >> 5)] >> (k & 31)) & 0xFu;
            if (!bits) continue;
            const int s = (y + color) & 1;
            const S *row = V + (size_t)y * g.S + 4;
            const float4 mid = Store<S>::load4(row + k);
            const float4 up = Store<S>::load4(row - g.S + k), dn = Store<S>::load4(row + g.S + k);
            float4 ex4 = Store<S>::load4(row + (s ? k + 4 : k - 4));
            const float ex = s ? ex4.x : ex4.w;
            const float4 c = Store<S>::load4(U + (size_t)y * g.S + 4 + k);
            const float4 q = Store<S>::load4(Q + (size_t)y * g.S + 4 + k);
            float l[4], rr[4];
            if (s) { l[0] = mid.x; l[1] = mid.y; l[2] = mid.z; l[3] = mid.w; rr[0] = mid.y; rr[1] = mid.z; rr[2] = mid.w; rr[3] = ex; }
            else { l[0] = ex; l[1] = mid.x; l[2] = mid.y; l[3] = mid.z; rr[0] = mid.x; rr[1] = mid.y; rr[2] = mid.z; rr[3] = mid.w; }
            const float cu[4] = {up.x, up.y, up.z, up.w}, cd[4] = {dn.x, dn.y, dn.z, dn.w};
            const float cc[4] = {c.x, c.y, c.z, c.w}, cq[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
            for (int e = 0; e < 4; e++)
                if (bits & (1u << e))
                    r = fmaxf(r, fabsf(fmaf(0.25f, (l[e] + rr[e]) + (cu[e] + cd[e]), cq[e] - cc[e])));
        }
    }
    block_max_atomic(r, out_max);
}

// T-fused SOR sweeps of the correction equation, storage S, FP32 arithmetic.
// Same register blocking as the FP32 kernel (8 rows x float4 of both colours
// per thread, 8 warps, halo 2T rows / ceil((T+1)/4) float4 columns); the
// right-hand side of the thread's rows is converted to FP32 once, at the start,
// into the thread's own slots of shared memory (re-read from global memory or
// L1 for every row of every half-sweep, half of those reads missed L1).
constexpr int kMxRows = 8, kMxWarps = 8;
constexpr size_t kMxQBytes = sizeof(float4) * 2 * kMxRows * kMxWarps * 32;   // dynamic shared memory (64 KB)

// One half-sweep of the correction equation for colour C (compile-time, so the
// register arrays stay in registers): e <- e + omega ((1/4) sum nbr + q - e).
template <int C, class S>
__device__ __forceinline__ void mx_half(float4 (&v)[2][kMxRows], const uint32_t (&m)[2], float omega,
                                        float4 (&s_top)[2][kMxWarps][32], float4 (&s_bot)[2][kMxWarps][32],
                                        const float4 *__restrict__ sq) {
    constexpr int RB = kMxRows, WARPS = kMxWarps, O = 1 - C;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    s_top[C][warp][lane] = v[O][0];
    s_bot[C][warp][lane] = v[O][RB - 1];
    __syncthreads();
    const float4 above = warp > 0 ? s_bot[C][warp - 1][lane] : z4;
    const float4 below = warp < WARPS - 1 ? s_top[C][warp + 1][lane] : z4;
#pragma unroll
    for (int r = 0; r < RB; r++) {
        const float4 mid = v[O][r];
        const float4 up = r == 0 ? above : v[O][r - 1];
        const float4 dn = r == RB - 1 ? below : v[O][r + 1];
        float l0, l1, l2, l3, r0, r1, r2, r3;
        if (((r + C) & 1) != 0) {   // rows start even
            const float ex = __shfl_down_sync(0xffffffffu, mid.x, 1);
            l0 = mid.x; l1 = mid.y; l2 = mid.z; l3 = mid.w; r0 = mid.y; r1 = mid.z; r2 = mid.w; r3 = ex;
        } else {
            const float ex = __shfl_up_sync(0xffffffffu, mid.w, 1);
            l0 = ex; l1 = mid.x; l2 = mid.y; l3 = mid.z; r0 = mid.x; r1 = mid.y; r2 = mid.z; r3 = mid.w;
        }
        const float4 q = sq[(C * RB + r) * (WARPS * 32) + threadIdx.x];
        float4 cv = v[C][r];
        const uint32_t bits = (m[C] >> (4 * r)) & 0xFu;
        const float n0 = fmaf(omega, fmaf(0.25f, (l0 + r0) + (up.x + dn.x), q.x - cv.x), cv.x);
        const float n1 = fmaf(omega, fmaf(0.25f, (l1 + r1) + (up.y + dn.y), q.y - cv.y), cv.y);
        const float n2 = fmaf(omega, fmaf(0.25f, (l2 + r2) + (up.z + dn.z), q.z - cv.z), cv.z);
        const float n3 = fmaf(omega, fmaf(0.25f, (l3 + r3) + (up.w + dn.w), q.w - cv.w), cv.w);
        cv.x = (bits & 1u) ? n0 : cv.x;
        cv.y = (bits & 2u) ? n1 : cv.y;
        cv.z = (bits & 4u) ? n2 : cv.z;
        cv.w = (bits & 8u) ? n3 : cv.w;
        v[C][r] = cv;
    }
}

template <int T, class S>
__global__ void __launch_bounds__(kMxWarps * 32, 2)
mx_tb_kernel(const S *__restrict__ Rin, const S *__restrict__ Bin, S *__restrict__ Rout, S *__restrict__ Bout,
             const S *__restrict__ Qr, const S *__restrict__ Qb, const uint32_t *__restrict__ MR,
             const uint32_t *__restrict__ MB, int ny, int W4, int Sst, int MW, const float *__restrict__ omega_p) {
    constexpr int RB = kMxRows, WARPS = kMxWarps;
    constexpr int HK4 = (T + 1 + 3) / 4, HY = 2 * T, KI4 = 32 - 2 * HK4, YI = WARPS * RB - 2 * HY;
    __shared__ float4 s_top[2][WARPS][32];
    __shared__ float4 s_bot[2][WARPS][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int k4 = (int)blockIdx.x * KI4 - HK4 + lane;
    const int y_tile = (int)blockIdx.y * YI;
    const int y0 = y_tile - HY + warp * RB;
    const bool kin = (k4 >= 0) && (k4 < W4);
    const int k = 4 * k4;
    extern __shared__ float4 sq[];   // [colour][row][thread]: the right-hand side of the thread's rows
    const float omega = *omega_p;
    float4 v[2][RB];
    uint32_t m[2] = {0u, 0u};
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int r = 0; r < RB; r++) {
        const int y = y0 + r;
        const bool in = kin && y >= 0 && y < ny;
        const size_t off = (size_t)(in ? y : 0) * Sst + 4 + (in ? k : 0);
        v[0][r] = in ? Store<S>::load4(Rin + off) : z4;
        v[1][r] = in ? Store<S>::load4(Bin + off) : z4;
        sq[r * (WARPS * 32) + threadIdx.x] = in ? Store<S>::load4(Qr + off) : z4;
        sq[(RB + r) * (WARPS * 32) + threadIdx.x] = in ? Store<S>::load4(Qb + off) : z4;
        if (in) {
            const size_t w = (size_t)y * MW + (k >> 5);
            m[0] |= ((MR[w] >> (k & 31)) & 0xFu) << (4 * r);
            m[1] |= ((MB[w] >> (k & 31)) & 0xFu) << (4 * r);
        }
    }
#pragma unroll 1
    for (int p = 0; p < T; p++) {   // red then black, colour-indexed exchange buffers
        mx_half<0, S>(v, m, omega, s_top, s_bot, sq);
        mx_half<1, S>(v, m, omega, s_top, s_bot, sq);
    }
    const bool kint = lane >= HK4 && lane < 32 - HK4 && kin;
    if (kint) {
#pragma unroll
        for (int r = 0; r < RB; r++) {
            const int y = y0 + r;
            if (y >= y_tile && y < y_tile + YI && y < ny) {
                const size_t off = (size_t)y * Sst + 4 + k;
                Store<S>::store4(Rout + off, v[0][r]);
                Store<S>::store4(Bout + off, v[1][r]);
            }
        }
    }
}

// ---- graph-driven inner solve --------------------------------------------------------
// One correction solve as a CUDA graph: a conditional while-node whose body is
// K/T sweep launches, the inner residual and this control kernel, which takes
// the host loop's decision on the device (relax_control, then the storage-floor
// stop: after five intervals a residual that fell by less than 2 % ends the
// solve) and sets the loop condition.  ctl->pad counts the intervals.
__global__ void mx_inner_control_kernel(RelaxCtl *ctl, unsigned int *rmax, cudaGraphConditionalHandle h) {
    RelaxCtl c = *ctl;
    const float rf = __uint_as_float(*rmax);
    *rmax = 0u;
    const double prev = c.r_prev;
    const int it = c.pad;
    c.sweeps += c.K;
    int go = relax_control(c, (double)rf, -1.0, c.K, -1.0);
    if (go && prev > 0.0 && it > 4 && rf > 0.98 * prev) go = 0;   // storage floor reached
    if (c.sweeps + c.K > c.max_sweeps) go = 0;
    c.pad = it + 1;
    c.go = go;
    *ctl = c;
    cudaGraphSetConditional(h, go ? 1u : 0u);
}

struct MxGraph {
    int dev, ny, W4, ssize;
    const void *key[5];
    cudaGraph_t graph;
    cudaGraphExec_t exec;
};
static std::mutex g_mx_graph_mutex;
static std::vector<MxGraph> g_mx_graphs;

template <int T, class S>
static int mx_build_inner_graph(RBLayout g, S *const (&e)[2][2], S *const (&q)[2], RelaxScalars *sc, int ny, int K,
                                MxGraph *out) {
    cudaGraph_t G = nullptr;
    TW_CUDA(cudaGraphCreate(&G, 0));
    cudaGraphConditionalHandle h;
    cudaError_t err = cudaGraphConditionalHandleCreate(&h, G, 1u, cudaGraphCondAssignDefault);
    if (err != cudaSuccess) { cudaGraphDestroy(G); set_cuda_error(err); return TW_ECUDA; }
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t cnode;
    err = cudaGraphAddNode(&cnode, G, nullptr, nullptr, 0, &cp);
    if (err != cudaSuccess) { cudaGraphDestroy(G); set_cuda_error(err); return TW_ECUDA; }
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    cudaStream_t cs;
    err = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (err != cudaSuccess) { cudaGraphDestroy(G); set_cuda_error(err); return TW_ECUDA; }
    err = cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
    if (err != cudaSuccess) { cudaStreamDestroy(cs); cudaGraphDestroy(G); set_cuda_error(err); return TW_ECUDA; }
    const int KI4 = 32 - 2 * ((T + 4) / 4), YI = kMxWarps * kMxRows - 4 * T;
    const dim3 tgrid(ceil_div(g.W4, KI4), ceil_div(ny, YI));
    const float *omega_dev = &sc->ctl.omega_f;
    pause_launch_count(true);
    int cur = 0;
    for (int i = 0; i < K / T; i++) {
        TW_LAUNCH((mx_tb_kernel<T, S>), tgrid, kMxWarps * 32, kMxQBytes, cs, e[cur][0], e[cur][1], e[1 - cur][0],
                  e[1 - cur][1], q[0], q[1], g.MR, g.MB, ny, g.W4, g.S, g.MW, omega_dev);
        cur = 1 - cur;
    }
    TW_LAUNCH((mx_inner_residual_kernel<S>), dim3(ceil_div(g.W4, 64), ceil_div(ny, 4)), dim3(64, 4), 0, cs, g, ny,
              e[cur][0], e[cur][1], q[0], q[1], &sc->max32);
    TW_LAUNCH(mx_inner_control_kernel, 1, 1, 0, cs, &sc->ctl, &sc->max32, h);
    pause_launch_count(false);
    cudaGraph_t captured = nullptr;
    err = cudaStreamEndCapture(cs, &captured);
    cudaStreamDestroy(cs);
    if (err != cudaSuccess) { cudaGraphDestroy(G); set_cuda_error(err); return TW_ECUDA; }
    cudaGraphExec_t exec;
    err = cudaGraphInstantiate(&exec, G, 0);
    if (err != cudaSuccess) { cudaGraphDestroy(G); set_cuda_error(err); return TW_ECUDA; }
    out->graph = G;
    out->exec = exec;
    return TW_OK;
}

// Run one correction solve through the cached graph of this layout; the
// control record sc->ctl must hold the solve's starting state.
template <int T, class S>
static int mx_inner_graph(RBLayout &g, S *const (&e)[2][2], S *const (&q)[2], RelaxScalars *sc, int ny, int K,
                          cudaStream_t s) {
    int dev = 0;
    TW_CUDA(cudaGetDevice(&dev));
    const void *key[5] = {sc, e[0][0], e[1][0], q[0], g.MR};
    std::lock_guard<std::mutex> lock(g_mx_graph_mutex);
    const int ssize = (int)(sizeof(S) + 8 * std::is_same<S, __half>::value);   // the storage type
    MxGraph *ent = nullptr;
    for (auto &m : g_mx_graphs)
        if (m.dev == dev && m.ny == ny && m.W4 == g.W4 && m.ssize == ssize && !memcmp(m.key, key, sizeof(key)))
            ent = &m;
    if (!ent) {
        if (g_mx_graphs.size() >= 8) {
            cudaGraphExecDestroy(g_mx_graphs.front().exec);
            cudaGraphDestroy(g_mx_graphs.front().graph);
            g_mx_graphs.erase(g_mx_graphs.begin());
        }
        MxGraph ne;
        ne.dev = dev; ne.ny = ny; ne.W4 = g.W4;
        ne.ssize = ssize;
        memcpy(ne.key, key, sizeof(key));
        const int er = mx_build_inner_graph<T, S>(g, e, q, sc, ny, K, &ne);
        if (er) return er;
        g_mx_graphs.push_back(ne);
        ent = &g_mx_graphs.back();
    }
    TW_CUDA(cudaGraphLaunch(ent->exec, s));
    return TW_OK;
}

// ---- driver ----------------------------------------------------------------------

template <class S>
static int mixed_solve(const uint8_t *occ, int nx, int ny, int gx, int gy, float *u, int mode, const hp_params *p,
                       hp_stats *st, RelaxLayout &R, cudaStream_t s) {
    RBLayout g = R.rb;
    S *e[2][2] = {{(S *)R.mx.e_r, (S *)R.mx.e_b}, {(S *)R.mx.e_r2, (S *)R.mx.e_b2}};
    S *q[2] = {(S *)R.mx.q_r, (S *)R.mx.q_b};
    double *x = R.mx.x;
    RelaxScalars *sc = R.scal;
    const size_t plane = (size_t)ny * g.S * sizeof(S);
    for (int i = 0; i < 2; i++) {
        TW_CUDA(cudaMemsetAsync(q[i], 0, plane, s));
        TW_CUDA(cudaMemsetAsync(e[0][i], 0, plane, s));
        TW_CUDA(cudaMemsetAsync(e[1][i], 0, plane, s));
    }
    TW_LAUNCH(mx_init_kernel, dim3(ceil_div(g.W2 + 31, 128), ny), 128, 0, s, occ, u, nx, ny, gx, gy, mode,
              (p->flags & HP_WARM_START) ? 1 : 0, g, x);
    TW_CHECK_LAUNCH();
    const int T = 4, K = 32;
    TW_CUDA(cudaFuncSetAttribute(mx_tb_kernel<T, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMxQBytes));
    // inner solves relax the correction residual by this factor (bounded by the storage precision)
    const double inner_drop = (sizeof(S) == 4) ? 1e-4 : (std::is_same<S, __half>::value ? 2e-3 : 1e-2);
    RelaxCtl c;   // omega state carried across the inner solves
    memset(&c, 0, sizeof(c));
    c.adapt = p->omega == 0.0;
    c.omega = c.adapt ? sor_initial_omega(nx, ny) : p->omega;
    c.omega_max = sor_omega_cap(nx, ny);
    // Each correction solve starts from the over-relaxation the earlier ones adapted to, not from
    // where the last one ended: a correction solve ends at its storage floor, where the controller
    // takes the stagnation for the FP32 rounding floor and backs omega off for good; carried into
    // the next solve, that left every later one at omega ~1.5 (FP16 on static2048: 44 outer steps).
    const int adapt0 = c.adapt;
    double omega_keep = c.omega;
    int sweeps = 0, launches = 0, checks = 0, outer = 0;
    bool graph_used = false;
    double r_inf = 0.0, corr = 0.0, corr_prev = 0.0;   // sizes of the last two outer updates (max |s e|)
    st->status = TW_NOT_CONVERGED;
    const dim3 rgrid(ceil_div(g.W4, 128), ny), rblock(128);
    const int KI4 = 32 - 2 * ((T + 4) / 4), YI = kMxWarps * kMxRows - 4 * T;
    const dim3 tgrid(ceil_div(g.W4, KI4), ceil_div(ny, YI));
    for (;;) {
        // 1. FP64 residual max of the master
        TW_CUDA(cudaMemsetAsync(&sc->max64, 0, sizeof(sc->max64) + sizeof(sc->sum64), s));
        TW_LAUNCH((mx_residual_kernel<S>), rgrid, rblock, 0, s, g, x, nx, ny, 0, (const double *)nullptr,
                  (S *)nullptr, (S *)nullptr, &sc->max64);
        TW_CHECK_LAUNCH();
        unsigned long long mb = 0;
        TW_CUDA(cudaMemcpyAsync(&mb, &sc->max64, sizeof(mb), cudaMemcpyDeviceToHost, s));
        TW_CUDA(cudaStreamSynchronize(s));
        memcpy(&r_inf, &mb, sizeof(double));
        double sum = 0.0;
        TW_CUDA(cudaMemcpyAsync(&sum, &sc->sum64, sizeof(sum), cudaMemcpyDeviceToHost, s));
        TW_CUDA(cudaStreamSynchronize(s));
        st->resid_l2 = sqrt(sum);
        checks++;
        // outer error estimate (etol > 0): the last update's size corr shrinks by q = corr / corr_prev
        // per outer step; the error left is taken as corr / (1 - q), the whole geometric tail including
        // a step of the last update's own size -- that update comes from an inexact, low-precision
        // correction solve, and the tail alone (corr q / (1 - q)) was measured below the true error
        // (q above 0.9, or no earlier update: not estimated yet)
        double est = DBL_MAX;
        if (corr_prev > 0.0 && corr > 0.0) {
            const double q = corr / corr_prev;
            if (q < 0.9) est = corr / (1.0 - q);
        } else if (outer > 0 && corr == 0.0) {
            est = 0.0;
        }
        if (p->etol > 0.0) st->err_est = est;
        const bool r_ok = (p->tol > 0.0 && r_inf <= p->tol) || r_inf == 0.0;
        if (r_ok && (p->etol <= 0.0 || est <= p->etol)) { st->status = TW_OK; break; }
        if (p->etol > 0.0 && p->tol <= 0.0 && est <= p->etol) { st->status = TW_OK; break; }
        if (sweeps >= p->max_sweeps) break;
        // 2. q = r / s in storage precision (s kept on the device in pad1[0])
        double *scale = &sc->pad1[0];
        TW_CUDA(cudaMemcpyAsync(scale, &r_inf, sizeof(double), cudaMemcpyHostToDevice, s));
        TW_LAUNCH((mx_residual_kernel<S>), rgrid, rblock, 0, s, g, x, nx, ny, 1, (const double *)scale, q[0], q[1],
                  &sc->max64);
        // 3. inner SOR on e (cold start at 0)
        TW_CUDA(cudaMemsetAsync(e[0][0], 0, plane, s));
        TW_CUDA(cudaMemsetAsync(e[0][1], 0, plane, s));
        int cur = 0;
        c.omega = omega_keep;
        c.adapt = adapt0;
        c.r_prev = -1.0;
        c.same_iv = 0;
        c.K = K;
        c.tol = inner_drop;    // |q| <= 1, so this is the relative drop
        c.status = TW_NOT_CONVERGED;
        c.omega_f = (float)c.omega;
        float *omega_dev = &sc->ctl.omega_f;
        // whole check intervals run in the inner graph (no host round trip per interval); a cap
        // closer than one interval, or HP_HOST_LOOP, keeps the host-driven loop below
        const bool graph = !(p->flags & HP_HOST_LOOP) && p->max_sweeps - sweeps >= K;
        if (graph) {
            c.sweeps = 0;
            c.checks = 0;
            c.pad = 0;
            c.max_sweeps = p->max_sweeps - sweeps;
            c.go = 1;
            TW_CUDA(cudaMemcpyAsync(&sc->ctl, &c, sizeof(c), cudaMemcpyHostToDevice, s));
            TW_CUDA(cudaMemsetAsync(&sc->max32, 0, sizeof(unsigned int), s));
            const int er = mx_inner_graph<T, S>(g, e, q, sc, ny, K, s);
            if (er) return er;
            TW_CUDA(cudaMemcpyAsync(&c, &sc->ctl, sizeof(c), cudaMemcpyDeviceToHost, s));
            TW_CUDA(cudaStreamSynchronize(s));
            sweeps += c.sweeps;
            checks += c.checks;
            launches += c.checks * (K / T);
            count_launches((unsigned long long)c.checks * (K / T + 2));
            graph_used = true;
        }
        for (int it = 0; !graph && sweeps < p->max_sweeps; it++) {
            TW_CUDA(cudaMemcpyAsync(omega_dev, &c.omega_f, sizeof(float), cudaMemcpyHostToDevice, s));
            int n = p->max_sweeps - sweeps < K ? p->max_sweeps - sweeps : K;
            for (int done = 0; done < n; done += T) {
                // a partial last launch is rounded up to T sweeps (the cap may be exceeded by < T)
                TW_LAUNCH((mx_tb_kernel<T, S>), tgrid, kMxWarps * 32, kMxQBytes, s, e[cur][0], e[cur][1], e[1 - cur][0],
                          e[1 - cur][1], q[0], q[1], g.MR, g.MB, ny, g.W4, g.S, g.MW, (const float *)omega_dev);
                cur = 1 - cur;
                launches++;
            }
            TW_CHECK_LAUNCH();
            sweeps += ((n + T - 1) / T) * T;
            TW_CUDA(cudaMemsetAsync(&sc->max32, 0, sizeof(unsigned int), s));
            TW_LAUNCH((mx_inner_residual_kernel<S>), dim3(ceil_div(g.W4, 64), ceil_div(ny, 4)), dim3(64, 4), 0, s, g,
                      ny, e[cur][0], e[cur][1], q[0], q[1], &sc->max32);
            float rf;
            int er = read_max_f32(&sc->max32, s, &rf);
            if (er) return er;
            checks++;
            const double prev = c.r_prev;
            if (!relax_control(c, (double)rf, -1.0, n, -1.0)) break;
            if (prev > 0.0 && it > 4 && rf > 0.98 * prev) break;   // storage floor reached
        }
        if (c.adapt && c.omega > omega_keep) omega_keep = c.omega;   // adapted upwards, not backed off
        // 4. x += s e, and the update's size
        unsigned long long *dmax = reinterpret_cast<unsigned long long *>(&sc->pad1[1]);
        TW_CUDA(cudaMemsetAsync(dmax, 0, sizeof(*dmax), s));
        TW_LAUNCH((mx_update_kernel<S>), dim3(ceil_div(nx, 256), ny), 256, 0, s, g, x, nx, ny, (const double *)scale,
                  e[cur][0], e[cur][1], dmax);
        TW_CHECK_LAUNCH();
        unsigned long long db = 0;
        TW_CUDA(cudaMemcpyAsync(&db, dmax, sizeof(db), cudaMemcpyDeviceToHost, s));
        TW_CUDA(cudaStreamSynchronize(s));
        corr_prev = corr;
        memcpy(&corr, &db, sizeof(double));
        outer++;
        if (outer > 64) break;
    }
    const size_t n = (size_t)nx * ny;
    TW_LAUNCH(mx_output_kernel, ceil_div(n, 256), 256, 0, s, x, u, n);
    TW_CHECK_LAUNCH();
    st->sweeps = sweeps;
    st->checks = checks;
    st->omega = c.omega;
    st->sweep_launches = launches;
    st->tblock = T;
    st->loop = graph_used ? HP_LOOP_GRAPH : HP_LOOP_HOST;
    st->resid_inf = r_inf;   // the FP64 master's residual (the FP32 output rounds it)
    return TW_OK;
}

int relax_mixed(const uint8_t *occ, int nx, int ny, int gx, int gy, float *u, int mode, const hp_params *p,
                hp_stats *st, RelaxLayout &R, cudaStream_t s) {
    switch (p->storage) {
        case HP_STORE_F16: return mixed_solve<__half>(occ, nx, ny, gx, gy, u, mode, p, st, R, s);
        case HP_STORE_BF16: return mixed_solve<__nv_bfloat16>(occ, nx, ny, gx, gy, u, mode, p, st, R, s);
        default: return mixed_solve<float>(occ, nx, ny, gx, gy, u, mode, p, st, R, s);
    }
}

}  // namespace tw
