// Learned warm start: a small encoder-decoder network that predicts
// log(u) (u = 1 - phi) from the occupancy and a goal-distance map, trained on
// fields the relaxation itself produced.  The relaxation then finishes from
// the prediction (hp_relax with HP_WARM_START), so the method's own relaxation
// still decides the final field and its residual.
//
// Network (fully convolutional, input H and W multiples of 8):
//   enc0  conv3x3 2->32, conv 32->32            @ H     (ReLU after every conv but the head)
//   enc1  avgpool2, conv 32->64, conv 64->64    @ H/2
//   enc2  avgpool2, conv 64->128, conv 128->128 @ H/4
//   enc3  avgpool2, conv 128->128, conv 128->128 @ H/8
//   dec2  up2, conv 128->128 (+ enc2, ReLU), conv 128->128 @ H/4
//   dec1  up2, conv 128->64  (+ enc1, ReLU), conv 64->64   @ H/2
//   dec0  up2, conv 64->32   (+ enc0, ReLU), conv 32->32   @ H
//   head  conv 32->1 (linear): the prediction p = log(u) / 30
// Inputs: channel 0 = 1 on obstacles/border/goal-free... (1 where occupied),
// channel 1 = distance to the goal / grid diagonal.
// Storage: activations and their gradients in BF16, weights in FP32 (rounded
// to BF16 when loaded), every product accumulated in FP32.
//
// Kernels: every convolution with 16k input channels and 32, 64 or 128 output
// channels, its data gradient included, runs on the 5th-generation tensor
// cores with tensor-memory accumulators (nn_conv_tc.cu: the wide form for
// W % 128 == 0, the narrow form for W = 16, 32, 64), and so does every weight
// gradient; all layers' BF16 tensor-core weights are arranged once per step.
// Here: the mma.sync implicit GEMM for other shapes, direct convolutions on
// CUDA cores (16x16 pixel tiles for 16 output channels, 18x18 input tiles per
// chunk of 8 input channels) for the 2-channel input layer and the 1-channel
// head, the CUDA-core weight gradient where W % 16 != 0, pooling, upsampling,
// loss and Adam.
#include <cuda_bf16.h>
#include <math.h>
#include <string.h>

#include <vector>

#include "common.cuh"
#include "nn_tc.cuh"

namespace tw {
namespace nn {

typedef __nv_bfloat16 bf16;

struct ConvSpec { int cin, cout, level; };
// layer order: enc0a enc0b enc1a enc1b enc2a enc2b enc3a enc3b dec2a dec2b dec1a dec1b dec0a dec0b head
static const ConvSpec kConvs[15] = {
    {2, 32, 0},    {32, 32, 0},  {32, 64, 1},   {64, 64, 1},   {64, 128, 2},  {128, 128, 2},
    {128, 128, 3}, {128, 128, 3}, {128, 128, 2}, {128, 128, 2}, {128, 64, 1},  {64, 64, 1},
    {64, 32, 0},   {32, 32, 0},  {32, 1, 0}};
constexpr int kNumConvs = 15;

static size_t conv_params(int i) { return (size_t)kConvs[i].cout * kConvs[i].cin * 9 + kConvs[i].cout; }
static size_t param_offset(int i) {
    size_t o = 0;
    for (int k = 0; k < i; k++) o += conv_params(k);
    return o;
}
static size_t total_params() { return param_offset(kNumConvs); }

// ---- kernels ----------------------------------------------------------------------

constexpr int TS = 16;   // pixel tile side
constexpr size_t kSplitKCap = (size_t)1 << 23;   // floats of split-K partial sums (32 MB of workspace)
constexpr int COB = 16;  // output channels per CTA (CUDA-core kernels)
constexpr int CIB = 8;   // input channels per staged chunk

__device__ __forceinline__ float bf(float v) { return __bfloat162float(__float2bfloat16(v)); }

// Y = act(conv3x3(X) + b + S): X [cin][H][W] bf16, Wt [cout][cin][3][3] fp32 (rounded to bf16),
// b [cout] (nullable), S [cout][H][W] bf16 (nullable), Y [cout][H][W] bf16.
// COB output channels per CTA, CIB input channels per staged chunk (the
// network's first layer has 2 input channels, its head 1 output channel).
template <int COB, int CIB>
__global__ void __launch_bounds__(256) conv3x3_fwd_kernel(const bf16 *__restrict__ X, const float *__restrict__ Wt,
                                                          const float *__restrict__ b, const bf16 *__restrict__ S,
                                                          bf16 *__restrict__ Y, int cin, int cout, int H, int W,
                                                          int relu) {
    __shared__ float xs[CIB][TS + 2][TS + 2];
    __shared__ float ws[COB][CIB][9];
    const int tx = threadIdx.x % TS, ty = threadIdx.x / TS;
    const int x0 = blockIdx.x * TS, y0 = blockIdx.y * TS, co0 = blockIdx.z * COB;
    const int x = x0 + tx, y = y0 + ty;
    float acc[COB];
#pragma unroll
    for (int c = 0; c < COB; c++) acc[c] = 0.0f;
    for (int ci0 = 0; ci0 < cin; ci0 += CIB) {
        __syncthreads();
        for (int i = threadIdx.x; i < CIB * (TS + 2) * (TS + 2); i += 256) {
            const int c = i / ((TS + 2) * (TS + 2)), r = i % ((TS + 2) * (TS + 2));
            const int yy = y0 + r / (TS + 2) - 1, xx = x0 + r % (TS + 2) - 1;
            float v = 0.0f;
            if (ci0 + c < cin && yy >= 0 && yy < H && xx >= 0 && xx < W)
                v = __bfloat162float(X[((size_t)(ci0 + c) * H + yy) * W + xx]);
            xs[c][r / (TS + 2)][r % (TS + 2)] = v;
        }
        for (int i = threadIdx.x; i < COB * CIB * 9; i += 256) {
            const int co = i / (CIB * 9), r = i % (CIB * 9), c = r / 9, k = r % 9;
            float v = 0.0f;
            if (co0 + co < cout && ci0 + c < cin) v = bf(Wt[((size_t)(co0 + co) * cin + ci0 + c) * 9 + k]);
            ws[co][c][k] = v;
        }
        __syncthreads();
#pragma unroll
        for (int c = 0; c < CIB; c++) {
            float in[9];
#pragma unroll
            for (int k = 0; k < 9; k++) in[k] = xs[c][ty + k / 3][tx + k % 3];
#pragma unroll
            for (int co = 0; co < COB; co++) {
                float a = acc[co];
#pragma unroll
                for (int k = 0; k < 9; k++) a = fmaf(in[k], ws[co][c][k], a);
                acc[co] = a;
            }
        }
    }
    if (x >= W || y >= H) return;
#pragma unroll
    for (int co = 0; co < COB; co++) {
        const int oc = co0 + co;
        if (oc >= cout) break;
        float v = acc[co] + (b ? b[oc] : 0.0f);
        const size_t o = ((size_t)oc * H + y) * W + x;
        if (S) v += __bfloat162float(S[o]);
        if (relu) v = fmaxf(v, 0.0f);
        Y[o] = __float2bfloat16(v);
    }
}

// Tensor-core form of conv3x3_fwd_kernel (the same Y, up to FP32 summation
// order) for cin a multiple of 16 and cout a multiple of NB: an implicit GEMM
// with M = pixels, N = output channels, K = 9 taps x cin, on BF16
// mma.sync.m16n8k16 with FP32 accumulators.  A CTA computes a 16 x 16 pixel
// tile for NB output channels; warp w owns pixel rows 2w and 2w + 1 (one m16
// tile each: 16 pixels along x) and all NB channels.  Per chunk of 16 input
// channels the 18 x 18 input tile is staged channel-last (a pixel's 16
// channels contiguous, stride 24 BF16 so that fragment loads are
// conflict-free) and the weights as [tap][co][ci]; a fragment register is
// then one 32-bit shared load.  Fragment layouts (m16n8k16, BF16): A row = pixel
// g or g + 8 of the lane's group g = lane / 4, columns 2t, 2t + 1 (+ 8) with
// t = lane % 4; B column = channel g, rows 2t, 2t + 1 (+ 8); C rows g, g + 8,
// columns 2t, 2t + 1.
constexpr int kTcStride = 24;   // BF16 per staged pixel / weight row (16 used)

__device__ __forceinline__ void mma_bf16_16816(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Split K: with splits > 1, blockIdx.z = channel block + (cout / NB) x split,
// each split takes its share of the 16-channel chunks and writes FP32 partial
// sums to part[split][cout][H][W] (no bias, skip or activation), which
// splitk_finalize_kernel adds up in split order.
template <int NB>
__global__ void __launch_bounds__(256) conv3x3_fwd_mma_kernel(const bf16 *__restrict__ X, const float *__restrict__ Wt,
                                                              const float *__restrict__ b, const bf16 *__restrict__ S,
                                                              bf16 *__restrict__ Y, int cin, int cout, int H, int W,
                                                              int relu, int splits, float *__restrict__ part) {
    constexpr int NT = NB / 8;
    __shared__ __align__(16) bf16 xs[(TS + 2) * (TS + 2) * kTcStride];
    __shared__ __align__(16) bf16 ws[9 * NB * kTcStride];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane >> 2, t4 = lane & 3;
    const int nzb = cout / NB, sp = blockIdx.z / nzb;
    const int x0 = blockIdx.x * TS, y0 = blockIdx.y * TS, co0 = (blockIdx.z % nzb) * NB;
    const int chunks = cin / 16, per = (chunks + splits - 1) / splits;
    const int c_begin = sp * per * 16, c_end = min(chunks, (sp + 1) * per) * 16;
    float acc[2][NT][4];
#pragma unroll
    for (int m = 0; m < 2; m++)
#pragma unroll
        for (int n = 0; n < NT; n++)
#pragma unroll
            for (int e = 0; e < 4; e++) acc[m][n][e] = 0.0f;

    for (int ci0 = c_begin; ci0 < c_end; ci0 += 16) {
        __syncthreads();
        // input tile, channel-last: xs[(yy * 18 + xx) * 24 + c]
        for (int i = threadIdx.x; i < 16 * (TS + 2) * (TS + 2); i += 256) {
            const int c = i / ((TS + 2) * (TS + 2)), r = i % ((TS + 2) * (TS + 2));
            const int yy = y0 + r / (TS + 2) - 1, xx = x0 + r % (TS + 2) - 1;
            bf16 v = __float2bfloat16(0.0f);
            if (yy >= 0 && yy < H && xx >= 0 && xx < W) v = X[((size_t)(ci0 + c) * H + yy) * W + xx];
            xs[r * kTcStride + c] = v;
        }
        // weights as [tap][co][ci], rounded to BF16
        for (int i = threadIdx.x; i < NB * 16 * 9; i += 256) {
            const int co = i / (16 * 9), r = i % (16 * 9), c = r / 9, k = r % 9;
            const float v = Wt[((size_t)(co0 + co) * cin + ci0 + c) * 9 + k];
            ws[(k * NB + co) * kTcStride + c] = __float2bfloat16(v);
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < 9; k++) {
            const int dy = k / 3, dx = k % 3;
            uint32_t a[2][4];
#pragma unroll
            for (int m = 0; m < 2; m++) {
                const int row = 2 * warp + m + dy;
                const bf16 *p0 = xs + (row * (TS + 2) + g + dx) * kTcStride + 2 * t4;
                const bf16 *p1 = p0 + 8 * kTcStride;   // pixel g + 8
                a[m][0] = *reinterpret_cast<const uint32_t *>(p0);
                a[m][1] = *reinterpret_cast<const uint32_t *>(p1);
                a[m][2] = *reinterpret_cast<const uint32_t *>(p0 + 8);
                a[m][3] = *reinterpret_cast<const uint32_t *>(p1 + 8);
            }
#pragma unroll
            for (int n = 0; n < NT; n++) {
                const bf16 *q = ws + (k * NB + n * 8 + g) * kTcStride + 2 * t4;
                const uint32_t b0 = *reinterpret_cast<const uint32_t *>(q);
                const uint32_t b1 = *reinterpret_cast<const uint32_t *>(q + 8);
                mma_bf16_16816(acc[0][n], a[0], b0, b1);
                mma_bf16_16816(acc[1][n], a[1], b0, b1);
            }
        }
    }
    // epilogue: bias, skip, ReLU, BF16 store
#pragma unroll
    for (int m = 0; m < 2; m++) {
        const int y = y0 + 2 * warp + m;
        if (y >= H) continue;
#pragma unroll
        for (int n = 0; n < NT; n++) {
#pragma unroll
            for (int e = 0; e < 4; e++) {
                const int x = x0 + g + (e >= 2 ? 8 : 0);
                const int oc = co0 + n * 8 + 2 * t4 + (e & 1);
                if (x >= W) continue;
                const size_t o = ((size_t)oc * H + y) * W + x;
                if (splits > 1) {
                    part[(size_t)sp * cout * H * W + o] = acc[m][n][e];
                    continue;
                }
                float v = acc[m][n][e] + (b ? b[oc] : 0.0f);
                if (S) v += __bfloat162float(S[o]);
                if (relu) v = fmaxf(v, 0.0f);
                Y[o] = __float2bfloat16(v);
            }
        }
    }
}

// Y = act(sum over splits of part + b + S), the splits added in index order.
__global__ void splitk_finalize_kernel(const float *__restrict__ part, int splits, const float *__restrict__ b,
                                       const bf16 *__restrict__ S, bf16 *__restrict__ Y, int cout, int H, int W,
                                       int relu) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y, oc = blockIdx.z;
    if (x >= W) return;
    const size_t o = ((size_t)oc * H + y) * W + x, plane = (size_t)cout * H * W;
    float v = 0.0f;
    for (int sp = 0; sp < splits; sp++) v += part[sp * plane + o];
    v += b ? b[oc] : 0.0f;
    if (S) v += __bfloat162float(S[o]);
    if (relu) v = fmaxf(v, 0.0f);
    Y[o] = __float2bfloat16(v);
}

// weight transform for the data gradient: Wt'[ci][co][8 - k] = Wt[co][ci][k]
__global__ void conv_transpose_weights_kernel(const float *__restrict__ Wt, float *__restrict__ Wtt, int cin, int cout) {
    const size_t n = (size_t)cin * cout * 9;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int k = (int)(i % 9), ci = (int)((i / 9) % cin), co = (int)(i / 9 / cin);
        Wtt[((size_t)ci * cout + co) * 9 + (8 - k)] = Wt[i];
    }
}

// Partial sums of dW[co][ci][k] = sum_p dY[co][p] X[ci][p + k - (1,1)] and
// db[co] = sum_p dY[co][p] over one chunk of rows: CTA (co block of 16, ci
// block of 8, row chunk z) writes its sums to part[z][co][ci][k] and (ci block
// 0) part_b[z][co]; conv3x3_bwd_weight_sum_kernel adds the chunks in order, so
// the gradients do not depend on the order CTAs finish in.
__global__ void __launch_bounds__(256) conv3x3_bwd_weight_kernel(const bf16 *__restrict__ X, const bf16 *__restrict__ dY,
                                                                 float *__restrict__ part, float *__restrict__ part_b,
                                                                 int cin, int cout, int H, int W, int rows_per_cta) {
    // thread t: weight index (co, c, k) = t for t < COB*CIB*9/...; accumulate over pixels
    const int co0 = blockIdx.x * COB, ci0 = blockIdx.y * CIB;
    const int ya = blockIdx.z * rows_per_cta, yb = min(H, ya + rows_per_cta);
    __shared__ float sdy[COB][TS * 4];
    __shared__ float sx[CIB][3][TS * 4 + 2];
    // 16*8*9 = 1152 weights; 256 threads hold 4.5 -> use 5 slots each
    float acc[5];
    float accb = 0.0f;
#pragma unroll
    for (int j = 0; j < 5; j++) acc[j] = 0.0f;
    for (int y = ya; y < yb; y++) {
        for (int xs0 = 0; xs0 < W; xs0 += TS * 4) {
            __syncthreads();
            for (int i = threadIdx.x; i < COB * TS * 4; i += 256) {
                const int co = i / (TS * 4), xx = xs0 + i % (TS * 4);
                sdy[co][i % (TS * 4)] = (co0 + co < cout && xx < W)
                                            ? __bfloat162float(dY[((size_t)(co0 + co) * H + y) * W + xx]) : 0.0f;
            }
            for (int i = threadIdx.x; i < CIB * 3 * (TS * 4 + 2); i += 256) {
                const int c = i / (3 * (TS * 4 + 2)), r = (i / (TS * 4 + 2)) % 3, xx = xs0 + i % (TS * 4 + 2) - 1;
                const int yy = y + r - 1;
                sx[c][r][i % (TS * 4 + 2)] = (ci0 + c < cin && yy >= 0 && yy < H && xx >= 0 && xx < W)
                                                 ? __bfloat162float(X[((size_t)(ci0 + c) * H + yy) * W + xx]) : 0.0f;
            }
            __syncthreads();
#pragma unroll
            for (int j = 0; j < 5; j++) {
                const int t = threadIdx.x + 256 * j;
                if (t >= COB * CIB * 9) break;
                const int co = t / (CIB * 9), c = (t / 9) % CIB, k = t % 9, ky = k / 3, kx = k % 3;
                float a = acc[j];
                for (int p = 0; p < TS * 4; p++) a = fmaf(sdy[co][p], sx[c][ky][p + kx], a);
                acc[j] = a;
            }
            if (blockIdx.y == 0 && threadIdx.x < COB)
                for (int p = 0; p < TS * 4; p++) accb += sdy[threadIdx.x][p];
        }
    }
    const size_t zo = (size_t)blockIdx.z * cout * cin * 9;
#pragma unroll
    for (int j = 0; j < 5; j++) {
        const int t = threadIdx.x + 256 * j;
        if (t >= COB * CIB * 9) break;
        const int co = t / (CIB * 9), c = (t / 9) % CIB, k = t % 9;
        if (co0 + co < cout && ci0 + c < cin) part[zo + ((size_t)(co0 + co) * cin + ci0 + c) * 9 + k] = acc[j];
    }
    if (blockIdx.y == 0 && threadIdx.x < COB && co0 + threadIdx.x < cout)
        part_b[(size_t)blockIdx.z * cout + co0 + threadIdx.x] = accb;
}

// dW += sum over the row chunks of part, db += sum of part_b, chunks in order.
__global__ void conv3x3_bwd_weight_sum_kernel(const float *__restrict__ part, const float *__restrict__ part_b,
                                              int chunks, float *__restrict__ dW, float *__restrict__ db, int cin,
                                              int cout) {
    const size_t n = (size_t)cout * cin * 9;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n + cout; i += (size_t)gridDim.x * blockDim.x) {
        if (i < n) {
            float v = 0.0f;
            for (int z = 0; z < chunks; z++) v += part[(size_t)z * n + i];
            dW[i] += v;
        } else if (db) {
            const size_t co = i - n;
            float v = 0.0f;
            for (int z = 0; z < chunks; z++) v += part_b[(size_t)z * cout + co];
            db[co] += v;
        }
    }
}

// dA = dY * (A > 0) in place on dY (A: the post-ReLU activation)
__global__ void relu_bwd_kernel(const bf16 *__restrict__ A, bf16 *__restrict__ dY, size_t n) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        if (!(__bfloat162float(A[i]) > 0.0f)) dY[i] = __float2bfloat16(0.0f);
}

// Pooling and upsampling kernels: grid (ceil(width / 256), rows, channels) of
// the tensor they write, so a thread finds its element without divisions.

__global__ void pool2_fwd_kernel(const bf16 *__restrict__ X, bf16 *__restrict__ Y, int C, int H, int W) {
    const int h = H / 2, w = W / 2;
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y, c = blockIdx.z;
    if (x >= w) return;
    const bf16 *p = X + ((size_t)c * H + 2 * y) * W + 2 * x;
    const float v = (__bfloat162float(p[0]) + __bfloat162float(p[1])) +
                    (__bfloat162float(p[W]) + __bfloat162float(p[W + 1]));
    Y[((size_t)c * h + y) * w + x] = __float2bfloat16(0.25f * v);
}

// gradient of the 2x2 average pool, accumulated into dX (dX += dY / 4 spread over the window)
__global__ void pool2_bwd_kernel(const bf16 *__restrict__ dY, bf16 *__restrict__ dX, int C, int H, int W) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y, c = blockIdx.z;
    if (x >= W) return;
    const float g = 0.25f * __bfloat162float(dY[((size_t)c * (H / 2) + y / 2) * (W / 2) + x / 2]);
    const size_t i = ((size_t)c * H + y) * W + x;
    dX[i] = __float2bfloat16(__bfloat162float(dX[i]) + g);
}

// X [C][H/2][W/2] -> Y [C][H][W] (nearest)
__global__ void up2_fwd_kernel(const bf16 *__restrict__ X, bf16 *__restrict__ Y, int C, int H, int W) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y, c = blockIdx.z;
    if (x >= W) return;
    Y[((size_t)c * H + y) * W + x] = X[((size_t)c * (H / 2) + y / 2) * (W / 2) + x / 2];
}

// dX [C][H/2][W/2] = sum of the 4 children of dY [C][H][W]
__global__ void up2_bwd_kernel(const bf16 *__restrict__ dY, bf16 *__restrict__ dX, int C, int H, int W) {
    const int h = H / 2, w = W / 2;
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y, c = blockIdx.z;
    if (x >= w) return;
    const bf16 *p = dY + ((size_t)c * H + 2 * y) * W + 2 * x;
    dX[((size_t)c * h + y) * w + x] = __float2bfloat16((__bfloat162float(p[0]) + __bfloat162float(p[1])) +
                                                       (__bfloat162float(p[W]) + __bfloat162float(p[W + 1])));
}

__global__ void add_inplace_kernel(bf16 *__restrict__ A, const bf16 *__restrict__ B, size_t n) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        A[i] = __float2bfloat16(__bfloat162float(A[i]) + __bfloat162float(B[i]));
}

// Input features: channel 0 = occupied (occ != 0), channel 1 = goal distance / diagonal.
__global__ void features_kernel(const uint8_t *__restrict__ occ, int H, int W, int gx, int gy, bf16 *__restrict__ X) {
    const size_t n = (size_t)H * W;
    const float diag = sqrtf((float)H * H + (float)W * W);
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % W), y = (int)(i / W);
        X[i] = __float2bfloat16(occ[i] != 0 ? 1.0f : 0.0f);
        X[n + i] = __float2bfloat16(sqrtf((float)(x - gx) * (x - gx) + (float)(y - gy) * (y - gy)) / diag);
    }
}

// Masked MSE over free cells: loss = sum m (p - t)^2 / sum m; dP = 2 m (p - t) / sum m (bf16).
__global__ void __launch_bounds__(256) mse_kernel(const bf16 *__restrict__ P, const float *__restrict__ T,
                                                  const uint8_t *__restrict__ occ, int gx, int gy, int W, size_t n,
                                                  float inv_count, bf16 *__restrict__ dP, float *__restrict__ loss) {
    float s = 0.0f;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const bool m = occ[i] == 0 && !((int)(i % W) == gx && (int)(i / W) == gy);
        const float d = m ? (__bfloat162float(P[i]) - T[i]) : 0.0f;
        s += d * d;
        dP[i] = __float2bfloat16(2.0f * d * inv_count);
    }
    // the CTA's sum into part[blockIdx.x] (fixed-shape reduction); loss_sum_kernel adds the CTAs in order
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    __shared__ float sw[8];
    if ((threadIdx.x & 31) == 0) sw[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.0f;
        for (int w = 0; w < 8; w++) t += sw[w];
        loss[blockIdx.x] = t * inv_count;
    }
}

// *loss = sum of the n per-CTA partials, in index order (one thread: n <= 4096).
__global__ void loss_sum_kernel(const float *__restrict__ part, int n, float *__restrict__ loss) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    float t = 0.0f;
    for (int i = 0; i < n; i++) t += part[i];
    *loss = t;
}

__global__ void adam_kernel(float *__restrict__ w, const float *__restrict__ g, float *__restrict__ m,
                            float *__restrict__ v, size_t n, float lr, float b1, float b2, float eps, float c1,
                            float c2) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.0f - b1) * gi;
        const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

// He-normal initialisation from a counter-based generator (SplitMix64 + Box-Muller), biases 0.
__device__ __forceinline__ unsigned long long splitmix(unsigned long long x) {
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}
__global__ void init_kernel(float *__restrict__ w, size_t n_w, size_t n_total, float stdv, unsigned long long seed,
                            size_t offset) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_total; i += (size_t)gridDim.x * blockDim.x) {
        if (i >= n_w) { w[i] = 0.0f; continue; }
        const unsigned long long a = splitmix(seed * 0x100000001B3ull + 2 * (offset + i));
        const unsigned long long b = splitmix(seed * 0x100000001B3ull + 2 * (offset + i) + 1);
        const float u1 = ((a >> 40) + 1) * (1.0f / 16777217.0f), u2 = (b >> 40) * (1.0f / 16777216.0f);
        w[i] = stdv * sqrtf(-2.0f * logf(u1)) * cosf(6.2831853f * u2);
    }
}

__global__ void to_u_kernel(const bf16 *__restrict__ P, const uint8_t *__restrict__ occ, int gx, int gy, int W,
                            size_t n, float *__restrict__ u) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const bool goal = (int)(i % W) == gx && (int)(i / W) == gy;
        float v = occ[i] != 0 ? 0.0f : expf(fminf(30.0f * __bfloat162float(P[i]), 0.0f));
        u[i] = goal ? 1.0f : v;
    }
}

// Coarse input for the warm start at stride s: a coarse cell is occupied when
// any of its s x s cells is, except the cell holding the goal, which stays
// free so that the network sees a reachable goal.
__global__ void occ_pool_kernel(const uint8_t *__restrict__ occ, int W, int s, int gxc, int gyc,
                                uint8_t *__restrict__ oc, int wc) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= wc) return;
    uint8_t v = 0;
    for (int dy = 0; dy < s; dy++)
        for (int dx = 0; dx < s; dx++) v |= occ[(size_t)(y * s + dy) * W + x * s + dx];
    oc[(size_t)y * wc + x] = (x == gxc && y == gyc) ? 0 : (v != 0);
}

// Full-resolution warm start from the coarse prediction: p bilinearly
// interpolated at each cell centre (cell-centred grids, clamped at the edges),
// u = exp(min(30 p, 0)), 0 on occupied cells, 1 at the goal.
__global__ void upsample_to_u_kernel(const bf16 *__restrict__ P, int hc, int wc, int s,
                                     const uint8_t *__restrict__ occ, int W, int gx, int gy,
                                     float *__restrict__ u) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= W) return;
    const size_t i = (size_t)y * W + x;
    if (occ[i] != 0) { u[i] = 0.0f; return; }
    if (x == gx && y == gy) { u[i] = 1.0f; return; }
    const float fx = fminf(fmaxf((x + 0.5f) / s - 0.5f, 0.0f), (float)(wc - 1));
    const float fy = fminf(fmaxf((y + 0.5f) / s - 0.5f, 0.0f), (float)(hc - 1));
    const int x0 = (int)fx, y0 = (int)fy;
    const int x1 = x0 + 1 < wc ? x0 + 1 : x0, y1 = y0 + 1 < hc ? y0 + 1 : y0;
    const float ax = fx - x0, ay = fy - y0;
    const float p00 = __bfloat162float(P[(size_t)y0 * wc + x0]), p01 = __bfloat162float(P[(size_t)y0 * wc + x1]);
    const float p10 = __bfloat162float(P[(size_t)y1 * wc + x0]), p11 = __bfloat162float(P[(size_t)y1 * wc + x1]);
    const float p = (1.0f - ay) * ((1.0f - ax) * p00 + ax * p01) + ay * ((1.0f - ax) * p10 + ax * p11);
    u[i] = expf(fminf(30.0f * p, 0.0f));
}

// ---- host-side network -------------------------------------------------------------

struct Act {   // activation buffers per level (bf16 [C][h][w])
    bf16 *in;                          // features [2][H][W]
    bf16 *e[4][2];                     // encoder conv outputs per level (a, b)
    bf16 *p[3];                        // pooled inputs of levels 1..3
    bf16 *u[3];                        // upsampled decoder inputs at levels 2, 1, 0
    bf16 *d[3][2];                     // decoder conv outputs at levels 2, 1, 0
    bf16 *out;                         // head output [1][H][W]
    bf16 *g0, *g1, *g2;                // gradient scratch (64 x H x W each)
    bf16 *sk[3];                       // gradients into the skip sources e[2][1], e[1][1], e[0][1]
    float *target;                     // [H][W] training target (log u / 30)
    float *wt;                         // transposed weights scratch
    bf16 *wtf, *wtb;                   // every layer's tensor-core weights: forward, transposed
    float *kpart;                      // split-K partial sums (kSplitKCap floats)
    float *loss;
};

static size_t lvl_px(int H, int W, int l) { return (size_t)(H >> l) * (W >> l); }

// Offset of layer li's tensor-core weights (BF16, 128-byte aligned slots) in Act::wtf / Act::wtb.
static size_t tc_w_off(int li) {
    size_t o = 0;
    for (int k = 0; k < li; k++) o += ((size_t)kConvs[k].cin * kConvs[k].cout * 9 + 63) & ~(size_t)63;
    return o;
}
// Channel counts the tensor-memory kernels take: the layer itself, and its transpose (the data gradient).
static bool tc_fwd_ok(int li) {
    const ConvSpec &c = kConvs[li];
    return c.cin % 16 == 0 && (c.cout == 32 || c.cout == 64 || c.cout == 128);
}
static bool tc_bwd_ok(int li) {
    const ConvSpec &c = kConvs[li];
    return c.cout % 16 == 0 && (c.cin == 32 || c.cin == 64 || c.cin == 128);
}

static size_t carve_act(Carver &cv, int H, int W, Act *A) {
    Act a;
    a.in = cv.take<bf16>(2 * lvl_px(H, W, 0));
    const int ch[4] = {32, 64, 128, 128};
    for (int l = 0; l < 4; l++) {
        a.e[l][0] = cv.take<bf16>(ch[l] * lvl_px(H, W, l));
        a.e[l][1] = cv.take<bf16>(ch[l] * lvl_px(H, W, l));
    }
    for (int l = 1; l < 4; l++) a.p[l - 1] = cv.take<bf16>(ch[l - 1] * lvl_px(H, W, l));
    const int uc[3] = {128, 128, 64};   // channels entering dec2, dec1, dec0
    const int ul[3] = {2, 1, 0};
    const int dc[3] = {128, 64, 32};
    for (int j = 0; j < 3; j++) {
        a.u[j] = cv.take<bf16>(uc[j] * lvl_px(H, W, ul[j]));
        a.d[j][0] = cv.take<bf16>(dc[j] * lvl_px(H, W, ul[j]));
        a.d[j][1] = cv.take<bf16>(dc[j] * lvl_px(H, W, ul[j]));
    }
    a.out = cv.take<bf16>(lvl_px(H, W, 0));
    const size_t gm = 64 * lvl_px(H, W, 0);   // the largest activation gradient (u[2]: 64 ch at full size)
    a.g0 = cv.take<bf16>(gm);
    a.g1 = cv.take<bf16>(gm);
    a.g2 = cv.take<bf16>(gm);
    a.sk[0] = cv.take<bf16>(128 * lvl_px(H, W, 2));
    a.sk[1] = cv.take<bf16>(64 * lvl_px(H, W, 1));
    a.sk[2] = cv.take<bf16>(32 * lvl_px(H, W, 0));
    a.target = cv.take<float>(lvl_px(H, W, 0));
    a.wt = cv.take<float>(128 * 128 * 9);
    a.wtf = cv.take<bf16>(tc_w_off(kNumConvs));
    a.wtb = cv.take<bf16>(tc_w_off(kNumConvs));
    a.kpart = cv.take<float>(kSplitKCap);
    a.loss = cv.take<float>(64);
    if (A) *A = a;
    return cv.need;
}

static unsigned blocks_for(size_t n) { return (unsigned)((n + 255) / 256 > 4096 ? 4096 : (n + 255) / 256); }

// Split-K factor of a tensor-core convolution: enough CTAs for two per SM of a
// 152-SM GPU when the pixel tiles alone are too few, at most one chunk of 16
// input channels per split, and at most cap_floats of FP32 partials.
static int splitk_plan(int cin, int cout, int H, int W, size_t cap_floats) {
    const int nb = cout % 64 == 0 ? 64 : 32;
    const long base = (long)ceil_div(W, TS) * ceil_div(H, TS) * (cout / nb);
    if (base >= 152) return 1;
    const int chunks = cin / 16;
    int sp = (int)((304 + base - 1) / base);
    if (sp > chunks) sp = chunks;
    while (sp > 1 && (size_t)sp * cout * H * W > cap_floats) sp--;
    if (sp < 1) return 1;
    const int per = (chunks + sp - 1) / sp;   // no empty split
    return (chunks + per - 1) / per;
}

// Floats of part the narrow tensor-memory form takes ahead of its partial sums
// (the re-arranged BF16 weights, rounded up to 256 bytes).
static size_t narrow_weight_floats(int cin, int cout) {
    return ((conv3x3_tc_scratch_bytes(cin, cout) + 255) & ~(size_t)255) / sizeof(float);
}

// The narrow tensor-memory form (W < 128) with its split-K finalisation: the
// weights at the start of part, the partial sums after them.
static int conv3x3_narrow(const bf16 *X, const float *Wt, const float *b, const bf16 *S, bf16 *Y, int cin, int cout,
                          int H, int W, int relu, cudaStream_t s, float *part, size_t part_floats,
                          const bf16 *wpre) {
    const size_t wf = wpre ? 0 : narrow_weight_floats(cin, cout);
    if (!part || part_floats < wf) return TW_EWORKSPACE;
    const int sp = conv3x3_tc_narrow_splits(cin, cout, H, W, part_floats - wf);
    float *pp = part + wf;
    void *wsc = wpre ? (void *)wpre : (void *)part;
    const int e = conv3x3_tc_narrow(X, Wt, b, S, Y, cin, cout, H, W, relu, sp, wsc, sp > 1 ? pp : nullptr, s,
                                    wpre != nullptr);
    if (e || sp == 1) return e;
    TW_LAUNCH(splitk_finalize_kernel, dim3(ceil_div(W, 256), H, cout), 256, 0, s, pp, sp, b, S, Y, cout, H, W, relu);
    return TW_OK;
}

// One 3x3 convolution: the tensor-core kernel where the channel counts allow
// it (impl WS_CONV_AUTO), or the one asked for.  part (nullable): scratch for
// split-K partial sums, part_floats long, which also holds the re-arranged
// weights of the tensor-memory kernels (WS_CONV_TC) unless wpre (nullable)
// holds them already arranged.
static int conv3x3(const bf16 *X, const float *Wt, const float *b, const bf16 *S, bf16 *Y, int cin, int cout, int H,
                   int W, int relu, int impl, cudaStream_t s, float *part = nullptr, size_t part_floats = 0,
                   const bf16 *wpre = nullptr) {
    const bool mma_ok = cin % 16 == 0 && cout % 32 == 0;
    if (impl == WS_CONV_MMA && !mma_ok) return TW_EINVAL;
    const bool room = part && part_floats * sizeof(float) >= conv3x3_tc_scratch_bytes(cin, cout);
    void *wsc = wpre ? (void *)wpre : (void *)part;
    if (impl == WS_CONV_TC) {
        if (conv3x3_tc_narrow_ok(cin, cout, H, W))
            return conv3x3_narrow(X, Wt, b, S, Y, cin, cout, H, W, relu, s, part, part_floats, wpre);
        if (!conv3x3_tc_ok(cin, cout, H, W)) return TW_EINVAL;
        if (!wpre && !room) return TW_EWORKSPACE;
        return conv3x3_tc(X, Wt, b, S, Y, cin, cout, H, W, relu, wsc, s, wpre != nullptr);
    }
    // the automatic choice: a tensor-memory kernel wherever its shape conditions hold and the
    // scratch for its re-arranged weights is there (inside the network), else mma.sync or CUDA cores
    if (impl == WS_CONV_AUTO && part && conv3x3_tc_ok(cin, cout, H, W) && (wpre || room))
        return conv3x3_tc(X, Wt, b, S, Y, cin, cout, H, W, relu, wsc, s, wpre != nullptr);
    if (impl == WS_CONV_AUTO && part && conv3x3_tc_narrow_ok(cin, cout, H, W) &&
        (wpre || part_floats >= narrow_weight_floats(cin, cout)))
        return conv3x3_narrow(X, Wt, b, S, Y, cin, cout, H, W, relu, s, part, part_floats, wpre);
    if (impl != WS_CONV_SIMT && mma_ok) {
        const int sp = part ? splitk_plan(cin, cout, H, W, part_floats) : 1;
        float *pp = sp > 1 ? part : nullptr;
        if (cout % 64 == 0) {
            dim3 grid(ceil_div(W, TS), ceil_div(H, TS), cout / 64 * sp);
            TW_LAUNCH(conv3x3_fwd_mma_kernel<64>, grid, 256, 0, s, X, Wt, b, S, Y, cin, cout, H, W, relu, sp, pp);
        } else {
            dim3 grid(ceil_div(W, TS), ceil_div(H, TS), cout / 32 * sp);
            TW_LAUNCH(conv3x3_fwd_mma_kernel<32>, grid, 256, 0, s, X, Wt, b, S, Y, cin, cout, H, W, relu, sp, pp);
        }
        if (sp > 1)
            TW_LAUNCH(splitk_finalize_kernel, dim3(ceil_div(W, 256), H, cout), 256, 0, s, part, sp, b, S, Y, cout, H,
                      W, relu);
        return TW_OK;
    }
    if (cout < 8) {
        dim3 grid(ceil_div(W, TS), ceil_div(H, TS), cout);
        TW_LAUNCH((conv3x3_fwd_kernel<1, CIB>), grid, 256, 0, s, X, Wt, b, S, Y, cin, cout, H, W, relu);
    } else if (cin <= 2) {
        dim3 grid(ceil_div(W, TS), ceil_div(H, TS), ceil_div(cout, COB));
        TW_LAUNCH((conv3x3_fwd_kernel<COB, 2>), grid, 256, 0, s, X, Wt, b, S, Y, cin, cout, H, W, relu);
    } else {
        dim3 grid(ceil_div(W, TS), ceil_div(H, TS), ceil_div(cout, COB));
        TW_LAUNCH((conv3x3_fwd_kernel<COB, CIB>), grid, 256, 0, s, X, Wt, b, S, Y, cin, cout, H, W, relu);
    }
    return TW_OK;
}

// Row chunks of the CUDA-core weight gradient: enough chunks for about four
// CTAs per SM of a 152-SM GPU (the layers it serves have few channels, so few
// channel blocks), as many as cap_floats of partial sums allow; 0 if even one
// chunk does not fit.
static int wgrad_simt_rows(int cin, int cout, int H, size_t cap_floats) {
    const size_t per = (size_t)cout * cin * 9 + cout;
    if (per > cap_floats) return 0;
    const long blocks = (long)ceil_div(cout, COB) * ceil_div(cin, CIB);
    long nz = (608 + blocks - 1) / blocks;
    if (nz > H) nz = H;
    int rows = ceil_div(H, (int)nz);
    while ((size_t)ceil_div(H, rows) * per > cap_floats) rows *= 2;
    return rows;
}

// dW += dL/dW, db += dL/db (db nullable) of one 3x3 convolution from its input X
// and output gradient dY: on the tensor cores (tcgen05, accumulators in tensor
// memory) where the channel counts and the width allow it and impl is
// WS_CONV_AUTO or WS_CONV_TC, else on CUDA cores (WS_CONV_SIMT, or AUTO
// elsewhere).  part: part_floats floats of scratch for the partial sums of the
// pixel chunks.  Either form adds the chunks in a fixed order: the result is
// the same on every run.
static int conv3x3_wgrad(const bf16 *X, const bf16 *dY, float *dW, float *db, int cin, int cout, int H, int W,
                         int impl, float *part, size_t part_floats, cudaStream_t s) {
    if (impl == WS_CONV_MMA) return TW_EINVAL;
    const bool tc_ok = conv3x3_wgrad_tc_ok(cin, cout, H, W);
    if (impl == WS_CONV_TC && !tc_ok) return TW_EINVAL;
    if (impl != WS_CONV_SIMT && tc_ok) return conv3x3_wgrad_tc(X, dY, dW, db, cin, cout, H, W, part, part_floats, s);
    const int rows = wgrad_simt_rows(cin, cout, H, part_floats);
    if (!part || rows < 1) return TW_EWORKSPACE;
    const size_t per = (size_t)cout * cin * 9 + cout;
    const int nz = ceil_div(H, rows);
    float *part_b = part + (size_t)nz * cout * cin * 9;
    dim3 gw(ceil_div(cout, COB), ceil_div(cin, CIB), nz);
    TW_LAUNCH(conv3x3_bwd_weight_kernel, gw, 256, 0, s, X, dY, part, part_b, cin, cout, H, W, rows);
    TW_LAUNCH(conv3x3_bwd_weight_sum_kernel, blocks_for(per), 256, 0, s, part, part_b, nz, dW, db, cin, cout);
    return TW_OK;
}

// Floats of scratch conv3x3_wgrad needs for the form impl selects.
static size_t conv3x3_wgrad_floats(int cin, int cout, int H, int W, int impl) {
    const size_t per = (size_t)cout * cin * 9 + cout;
    if (impl != WS_CONV_SIMT && conv3x3_wgrad_tc_ok(cin, cout, H, W)) {
        int chunk = 0;
        return (size_t)conv3x3_wgrad_tc_plan(cin, cout, H, W, (size_t)-1, &chunk) * per;
    }
    return (size_t)ceil_div(H, wgrad_simt_rows(cin, cout, H, (size_t)-1)) * per;
}

// Every layer's tensor-core weights (forward and, with bwd, transposed) in one launch;
// the convolutions of the step then read them from wtf / wtb.
static void prepare_tc_weights(const float *P, Act &A, bool bwd, cudaStream_t s) {
    TcPrepTable t;
    memset(&t, 0, sizeof(t));
    t.n = kNumConvs;
    for (int li = 0; li < kNumConvs; li++) {
        t.poff[li] = (long long)param_offset(li);
        t.cin[li] = kConvs[li].cin;
        t.cout[li] = kConvs[li].cout;
        t.foff[li] = tc_fwd_ok(li) ? (long long)tc_w_off(li) : -1;
        t.boff[li] = bwd && tc_bwd_ok(li) ? (long long)tc_w_off(li) : -1;
        t.total += 2LL * kConvs[li].cin * kConvs[li].cout * 9;
    }
    conv_tc_prepare_weights(P, t, A.wtf, A.wtb, s);
}

static void conv_fwd(const bf16 *X, const float *params, int li, const bf16 *S, bf16 *Y, int H, int W, int relu,
                     float *kpart, const bf16 *wtf, cudaStream_t s, bool bias = true) {
    const ConvSpec &c = kConvs[li];
    const float *Wt = params + param_offset(li);
    const float *b = bias ? Wt + (size_t)c.cout * c.cin * 9 : nullptr;
    conv3x3(X, Wt, b, S, Y, c.cin, c.cout, H, W, relu, WS_CONV_AUTO, s, kpart, kSplitKCap,
            tc_fwd_ok(li) ? wtf + tc_w_off(li) : nullptr);
}

// The forward pass; every intermediate is kept for the backward pass.
static void forward(const float *P, Act &A, int H, int W, cudaStream_t s) {
    const int ch[4] = {32, 64, 128, 128};
    // encoder
    conv_fwd(A.in, P, 0, nullptr, A.e[0][0], H, W, 1, A.kpart, A.wtf, s);
    conv_fwd(A.e[0][0], P, 1, nullptr, A.e[0][1], H, W, 1, A.kpart, A.wtf, s);
    for (int l = 1; l < 4; l++) {
        const int h = H >> l, w = W >> l;
        TW_LAUNCH(pool2_fwd_kernel, dim3(ceil_div(w, 256), h, ch[l - 1]), 256, 0, s, A.e[l - 1][1], A.p[l - 1],
                  ch[l - 1], H >> (l - 1), W >> (l - 1));
        conv_fwd(A.p[l - 1], P, 2 * l, nullptr, A.e[l][0], h, w, 1, A.kpart, A.wtf, s);
        conv_fwd(A.e[l][0], P, 2 * l + 1, nullptr, A.e[l][1], h, w, 1, A.kpart, A.wtf, s);
    }
    // decoder: level 2, 1, 0
    const bf16 *prev = A.e[3][1];
    const int pc[3] = {128, 128, 64};
    for (int j = 0; j < 3; j++) {
        const int l = 2 - j, h = H >> l, w = W >> l;
        TW_LAUNCH(up2_fwd_kernel, dim3(ceil_div(w, 256), h, pc[j]), 256, 0, s, prev, A.u[j], pc[j], h, w);
        conv_fwd(A.u[j], P, 8 + 2 * j, A.e[l][1], A.d[j][0], h, w, 1, A.kpart, A.wtf, s);
        conv_fwd(A.d[j][0], P, 9 + 2 * j, nullptr, A.d[j][1], h, w, 1, A.kpart, A.wtf, s);
        prev = A.d[j][1];
    }
    conv_fwd(A.d[2][1], P, 14, nullptr, A.out, H, W, 0, A.kpart, A.wtf, s);
}

// Gradient through one conv layer: dY (its output gradient, ReLU already applied)
// -> dX (overwritten, or accumulated when accumulate != 0) and dW/db (accumulated).
static void conv_bwd(const bf16 *X, const float *P, float *G, int li, const bf16 *dY, bf16 *dX, bf16 *tmp, int H,
                     int W, float *wt, float *kpart, const bf16 *wtb, int accumulate, cudaStream_t s) {
    const ConvSpec &c = kConvs[li];
    const float *Wt = P + param_offset(li);
    float *dW = G + param_offset(li);
    float *db = dW + (size_t)c.cout * c.cin * 9;
    conv3x3_wgrad(X, dY, dW, db, c.cin, c.cout, H, W, WS_CONV_AUTO, kpart, kSplitKCap, s);
    if (!dX) return;
    // dX = conv3x3(dY, W^T) with cin/cout swapped: a forward conv of the transposed layer, whose
    // tensor-core weights the step prepared; the FP32 transpose only for the other kernels
    const bool tcx = wtb && tc_bwd_ok(li) &&
                     (conv3x3_tc_ok(c.cout, c.cin, H, W) || conv3x3_tc_narrow_ok(c.cout, c.cin, H, W));
    if (!tcx)
        TW_LAUNCH(conv_transpose_weights_kernel, blocks_for((size_t)c.cin * c.cout * 9), 256, 0, s, Wt, wt, c.cin,
                  c.cout);
    bf16 *dst = accumulate ? tmp : dX;
    conv3x3(dY, wt, nullptr, nullptr, dst, c.cout, c.cin, H, W, 0, WS_CONV_AUTO, s, kpart, kSplitKCap,
            tcx ? wtb + tc_w_off(li) : nullptr);
    if (accumulate)
        TW_LAUNCH(add_inplace_kernel, blocks_for((size_t)c.cin * H * W), 256, 0, s, dX, tmp, (size_t)c.cin * H * W);
}

// Backward pass from dOut (gradient of the head output) to the parameter gradients G.
static void backward(const float *P, float *G, Act &A, int H, int W, cudaStream_t s, bf16 *d_out,
                     std::vector<bf16 *> &scratch) {
    // scratch buffers: dA (current), dB, skip gradients per level, tmp
    bf16 *dcur = scratch[0], *dnext = scratch[1], *tmp = scratch[2];
    bf16 *dskip[3] = {scratch[3], scratch[4], scratch[5]};   // gradients into e[2][1], e[1][1], e[0][1]
    // head (linear): dOut -> d(d[2][1])
    conv_bwd(A.d[2][1], P, G, 14, d_out, dcur, tmp, H, W, A.wt, A.kpart, A.wtb, 0, s);
    const int dc[3] = {128, 64, 32}, pc[3] = {128, 128, 64};
    for (int j = 2; j >= 0; j--) {
        const int l = 2 - j, h = H >> l, w = W >> l;
        // dcur: gradient of d[j][1] (post-ReLU output of conv 9 + 2j)
        TW_LAUNCH(relu_bwd_kernel, blocks_for(dc[j] * lvl_px(H, W, l)), 256, 0, s, A.d[j][1], dcur,
                  (size_t)dc[j] * lvl_px(H, W, l));
        conv_bwd(A.d[j][0], P, G, 9 + 2 * j, dcur, dnext, tmp, h, w, A.wt, A.kpart, A.wtb, 0, s);   // -> grad of d[j][0]
        TW_LAUNCH(relu_bwd_kernel, blocks_for(dc[j] * lvl_px(H, W, l)), 256, 0, s, A.d[j][0], dnext,
                  (size_t)dc[j] * lvl_px(H, W, l));
        // d[j][0] = relu(conv(u[j]) + e[l][1]): the skip receives the same gradient
        cudaMemcpyAsync(dskip[j], dnext, sizeof(bf16) * dc[j] * lvl_px(H, W, l), cudaMemcpyDeviceToDevice, s);
        conv_bwd(A.u[j], P, G, 8 + 2 * j, dnext, dcur, tmp, h, w, A.wt, A.kpart, A.wtb, 0, s);      // -> grad of u[j]
        // u[j] = up2(prev): gradient to prev (level l + 1)
        TW_LAUNCH(up2_bwd_kernel, dim3(ceil_div(w / 2, 256), h / 2, pc[j]), 256, 0, s, dcur, dnext, pc[j], h, w);
        bf16 *t = dcur; dcur = dnext; dnext = t;   // dcur: gradient of the previous decoder output
    }
    // dcur: gradient of e[3][1]; walk the encoder down, adding the skip gradients
    const int ch[4] = {32, 64, 128, 128};
    for (int l = 3; l >= 0; l--) {
        const int h = H >> l, w = W >> l;
        if (l <= 2)
            TW_LAUNCH(add_inplace_kernel, blocks_for(ch[l] * lvl_px(H, W, l)), 256, 0, s, dcur, dskip[2 - l],
                      (size_t)ch[l] * lvl_px(H, W, l));
        TW_LAUNCH(relu_bwd_kernel, blocks_for(ch[l] * lvl_px(H, W, l)), 256, 0, s, A.e[l][1], dcur,
                  (size_t)ch[l] * lvl_px(H, W, l));
        conv_bwd(A.e[l][0], P, G, 2 * l + 1, dcur, dnext, tmp, h, w, A.wt, A.kpart, A.wtb, 0, s);   // grad of e[l][0]
        TW_LAUNCH(relu_bwd_kernel, blocks_for(ch[l] * lvl_px(H, W, l)), 256, 0, s, A.e[l][0], dnext,
                  (size_t)ch[l] * lvl_px(H, W, l));
        const bf16 *xin = l == 0 ? A.in : A.p[l - 1];
        if (l == 0) {
            conv_bwd(xin, P, G, 0, dnext, nullptr, tmp, h, w, A.wt, A.kpart, A.wtb, 0, s);
        } else {
            conv_bwd(xin, P, G, 2 * l, dnext, dcur, tmp, h, w, A.wt, A.kpart, A.wtb, 0, s);          // grad of p[l-1]
            // p[l-1] = pool2(e[l-1][1]): spread into a zeroed gradient of e[l-1][1]
            cudaMemsetAsync(dnext, 0, sizeof(bf16) * ch[l - 1] * lvl_px(H, W, l - 1), s);
            TW_LAUNCH(pool2_bwd_kernel, dim3(ceil_div(W >> (l - 1), 256), H >> (l - 1), ch[l - 1]), 256, 0, s, dcur,
                      dnext, ch[l - 1], H >> (l - 1), W >> (l - 1));
            bf16 *t = dcur; dcur = dnext; dnext = t;
        }
    }
}

__global__ void make_target_kernel(const float *__restrict__ u, float *__restrict__ t, size_t n) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        t[i] = fmaxf(logf(fmaxf(u[i], 1e-30f)), -30.0f * 2.302585093f) / 30.0f;
}

__global__ void bf16_to_f32_kernel(const bf16 *__restrict__ a, float *__restrict__ b, size_t n) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        b[i] = __bfloat162float(a[i]);
}
__global__ void count_free_kernel(const uint8_t *__restrict__ occ, int gx, int gy, int W, size_t n, float *out) {
    float c = 0.0f;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        c += (occ[i] == 0 && !((int)(i % W) == gx && (int)(i / W) == gy)) ? 1.0f : 0.0f;
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(out, c);
}

static bool valid_hw(int H, int W) { return H >= 16 && W >= 16 && H % 8 == 0 && W % 8 == 0 && H <= 8192 && W <= 8192; }

}  // namespace nn
}  // namespace tw

using namespace tw;
using namespace tw::nn;

extern "C" size_t ws_unet_param_count(void) { return total_params(); }

extern "C" size_t ws_unet_workspace_size(int H, int W) {
    if (!valid_hw(H, W)) return 0;
    Carver cv;
    return carve_act(cv, H, W, nullptr);
}

static bool valid_stride(int H, int W, int s) {
    return (s == 1 || s == 2 || s == 4) && H % s == 0 && W % s == 0 && valid_hw(H / s, W / s) && H <= 8192 &&
           W <= 8192;
}

// the network's buffers at the coarse size, then the coarse occupancy
static size_t carve_warm(Carver &cv, int H, int W, int s, Act *A, uint8_t **oc) {
    carve_act(cv, H / s, W / s, A);
    uint8_t *o = cv.take<uint8_t>((size_t)(H / s) * (W / s));
    if (oc) *oc = o;
    return cv.need;
}

extern "C" size_t ws_unet_warm_start_workspace_size(int H, int W, int stride) {
    if (!valid_stride(H, W, stride)) return 0;
    Carver cv;
    return carve_warm(cv, H, W, stride, nullptr, nullptr);
}

extern "C" int ws_unet_warm_start(const float *params, const uint8_t *occ, int H, int W, int gx, int gy, int stride,
                                  float *u_out, void *workspace, size_t workspace_bytes, void *stream) {
    if (!params || !occ || !u_out || !valid_stride(H, W, stride) || gx < 0 || gy < 0 || gx >= W || gy >= H)
        return TW_EINVAL;
    if (!workspace || !ws_aligned(workspace)) return TW_EWORKSPACE;
    Carver cv(workspace, workspace_bytes);
    Act A;
    uint8_t *oc = nullptr;
    carve_warm(cv, H, W, stride, &A, &oc);
    if (!cv.ok()) return TW_EWORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    const int hc = H / stride, wc = W / stride, gxc = gx / stride, gyc = gy / stride;
    const uint8_t *oin = occ;
    if (stride > 1) {
        TW_LAUNCH(occ_pool_kernel, dim3(ceil_div(wc, 256), hc), 256, 0, s, occ, W, stride, gxc, gyc, oc, wc);
        oin = oc;
    }
    const size_t nc = (size_t)hc * wc;
    TW_LAUNCH(features_kernel, blocks_for(nc), 256, 0, s, oin, hc, wc, gxc, gyc, A.in);
    prepare_tc_weights(params, A, false, s);
    forward(params, A, hc, wc, s);
    TW_LAUNCH(upsample_to_u_kernel, dim3(ceil_div(W, 256), H), 256, 0, s, A.out, hc, wc, stride, occ, W, gx, gy,
              u_out);
    TW_CHECK_LAUNCH();
    return TW_OK;
}

extern "C" int ws_unet_init(float *params, unsigned long long seed, void *stream) {
    if (!params) return TW_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    for (int i = 0; i < kNumConvs; i++) {
        const ConvSpec &c = kConvs[i];
        const size_t nw = (size_t)c.cout * c.cin * 9;
        const float stdv = (i == kNumConvs - 1) ? sqrtf(1.0f / (9.0f * c.cin)) : sqrtf(2.0f / (9.0f * c.cin));
        TW_LAUNCH(init_kernel, blocks_for(conv_params(i)), 256, 0, s, params + param_offset(i), nw, conv_params(i),
                  stdv, seed, param_offset(i));
    }
    TW_CHECK_LAUNCH();
    return TW_OK;
}

extern "C" int ws_make_target(const float *u, size_t n, float *target, void *stream) {
    if (!u || !target) return TW_EINVAL;
    TW_LAUNCH(make_target_kernel, blocks_for(n), 256, 0, (cudaStream_t)stream, u, target, n);
    TW_CHECK_LAUNCH();
    return TW_OK;
}

extern "C" int ws_unet_forward(const float *params, const uint8_t *occ, int H, int W, int gx, int gy, float *u_out,
                               float *pred_out, void *workspace, size_t workspace_bytes, void *stream) {
    if (!params || !occ || !valid_hw(H, W) || gx < 0 || gy < 0 || gx >= W || gy >= H) return TW_EINVAL;
    if (!workspace || !ws_aligned(workspace)) return TW_EWORKSPACE;
    Carver cv(workspace, workspace_bytes);
    Act A;
    carve_act(cv, H, W, &A);
    if (!cv.ok()) return TW_EWORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t n = (size_t)H * W;
    TW_LAUNCH(features_kernel, blocks_for(n), 256, 0, s, occ, H, W, gx, gy, A.in);
    prepare_tc_weights(params, A, false, s);
    forward(params, A, H, W, s);
    if (u_out) TW_LAUNCH(to_u_kernel, blocks_for(n), 256, 0, s, A.out, occ, gx, gy, W, n, u_out);
    if (pred_out) {
        TW_LAUNCH(bf16_to_f32_kernel, blocks_for(n), 256, 0, s, A.out, pred_out, n);
    }
    TW_CHECK_LAUNCH();
    return TW_OK;
}

extern "C" int ws_unet_train_step(float *params, float *grads, float *adam_m, float *adam_v, int step, float lr,
                                  const uint8_t *occ, int H, int W, int gx, int gy, const float *target,
                                  float *loss_host, void *workspace, size_t workspace_bytes, void *stream) {
    if (!params || !grads || !occ || !target || !valid_hw(H, W) || gx < 0 || gy < 0 || gx >= W || gy >= H ||
        (adam_m && (!adam_v || step < 1 || !(lr > 0.0f))))
        return TW_EINVAL;
    if (!workspace || !ws_aligned(workspace)) return TW_EWORKSPACE;
    Carver cv(workspace, workspace_bytes);
    Act A;
    carve_act(cv, H, W, &A);
    if (!cv.ok()) return TW_EWORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t n = (size_t)H * W;
    TW_LAUNCH(features_kernel, blocks_for(n), 256, 0, s, occ, H, W, gx, gy, A.in);
    prepare_tc_weights(params, A, true, s);
    forward(params, A, H, W, s);
    // free-cell count for the loss normalisation (the mask: occ == 0 and not the goal)
    TW_CUDA(cudaMemsetAsync(A.loss, 0, 2 * sizeof(float), s));
    TW_LAUNCH(count_free_kernel, blocks_for(n), 256, 0, s, occ, gx, gy, W, n, A.loss + 1);
    float cnt = 0.0f;
    TW_CUDA(cudaMemcpyAsync(&cnt, A.loss + 1, sizeof(float), cudaMemcpyDeviceToHost, s));
    TW_CUDA(cudaStreamSynchronize(s));
    const float inv = cnt > 0.0f ? 1.0f / cnt : 0.0f;
    bf16 *d_out = A.g2;   // head-output gradient
    TW_LAUNCH(mse_kernel, blocks_for(n), 256, 0, s, A.out, target, occ, gx, gy, W, n, inv, d_out, A.kpart);
    TW_LAUNCH(loss_sum_kernel, 1, 32, 0, s, A.kpart, (int)blocks_for(n), A.loss);
    TW_CUDA(cudaMemsetAsync(grads, 0, sizeof(float) * total_params(), s));
    // backward needs its own scratch: dcur, dnext, tmp (64 x H x W), and the skip gradients
    std::vector<bf16 *> scratch = {A.g0, A.g1, A.g2, A.sk[0], A.sk[1], A.sk[2]};
    backward(params, grads, A, H, W, s, d_out, scratch);
    if (adam_m) {
        const float b1 = 0.9f, b2 = 0.999f;
        const float c1 = 1.0f - powf(b1, (float)step), c2 = 1.0f - powf(b2, (float)step);
        TW_LAUNCH(adam_kernel, blocks_for(total_params()), 256, 0, s, params, grads, adam_m, adam_v, total_params(),
                  lr, b1, b2, 1e-8f, c1, c2);
    }
    TW_CHECK_LAUNCH();
    if (loss_host) {
        TW_CUDA(cudaMemcpyAsync(loss_host, A.loss, sizeof(float), cudaMemcpyDeviceToHost, s));
        TW_CUDA(cudaStreamSynchronize(s));
    }
    return TW_OK;
}

extern "C" size_t ws_conv3x3_workspace_size(int cin, int cout, int H, int W, int impl) {
    using namespace tw::nn;
    if (impl != WS_CONV_TC || cin < 1 || cout < 1 || H < 1 || W < 1) return 0;
    if (conv3x3_tc_narrow_ok(cin, cout, H, W)) {
        const int sp = conv3x3_tc_narrow_splits(cin, cout, H, W, (size_t)-1);
        return narrow_weight_floats(cin, cout) * sizeof(float) + (sp > 1 ? (size_t)sp * cout * H * W * sizeof(float) : 0);
    }
    if (!conv3x3_tc_ok(cin, cout, H, W)) return 0;
    return (conv3x3_tc_scratch_bytes(cin, cout) + 255) & ~(size_t)255;
}

extern "C" int ws_conv3x3(const void *X, const float *Wt, const float *b, const void *S, void *Y, int cin, int cout,
                          int H, int W, int relu, int impl, void *workspace, size_t workspace_bytes, void *stream) {
    using namespace tw::nn;
    if (!X || !Wt || !Y || cin < 1 || cout < 1 || H < 1 || W < 1 || H > 65536 || W > 65536 ||
        (impl != WS_CONV_AUTO && impl != WS_CONV_SIMT && impl != WS_CONV_MMA && impl != WS_CONV_TC))
        return TW_EINVAL;
    if (impl == WS_CONV_TC && (!workspace || !ws_aligned(workspace))) return TW_EWORKSPACE;
    int e = conv3x3((const bf16 *)X, Wt, b, (const bf16 *)S, (bf16 *)Y, cin, cout, H, W, relu ? 1 : 0, impl,
                    (cudaStream_t)stream, impl == WS_CONV_TC ? (float *)workspace : nullptr,
                    impl == WS_CONV_TC ? workspace_bytes / sizeof(float) : 0);
    if (e) return e;
    TW_CHECK_LAUNCH();
    return TW_OK;
}

extern "C" size_t ws_conv3x3_wgrad_workspace_size(int cin, int cout, int H, int W, int impl) {
    using namespace tw::nn;
    if (cin < 1 || cout < 1 || H < 1 || W < 1 || H > 65536 || W > 65536 ||
        (impl != WS_CONV_AUTO && impl != WS_CONV_SIMT && impl != WS_CONV_TC) ||
        (impl == WS_CONV_TC && !conv3x3_wgrad_tc_ok(cin, cout, H, W)))
        return 0;
    return (conv3x3_wgrad_floats(cin, cout, H, W, impl) * sizeof(float) + 255) & ~(size_t)255;
}

extern "C" int ws_conv3x3_wgrad(const void *X, const void *dY, float *dW, float *db, int cin, int cout, int H, int W,
                                int impl, void *workspace, size_t workspace_bytes, void *stream) {
    using namespace tw::nn;
    if (!X || !dY || !dW || cin < 1 || cout < 1 || H < 1 || W < 1 || H > 65536 || W > 65536 ||
        (impl != WS_CONV_AUTO && impl != WS_CONV_SIMT && impl != WS_CONV_TC) ||
        (impl == WS_CONV_TC && !conv3x3_wgrad_tc_ok(cin, cout, H, W)))
        return TW_EINVAL;
    if (!workspace || !ws_aligned(workspace) ||
        workspace_bytes < conv3x3_wgrad_floats(cin, cout, H, W, impl) * sizeof(float))
        return TW_EWORKSPACE;
    int e = conv3x3_wgrad((const bf16 *)X, (const bf16 *)dY, dW, db, cin, cout, H, W, impl, (float *)workspace,
                          workspace_bytes / sizeof(float), (cudaStream_t)stream);
    if (e) return e;
    TW_CHECK_LAUNCH();
    return TW_OK;
}

extern "C" int ws_conv_check(int *timed_out) {
    using namespace tw::nn;
    if (!timed_out) return TW_EINVAL;
    return conv3x3_tc_error(timed_out);
}
