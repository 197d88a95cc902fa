// 3x3 convolution of the warm-start network on the 5th-generation tensor
// cores: an implicit GEMM issued with tcgen05.mma, accumulators in tensor
// memory (TMEM), operands staged in shared memory.
//
// GEMM view of one CTA: M = 128 output pixels of one image row (x0 .. x0+127)
// for each of MT consecutive rows (MT accumulators), N = cout, K = 9 taps x cin,
// consumed 16 input channels (one "chunk") at a time.  Per chunk the CTA stages
//   A: the chunk's 16 channels of MT + 2 input rows x 130 pixels (the tile and
//      its one-pixel halo), channel-last, as two 8-channel halves
//      [half][row][pixel][8 channels] (16 bytes per pixel and half): every
//      8 x 8 block of (pixels, channels) is one contiguous 128-byte core matrix
//      of the no-swizzle K-major operand layout, so the operand of tap (dy, dx)
//      and output row t is the same array started (t + dy) * 130 + dx pixels
//      in: a shift by whole 16-byte rows, no data movement per tap;
//   B: the chunk's weights, pre-arranged once per layer as
//      [tap][half][cout][8 channels] BF16 (conv_tc_weights_kernel).
// One elected thread issues the 9 x MT MMAs of a chunk (M = 128, N = cout,
// K = 16, BF16 in, FP32 accumulate) and commits them to the stage's mbarrier;
// meanwhile every thread stages the next chunk into the other stage
// (double buffering).  The epilogue reads each accumulator row from TMEM
// (warp w owns TMEM lanes 32 (w % 4) .. + 31, i.e. pixels), adds bias and skip,
// applies ReLU and stores BF16 in the network's [cout][H][W] layout.
//
// Every wait is bounded (one second of %globaltimer); a timeout sets
// g_conv_tc_error, skips the remaining work, waits (bounded) for the MMAs
// already issued and frees the TMEM before returning.
#include <cuda_bf16.h>
#include <stdint.h>

#include "common.cuh"
#include "nn_tc.cuh"

namespace tw {
namespace nn {

__device__ int g_conv_tc_error;   // 1 after a bounded wait timed out

namespace tc {

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t globaltimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n"
        " .reg .pred p;\n"
        " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n"
        "}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for the phase with the given parity to complete; false after one second.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
    const uint64_t t0 = globaltimer();
    while (!mbar_try_wait(bar, parity))
        if (globaltimer() - t0 > 1000000000ull) return false;
    return true;
}

// One thread: expect tx bytes on *bar, then copy bytes (multiple of 16, both
// addresses 16-byte aligned) from global to shared memory with the bulk-copy
// engine; the barrier's phase completes when they have landed.
__device__ __forceinline__ void bulk_load(void *dst_smem, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst_smem)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// Generic-proxy shared-memory writes -> visible to the tensor core's (async proxy) reads.
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// TMEM allocation (one whole warp); the base address is written to *dst.
__device__ __forceinline__ void tmem_alloc(uint32_t *dst, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)), "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// Shared-memory matrix descriptor, no swizzle: start address, the byte
// offset between core matrices along K (leading) and along M/N (stride),
// descriptor version 1 (bits 46-47).
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}

// Instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1), BF16 A
// and B (bits 7-9 and 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 in
// bits 17-22, M >> 4 in bits 24-28.
template <int M, int N>
struct IDesc {
    static constexpr uint32_t value = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
                                      ((uint32_t)(M >> 4) << 24);
};

// D[tmem] (+)= A[smem] x B[smem]^T, one elected thread.
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n"
        " .reg .pred p;\n"
        " setp.ne.u32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n"
        "}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// Arrive on *bar once every tcgen05.mma issued so far by this thread has completed.
__device__ __forceinline__ void mma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

// 16 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 16; j++) v[j] = __uint_as_float(r[j]);
}

}  // namespace tc

// Weights Wt [cout][cin][3][3] FP32 -> Wb [cin/16][9][2][cout][8] BF16: for
// chunk c, tap k and half h, the cout x 8 block of input channels
// 16c + 8h .. 16c + 8h + 7, one 16-byte row per output channel.
__global__ void conv_tc_weights_kernel(const float *__restrict__ Wt, bf16 *__restrict__ Wb, int cin, int cout) {
    const size_t n = (size_t)cin * cout * 9;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        // i enumerates the destination: ((((chunk * 9 + k) * 2 + h) * cout + co) * 8 + e)
        const int e = (int)(i % 8);
        size_t r = i / 8;
        const int co = (int)(r % cout);
        r /= cout;
        const int h = (int)(r % 2);
        r /= 2;
        const int k = (int)(r % 9);
        const int chunk = (int)(r / 9);
        const int ci = 16 * chunk + 8 * h + e;
        Wb[i] = __float2bfloat16(Wt[((size_t)co * cin + ci) * 9 + k]);
    }
}

__global__ void conv_tc_weights_all_kernel(const float *__restrict__ P, bf16 *__restrict__ wf, bf16 *__restrict__ wb,
                                           TcPrepTable t) {
    for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < t.total;
         g += (long long)gridDim.x * blockDim.x) {
        long long i = g;
        int l = 0;
        for (; l < t.n; l++) {
            const long long n2 = 2LL * t.cin[l] * t.cout[l] * 9;
            if (i < n2) break;
            i -= n2;
        }
        if (l >= t.n) continue;
        const long long n = (long long)t.cin[l] * t.cout[l] * 9;
        const bool bwd = i >= n;
        if (bwd) i -= n;
        const long long off = bwd ? t.boff[l] : t.foff[l];
        if (off < 0) continue;
        // the arranged layer: cin_a -> cout_a
        const int cin_a = bwd ? t.cout[l] : t.cin[l], cout_a = bwd ? t.cin[l] : t.cout[l];
        const int e = (int)(i % 8);
        long long r = i / 8;
        const int co = (int)(r % cout_a);
        r /= cout_a;
        const int h = (int)(r % 2);
        r /= 2;
        const int k = (int)(r % 9);
        const int chunk = (int)(r / 9);
        const int ci = 16 * chunk + 8 * h + e;
        const float *W = P + t.poff[l];
        const float v = bwd ? W[((size_t)ci * t.cin[l] + co) * 9 + (8 - k)] : W[((size_t)co * t.cin[l] + ci) * 9 + k];
        (bwd ? wb : wf)[off + i] = __float2bfloat16(v);
    }
}

int conv_tc_prepare_weights(const float *P, const TcPrepTable &t, bf16 *wf, bf16 *wb, cudaStream_t s) {
    TW_LAUNCH(conv_tc_weights_all_kernel, (unsigned)((t.total + 255) / 256 > 2048 ? 2048 : (t.total + 255) / 256), 256,
              0, s, P, wf, wb, t);
    return TW_OK;
}

template <int N, int MT>
struct TcShape {
    static constexpr int PX = 130;                                  // 128 pixels + halo
    static constexpr int ROWS = MT + 2;                             // input rows per tile
    static constexpr uint32_t A_HALF = ROWS * PX * 16;              // bytes of one 8-channel half
    static constexpr uint32_t A_BYTES = 2 * A_HALF;
    static constexpr uint32_t B_TAP = 2 * N * 16;                   // bytes of one tap's weights
    static constexpr uint32_t B_BYTES = 9 * B_TAP;
    static constexpr uint32_t STAGE = A_BYTES + B_BYTES;
    static constexpr uint32_t SMEM = 2 * STAGE;
    static constexpr uint32_t NCOL = MT * N <= 32 ? 32 : (MT * N <= 64 ? 64 : (MT * N <= 128 ? 128 : (MT * N <= 256 ? 256 : 512)));
    static_assert(MT * N <= 512, "accumulators exceed the tensor memory");
    static_assert(A_HALF % 16 == 0 && B_TAP % 16 == 0 && STAGE % 16 == 0, "16-byte operand alignment");
};

// Y = act(conv3x3(X) + b + S) for W % 128 == 0, H % MT == 0, cin % 16 == 0,
// cout == N; kTcThreads threads; grid (W / 128, H / MT).  Per chunk i (stage i % 2):
// once the MMAs of chunk i - 2 are done, thread 0 starts the bulk copy of the
// chunk's weights into the stage, every thread writes the chunk's input tile
// from the registers it loaded during the previous chunk and issues the loads
// of the next chunk's tile (in flight while this chunk's MMAs run); after a
// barrier thread 0 waits for the weights and issues the MMAs.
constexpr int kTcThreads = 256;   // 8 warps: more tile loads in flight per SM
template <int N, int MT>
__global__ void __launch_bounds__(kTcThreads, 2) conv3x3_tc_kernel(const bf16 *__restrict__ X, const uint4 *__restrict__ Wb,
                                                         const float *__restrict__ b, const bf16 *__restrict__ S,
                                                         bf16 *__restrict__ Y, int cin, int H, int W, int relu) {
    using Sh = TcShape<N, MT>;
    constexpr int NITEMS = 2 * Sh::ROWS * Sh::PX;          // (half, row, pixel) items of a tile
    constexpr int ITEMS = (NITEMS + kTcThreads - 1) / kTcThreads;   // per thread
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ uint64_t mma_done[2], b_full[2];
    __shared__ uint32_t tmem_base_sh;
    __shared__ int abort_sh;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int x0 = blockIdx.x * 128, y0 = blockIdx.y * MT;
    const int chunks = cin / 16;
    const size_t plane = (size_t)H * W;

    if (warp == 0) tc::tmem_alloc(&tmem_base_sh, Sh::NCOL);
    if (tid == 0) {
        for (int k = 0; k < 2; k++) {
            tc::mbar_init(&mma_done[k], 1);
            tc::mbar_init(&b_full[k], 1);
        }
        tc::fence_mbar_init();
        abort_sh = 0;
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tmem_base_sh;
    const uint32_t sbase = tc::smem_u32(smem);

    // this thread's items: source offsets (or -1 outside the image / past the tile) and shared offsets
    long long src_off[ITEMS];
    uint32_t dst_off[ITEMS];
#pragma unroll
    for (int j = 0; j < ITEMS; j++) {
        const int it = tid + kTcThreads * j;
        src_off[j] = -1;
        dst_off[j] = 0xFFFFFFFFu;
        if (it < NITEMS) {
            const int h = it / (Sh::ROWS * Sh::PX), rem = it - h * (Sh::ROWS * Sh::PX);
            const int r = rem / Sh::PX, p = rem - r * Sh::PX;
            const int y = y0 - 1 + r, x = x0 - 1 + p;
            dst_off[j] = h * Sh::A_HALF + (r * Sh::PX + p) * 16;
            if (y >= 0 && y < H && x >= 0 && x < W) src_off[j] = (long long)(8 * h) * plane + (long long)y * W + x;
        }
    }
    const unsigned short *Xs = reinterpret_cast<const unsigned short *>(X);
    uint32_t ra[ITEMS][4];   // the prefetched tile: 8 channels per item, packed in pairs
    auto load_tile = [&](int chunk) {
        const unsigned short *base = Xs + (size_t)(16 * chunk) * plane;
#pragma unroll
        for (int j = 0; j < ITEMS; j++) {
#pragma unroll
            for (int c = 0; c < 8; c += 2) {
                uint32_t lo = 0u, hi = 0u;
                if (src_off[j] >= 0) {
                    lo = __ldg(base + src_off[j] + (size_t)c * plane);
                    hi = __ldg(base + src_off[j] + (size_t)(c + 1) * plane);
                }
                ra[j][c >> 1] = lo | (hi << 16);
            }
        }
    };
    load_tile(0);
    int issued = 0;
    for (int i = 0; i < chunks; i++) {
        const int st = i & 1;
        // the stage's previous chunk (i - 2) must have been consumed by its MMAs
        if (i >= 2 && !tc::mbar_wait(&mma_done[st], (uint32_t)(((i >> 1) - 1) & 1))) abort_sh = 1;
        uint8_t *sA = smem + st * Sh::STAGE;
        if (tid == 0 && !abort_sh)
            tc::bulk_load(sA + Sh::A_BYTES, Wb + (size_t)i * (Sh::B_BYTES / 16), Sh::B_BYTES, &b_full[st]);
#pragma unroll
        for (int j = 0; j < ITEMS; j++)
            if (dst_off[j] != 0xFFFFFFFFu)
                *reinterpret_cast<uint4 *>(sA + dst_off[j]) = make_uint4(ra[j][0], ra[j][1], ra[j][2], ra[j][3]);
        if (i + 1 < chunks) load_tile(i + 1);
        tc::fence_proxy_async_smem();
        __syncthreads();
        if (abort_sh) break;
        if (tid == 0) {
            if (!tc::mbar_wait(&b_full[st], (uint32_t)((i >> 1) & 1))) {
                abort_sh = 1;
            } else {
                tc::fence_after_sync();
                const uint32_t a0 = sbase + st * Sh::STAGE, b0 = a0 + Sh::A_BYTES;
#pragma unroll 1
                for (int t = 0; t < MT; t++) {
#pragma unroll
                    for (int k = 0; k < 9; k++) {
                        const int dy = k / 3, dx = k - 3 * (k / 3);
                        const uint64_t ad = tc::smem_desc(a0 + ((t + dy) * Sh::PX + dx) * 16, Sh::A_HALF, 128);
                        const uint64_t bd = tc::smem_desc(b0 + k * Sh::B_TAP, N * 16, 128);
                        tc::mma_bf16(tmem + (uint32_t)(t * N), ad, bd, tc::IDesc<128, N>::value,
                                     (i > 0 || k > 0) ? 1u : 0u);
                    }
                }
                tc::mma_commit(&mma_done[st]);
            }
        }
        issued = i + 1;
    }
    __syncthreads();   // thread 0's abort (a weight copy that never landed) is seen by all
    // the last issued chunk's commit covers every MMA issued before it
    bool done = true;
    if (issued > 0 && !abort_sh) {
        const int last = issued - 1;
        done = tc::mbar_wait(&mma_done[last & 1], (uint32_t)((last >> 1) & 1));
    }
    if (!done || abort_sh) {
        if (tid == 0) atomicExch(&g_conv_tc_error, 1);
        // the MMAs already issued must finish before the tensor memory is released (bounded)
        if (issued > 0) tc::mbar_wait(&mma_done[(issued - 1) & 1], (uint32_t)(((issued - 1) >> 1) & 1));
    } else {
        tc::fence_after_sync();
        // warp w reads TMEM lanes 32 (w % 4) .. + 31 (its pixels); warps 0-3 and 4-7 take alternate
        // 16-column blocks of the MT accumulators
        const int wl = warp & 3, wh = warp >> 2;
        const int x = x0 + 32 * wl + lane;
#pragma unroll 1
        for (int t = 0; t < MT; t++) {
            const int y = y0 + t;
#pragma unroll 1
            for (int c0 = 16 * wh; c0 < N; c0 += 16 * (kTcThreads / 128)) {
                float v[16];
                tc::tmem_ld16(tmem + ((uint32_t)(32 * wl) << 16) + (uint32_t)(t * N + c0), v);
#pragma unroll
                for (int j = 0; j < 16; j++) {
                    const int co = c0 + j;
                    const size_t o = (size_t)co * plane + (size_t)y * W + x;
                    float val = v[j] + (b ? b[co] : 0.0f);
                    if (S) val += __bfloat162float(S[o]);
                    if (relu) val = fmaxf(val, 0.0f);
                    Y[o] = __float2bfloat16(val);
                }
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, Sh::NCOL);
}

// Output rows per CTA for cout = n (measured on GB300: four rows gain 10-15 % at cout 32 and 64;
// at cout 128 their 512 accumulator columns leave one CTA per SM and two rows are faster).
static constexpr int tc_rows(int n) { return n == 128 ? 2 : 4; }

template <int N>
static int launch_tc(const bf16 *X, const bf16 *Wb, const float *b, const bf16 *S, bf16 *Y, int cin, int H, int W,
                     int relu, cudaStream_t s) {
    // output rows per CTA: 4 where the accumulators leave room for two CTAs per SM, else 2
    constexpr int MT = tc_rows(N);
    using Sh = TcShape<N, MT>;
    static bool attr_set[64] = {};   // per device: the dynamic shared-memory opt-in
    int dev = 0;
    TW_CUDA(cudaGetDevice(&dev));
    if (dev >= 0 && dev < 64 && !attr_set[dev]) {
        TW_CUDA(cudaFuncSetAttribute(conv3x3_tc_kernel<N, MT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)Sh::SMEM));
        attr_set[dev] = true;
    }
    dim3 grid(W / 128, H / MT);
    TW_LAUNCH((conv3x3_tc_kernel<N, MT>), grid, kTcThreads, Sh::SMEM, s, X, reinterpret_cast<const uint4 *>(Wb), b, S, Y,
              cin, H, W, relu);
    return TW_OK;
}

// Shape conditions of the tensor-memory convolution.
bool conv3x3_tc_ok(int cin, int cout, int H, int W) {
    return cin % 16 == 0 && cin >= 16 && (cout == 32 || cout == 64 || cout == 128) && W % 128 == 0 && H % tc_rows(cout) == 0;
}

// Bytes of BF16 scratch for the re-arranged weights of a cin -> cout layer.
size_t conv3x3_tc_scratch_bytes(int cin, int cout) { return (size_t)cin * cout * 9 * sizeof(bf16); }

// Y = act(conv3x3(X, Wt) + b + S) on the tensor cores; scratch holds
// conv3x3_tc_scratch_bytes(cin, cout) bytes (16-byte aligned), where the
// weights are re-arranged, or (prearranged) already holds them in that layout.
int conv3x3_tc(const bf16 *X, const float *Wt, const float *b, const bf16 *S, bf16 *Y, int cin, int cout, int H,
               int W, int relu, void *scratch, cudaStream_t s, bool prearranged) {
    if (!conv3x3_tc_ok(cin, cout, H, W) || !scratch || ((uintptr_t)scratch & 15)) return TW_EINVAL;
    bf16 *Wb = (bf16 *)scratch;
    const size_t n = (size_t)cin * cout * 9;
    if (!prearranged)
        TW_LAUNCH(conv_tc_weights_kernel, (unsigned)((n + 255) / 256 > 1024 ? 1024 : (n + 255) / 256), 256, 0, s, Wt,
                  Wb, cin, cout);
    switch (cout) {
        case 32: return launch_tc<32>(X, Wb, b, S, Y, cin, H, W, relu, s);
        case 64: return launch_tc<64>(X, Wb, b, S, Y, cin, H, W, relu, s);
        default: return launch_tc<128>(X, Wb, b, S, Y, cin, H, W, relu, s);
    }
}

// ---- the same convolution for images narrower than 128 pixels ------------------
//
// W in {16, 32, 64}: one M block of 128 pixels spans R = 128 / W image rows, and
// a CTA computes NMB such blocks (NMB * R rows).  The tap shift in x cannot be a
// whole-row offset of one haloed tile here (the halo columns would sit between
// the rows of an M block), so per 16-channel chunk the input rows are written
// channel-last three times, shifted by dx - 1 pixels with zeros at the row ends:
// copy dx holds X[y][x + dx - 1], rows contiguous with pitch W, so the operand of
// tap (dy, dx) for block t is copy dx started (t * R + dy) * W pixels in.  The
// weights are the wide kernel's per-chunk layout, brought by the bulk-copy
// engine.  Split K: CTA (block, split) takes its share of the chunks; with more
// than one split it writes FP32 partial sums part[split][cout][H][W] (added in
// split order by the caller's finalisation, which also applies bias, skip and
// activation), else the finished BF16 output.
constexpr int kNarrowMB = 2;   // M blocks (of 128 pixels) per CTA

template <int N>
struct TcNarrowShape {
    static constexpr int PXMAX = kNarrowMB * 128 + 2 * 64;          // tile pixels at W = 64 (the widest)
    static constexpr uint32_t A_BYTES = 3 * 2 * PXMAX * 16;         // 3 shifted copies x 2 halves
    static constexpr uint32_t B_TAP = 2 * N * 16;
    static constexpr uint32_t B_BYTES = 9 * B_TAP;
    static constexpr uint32_t STAGE = A_BYTES + B_BYTES;
    static constexpr uint32_t SMEM = 2 * STAGE;
    static constexpr uint32_t NCOL = kNarrowMB * N <= 64 ? 64 : (kNarrowMB * N <= 128 ? 128 : 256);
    static constexpr int ITEMS = (2 * PXMAX + kTcThreads - 1) / kTcThreads;
    static_assert(STAGE % 16 == 0 && A_BYTES % 16 == 0, "16-byte operand alignment");
};

template <int N>
__global__ void __launch_bounds__(kTcThreads, N == 128 ? 1 : 2)
    conv3x3_tc_narrow_kernel(const bf16 *__restrict__ X, const uint4 *__restrict__ Wb, const float *__restrict__ b,
                             const bf16 *__restrict__ S, bf16 *__restrict__ Y, float *__restrict__ part, int cin,
                             int H, int W, int relu, int splits) {
    using Sh = TcNarrowShape<N>;
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ uint64_t mma_done[2], b_full[2];
    __shared__ uint32_t tmem_base_sh;
    __shared__ int abort_sh;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int R = 128 / W;                       // image rows per M block
    const int rows = kNarrowMB * R + 2;          // staged rows (one halo row above and below)
    const int y0 = blockIdx.x * kNarrowMB * R;
    const int chunks = cin / 16, per = (chunks + splits - 1) / splits;
    const int cb = blockIdx.y * per, ce = min(chunks, cb + per);
    const uint32_t half = (uint32_t)(rows * W) * 16u;   // bytes of one 8-channel half of one copy
    const size_t plane = (size_t)H * W;

    if (warp == 0) tc::tmem_alloc(&tmem_base_sh, Sh::NCOL);
    if (tid == 0) {
        for (int k = 0; k < 2; k++) {
            tc::mbar_init(&mma_done[k], 1);
            tc::mbar_init(&b_full[k], 1);
        }
        tc::fence_mbar_init();
        abort_sh = 0;
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tmem_base_sh;
    const uint32_t sbase = tc::smem_u32(smem);

    // this thread's items (half, row, x): source offsets (-1 outside the image) and positions
    const int nitems = 2 * rows * W;
    long long src_off[Sh::ITEMS];
    int pos[Sh::ITEMS];   // h * rows * W + r * W + x, or -1 past the tile
#pragma unroll
    for (int j = 0; j < Sh::ITEMS; j++) {
        const int it = tid + kTcThreads * j;
        src_off[j] = -1;
        pos[j] = -1;
        if (it < nitems) {
            const int h = it / (rows * W), rem = it - h * (rows * W);
            const int r = rem / W, x = rem - r * W;
            const int y = y0 - 1 + r;
            pos[j] = it;
            if (y >= 0 && y < H) src_off[j] = (long long)(8 * h) * plane + (long long)y * W + x;
        }
    }
    const unsigned short *Xs = reinterpret_cast<const unsigned short *>(X);
    uint32_t ra[Sh::ITEMS][4];
    auto load_tile = [&](int chunk) {
        const unsigned short *base = Xs + (size_t)(16 * chunk) * plane;
#pragma unroll
        for (int j = 0; j < Sh::ITEMS; j++) {
#pragma unroll
            for (int c = 0; c < 8; c += 2) {
                uint32_t lo = 0u, hi = 0u;
                if (src_off[j] >= 0) {
                    lo = __ldg(base + src_off[j] + (size_t)c * plane);
                    hi = __ldg(base + src_off[j] + (size_t)(c + 1) * plane);
                }
                ra[j][c >> 1] = lo | (hi << 16);
            }
        }
    };
    if (cb < ce) load_tile(cb);
    int issued = 0;
    for (int i = cb; i < ce; i++) {
        const int li = i - cb, st = li & 1;
        if (li >= 2 && !tc::mbar_wait(&mma_done[st], (uint32_t)(((li >> 1) - 1) & 1))) abort_sh = 1;
        uint8_t *sA = smem + st * Sh::STAGE;
        if (tid == 0 && !abort_sh)
            tc::bulk_load(sA + Sh::A_BYTES, Wb + (size_t)i * (Sh::B_BYTES / 16), Sh::B_BYTES, &b_full[st]);
#pragma unroll
        for (int j = 0; j < Sh::ITEMS; j++) {
            if (pos[j] < 0) continue;
            const int h = pos[j] / (rows * W), rem = pos[j] - h * (rows * W);
            const int x = rem % W;
            const uint4 v = make_uint4(ra[j][0], ra[j][1], ra[j][2], ra[j][3]);
            const uint4 zero = make_uint4(0u, 0u, 0u, 0u);
            uint8_t *p = sA + h * half + (uint32_t)rem * 16u;   // copy 0, this pixel's slot
            // copy dx holds X[x + dx - 1]: this pixel is copy 1 at x, copy 0 at x + 1, copy 2 at x - 1
            *reinterpret_cast<uint4 *>(p + 2 * half) = v;
            if (x + 1 < W) *reinterpret_cast<uint4 *>(p + 16) = v;
            if (x == 0) *reinterpret_cast<uint4 *>(p) = zero;
            if (x >= 1) *reinterpret_cast<uint4 *>(p + 4 * half - 16) = v;
            if (x == W - 1) *reinterpret_cast<uint4 *>(p + 4 * half) = zero;
        }
        if (i + 1 < ce) load_tile(i + 1);
        tc::fence_proxy_async_smem();
        __syncthreads();
        if (abort_sh) break;
        if (tid == 0) {
            if (!tc::mbar_wait(&b_full[st], (uint32_t)((li >> 1) & 1))) {
                abort_sh = 1;
            } else {
                tc::fence_after_sync();
                const uint32_t a0 = sbase + st * Sh::STAGE, b0 = a0 + Sh::A_BYTES;
#pragma unroll 1
                for (int t = 0; t < kNarrowMB; t++) {
#pragma unroll
                    for (int k = 0; k < 9; k++) {
                        const int dy = k / 3, dx = k - 3 * (k / 3);
                        const uint64_t ad =
                            tc::smem_desc(a0 + dx * 2 * half + (uint32_t)((t * R + dy) * W) * 16u, half, 128);
                        const uint64_t bd = tc::smem_desc(b0 + k * Sh::B_TAP, N * 16, 128);
                        tc::mma_bf16(tmem + (uint32_t)(t * N), ad, bd, tc::IDesc<128, N>::value,
                                     (li > 0 || k > 0) ? 1u : 0u);
                    }
                }
                tc::mma_commit(&mma_done[st]);
            }
        }
        issued = li + 1;
    }
    __syncthreads();
    bool done = true;
    if (issued > 0 && !abort_sh) {
        const int last = issued - 1;
        done = tc::mbar_wait(&mma_done[last & 1], (uint32_t)((last >> 1) & 1));
    }
    if (!done) abort_sh = 1;
    __syncthreads();
    if (abort_sh) {
        if (tid == 0) atomicExch(&g_conv_tc_error, 1);
        if (issued > 0) tc::mbar_wait(&mma_done[(issued - 1) & 1], (uint32_t)(((issued - 1) >> 1) & 1));
    } else {
        tc::fence_after_sync();
        const int wl = warp & 3, wh = warp >> 2;
        const int pix = 32 * wl + lane;   // TMEM lane = pixel of the M block
#pragma unroll 1
        for (int t = 0; t < kNarrowMB; t++) {
            const int y = y0 + t * R + pix / W, x = pix % W;
#pragma unroll 1
            for (int c0 = 16 * wh; c0 < N; c0 += 16 * (kTcThreads / 128)) {
                float v[16];
                tc::tmem_ld16(tmem + ((uint32_t)(32 * wl) << 16) + (uint32_t)(t * N + c0), v);
                if (issued == 0) {
#pragma unroll
                    for (int j = 0; j < 16; j++) v[j] = 0.0f;   // a split without chunks adds nothing
                }
#pragma unroll
                for (int j = 0; j < 16; j++) {
                    const int co = c0 + j;
                    const size_t o = (size_t)co * plane + (size_t)y * W + x;
                    if (splits > 1) {
                        part[(size_t)blockIdx.y * N * plane + o] = v[j];
                    } else {
                        float val = v[j] + (b ? b[co] : 0.0f);
                        if (S) val += __bfloat162float(S[o]);
                        if (relu) val = fmaxf(val, 0.0f);
                        Y[o] = __float2bfloat16(val);
                    }
                }
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, Sh::NCOL);
}

// Shape conditions of the narrow tensor-memory convolution.
bool conv3x3_tc_narrow_ok(int cin, int cout, int H, int W) {
    return cin % 16 == 0 && cin >= 16 && (cout == 32 || cout == 64 || cout == 128) &&
           (W == 16 || W == 32 || W == 64) && H % (kNarrowMB * 128 / W) == 0;
}

// Splits of the narrow form: enough CTAs for two per SM of a 152-SM GPU, at most
// one per 16-channel chunk, no empty split, and partial sums within part_floats.
int conv3x3_tc_narrow_splits(int cin, int cout, int H, int W, size_t part_floats) {
    const int base = H / (kNarrowMB * 128 / W);
    const int chunks = cin / 16;
    int sp = (304 + base - 1) / base;
    if (sp > chunks) sp = chunks;
    while (sp > 1 && (size_t)sp * cout * H * W > part_floats) sp--;
    if (sp < 1) sp = 1;
    const int per = (chunks + sp - 1) / sp;
    return (chunks + per - 1) / per;
}

template <int N>
static int launch_tc_narrow(const bf16 *X, const bf16 *Wb, const float *b, const bf16 *S, bf16 *Y, float *part,
                            int cin, int H, int W, int relu, int splits, cudaStream_t s) {
    using Sh = TcNarrowShape<N>;
    static bool attr_set[64] = {};
    int dev = 0;
    TW_CUDA(cudaGetDevice(&dev));
    if (dev >= 0 && dev < 64 && !attr_set[dev]) {
        TW_CUDA(cudaFuncSetAttribute(conv3x3_tc_narrow_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)Sh::SMEM));
        attr_set[dev] = true;
    }
    dim3 grid(H / (kNarrowMB * 128 / W), splits);
    TW_LAUNCH((conv3x3_tc_narrow_kernel<N>), grid, kTcThreads, Sh::SMEM, s, X, reinterpret_cast<const uint4 *>(Wb), b,
              S, Y, part, cin, H, W, relu, splits);
    return TW_OK;
}

// The narrow form: wscratch holds conv3x3_tc_scratch_bytes(cin, cout) bytes for the
// re-arranged weights (16-byte aligned; already arranged if prearranged); with
// splits > 1 the kernel writes FP32 partial sums to part[split][cout][H][W] and
// the caller finalises them.
int conv3x3_tc_narrow(const bf16 *X, const float *Wt, const float *b, const bf16 *S, bf16 *Y, int cin, int cout, int H,
                      int W, int relu, int splits, void *wscratch, float *part, cudaStream_t s, bool prearranged) {
    if (!conv3x3_tc_narrow_ok(cin, cout, H, W) || !wscratch || ((uintptr_t)wscratch & 15) || splits < 1 ||
        (splits > 1 && !part))
        return TW_EINVAL;
    bf16 *Wb = (bf16 *)wscratch;
    const size_t n = (size_t)cin * cout * 9;
    if (!prearranged)
        TW_LAUNCH(conv_tc_weights_kernel, (unsigned)((n + 255) / 256 > 1024 ? 1024 : (n + 255) / 256), 256, 0, s, Wt,
                  Wb, cin, cout);
    switch (cout) {
        case 32: return launch_tc_narrow<32>(X, Wb, b, S, Y, part, cin, H, W, relu, splits, s);
        case 64: return launch_tc_narrow<64>(X, Wb, b, S, Y, part, cin, H, W, relu, splits, s);
        default: return launch_tc_narrow<128>(X, Wb, b, S, Y, part, cin, H, W, relu, splits, s);
    }
}

// Reads and clears the timeout flag of the current device (1 if a bounded wait gave up).
int conv3x3_tc_error(int *flag) {
    int h = 0;
    TW_CUDA(cudaMemcpyFromSymbol(&h, g_conv_tc_error, sizeof(int)));
    if (h) {
        const int zero = 0;
        TW_CUDA(cudaMemcpyToSymbol(g_conv_tc_error, &zero, sizeof(int)));
    }
    *flag = h;
    return TW_OK;
}


// ---- weight gradient on the tensor cores ---------------------------------------
//
// dW[co][ci][ky][kx] = sum_p dY[co][p] X[ci][p + (ky - 1, kx - 1)] (zero outside
// the image) and db[co] = sum_p dY[co][p]: for each tap a GEMM whose K runs over
// the pixels.  CTA (ky, z) owns the three taps (ky, 0..2) and the pixel chunk z
// (consecutive pixels in row-major order), 64 pixels per stage.  The operands are
// staged K-major without swizzle: 8 consecutive pixels of one channel (16 bytes,
// one aligned copy from the network's [c][H][W] layout) form one row of a core
// matrix; channel group g and pixel group j sit at g * SBO + j * 128 bytes.
// Every thread copies its share of a stage with cp.async (16 bytes, zero-filled
// outside the tensor) into a ring of four stages, two stages ahead of the one
// the tensor cores consume: dY, and X at the row of tap ky with one extra pixel
// group on each side (groups -1 .. 8).  Once a stage has landed, the threads
// build the two copies of X shifted by one pixel (taps kx = 0 and 2) from the
// landed groups and their neighbours (zero across the image's left and right
// edges), so that every tap's operand starts on a 16-byte boundary; the
// unshifted tap reads the landed X directly.  M = 128 rows: X where cin is 128
// and cout at most 64, else dY (its rows beyond cout unused); N the other side's
// channel count rounded up to 32, 64 or 128 (columns beyond it unused); the
// three taps' accumulators lie side by side in tensor memory.  Each CTA writes its chunk's
// sums to part[z][k][m][n] (m the M row, n the N column), the bias sums (CTAs
// with ky = 0) to part_b[z][co]; conv_wgrad_tc_sum_kernel adds the chunks in
// order, so the result does not depend on the order the CTAs finish in.
constexpr int kWgPx = 64;          // pixels per stage
constexpr int kWgThreads = 256;
constexpr int kWgRing = 4;         // stages of copies in flight or landed
constexpr int kWgAhead = 2;        // stages copied ahead of the one consumed

template <bool XA, int N>
struct WgShape {
    static constexpr int DROWS = XA ? N : 128;                   // dY rows (128 on the M side)
    static constexpr int XROWS = XA ? 128 : N;                   // X rows
    static constexpr uint32_t D_BYTES = DROWS * 128;             // 8 groups of 8 pixels per channel
    static constexpr uint32_t X1_SBO = 10 * 128;                 // 10 groups (-1 .. 8) per channel group
    static constexpr uint32_t X1_BYTES = XROWS * 160;
    static constexpr uint32_t SLOT = D_BYTES + X1_BYTES;         // one ring stage
    static constexpr uint32_t XS_PLANE = XROWS * 128;            // one shifted copy
    static constexpr uint32_t XS_BUF = 2 * XS_PLANE;             // kx = 0 and 2
    static constexpr uint32_t SMEM = kWgRing * SLOT + 2 * XS_BUF;
    static constexpr uint32_t NCOL = 3 * N <= 128 ? 128 : (3 * N <= 256 ? 256 : 512);
    static constexpr int QD = DROWS * 8 / kWgThreads;            // dY groups per thread (at most)
    static constexpr int QX1 = (XROWS * 10 + kWgThreads - 1) / kWgThreads;   // X groups per thread (at most)
    // CTAs one SM holds (233472 bytes of shared memory, 512 tensor-memory columns)
    static constexpr int RES = (233472 / (SMEM + 2048)) < (512 / NCOL) ? (233472 / (SMEM + 2048)) : (512 / NCOL);
    static_assert(3 * N <= 512, "accumulators exceed the tensor memory");
    static_assert(SLOT % 1024 == 0 && XS_PLANE % 1024 == 0, "stage alignment");
    static_assert(SMEM <= 227 * 1024, "shared memory");
};

namespace tc {
// 16-byte global -> shared copy; src_bytes = 0 fills zeros without reading.
__device__ __forceinline__ void cp_async16(void *dst_smem, const void *src, uint32_t src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(dst_smem)), "l"(src), "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int n>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(n) : "memory"); }
}  // namespace tc

template <bool XA, int N>
__global__ void __launch_bounds__(kWgThreads, 1)
    conv3x3_wgrad_tc_kernel(const bf16 *__restrict__ X, const bf16 *__restrict__ dY, float *__restrict__ part,
                            float *__restrict__ part_b, int cin, int cout, int H, int W, int chunk_px) {
    using Sh = WgShape<XA, N>;
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ uint64_t mma_done[2];
    __shared__ uint32_t tmem_base_sh;
    __shared__ int abort_sh;
    __shared__ float bias_sh[4][4][8];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int ky = blockIdx.x, z = blockIdx.y;
    const long plane = (long)H * W;
    const long pa = (long)z * chunk_px;
    const long pb = pa + chunk_px < plane ? pa + chunk_px : plane;
    const int nst = (int)((pb - pa + kWgPx - 1) / kWgPx);
    const int ma = XA ? cin : cout;   // rows of the M side that hold data
    const long xoff = (long)(ky - 1) * W;   // X pixel of dY pixel p: p + xoff (+ kx - 1)

    if (warp == 0) tc::tmem_alloc(&tmem_base_sh, Sh::NCOL);
    if (tid == 0) {
        tc::mbar_init(&mma_done[0], 1);
        tc::mbar_init(&mma_done[1], 1);
        tc::fence_mbar_init();
        abort_sh = 0;
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tmem_base_sh;
    const uint32_t sbase = tc::smem_u32(smem);
    uint8_t *const xs_buf = smem + kWgRing * Sh::SLOT;

    // copies of stage i into ring slot i % kWgRing: dY group (c, j) at ((c / 8) * 8 + j) * 128 + (c % 8) * 16,
    // X group (c, j), j = -1 .. 8, at ((c / 8) * 10 + j + 1) * 128 + (c % 8) * 16
    auto issue_stage = [&](int i) {
        uint8_t *sD = smem + (i % kWgRing) * Sh::SLOT;
        uint8_t *sX = sD + Sh::D_BYTES;
        const long p0 = pa + (long)i * kWgPx;
#pragma unroll
        for (int q = 0; q < Sh::QD; q++) {
            const int u = tid + kWgThreads * q;
            const int c = (u >> 6) * 8 + (u & 7), j = (u >> 3) & 7;
            if (c < cout) {
                const long p = p0 + 8 * j;
                const bool in = p < pb;
                tc::cp_async16(sD + u * 16, in ? (const void *)(dY + (size_t)c * plane + p) : (const void *)dY,
                               in ? 16u : 0u);
            }
        }
#pragma unroll
        for (int q = 0; q < Sh::QX1; q++) {
            const int v = tid + kWgThreads * q;
            const int c = (v / 80) * 8 + (v & 7), jj = (v >> 3) % 10;
            if (c < cin) {
                const long px = p0 + 8 * (jj - 1) + xoff;
                const bool in = px >= 0 && px < plane;
                tc::cp_async16(sX + v * 16, in ? (const void *)(X + (size_t)c * plane + px) : (const void *)X,
                               in ? 16u : 0u);
            }
        }
    };

    // this thread's groups when building the shifted copies: pixel group jg, channels cb + 32 q
    const int jg = (tid >> 3) & 7;
    const int cb = (tid >> 6) * 8 + (tid & 7);
    const int nqd = (cout + 31) / 32, nqx = (cin + 31) / 32;
    float bsum[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    const bool with_bias = ky == 0;

#pragma unroll 1
    for (int i = 0; i < kWgAhead; i++) {
        if (i < nst) issue_stage(i);
        tc::cp_async_commit();
    }
    int issued = 0;
    for (int i = 0; i < nst; i++) {
        const int st = i & 1;
        // MMAs of stage i - 2 read ring slot (i + 2) % 4 and shifted buffer st
        if (i >= 2 && !tc::mbar_wait(&mma_done[st], (uint32_t)(((i >> 1) - 1) & 1))) abort_sh = 1;
        if (i + kWgAhead < nst) issue_stage(i + kWgAhead);
        tc::cp_async_commit();
        tc::cp_async_wait<kWgAhead>();   // stage i has landed (this thread's copies)
        __syncthreads();                 // ... and every other thread's
        const uint8_t *sD = smem + (i % kWgRing) * Sh::SLOT;
        const uint8_t *sX = sD + Sh::D_BYTES;
        uint8_t *sS = xs_buf + st * Sh::XS_BUF;
        const long p = pa + (long)i * kWgPx + 8 * jg;
        const int x = (int)(p % W);
#pragma unroll
        for (int q = 0; q < 4; q++) {
            const int c = cb + 32 * q;
            if (q < nqx && c < cin) {
                const uint8_t *g = sX + (((c >> 3) * 10 + jg + 1) * 128 + (c & 7) * 16);
                const uint4 v = *reinterpret_cast<const uint4 *>(g);
                const uint32_t a = x > 0 ? *reinterpret_cast<const unsigned short *>(g - 128 + 14) : 0u;
                const uint32_t b = x + 8 < W ? *reinterpret_cast<const unsigned short *>(g + 128) : 0u;
                const uint32_t off = (uint32_t)(tid + 256 * q) * 16u;
                // kx = 0: pixels x - 1 .. x + 6; kx = 2: x + 1 .. x + 8
                *reinterpret_cast<uint4 *>(sS + off) =
                    make_uint4(__byte_perm(a, v.x, 0x5410), __byte_perm(v.x, v.y, 0x5432),
                               __byte_perm(v.y, v.z, 0x5432), __byte_perm(v.z, v.w, 0x5432));
                *reinterpret_cast<uint4 *>(sS + Sh::XS_PLANE + off) =
                    make_uint4(__byte_perm(v.x, v.y, 0x5432), __byte_perm(v.y, v.z, 0x5432),
                               __byte_perm(v.z, v.w, 0x5432), __byte_perm(v.w, b, 0x5432));
            }
            if (with_bias && q < nqd && c < cout) {
                const uint4 d = *reinterpret_cast<const uint4 *>(sD + (uint32_t)(tid + 256 * q) * 16u);
                const uint32_t w[4] = {d.x, d.y, d.z, d.w};
                float t = 0.0f;
#pragma unroll
                for (int e = 0; e < 4; e++) t += __uint_as_float(w[e] << 16) + __uint_as_float(w[e] & 0xFFFF0000u);
                bsum[q] += t;
            }
        }
        tc::fence_proxy_async_smem();
        __syncthreads();
        if (abort_sh) break;
        if (tid == 0) {
            tc::fence_after_sync();
            const long left = pb - (pa + (long)i * kWgPx);
            const int ks = (int)((left < kWgPx ? left : kWgPx) / 16);   // K steps of 16 pixels
            const uint32_t d0 = sbase + (uint32_t)((i % kWgRing) * Sh::SLOT), x1 = d0 + Sh::D_BYTES + 128;
            const uint32_t s0 = sbase + kWgRing * Sh::SLOT + st * Sh::XS_BUF;
            for (int s = 0; s < ks; s++) {
                const uint64_t dd = tc::smem_desc(d0 + 256 * s, 128, 1024);
#pragma unroll
                for (int kx = 0; kx < 3; kx++) {
                    const uint64_t xd = kx == 1 ? tc::smem_desc(x1 + 256 * s, 128, Sh::X1_SBO)
                                                : tc::smem_desc(s0 + (kx >> 1) * Sh::XS_PLANE + 256 * s, 128, 1024);
                    tc::mma_bf16(tmem + (uint32_t)(kx * N), XA ? xd : dd, XA ? dd : xd, tc::IDesc<128, N>::value,
                                 (i > 0 || s > 0) ? 1u : 0u);
                }
            }
            tc::mma_commit(&mma_done[st]);
        }
        issued = i + 1;
    }
    tc::cp_async_wait<0>();
    __syncthreads();
    bool done = true;
    if (issued > 0 && !abort_sh) {
        const int last = issued - 1;
        done = tc::mbar_wait(&mma_done[last & 1], (uint32_t)((last >> 1) & 1));
    }
    if (!done) abort_sh = 1;
    __syncthreads();   // one outcome for the whole CTA (the epilogue below synchronises)
    if (abort_sh) {
        if (tid == 0) atomicExch(&g_conv_tc_error, 1);
        if (issued > 0) tc::mbar_wait(&mma_done[(issued - 1) & 1], (uint32_t)(((issued - 1) >> 1) & 1));
    } else {
        tc::fence_after_sync();
        const int wl = warp & 3, wh = warp >> 2;
        const int m = 32 * wl + lane;
        const int nb = XA ? cout : cin;   // columns of a tap that hold data
        const size_t tap = (size_t)ma * nb;
#pragma unroll 1
        for (int c0 = 16 * wh; c0 < 3 * N; c0 += 32) {
            float v[16];
            tc::tmem_ld16(tmem + ((uint32_t)(32 * wl) << 16) + (uint32_t)c0, v);
            const int k = 3 * ky + c0 / N, n0 = c0 % N;
            if (m < ma && n0 < nb) {
                float *o = part + ((size_t)z * 9 + k) * tap + (size_t)m * nb + n0;
                if (nb == N) {
#pragma unroll
                    for (int e = 0; e < 4; e++)
                        reinterpret_cast<float4 *>(o)[e] = make_float4(v[4 * e], v[4 * e + 1], v[4 * e + 2], v[4 * e + 3]);
                } else {
#pragma unroll
                    for (int e = 0; e < 16; e++)
                        if (n0 + e < nb) o[e] = v[e];
                }
            }
        }
        if (with_bias) {
            // threads with the same channels differ in the pixel group: lane bits 3-4 and the warp's parity
#pragma unroll
            for (int q = 0; q < 4; q++) {
                float t = bsum[q];
                t += __shfl_xor_sync(0xffffffffu, t, 8);
                t += __shfl_xor_sync(0xffffffffu, t, 16);
                if ((warp & 1) && lane < 8) bias_sh[warp >> 1][q][lane] = t;
                bsum[q] = t;
            }
            __syncthreads();
            if (!(warp & 1) && lane < 8)
#pragma unroll
                for (int q = 0; q < 4; q++) {
                    const int c = cb + 32 * q;
                    if (q < nqd && c < cout) part_b[(size_t)z * cout + c] = bsum[q] + bias_sh[warp >> 1][q][lane];
                }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, Sh::NCOL);
}

// dW += sum over the chunks of part (layout [z][k][m][n]), db += sum of part_b.
// A block takes 32 consecutive sums; its warp w adds chunks w, w + 8, ... in
// order, and lane i of warp 0 adds the eight warps' results in order: a fixed
// order, whatever the timing.
__global__ void __launch_bounds__(256) conv_wgrad_tc_sum_kernel(const float *__restrict__ part,
                                                                const float *__restrict__ part_b, int chunks,
                                                                float *__restrict__ dW, float *__restrict__ db, int cin,
                                                                int cout, int xa) {
    __shared__ float acc[8][32];
    const int ma = xa ? cin : cout, nb = xa ? cout : cin;
    const size_t n = (size_t)cout * cin * 9, tap = (size_t)ma * nb;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const size_t i = (size_t)blockIdx.x * 32 + lane;
    float v = 0.0f;
    if (i < n) {
        for (int z = w; z < chunks; z += 8) v += part[(size_t)z * n + i];
    } else if (i < n + cout) {
        for (int z = w; z < chunks; z += 8) v += part_b[(size_t)z * cout + (i - n)];
    }
    acc[w][lane] = v;
    __syncthreads();
    if (w != 0 || i >= n + cout) return;
    float t = acc[0][lane];
#pragma unroll
    for (int j = 1; j < 8; j++) t += acc[j][lane];
    if (i < n) {
        const int k = (int)(i / tap), m = (int)((i / nb) % ma), c = (int)(i % nb);
        const int co = xa ? c : m, ci = xa ? m : c;
        dW[((size_t)co * cin + ci) * 9 + k] += t;
    } else if (db) {
        db[i - n] += t;
    }
}

// Shape conditions of the tensor-memory weight gradient.
// Channel counts up to 128 on either side: the M side (128 rows) and the N
// side (32, 64 or 128 columns) are padded, and what the padding rows and
// columns accumulate is never stored.
bool conv3x3_wgrad_tc_ok(int cin, int cout, int H, int W) {
    return cin >= 1 && cin <= 128 && cout >= 1 && cout <= 128 && W % 16 == 0 && W >= 16 && H >= 1 &&
           (size_t)H * W <= ((size_t)1 << 31);
}

// Which side is M: X where it has all 128 rows and dY fits N = 64 (half the MMA
// work of padding dY to 128), else dY.
static bool wgrad_tc_xa(int cin, int cout) { return cin == 128 && cout <= 64; }
static int wgrad_tc_n(int c) { return c <= 32 ? 32 : c <= 64 ? 64 : 128; }

// CTAs per SM of the weight-gradient form a cin -> cout layer uses.
static int wgrad_tc_res(int cin, int cout) {
    if (wgrad_tc_xa(cin, cout)) return wgrad_tc_n(cout) == 32 ? WgShape<true, 32>::RES : WgShape<true, 64>::RES;
    const int n = wgrad_tc_n(cin);
    return n == 32 ? WgShape<false, 32>::RES : n == 64 ? WgShape<false, 64>::RES : WgShape<false, 128>::RES;
}

// Pixel chunks of the weight gradient: about 50 chunks per CTA an SM holds
// (three CTAs each, one per kernel row: 150 per wave on a 152-SM GPU), at least
// one stage each, and at most cap_floats of FP32 partial sums.  Returns the
// number of chunks, *chunk_px their size.
int conv3x3_wgrad_tc_plan(int cin, int cout, int H, int W, size_t cap_floats, int *chunk_px) {
    const long px = (long)H * W;
    const size_t per = (size_t)9 * cin * cout + cout;
    long zc = (px + kWgPx - 1) / kWgPx;
    const long target = 50L * wgrad_tc_res(cin, cout);
    if (zc > target) zc = target;
    if ((size_t)zc > cap_floats / per) zc = (long)(cap_floats / per);
    if (zc < 1) return 0;
    long ch = (px + zc - 1) / zc;
    ch = (ch + kWgPx - 1) / kWgPx * kWgPx;
    *chunk_px = (int)ch;
    return (int)((px + ch - 1) / ch);
}

template <bool XA, int N>
static int launch_wgrad_tc(const bf16 *X, const bf16 *dY, float *part, float *part_b, int cin, int cout, int H, int W,
                           int nz, int chunk_px, cudaStream_t s) {
    using Sh = WgShape<XA, N>;
    static bool attr_set[64] = {};
    int dev = 0;
    TW_CUDA(cudaGetDevice(&dev));
    if (dev >= 0 && dev < 64 && !attr_set[dev]) {
        TW_CUDA(cudaFuncSetAttribute(conv3x3_wgrad_tc_kernel<XA, N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)Sh::SMEM));
        attr_set[dev] = true;
    }
    TW_LAUNCH((conv3x3_wgrad_tc_kernel<XA, N>), dim3(3, nz), kWgThreads, Sh::SMEM, s, X, dY, part, part_b, cin, cout,
              H, W, chunk_px);
    return TW_OK;
}

// dW += dL/dW, db += dL/db (db nullable) of a 3x3 convolution from its input X
// (BF16 [cin][H][W]) and output gradient dY (BF16 [cout][H][W]) on the tensor
// cores; part: part_floats floats of scratch (16-byte aligned) for the chunks'
// partial sums.
int conv3x3_wgrad_tc(const bf16 *X, const bf16 *dY, float *dW, float *db, int cin, int cout, int H, int W,
                     float *part, size_t part_floats, cudaStream_t s) {
    if (!conv3x3_wgrad_tc_ok(cin, cout, H, W) || (((uintptr_t)X | (uintptr_t)dY) & 15)) return TW_EINVAL;
    int chunk = 0;
    const int nz = conv3x3_wgrad_tc_plan(cin, cout, H, W, part_floats, &chunk);
    if (!part || ((uintptr_t)part & 15) || nz < 1) return TW_EWORKSPACE;
    float *part_b = part + (size_t)nz * 9 * cin * cout;
    int e;
    const bool xa = wgrad_tc_xa(cin, cout);
    if (xa) {
        e = wgrad_tc_n(cout) == 32 ? launch_wgrad_tc<true, 32>(X, dY, part, part_b, cin, cout, H, W, nz, chunk, s)
                                   : launch_wgrad_tc<true, 64>(X, dY, part, part_b, cin, cout, H, W, nz, chunk, s);
    } else {
        const int n = wgrad_tc_n(cin);
        e = n == 32   ? launch_wgrad_tc<false, 32>(X, dY, part, part_b, cin, cout, H, W, nz, chunk, s)
            : n == 64 ? launch_wgrad_tc<false, 64>(X, dY, part, part_b, cin, cout, H, W, nz, chunk, s)
                      : launch_wgrad_tc<false, 128>(X, dY, part, part_b, cin, cout, H, W, nz, chunk, s);
    }
    if (e) return e;
    const size_t n = (size_t)cout * cin * 9 + cout;
    TW_LAUNCH(conv_wgrad_tc_sum_kernel, (unsigned)((n + 31) / 32), 256, 0, s, part, part_b, nz, dW, db, cin, cout,
              xa ? 1 : 0);
    return TW_OK;
}

}  // namespace nn
}  // namespace tw
