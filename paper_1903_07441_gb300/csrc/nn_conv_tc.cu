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
// (warp w owns TMEM lanes 32w .. 32w + 31, i.e. pixels), adds bias and skip,
// applies ReLU and stores BF16 in the network's [cout][H][W] layout.
//
// Every wait is bounded (one second of %globaltimer); a timeout sets
// g_conv_tc_error, skips the remaining work, waits (bounded) for the MMAs
// already issued and frees the TMEM before returning.
#include <cuda_bf16.h>
#include <stdint.h>

#include "common.cuh"

namespace tw {
namespace nn {

typedef __nv_bfloat16 bf16;

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
// cout == N; 128 threads; grid (W / 128, H / MT).
template <int N, int MT>
__global__ void __launch_bounds__(128) conv3x3_tc_kernel(const bf16 *__restrict__ X, const uint4 *__restrict__ Wb,
                                                         const float *__restrict__ b, const bf16 *__restrict__ S,
                                                         bf16 *__restrict__ Y, int cin, int H, int W, int relu) {
    using Sh = TcShape<N, MT>;
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ uint64_t bars[2];
    __shared__ uint32_t tmem_base_sh;
    __shared__ int abort_sh;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int x0 = blockIdx.x * 128, y0 = blockIdx.y * MT;
    const int chunks = cin / 16;
    const size_t plane = (size_t)H * W;

    if (warp == 0) tc::tmem_alloc(&tmem_base_sh, Sh::NCOL);
    if (tid == 0) {
        tc::mbar_init(&bars[0], 1);
        tc::mbar_init(&bars[1], 1);
        tc::fence_mbar_init();
        abort_sh = 0;
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tmem_base_sh;
    const uint32_t sbase = tc::smem_u32(smem);
    int issued = 0;   // chunks whose MMAs were issued (thread 0's view; uniform through the barriers)

    for (int i = 0; i < chunks; i++) {
        const int st = i & 1;
        // the stage's previous chunk (i - 2) must have been consumed by its MMAs
        if (i >= 2 && !tc::mbar_wait(&bars[st], (uint32_t)(((i >> 1) - 1) & 1))) abort_sh = 1;
        uint8_t *sA = smem + st * Sh::STAGE;
        uint8_t *sB = sA + Sh::A_BYTES;
        // A: channel-last copy of 16 channels x ROWS rows x 130 pixels (zero outside the image)
        const int ci0 = 16 * i;
        for (int it = tid; it < 2 * Sh::ROWS * Sh::PX; it += 128) {
            const int h = it / (Sh::ROWS * Sh::PX), rem = it - h * (Sh::ROWS * Sh::PX);
            const int r = rem / Sh::PX, p = rem - r * Sh::PX;
            const int y = y0 - 1 + r, x = x0 - 1 + p;
            uint32_t w[4] = {0u, 0u, 0u, 0u};
            if (y >= 0 && y < H && x >= 0 && x < W) {
                const unsigned short *src =
                    reinterpret_cast<const unsigned short *>(X) + (size_t)(ci0 + 8 * h) * plane + (size_t)y * W + x;
#pragma unroll
                for (int c = 0; c < 8; c += 2)
                    w[c >> 1] = (uint32_t)__ldg(src + (size_t)c * plane) |
                                ((uint32_t)__ldg(src + (size_t)(c + 1) * plane) << 16);
            }
            *reinterpret_cast<uint4 *>(sA + h * Sh::A_HALF + (r * Sh::PX + p) * 16) = make_uint4(w[0], w[1], w[2], w[3]);
        }
        // B: the chunk's pre-arranged weights, a contiguous copy
        const uint4 *wsrc = Wb + (size_t)i * (Sh::B_BYTES / 16);
        for (int it = tid; it < (int)(Sh::B_BYTES / 16); it += 128) reinterpret_cast<uint4 *>(sB)[it] = __ldg(wsrc + it);
        tc::fence_proxy_async_smem();
        __syncthreads();
        if (abort_sh) break;
        if (tid == 0) {
            tc::fence_after_sync();
            const uint32_t a0 = sbase + st * Sh::STAGE, b0 = a0 + Sh::A_BYTES;
#pragma unroll 1
            for (int t = 0; t < MT; t++) {
#pragma unroll
                for (int k = 0; k < 9; k++) {
                    const int dy = k / 3, dx = k - 3 * (k / 3);
                    const uint64_t ad = tc::smem_desc(a0 + ((t + dy) * Sh::PX + dx) * 16, Sh::A_HALF, 128);
                    const uint64_t bd = tc::smem_desc(b0 + k * Sh::B_TAP, N * 16, 128);
                    tc::mma_bf16(tmem + (uint32_t)(t * N), ad, bd, tc::IDesc<128, N>::value, (i > 0 || k > 0) ? 1u : 0u);
                }
            }
            tc::mma_commit(&bars[st]);
        }
        issued = i + 1;
    }
    // the last issued chunk's commit covers every MMA issued before it
    bool done = true;
    if (issued > 0) {
        const int last = issued - 1;
        done = tc::mbar_wait(&bars[last & 1], (uint32_t)((last >> 1) & 1));
    }
    if (!done || abort_sh) {
        if (tid == 0) atomicExch(&g_conv_tc_error, 1);
    } else {
        tc::fence_after_sync();
        const int x = x0 + 32 * warp + lane;
#pragma unroll 1
        for (int t = 0; t < MT; t++) {
            const int y = y0 + t;
#pragma unroll 1
            for (int c0 = 0; c0 < N; c0 += 16) {
                float v[16];
                tc::tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(t * N + c0), v);
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

template <int N>
static int launch_tc(const bf16 *X, const bf16 *Wb, const float *b, const bf16 *S, bf16 *Y, int cin, int H, int W,
                     int relu, cudaStream_t s) {
    constexpr int MT = 2;
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
    TW_LAUNCH((conv3x3_tc_kernel<N, MT>), grid, 128, Sh::SMEM, s, X, reinterpret_cast<const uint4 *>(Wb), b, S, Y,
              cin, H, W, relu);
    return TW_OK;
}

// Shape conditions of the tensor-memory convolution.
bool conv3x3_tc_ok(int cin, int cout, int H, int W) {
    return cin % 16 == 0 && cin >= 16 && (cout == 32 || cout == 64 || cout == 128) && W % 128 == 0 && H % 2 == 0;
}

// Bytes of BF16 scratch for the re-arranged weights of a cin -> cout layer.
size_t conv3x3_tc_scratch_bytes(int cin, int cout) { return (size_t)cin * cout * 9 * sizeof(bf16); }

// Y = act(conv3x3(X, Wt) + b + S) on the tensor cores; scratch holds
// conv3x3_tc_scratch_bytes(cin, cout) bytes (16-byte aligned).
int conv3x3_tc(const bf16 *X, const float *Wt, const float *b, const bf16 *S, bf16 *Y, int cin, int cout, int H,
               int W, int relu, void *scratch, cudaStream_t s) {
    if (!conv3x3_tc_ok(cin, cout, H, W) || !scratch || ((uintptr_t)scratch & 15)) return TW_EINVAL;
    bf16 *Wb = (bf16 *)scratch;
    const size_t n = (size_t)cin * cout * 9;
    TW_LAUNCH(conv_tc_weights_kernel, (unsigned)((n + 255) / 256 > 1024 ? 1024 : (n + 255) / 256), 256, 0, s, Wt, Wb,
              cin, cout);
    switch (cout) {
        case 32: return launch_tc<32>(X, Wb, b, S, Y, cin, H, W, relu, s);
        case 64: return launch_tc<64>(X, Wb, b, S, Y, cin, H, W, relu, s);
        default: return launch_tc<128>(X, Wb, b, S, Y, cin, H, W, relu, s);
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

}  // namespace nn
}  // namespace tw
