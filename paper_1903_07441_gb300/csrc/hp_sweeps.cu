// Red-black SOR sweeps on the colour-split layout.
//
// rb_sweeps(n, T): n full sweeps (red half-sweep, then black half-sweep).
//  * T == 1: one global-memory half-sweep per launch (rb_half_sweep_kernel),
//    4 cells per thread with 128-bit loads.  Kept as the unfused form.
//  * T >= 2: rb_tb_kernel fuses T full sweeps (2T half-sweeps) per launch.
// Both evaluate the SOR update in the same order,
//     t = fma(1/4, (l + r) + (u + d), -c),   c' = fma(omega, t, c),
// so the fused and unfused forms give identical results.
//
// rb_tb_kernel: register-blocked temporal blocking.  A CTA owns a tile of
// 32 float4 columns (128 entries of each colour = 256 cells) x WARPS*RB rows,
// halo included.  Lane l of warp w holds, in registers, RB consecutive rows
// of float4 column l for BOTH colours.  A half-sweep then needs:
//   * up/down neighbours: in the thread's own registers, except for its first
//     and last row, which come from the warps above/below through a small
//     double-buffered shared-memory exchange (one barrier per half-sweep);
//   * left/right neighbours: the same float4 plus one value of the adjacent
//     lane (one warp shuffle per row).  Every thread's first row is even (tile
//     origins, halos and RB are even), so which side the extra value comes
//     from is known at compile time for every unrolled row.
// Each cell is read from global memory once and written once per launch: the
// algorithmic traffic of a launch is one read + one write of the field plus
// the 1-bit mask, for T sweeps.  Halo cells are recomputed redundantly
// (garbage from the tile edge advances one cell per half-sweep and never
// reaches the interior that is stored).
#include "common.cuh"
#include "hp_internal.cuh"

namespace tw {

__device__ __forceinline__ float sor1(float c, float l, float r, float u, float d, float omega) {
    const float t = fmaf(0.25f, (l + r) + (u + d), -c);
    return fmaf(omega, t, c);
}

// One half-sweep of colour COLOR, global memory, 4 cells per thread (float4).
template <int COLOR>
__global__ void __launch_bounds__(256) rb_half_sweep_kernel(RBLayout L, int ny, float omega) {
    int k4 = blockIdx.x * blockDim.x + threadIdx.x;
    int y = blockIdx.y * blockDim.y + threadIdx.y + 1;
    if (k4 >= L.W4 || y >= ny - 1) return;
    float *U = COLOR ? L.B : L.R;
    const float *V = COLOR ? L.R : L.B;
    const uint32_t *M = COLOR ? L.MB : L.MR;
    int k = 4 * k4;
    uint32_t bits = (M[(size_t)y * L.MW + (k >> 5)] >> (k & 31)) & 0xFu;
    if (!bits) return;
    int s = (y + COLOR) & 1;
    float4 nb[4];
    rb_load_neighbours(V, L.S, y, k, s, nb);
    float4 *up = reinterpret_cast<float4 *>(U + (size_t)y * L.S + 4 + k);
    float4 c = *up;
    c.x = (bits & 1u) ? sor1(c.x, nb[0].x, nb[1].x, nb[2].x, nb[3].x, omega) : c.x;
    c.y = (bits & 2u) ? sor1(c.y, nb[0].y, nb[1].y, nb[2].y, nb[3].y, omega) : c.y;
    c.z = (bits & 4u) ? sor1(c.z, nb[0].z, nb[1].z, nb[2].z, nb[3].z, omega) : c.z;
    c.w = (bits & 8u) ? sor1(c.w, nb[0].w, nb[1].w, nb[2].w, nb[3].w, omega) : c.w;
    *up = c;
}

int rb_sweeps_simple(RBLayout &L, int ny, int n, float omega, cudaStream_t s, int *launches) {
    dim3 b(64, 4), gr(ceil_div(L.W4, 64), ceil_div(ny - 2, 4));
    for (int i = 0; i < n; i++) {
        TW_LAUNCH((rb_half_sweep_kernel<0>), gr, b, 0, s, L, ny, omega);
        TW_LAUNCH((rb_half_sweep_kernel<1>), gr, b, 0, s, L, ny, omega);
    }
    TW_CHECK_LAUNCH();
    *launches += 2 * n;
    return TW_OK;
}

// SOR update of one float4 row; S = parity of the row for the colour updated
// (1: neighbours k..k+4, extra value from the next lane; 0: k-1..k+3, from the
// previous lane).
template <int S>
__device__ __forceinline__ float4 sor_row(float4 c, const float4 mid, const float4 up, const float4 dn,
                                          uint32_t bits, float omega) {
    float l0, l1, l2, l3, r0, r1, r2, r3;
    if (S) {
        const float ex = __shfl_down_sync(0xffffffffu, mid.x, 1);
        l0 = mid.x; l1 = mid.y; l2 = mid.z; l3 = mid.w;
        r0 = mid.y; r1 = mid.z; r2 = mid.w; r3 = ex;
    } else {
        const float ex = __shfl_up_sync(0xffffffffu, mid.w, 1);
        l0 = ex; l1 = mid.x; l2 = mid.y; l3 = mid.z;
        r0 = mid.x; r1 = mid.y; r2 = mid.z; r3 = mid.w;
    }
    const float n0 = sor1(c.x, l0, r0, up.x, dn.x, omega);
    const float n1 = sor1(c.y, l1, r1, up.y, dn.y, omega);
    const float n2 = sor1(c.z, l2, r2, up.z, dn.z, omega);
    const float n3 = sor1(c.w, l3, r3, up.w, dn.w, omega);
    c.x = (bits & 1u) ? n0 : c.x;
    c.y = (bits & 2u) ? n1 : c.y;
    c.z = (bits & 4u) ? n2 : c.z;
    c.w = (bits & 8u) ? n3 : c.w;
    return c;
}

template <int T, int RB, int WARPS>
struct TBShape {
    static constexpr int HK4 = (T + 1 + 3) / 4;       // halo, float4 columns per side
    static constexpr int HY = 2 * T;                   // halo rows per side
    static constexpr int KI4 = 32 - 2 * HK4;           // interior float4 columns
    static constexpr int YT = WARPS * RB;              // rows per tile (with halo)
    static constexpr int YI = YT - 2 * HY;             // interior rows
    static_assert(KI4 > 0 && YI > 0, "tile too small for the blocking depth");
    static_assert(YI % 2 == 0 && HY % 2 == 0 && RB % 2 == 0, "thread rows must start on even rows");
};

template <int COLOR, int RB, int WARPS>
__device__ __forceinline__ void tb_half_sweep(float4 (&v)[2][RB], const uint32_t m, float4 above, float4 below,
                                              float omega) {
    constexpr int O = 1 - COLOR;
#pragma unroll
    for (int r = 0; r < RB; r++) {
        const float4 up = (r == 0) ? above : v[O][r - 1];
        const float4 dn = (r == RB - 1) ? below : v[O][r + 1];
        // rows start even, so the parity of row r for colour COLOR is (r + COLOR) & 1
        if (((r + COLOR) & 1) != 0)
            v[COLOR][r] = sor_row<1>(v[COLOR][r], v[O][r], up, dn, (m >> (4 * r)) & 0xFu, omega);
        else
            v[COLOR][r] = sor_row<0>(v[COLOR][r], v[O][r], up, dn, (m >> (4 * r)) & 0xFu, omega);
    }
}

template <int T, int RB, int WARPS, int MINB>
__global__ void __launch_bounds__(WARPS * 32, MINB)
rb_tb_kernel(const float *__restrict__ Rin, const float *__restrict__ Bin, float *__restrict__ Rout,
             float *__restrict__ Bout, const uint32_t *__restrict__ MR, const uint32_t *__restrict__ MB,
             int ny, int W4, int S, int MW, float omega_arg, const float *__restrict__ omega_dev) {
    using Sh = TBShape<T, RB, WARPS>;
    // the graph-driven loop keeps omega in device memory (it adapts on the device)
    const float omega = omega_dev ? *omega_dev : omega_arg;
    __shared__ float4 s_top[2][WARPS][32];
    __shared__ float4 s_bot[2][WARPS][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int k4 = (int)blockIdx.x * Sh::KI4 - Sh::HK4 + lane;
    const int y_tile = (int)blockIdx.y * Sh::YI;
    const int y0 = y_tile - Sh::HY + warp * RB;   // even
    const bool kin = (k4 >= 0) && (k4 < W4);
    const int k = 4 * k4;

    float4 v[2][RB];
    uint32_t m[2] = {0u, 0u};  // bit 4*r + e: cell e of row r is free
#pragma unroll
    for (int r = 0; r < RB; r++) {
        const int y = y0 + r;
        const bool in = kin && y >= 0 && y < ny;
        const size_t off = (size_t)(in ? y : 0) * S + 4 + (in ? k : 0);
        v[0][r] = in ? __ldg(reinterpret_cast<const float4 *>(Rin + off)) : make_float4(0.f, 0.f, 0.f, 0.f);
        v[1][r] = in ? __ldg(reinterpret_cast<const float4 *>(Bin + off)) : make_float4(0.f, 0.f, 0.f, 0.f);
        if (in) {
            const size_t w = (size_t)y * MW + (k >> 5);
            m[0] |= ((__ldg(MR + w) >> (k & 31)) & 0xFu) << (4 * r);
            m[1] |= ((__ldg(MB + w) >> (k & 31)) & 0xFu) << (4 * r);
        }
    }
    const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);

#pragma unroll 1
    for (int p = 0; p < T; p++) {
        // red half-sweep: exchange black's first/last rows with the warps above/below
        s_top[0][warp][lane] = v[1][0];
        s_bot[0][warp][lane] = v[1][RB - 1];
        __syncthreads();
        tb_half_sweep<0, RB, WARPS>(v, m[0], warp > 0 ? s_bot[0][warp - 1][lane] : zero,
                                    warp < WARPS - 1 ? s_top[0][warp + 1][lane] : zero, omega);
        // black half-sweep: exchange red's first/last rows
        s_top[1][warp][lane] = v[0][0];
        s_bot[1][warp][lane] = v[0][RB - 1];
        __syncthreads();
        tb_half_sweep<1, RB, WARPS>(v, m[1], warp > 0 ? s_bot[1][warp - 1][lane] : zero,
                                    warp < WARPS - 1 ? s_top[1][warp + 1][lane] : zero, omega);
    }

    // store the interior
    const bool kint = lane >= Sh::HK4 && lane < 32 - Sh::HK4 && kin;
    if (kint) {
#pragma unroll
        for (int r = 0; r < RB; r++) {
            const int y = y0 + r;
            if (y >= y_tile && y < y_tile + Sh::YI && y < ny) {
                const size_t off = (size_t)y * S + 4 + k;
                *reinterpret_cast<float4 *>(Rout + off) = v[0][r];
                *reinterpret_cast<float4 *>(Bout + off) = v[1][r];
            }
        }
    }
}

constexpr int kTBRows = 8;    // rows per thread
constexpr int kTBWarps = 8;   // warps per CTA
constexpr int kTBMinBlocks = 1;

template <int T>
static void launch_tb(RBLayout &L, int ny, float omega, cudaStream_t s) {
    using Sh = TBShape<T, kTBRows, kTBWarps>;
    dim3 grid(ceil_div(L.W4, Sh::KI4), ceil_div(ny, Sh::YI));
    TW_LAUNCH((rb_tb_kernel<T, kTBRows, kTBWarps, kTBMinBlocks>), grid, kTBWarps * 32, 0, s, L.R, L.B, L.R2,
              L.B2, L.MR, L.MB, ny, L.W4, L.S, L.MW, omega, (const float *)nullptr);
    float *t = L.R; L.R = L.R2; L.R2 = t;
    t = L.B; L.B = L.B2; L.B2 = t;
}

int rb_sweeps(RBLayout &L, int nx, int ny, int n, int T, float omega, cudaStream_t s, int *launches) {
    (void)nx;
    if (T <= 1 || !L.R2) return rb_sweeps_simple(L, ny, n, omega, s, launches);
    if (T > 4) T = 4;
    int left = n;
    while (left > 0) {
        int t = left >= T ? T : left;
        if (t == 4) launch_tb<4>(L, ny, omega, s);
        else if (t == 3) launch_tb<3>(L, ny, omega, s);
        else if (t == 2) launch_tb<2>(L, ny, omega, s);
        else launch_tb<1>(L, ny, omega, s);
        left -= t;
        (*launches)++;
    }
    TW_CHECK_LAUNCH();
    return TW_OK;
}

// Kernel entry and launch shape of the T-fused sweep, for graph construction.
void tb_kernel_node(int T, RBLayout &L, int ny, void **func, dim3 *grid, dim3 *block) {
    switch (T) {
        case 4: { using Sh = TBShape<4, kTBRows, kTBWarps>;
                  *func = (void *)rb_tb_kernel<4, kTBRows, kTBWarps, kTBMinBlocks>;
                  *grid = dim3(ceil_div(L.W4, Sh::KI4), ceil_div(ny, Sh::YI)); break; }
        case 3: { using Sh = TBShape<3, kTBRows, kTBWarps>;
                  *func = (void *)rb_tb_kernel<3, kTBRows, kTBWarps, kTBMinBlocks>;
                  *grid = dim3(ceil_div(L.W4, Sh::KI4), ceil_div(ny, Sh::YI)); break; }
        default: { using Sh = TBShape<2, kTBRows, kTBWarps>;
                   *func = (void *)rb_tb_kernel<2, kTBRows, kTBWarps, kTBMinBlocks>;
                   *grid = dim3(ceil_div(L.W4, Sh::KI4), ceil_div(ny, Sh::YI)); break; }
    }
    *block = dim3(kTBWarps * 32);
}

}  // namespace tw
