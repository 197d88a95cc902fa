// Red-black SOR sweeps on the colour-split layout.
//
// rb_sweeps(n, T): n full sweeps (red half-sweep, then black half-sweep).
//  * T == 1: one global-memory half-sweep per launch (rb_half_sweep_kernel),
//    4 cells per thread with 128-bit loads.  Kept as the unfused form.
//  * T >= 2: rb_tb_kernel fuses T full sweeps (2T half-sweeps) per launch.
//
// rb_tb_kernel: register-blocked temporal blocking.  A CTA owns a tile of
// 32 float4 columns (128 entries of each colour = 256 cells) x WARPS*RB rows,
// halo included.  Lane l of warp w holds, in registers, RB consecutive rows
// of float4 column l for BOTH colours.  A half-sweep then needs:
//   * up/down neighbours: in the thread's own registers, except for its first
//     and last row, which come from the warps above/below through a small
//     double-buffered shared-memory exchange (one barrier per half-sweep);
//   * left/right neighbours: the same float4 plus one value of the adjacent
//     lane (one warp shuffle per row; the direction depends on the row parity).
// Each cell is read from global memory once and written once per launch: the
// algorithmic traffic of a launch is one read + one write of the field plus
// the 1-bit mask, for T sweeps.  Halo cells are recomputed redundantly
// (garbage from the tile edge advances one cell per half-sweep and never
// reaches the interior that is stored).
#include "common.cuh"
#include "hp_internal.cuh"

namespace tw {

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
    c.x = (bits & 1u) ? fmaf(omega, rb_avg(nb, 0) - c.x, c.x) : c.x;
    c.y = (bits & 2u) ? fmaf(omega, rb_avg(nb, 1) - c.y, c.y) : c.y;
    c.z = (bits & 4u) ? fmaf(omega, rb_avg(nb, 2) - c.z, c.z) : c.z;
    c.w = (bits & 8u) ? fmaf(omega, rb_avg(nb, 3) - c.w, c.w) : c.w;
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

__device__ __forceinline__ float4 sor4(float4 c, const float4 &l, const float4 &r, const float4 &u,
                                       const float4 &d, uint32_t bits, float omega) {
    float ax = 0.25f * ((l.x + r.x) + (u.x + d.x));
    float ay = 0.25f * ((l.y + r.y) + (u.y + d.y));
    float az = 0.25f * ((l.z + r.z) + (u.z + d.z));
    float aw = 0.25f * ((l.w + r.w) + (u.w + d.w));
    c.x = (bits & 1u) ? fmaf(omega, ax - c.x, c.x) : c.x;
    c.y = (bits & 2u) ? fmaf(omega, ay - c.y, c.y) : c.y;
    c.z = (bits & 4u) ? fmaf(omega, az - c.z, c.z) : c.z;
    c.w = (bits & 8u) ? fmaf(omega, aw - c.w, c.w) : c.w;
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
};

template <int T, int RB, int WARPS>
__global__ void __launch_bounds__(WARPS * 32)
rb_tb_kernel(const float *__restrict__ Rin, const float *__restrict__ Bin, float *__restrict__ Rout,
             float *__restrict__ Bout, const uint32_t *__restrict__ MR, const uint32_t *__restrict__ MB,
             int ny, int W4, int S, int MW, float omega) {
    using Sh = TBShape<T, RB, WARPS>;
    __shared__ float4 s_top[2][WARPS][32];
    __shared__ float4 s_bot[2][WARPS][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int k4 = (int)blockIdx.x * Sh::KI4 - Sh::HK4 + lane;
    const int y_tile = (int)blockIdx.y * Sh::YI;
    const int y0 = y_tile - Sh::HY + warp * RB;
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

#pragma unroll 1
    for (int p = 0; p < 2 * T; p++) {
        const int c = p & 1;      // colour updated in this half-sweep (red first)
        const int buf = p & 1;
        // publish the other colour's first and last rows for the warps above/below
        s_top[buf][warp][lane] = c ? v[0][0] : v[1][0];
        s_bot[buf][warp][lane] = c ? v[0][RB - 1] : v[1][RB - 1];
        __syncthreads();
        const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 above = warp > 0 ? s_bot[buf][warp - 1][lane] : zero;
        const float4 below = warp < WARPS - 1 ? s_top[buf][warp + 1][lane] : zero;
        if (c == 0) {
#pragma unroll
            for (int r = 0; r < RB; r++) {
                const int s = (y0 + r) & 1;
                const float4 mid = v[1][r];
                const float4 up = (r == 0) ? above : v[1][r - 1];
                const float4 dn = (r == RB - 1) ? below : v[1][r + 1];
                float4 lft, rgt;
                if (s) {
                    const float ex = __shfl_down_sync(0xffffffffu, mid.x, 1);
                    lft = mid;
                    rgt = make_float4(mid.y, mid.z, mid.w, ex);
                } else {
                    const float ex = __shfl_up_sync(0xffffffffu, mid.w, 1);
                    lft = make_float4(ex, mid.x, mid.y, mid.z);
                    rgt = mid;
                }
                v[0][r] = sor4(v[0][r], lft, rgt, up, dn, (m[0] >> (4 * r)) & 0xFu, omega);
            }
        } else {
#pragma unroll
            for (int r = 0; r < RB; r++) {
                const int s = (y0 + r + 1) & 1;
                const float4 mid = v[0][r];
                const float4 up = (r == 0) ? above : v[0][r - 1];
                const float4 dn = (r == RB - 1) ? below : v[0][r + 1];
                float4 lft, rgt;
                if (s) {
                    const float ex = __shfl_down_sync(0xffffffffu, mid.x, 1);
                    lft = mid;
                    rgt = make_float4(mid.y, mid.z, mid.w, ex);
                } else {
                    const float ex = __shfl_up_sync(0xffffffffu, mid.w, 1);
                    lft = make_float4(ex, mid.x, mid.y, mid.z);
                    rgt = mid;
                }
                v[1][r] = sor4(v[1][r], lft, rgt, up, dn, (m[1] >> (4 * r)) & 0xFu, omega);
            }
        }
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

template <int T>
static void launch_tb(RBLayout &L, int ny, float omega, cudaStream_t s) {
    using Sh = TBShape<T, kTBRows, kTBWarps>;
    dim3 grid(ceil_div(L.W4, Sh::KI4), ceil_div(ny, Sh::YI));
    TW_LAUNCH((rb_tb_kernel<T, kTBRows, kTBWarps>), grid, kTBWarps * 32, 0, s, L.R, L.B, L.R2, L.B2, L.MR,
              L.MB, ny, L.W4, L.S, L.MW, omega);
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

}  // namespace tw
