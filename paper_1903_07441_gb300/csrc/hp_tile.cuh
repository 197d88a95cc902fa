// Register-blocked, temporally blocked red-black SOR tile (shared by the
// single-field and the batched sweep kernels; see hp_sweeps.cu for the design).
#pragma once
#include "hp_internal.cuh"

namespace tw {

__device__ __forceinline__ float sor1(float c, float l, float r, float u, float d, float omega) {
    const float t = fmaf(0.25f, (l + r) + (u + d), -c);
    return fmaf(omega, t, c);
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

// One tile of the T-fused sweep: tile (bx, by) of a colour-split field.
// Shared by the single-field kernel and the batched persistent kernel.
template <int T, int RB, int WARPS>
__device__ __forceinline__ void tb_tile(const float *__restrict__ Rin, const float *__restrict__ Bin,
                                        float *__restrict__ Rout, float *__restrict__ Bout,
                                        const uint32_t *__restrict__ MR, const uint32_t *__restrict__ MB, int ny,
                                        int W4, int S, int MW, float omega, int bx, int by,
                                        float4 (&s_top)[2][WARPS][32], float4 (&s_bot)[2][WARPS][32]) {
    using Sh = TBShape<T, RB, WARPS>;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int k4 = bx * Sh::KI4 - Sh::HK4 + lane;
    const int y_tile = by * Sh::YI;
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

}  // namespace tw
