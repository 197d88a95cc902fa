// Register-blocked, temporally blocked red-black SOR tile (shared by the
// single-field and the batched sweep kernels; see hp_sweeps.cu for the design).
#pragma once
#include "hp_internal.cuh"

namespace tw {

// One Eq. 1 update's size, (1/4)((l + r) + (u + d)) - c: the SOR step before
// the factor omega, and (in magnitude) the residual of the cell.  Every kernel
// of the split layout evaluates it in this form so that their residuals agree
// bit for bit.
__device__ __forceinline__ float rb_step(float c, float l, float r, float u, float d) {
    return fmaf(0.25f, (l + r) + (u + d), -c);
}

__device__ __forceinline__ float sor1(float c, float l, float r, float u, float d, float omega) {
    return fmaf(omega, rb_step(c, l, r, u, d), c);
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

// Residual max over the masked cells of one float4 row (same neighbour
// pattern as sor_row).
template <int S>
__device__ __forceinline__ float resid_row(const float4 c, const float4 mid, const float4 up, const float4 dn,
                                           uint32_t bits, float acc) {
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
    if (bits & 1u) acc = fmaxf(acc, fabsf(rb_step(c.x, l0, r0, up.x, dn.x)));
    if (bits & 2u) acc = fmaxf(acc, fabsf(rb_step(c.y, l1, r1, up.y, dn.y)));
    if (bits & 4u) acc = fmaxf(acc, fabsf(rb_step(c.z, l2, r2, up.z, dn.z)));
    if (bits & 8u) acc = fmaxf(acc, fabsf(rb_step(c.w, l3, r3, up.w, dn.w)));
    return acc;
}

// Block-wide max of two non-negative floats, one atomicMax per CTA on each
// one's bits (out_b may be null: b is then not reduced).
__device__ __forceinline__ void block_max2_atomic(float a, unsigned int *out_a, float b, unsigned int *out_b) {
    __shared__ float sa[32], sb[32];
    a = sane(a);
    b = sane(b);
    for (int o = 16; o > 0; o >>= 1) {
        a = fmaxf(a, __shfl_xor_sync(0xffffffffu, a, o));
        b = fmaxf(b, __shfl_xor_sync(0xffffffffu, b, o));
    }
    const int t = threadIdx.y * blockDim.x + threadIdx.x;
    const int nt = blockDim.x * blockDim.y;
    if ((t & 31) == 0) {
        sa[t >> 5] = a;
        sb[t >> 5] = b;
    }
    __syncthreads();
    if (t < 32) {
        const bool in = t < (nt + 31) / 32;
        a = in ? sa[t] : 0.0f;
        b = in ? sb[t] : 0.0f;
        for (int o = 16; o > 0; o >>= 1) {
            a = fmaxf(a, __shfl_xor_sync(0xffffffffu, a, o));
            b = fmaxf(b, __shfl_xor_sync(0xffffffffu, b, o));
        }
        if (t == 0 && a > 0.0f) atomicMax(out_a, __float_as_uint(a));
        if (t == 0 && out_b && b > 0.0f) atomicMax(out_b, __float_as_uint(b));
    }
}

// One CTA (64 x 4 threads; each thread one float4 of each colour in
// kResidRows rows, strided by 4) of the FP32 residual check: atomicMax of the
// CTA's residual max into *out_max and, if l2part is given, the CTA's sum of
// squared residuals, reduced in a fixed order, into l2part[CTA index].
// snap (the snapshot state, see RelaxCtl::snap) 1: copy the planes into the
// snapshot planes L.R3/L.B3; 2: also atomicMax of the largest change of a free
// cell since the snapshot into *out_dmax.  Each thread reads and rewrites only
// the snapshot entries of its own cells.
constexpr int kResidRows = 4;
__device__ __forceinline__ void rb_residual_cta(const RBLayout &L, int ny, unsigned int *out_max, float *l2part,
                                                int snap, unsigned int *out_dmax) {
    const int k4 = blockIdx.x * blockDim.x + threadIdx.x;
    float r = 0.0f, q = 0.0f, dm = 0.0f;
#pragma unroll
    for (int i = 0; i < kResidRows; i++) {
    const int y = (blockIdx.y * kResidRows + i) * blockDim.y + threadIdx.y + 1;
    if (k4 < L.W4 && y < ny - 1) {
        const int k = 4 * k4;
#pragma unroll
        for (int color = 0; color < 2; color++) {
            const float *U = color ? L.B : L.R;
            const float *V = color ? L.R : L.B;
            const uint32_t *M = color ? L.MB : L.MR;
            const uint32_t bits = (M[(size_t)y * L.MW + (k >> 5)] >> (k & 31)) & 0xFu;
            if (!bits) continue;
            const int s = (y + color) & 1;
            float4 nb[4];
            rb_load_neighbours(V, L.S, y, k, s, nb);
            const float4 c = *reinterpret_cast<const float4 *>(U + (size_t)y * L.S + 4 + k);
            const float t0 = rb_step(c.x, nb[0].x, nb[1].x, nb[2].x, nb[3].x);
            const float t1 = rb_step(c.y, nb[0].y, nb[1].y, nb[2].y, nb[3].y);
            const float t2 = rb_step(c.z, nb[0].z, nb[1].z, nb[2].z, nb[3].z);
            const float t3 = rb_step(c.w, nb[0].w, nb[1].w, nb[2].w, nb[3].w);
            if (bits & 1u) { r = fmaxf(r, fabsf(t0)); q = fmaf(t0, t0, q); }
            if (bits & 2u) { r = fmaxf(r, fabsf(t1)); q = fmaf(t1, t1, q); }
            if (bits & 4u) { r = fmaxf(r, fabsf(t2)); q = fmaf(t2, t2, q); }
            if (bits & 8u) { r = fmaxf(r, fabsf(t3)); q = fmaf(t3, t3, q); }
            if (snap) {
                float4 *P = reinterpret_cast<float4 *>((color ? L.B3 : L.R3) + (size_t)y * L.S + 4 + k);
                if (snap == 2) {
                    const float4 p = *P;
                    if (bits & 1u) dm = fmaxf(dm, fabsf(c.x - p.x));
                    if (bits & 2u) dm = fmaxf(dm, fabsf(c.y - p.y));
                    if (bits & 4u) dm = fmaxf(dm, fabsf(c.z - p.z));
                    if (bits & 8u) dm = fmaxf(dm, fabsf(c.w - p.w));
                }
                *P = c;
            }
        }
    }
    }
    if (l2part) {   // fixed-order CTA sum: the same partials in every run
        __shared__ float sq[8];
        for (int o = 16; o > 0; o >>= 1) q += __shfl_xor_sync(0xffffffffu, q, o);
        const int t = threadIdx.y * blockDim.x + threadIdx.x;
        if ((t & 31) == 0) sq[t >> 5] = q;
        __syncthreads();
        if (t < 32) {
            float v = t < (int)((blockDim.x * blockDim.y + 31) / 32) ? sq[t] : 0.0f;
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (t == 0) l2part[blockIdx.y * gridDim.x + blockIdx.x] = v;
        }
    }
    if (snap == 2)
        block_max2_atomic(r, out_max, dm, out_dmax);
    else
        block_max_atomic(r, out_max);
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

// Free-cell bits of a thread's rows: the 4 bits of row r in byte r % 4 of
// word r / 4, so that each row's bits are one byte-aligned field.
template <int RB>
struct TBMask {
    uint32_t w[(RB + 3) / 4];
    __device__ __forceinline__ uint32_t row(int r) const { return (w[r >> 2] >> (8 * (r & 3))) & 0xFu; }
};

// Row exchange between the warps of a tile, double-buffered by colour.  top
// holds each warp's first row at index warp, bot its last row at index
// warp + 1; bot[c][0] and top[c][WARPS] stay zero, so that every warp reads
// its neighbours' rows without a branch (the rows beyond the tile are halo,
// whose values never reach the stored interior).
template <int WARPS>
struct TBShared {
    float4 top[2][WARPS + 1][32];
    float4 bot[2][WARPS + 1][32];
};

// Zero the two boundary slots; call before the first barrier of a tile.
template <int WARPS>
__device__ __forceinline__ void tb_shared_init(TBShared<WARPS> &sh) {
    const int t = threadIdx.x;
    if (t < 64) {
        const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
        sh.bot[t >> 5][0][t & 31] = z;
        sh.top[t >> 5][WARPS][t & 31] = z;
    }
}

template <int COLOR, int RB, int WARPS>
__device__ __forceinline__ void tb_half_sweep(float4 (&v)[2][RB], const TBMask<RB> &m, float4 above, float4 below,
                                              float omega) {
    constexpr int O = 1 - COLOR;
#pragma unroll
    for (int r = 0; r < RB; r++) {
        const float4 up = (r == 0) ? above : v[O][r - 1];
        const float4 dn = (r == RB - 1) ? below : v[O][r + 1];
        // rows start even, so the parity of row r for colour COLOR is (r + COLOR) & 1
        if (((r + COLOR) & 1) != 0)
            v[COLOR][r] = sor_row<1>(v[COLOR][r], v[O][r], up, dn, m.row(r), omega);
        else
            v[COLOR][r] = sor_row<0>(v[COLOR][r], v[O][r], up, dn, m.row(r), omega);
    }
}

// Load a thread's RB rows of float4 column k4 of both colours, and their
// free-cell bits.  Rows and columns outside the field read as zero with no
// free bit, so they never change.
template <int RB>
__device__ __forceinline__ void tb_load(float4 (&v)[2][RB], TBMask<RB> (&m)[2], const float *__restrict__ Rin,
                                        const float *__restrict__ Bin, const uint32_t *__restrict__ MR,
                                        const uint32_t *__restrict__ MB, int y0, int k4, bool kin, int ny, int S,
                                        int MW) {
    const int k = 4 * k4;
    // the mask words first: they are small and gate the first half-sweep, so
    // they should not queue behind the tile's field rows
    uint32_t mr[RB], mb[RB];
#pragma unroll
    for (int r = 0; r < RB; r++) {
        const int y = y0 + r;
        const bool in = kin && y >= 0 && y < ny;
        const size_t w = (size_t)(in ? y : 0) * MW + (in ? (k >> 5) : 0);
        mr[r] = in ? __ldg(MR + w) : 0u;
        mb[r] = in ? __ldg(MB + w) : 0u;
    }
#pragma unroll
    for (int r = 0; r < RB; r++) {
        const int y = y0 + r;
        const bool in = kin && y >= 0 && y < ny;
        const size_t off = (size_t)(in ? y : 0) * S + 4 + (in ? k : 0);
        v[0][r] = in ? __ldg(reinterpret_cast<const float4 *>(Rin + off)) : make_float4(0.f, 0.f, 0.f, 0.f);
        v[1][r] = in ? __ldg(reinterpret_cast<const float4 *>(Bin + off)) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int i = 0; i < (RB + 3) / 4; i++) {
        m[0].w[i] = 0u;
        m[1].w[i] = 0u;
    }
#pragma unroll
    for (int r = 0; r < RB; r++) {
        m[0].w[r >> 2] |= ((mr[r] >> (k & 31)) & 0xFu) << (8 * (r & 3));
        m[1].w[r >> 2] |= ((mb[r] >> (k & 31)) & 0xFu) << (8 * (r & 3));
    }
}

// Half-sweep of colour COLOR of the CTA's registers: first the other colour's
// first/last rows are exchanged with the warps above/below through shared
// memory (double-buffered by colour, one barrier).
template <int COLOR, int RB, int WARPS>
__device__ __forceinline__ void tb_exchange_half_sweep(float4 (&v)[2][RB], const TBMask<RB> &m, float omega,
                                                       TBShared<WARPS> &sh) {
    constexpr int O = 1 - COLOR;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    sh.top[COLOR][warp][lane] = v[O][0];
    sh.bot[COLOR][warp + 1][lane] = v[O][RB - 1];
    __syncthreads();
    tb_half_sweep<COLOR, RB, WARPS>(v, m, sh.bot[COLOR][warp][lane], sh.top[COLOR][warp + 1][lane], omega);
}

// One full red-black sweep of the CTA's registers.
template <int RB, int WARPS>
__device__ __forceinline__ void tb_full_sweep(float4 (&v)[2][RB], const TBMask<RB> (&m)[2], float omega,
                                              TBShared<WARPS> &sh) {
    tb_exchange_half_sweep<0, RB, WARPS>(v, m[0], omega, sh);
    tb_exchange_half_sweep<1, RB, WARPS>(v, m[1], omega, sh);
}

// Store colour C's rows of the tile interior [y_tile, y_tile + YI) held by the thread.
template <int C, int RB>
__device__ __forceinline__ void tb_store_colour(const float4 (&v)[2][RB], float *__restrict__ P, int y0, int y_tile,
                                                int YI, int k4, bool lane_int, int ny, int S) {
    if (!lane_int) return;
#pragma unroll
    for (int r = 0; r < RB; r++) {
        const int y = y0 + r;
        if (y >= y_tile && y < y_tile + YI && y < ny)
            *reinterpret_cast<float4 *>(P + (size_t)y * S + 4 + 4 * k4) = v[C][r];
    }
}

// Store the rows of the tile interior [y_tile, y_tile + YI) held by the thread.
template <int RB>
__device__ __forceinline__ void tb_store(const float4 (&v)[2][RB], float *__restrict__ Rout,
                                         float *__restrict__ Bout, int y0, int y_tile, int YI, int k4,
                                         bool lane_int, int ny, int S) {
    tb_store_colour<0, RB>(v, Rout, y0, y_tile, YI, k4, lane_int, ny, S);
    tb_store_colour<1, RB>(v, Bout, y0, y_tile, YI, k4, lane_int, ny, S);
}

// One tile of the T-fused sweep: tile (bx, by) of a colour-split field.
// Shared by the single-field kernel and the batched persistent kernel.
template <int T, int RB, int WARPS>
__device__ __forceinline__ void tb_tile(const float *__restrict__ Rin, const float *__restrict__ Bin,
                                        float *__restrict__ Rout, float *__restrict__ Bout,
                                        const uint32_t *__restrict__ MR, const uint32_t *__restrict__ MB, int ny,
                                        int W4, int S, int MW, float omega, int bx, int by, TBShared<WARPS> &sh) {
    using Sh = TBShape<T, RB, WARPS>;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int k4 = bx * Sh::KI4 - Sh::HK4 + lane;
    const int y_tile = by * Sh::YI;
    const int y0 = y_tile - Sh::HY + warp * RB;   // even
    const bool kin = (k4 >= 0) && (k4 < W4);

    float4 v[2][RB];
    TBMask<RB> m[2];
    tb_shared_init<WARPS>(sh);
    tb_load<RB>(v, m, Rin, Bin, MR, MB, y0, k4, kin, ny, S, MW);
#pragma unroll 1
    for (int p = 0; p < T; p++) tb_full_sweep<RB, WARPS>(v, m, omega, sh);
    tb_store<RB>(v, Rout, Bout, y0, y_tile, Sh::YI, k4, kin && lane >= Sh::HK4 && lane < 32 - Sh::HK4, ny, S);
}

}  // namespace tw
