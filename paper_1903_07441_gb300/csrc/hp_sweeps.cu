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
#include <string.h>

#include <mutex>
#include <vector>

#include "common.cuh"
#include "hp_internal.cuh"
#include "hp_tile.cuh"

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

template <int T, int RB, int WARPS, int MINB>
__global__ void __launch_bounds__(WARPS * 32, MINB)
rb_tb_kernel(const float *__restrict__ Rin, const float *__restrict__ Bin, float *__restrict__ Rout,
             float *__restrict__ Bout, const uint32_t *__restrict__ MR, const uint32_t *__restrict__ MB,
             int ny, int W4, int S, int MW, float omega_arg, const float *__restrict__ omega_dev) {
    __shared__ TBShared<WARPS> sh;
    // Programmatic dependent launch: consecutive sweep launches are chained so
    // that the next launch is scheduled while this one runs; each waits here for
    // the grid it depends on to complete (and its writes to be visible) before
    // touching memory.  Without such a dependency both instructions are no-ops.
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    // the graph-driven loop keeps omega in device memory (it adapts on the device)
    const float omega = omega_dev ? *omega_dev : omega_arg;
    tb_tile<T, RB, WARPS>(Rin, Bin, Rout, Bout, MR, MB, ny, W4, S, MW, omega, (int)blockIdx.x, (int)blockIdx.y, sh);
}

// Tile shape per blocking depth.  T <= 4: 8 rows x 8 warps (256 x 64 cells
// with halo, two CTAs per SM).  5 <= T <= 7: 14 rows x 12 warps (256 x 168
// cells, one CTA per SM, up to 168 registers a thread): the column halo is two
// float4 for every T in 4..7 (T + 1 <= 8 entries) and the taller tile keeps
// the row halo (2T per side) to 1.2x, so a 2048 x 2048 field is 10 x 15 = 150
// tiles -- one wave on 152 SMs -- and each launch carries 7 sweeps.
template <int T>
struct TBCfg {
    static constexpr int RB = T <= 4 ? 8 : 14;
    static constexpr int WARPS = T <= 4 ? 8 : 12;
    static constexpr int MINB = T <= 4 ? 2 : 1;   // CTAs per SM the register budget must allow
    using Sh = TBShape<T, RB, WARPS>;
};

// Launched with programmatic stream serialisation: back-to-back sweep launches
// overlap the next launch's scheduling with the current one's run (the kernel
// waits for its predecessor before its first memory access).
template <int T>
static void launch_tb(RBLayout &L, int ny, float omega, const float *omega_dev, cudaStream_t s) {
    using C = TBCfg<T>;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(ceil_div(L.W4, C::Sh::KI4), ceil_div(ny, C::Sh::YI));
    cfg.blockDim = dim3(C::WARPS * 32);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, rb_tb_kernel<T, C::RB, C::WARPS, C::MINB>, (const float *)L.R, (const float *)L.B,
                       L.R2, L.B2, (const uint32_t *)L.MR, (const uint32_t *)L.MB, ny, L.W4, L.S, L.MW, omega,
                       omega_dev);
    count_launches(1);
    float *t = L.R; L.R = L.R2; L.R2 = t;
    t = L.B; L.B = L.B2; L.B2 = t;
}

int rb_sweeps(RBLayout &L, int nx, int ny, int n, int T, float omega, cudaStream_t s, int *launches,
              const float *omega_dev) {
    (void)nx;
    if (T <= 1 || !L.R2) return rb_sweeps_simple(L, ny, n, omega, s, launches);
    if (T > kMaxTBlock) T = kMaxTBlock;
    int left = n;
    while (left > 0) {
        int t = left >= T ? T : left;
        switch (t) {
            case 7: launch_tb<7>(L, ny, omega, omega_dev, s); break;
            case 6: launch_tb<6>(L, ny, omega, omega_dev, s); break;
            case 5: launch_tb<5>(L, ny, omega, omega_dev, s); break;
            case 4: launch_tb<4>(L, ny, omega, omega_dev, s); break;
            case 3: launch_tb<3>(L, ny, omega, omega_dev, s); break;
            case 2: launch_tb<2>(L, ny, omega, omega_dev, s); break;
            default: launch_tb<1>(L, ny, omega, omega_dev, s); break;
        }
        left -= t;
        (*launches)++;
    }
    TW_CHECK_LAUNCH();
    return TW_OK;
}

struct SweepGraph {
    int dev, ny, n, T, W4, S, MW;
    const void *key[7];
    cudaGraphExec_t exec;
    int launches;
    bool swap;
};
static std::mutex g_sweep_graph_mutex;
static std::vector<SweepGraph> g_sweep_graphs;

int rb_sweeps_graph(RBLayout &L, int nx, int ny, int n, int T, const float *omega_dev, cudaStream_t s,
                    int *launches) {
    int dev = 0;
    TW_CUDA(cudaGetDevice(&dev));
    const void *key[7] = {L.R, L.B, L.R2, L.B2, L.MR, L.MB, omega_dev};   // with the row geometry below
    std::lock_guard<std::mutex> lock(g_sweep_graph_mutex);
    SweepGraph *ent = nullptr;
    for (auto &g : g_sweep_graphs)
        if (g.dev == dev && g.ny == ny && g.n == n && g.T == T && g.W4 == L.W4 && g.S == L.S && g.MW == L.MW &&
            !memcmp(g.key, key, sizeof(key)))
            ent = &g;
    if (!ent) {
        if (g_sweep_graphs.size() >= 8) {
            cudaGraphExecDestroy(g_sweep_graphs.front().exec);
            g_sweep_graphs.erase(g_sweep_graphs.begin());
        }
        cudaStream_t cs;
        TW_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) { cudaStreamDestroy(cs); set_cuda_error(e); return TW_ECUDA; }
        RBLayout Lc = L;
        int nl = 0;
        pause_launch_count(true);
        const int err = rb_sweeps(Lc, nx, ny, n, T, 1.0f, cs, &nl, omega_dev);
        pause_launch_count(false);
        cudaGraph_t g = nullptr;
        e = cudaStreamEndCapture(cs, &g);
        cudaStreamDestroy(cs);
        if (err || e != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            if (e != cudaSuccess) set_cuda_error(e);
            return err ? err : TW_ECUDA;
        }
        SweepGraph ne;
        ne.dev = dev; ne.ny = ny; ne.n = n; ne.T = T;
        ne.W4 = L.W4; ne.S = L.S; ne.MW = L.MW;
        memcpy(ne.key, key, sizeof(key));
        e = cudaGraphInstantiate(&ne.exec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) { set_cuda_error(e); return TW_ECUDA; }
        ne.launches = nl;
        ne.swap = Lc.R != L.R;
        g_sweep_graphs.push_back(ne);
        ent = &g_sweep_graphs.back();
    }
    TW_CUDA(cudaGraphLaunch(ent->exec, s));
    *launches += ent->launches;
    count_launches((unsigned long long)ent->launches);
    if (ent->swap) {
        float *t = L.R; L.R = L.R2; L.R2 = t;
        t = L.B; L.B = L.B2; L.B2 = t;
    }
    return TW_OK;
}

int tb_tiles(int T, int nx, int ny) {
    RBLayout L = rb_layout(nx, ny);
    int kx, yi;
    switch (T) {
        case 7: kx = TBCfg<7>::Sh::KI4; yi = TBCfg<7>::Sh::YI; break;
        case 6: kx = TBCfg<6>::Sh::KI4; yi = TBCfg<6>::Sh::YI; break;
        case 5: kx = TBCfg<5>::Sh::KI4; yi = TBCfg<5>::Sh::YI; break;
        case 4: kx = TBCfg<4>::Sh::KI4; yi = TBCfg<4>::Sh::YI; break;
        case 3: kx = TBCfg<3>::Sh::KI4; yi = TBCfg<3>::Sh::YI; break;
        default: kx = TBCfg<2>::Sh::KI4; yi = TBCfg<2>::Sh::YI; break;
    }
    return (int)(ceil_div(L.W4, kx) * ceil_div(ny, yi));
}

template <int T>
static void node_of(RBLayout &L, int ny, void **func, dim3 *grid, dim3 *block) {
    using C = TBCfg<T>;
    *func = (void *)rb_tb_kernel<T, C::RB, C::WARPS, C::MINB>;
    *grid = dim3(ceil_div(L.W4, C::Sh::KI4), ceil_div(ny, C::Sh::YI));
    *block = dim3(C::WARPS * 32);
}

// Kernel entry and launch shape of the T-fused sweep, for graph construction.
void tb_kernel_node(int T, RBLayout &L, int ny, void **func, dim3 *grid, dim3 *block) {
    switch (T) {
        case 7: node_of<7>(L, ny, func, grid, block); break;
        case 6: node_of<6>(L, ny, func, grid, block); break;
        case 5: node_of<5>(L, ny, func, grid, block); break;
        case 4: node_of<4>(L, ny, func, grid, block); break;
        case 3: node_of<3>(L, ny, func, grid, block); break;
        default: node_of<2>(L, ny, func, grid, block); break;
    }
}

}  // namespace tw
