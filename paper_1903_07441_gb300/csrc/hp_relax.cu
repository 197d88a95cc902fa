// Harmonic potential field relaxation (Sec. 3.1, Eqs. 1-2; Alg. 1 "Path Planning").
//
// The field is stored as u = 1 - phi: goal 1, obstacles and border 0.  The
// equation is linear, so the same 5-point average applies; tiny u keeps its
// relative precision far from the goal, where phi rounds to 1.
//
// Forms:
//  * HP_JACOBI -- the plain comparison form: Eq. 1 in FP32, one sweep per
//    launch, 16x16 thread blocks with one thread per cell (the paper's launch
//    shape), global loads, ping-pong buffers.
//  * HP_RBSOR  -- red-black SOR in FP32 on a colour-split layout: the red
//    cells (x + y even) and the black cells are packed into two arrays of
//    ny rows x ceil(nx/2) entries, so every half-sweep reads its own colour
//    and the other colour with unit-stride 128-bit loads.  One Dirichlet bit
//    per cell (free = 1) rides along.  Red-black is the parallel ordering of
//    Eq. 2's Gauss-Seidel family and has the same fixed point.  T full sweeps
//    are fused per launch in shared memory (temporal blocking).
//  * HP_MIXED  -- defect correction (see hp_mixed.cu).
//
// The stopping test is the 1/4-scaled residual max |(1/4) sum_nbr u - u| over
// free cells, reduced with warp shuffles and one atomic per CTA every K
// sweeps; the final residual is recomputed in FP64 on the stored output.
#include <math.h>
#include <string.h>

#include "common.cuh"
#include "hp_internal.cuh"
#include "hp_tile.cuh"

namespace tw {

// ---------------------------------------------------------------------------
// plain FP32 Jacobi (Eq. 1)
// ---------------------------------------------------------------------------

__global__ void jacobi_init_kernel(const uint8_t *__restrict__ occ, int nx, int ny, int gx, int gy,
                                   float *__restrict__ u, int warm) {
    int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= nx || y >= ny) return;
    size_t c = (size_t)y * nx + x;
    bool goal = (x == gx && y == gy);
    bool fixed = goal || occ[c] != 0 || x == 0 || y == 0 || x == nx - 1 || y == ny - 1;
    if (gx < 0) {  // general Dirichlet: occ is the fixed mask and u already holds its values
        return;
    }
    if (goal) u[c] = 1.0f;
    else if (fixed) u[c] = 0.0f;
    else if (!warm) u[c] = 0.5f;
}

// gx < 0: `occ` is a general fixed mask; otherwise the planner's occupancy + goal.
__global__ void __launch_bounds__(256) jacobi_sweep_kernel(const uint8_t *__restrict__ occ, int nx, int ny,
                                                           int gx, int gy, const float *__restrict__ src,
                                                           float *__restrict__ dst) {
    int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= nx || y >= ny) return;
    size_t c = (size_t)y * nx + x;
    bool fixed = occ[c] != 0 || (x == gx && y == gy) || x == 0 || y == 0 || x == nx - 1 || y == ny - 1;
    if (fixed) {
        dst[c] = src[c];
        return;
    }
    float a = (src[c + 1] + src[c - 1]) + (src[c + nx] + src[c - nx]);
    dst[c] = 0.25f * a;
}

// FP32 residual max of a full-layout field (warp-shuffle max, one atomic per CTA).
__global__ void __launch_bounds__(256) full_residual_kernel(const uint8_t *__restrict__ occ, int nx, int ny,
                                                            int gx, int gy, const float *__restrict__ u,
                                                            unsigned int *__restrict__ out_max) {
    int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y;
    float r = 0.0f;
    if (x > 0 && y > 0 && x < nx - 1 && y < ny - 1) {
        size_t c = (size_t)y * nx + x;
        if (!(occ[c] != 0 || (x == gx && y == gy))) {
            float a = 0.25f * ((u[c + 1] + u[c - 1]) + (u[c + nx] + u[c - nx]));
            r = fabsf(a - u[c]);
        }
    }
    block_max_atomic(r, out_max);
}

// FP64-accurate residual (max and sum of squares) of a full-layout FP32 field.
// A 32 x 8 CTA covers 32 x (8 * kResRows) cells, kResRows rows per thread, so
// that the block reduction is amortised over several cells.
constexpr int kResRows = 4;
__global__ void __launch_bounds__(256) full_residual_f64_kernel(const uint8_t *__restrict__ occ, int nx, int ny,
                                                                int gx, int gy, const float *__restrict__ u,
                                                                unsigned long long *__restrict__ out_max,
                                                                double *__restrict__ out_sum) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    float hi = 0.0f, lo = 0.0f, q = 0.0f;
#pragma unroll
    for (int i = 0; i < kResRows; i++) {
        const int y = (blockIdx.y * kResRows + i) * blockDim.y + threadIdx.y;
        if (x > 0 && y > 0 && x < nx - 1 && y < ny - 1) {
            const size_t c = (size_t)y * nx + x;
            if (!(occ[c] != 0 || (x == gx && y == gy))) {
                float h, l;
                resid_pair(u[c + 1], u[c - 1], u[c + nx], u[c - nx], u[c], h, l);
                pair_max(hi, lo, h, l);
                q = fmaf(h, h, q);
            }
        }
    }
    block_max_sum_pair(hi, lo, q, out_max, out_sum);
}

__global__ void goal_check_kernel(const uint8_t *__restrict__ occ, int nx, int gx, int gy, int *flag) {
    if (threadIdx.x == 0 && blockIdx.x == 0) *flag = occ[(size_t)gy * nx + gx] != 0;
}

__global__ void to_phi_kernel(float *__restrict__ u, size_t n) {
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) u[i] = 1.0f - u[i];
}

// ---------------------------------------------------------------------------
// colour-split layout
// ---------------------------------------------------------------------------

// Pack: full field (or init rule) -> red/black arrays + free-cell bits.
// Thread per (y, k); each warp covers 32 consecutive k of one row so that the
// mask word is one ballot.  mode 0: planner (occ + goal, cold init unless warm);
// mode 1: general Dirichlet (occ = fixed mask, values from u_in).
__global__ void rb_pack_kernel(const uint8_t *__restrict__ occ, const float *__restrict__ u_in, int nx,
                               int ny, int gx, int gy, int mode, int warm, RBLayout L) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    int y = blockIdx.y;
    if (y >= ny) return;
    int lane = threadIdx.x & 31;
#pragma unroll
    for (int color = 0; color < 2; color++) {
        int x = 2 * k + ((y + color) & 1);
        float v = 0.0f;
        bool free_cell = false;
        if (k < L.W2 && x < nx) {
            size_t c = (size_t)y * nx + x;
            bool border = x == 0 || y == 0 || x == nx - 1 || y == ny - 1;
            if (mode == 0) {
                bool goal = (x == gx && y == gy);
                bool fixed = goal || border || occ[c] != 0;
                free_cell = !fixed;
                v = goal ? 1.0f : (fixed ? 0.0f : (warm ? u_in[c] : 0.5f));
            } else {
                free_cell = !(border || occ[c] != 0);
                v = u_in[c];
            }
        }
        unsigned bits = __ballot_sync(0xffffffffu, free_cell);
        if (k < L.W2) {
            float *arr = color ? L.B : L.R;
            arr[(size_t)y * L.S + 4 + k] = v;
        }
        if (lane == 0 && k < L.W2 + 31) {
            uint32_t *M = color ? L.MB : L.MR;
            int w = k >> 5;
            if (w < L.MW) M[(size_t)y * L.MW + w] = bits;
        }
    }
}

// alt (nullable, device): when *alt != 0 the solution is in the second
// ping-pong pair (a polished copy the graph-driven loop accepted).
__global__ void rb_unpack_kernel(RBLayout L, int nx, int ny, float *__restrict__ out, int to_phi,
                                 const int *__restrict__ alt) {
    int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= nx || y >= ny) return;
    int color = (x + y) & 1;
    int k = x >> 1;
    const bool a = alt && *alt;
    const float *arr = color ? (a ? L.B2 : L.B) : (a ? L.R2 : L.R);
    float v = arr[(size_t)y * L.S + 4 + k];
    out[(size_t)y * nx + x] = to_phi ? 1.0f - v : v;
}

// FP32 residual max over both colours of the split layout (one atomicMax per
// CTA), if l2part is given each CTA's sum of squared residuals, and the
// snapshot work of the error estimate (snap_dev, when given, overrides
// snap_arg: the graph-driven loop keeps the state on the device).
__global__ void __launch_bounds__(256) rb_residual_kernel(RBLayout L, int ny, unsigned int *out_max, float *l2part,
                                                          int snap_arg, const int *snap_dev, unsigned int *out_dmax) {
    rb_residual_cta(L, ny, out_max, l2part, snap_dev ? *snap_dev : snap_arg, out_dmax);
}

// The 2-norm of the last check's residual from its per-CTA partials (one CTA
// of kPartThreads threads, the reduction the graph's control kernel uses).
__global__ void __launch_bounds__(kPartThreads) l2_finalize_kernel(const float *__restrict__ part, int n,
                                                                   double *out) {
    const double s = block_sum_partials(part, n, threadIdx.x);
    if (threadIdx.x == 0) *out = sqrt(s);
}

// ---------------------------------------------------------------------------
// host driver
// ---------------------------------------------------------------------------

__global__ void timing_gate_kernel(unsigned long long ns) {
    unsigned long long t0, t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    for (int i = 0; i < (1 << 20); i++) {
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
        if (t - t0 >= ns) break;
        __nanosleep(256);
    }
}

void timing_gate(cudaStream_t s) { TW_LAUNCH(timing_gate_kernel, 1, 1, 0, s, 30000ull); }

RBLayout rb_layout(int nx, int ny) {
    RBLayout L;
    memset(&L, 0, sizeof(L));
    int half = (nx + 1) / 2;
    L.W2 = (half + 3) & ~3;
    L.W4 = L.W2 / 4;
    L.S = L.W2 + 8;
    L.MW = (L.W2 + 31) / 32;
    return L;
}

size_t carve_rb(Carver &cv, int nx, int ny, RBLayout *out, bool pingpong, bool snapshot) {
    RBLayout L = rb_layout(nx, ny);
    size_t plane = (size_t)ny * L.S;
    L.R = cv.take<float>(plane);
    L.B = cv.take<float>(plane);
    L.MR = cv.take<uint32_t>((size_t)ny * L.MW);
    L.MB = cv.take<uint32_t>((size_t)ny * L.MW);
    if (pingpong) {
        L.R2 = cv.take<float>(plane);
        L.B2 = cv.take<float>(plane);
    }
    if (snapshot) {   // written before it is read: no clearing needed
        L.R3 = cv.take<float>(plane);
        L.B3 = cv.take<float>(plane);
    }
    if (out) *out = L;
    return cv.need;
}

static size_t carve_relax(Carver &cv, int nx, int ny, const hp_params *p, RelaxLayout *out) {
    RelaxLayout R;
    memset(&R, 0, sizeof(R));
    R.scal = cv.take<RelaxScalars>(1);
    int method = p ? p->method : HP_RBSOR;
    if (method == HP_JACOBI) {
        R.tmp = cv.take<float>((size_t)nx * ny);
    } else if (method == HP_RBSOR) {
        carve_rb(cv, nx, ny, &R.rb, true, p && p->etol > 0.0);
        R.l2part = cv.take<float>((size_t)rb_residual_blocks(R.rb, ny));
    } else {
        carve_mixed(cv, nx, ny, p ? p->storage : HP_STORE_F16, &R);
    }
    if (out) *out = R;
    return cv.need;
}

static bool valid_params(const hp_params *p) {
    return p && (p->method == HP_JACOBI || p->method == HP_RBSOR || p->method == HP_MIXED) &&
           (p->storage == HP_STORE_F32 || p->storage == HP_STORE_F16 || p->storage == HP_STORE_BF16) &&
           isfinite(p->omega) && (p->omega == 0.0 || (p->omega > 0.0 && p->omega < 2.0)) &&
           isfinite(p->tol) && p->tol >= 0.0 && p->max_sweeps >= 1 && p->check_every >= 0 &&
           p->tblock >= 0 && p->tblock <= 16 && isfinite(p->etol) && p->etol >= 0.0;
}

// First omega of an adaptive solve, by the longer side n, and never above
// sor_omega_cap.  The adaptation only raises omega, so the start stays below
// the optimum of cluttered scenes (30-45 % obstacles: 1.94-1.97 at
// 1024-2048, about 1.94 at 256-512).
double sor_initial_omega(int nx, int ny) {
    int n = nx > ny ? nx : ny;
    const double w = n >= 1024 ? 1.9 : (n >= 256 ? 1.85 : 1.75);
    const double cap = sor_omega_cap(nx, ny);
    return w < cap ? w : cap;
}

// Upper bound on omega_opt for any occupancy of an nx x ny grid: the Jacobi
// matrix of the free cells is a principal submatrix of the (nonnegative)
// Jacobi matrix of the empty box, so its spectral radius is at most the box's,
// mu = (cos(pi / (nx - 1)) + cos(pi / (ny - 1))) / 2 (Perron-Frobenius), and
// omega_opt = 2 / (1 + sqrt(1 - mu^2)) grows with mu.  Without the cap the
// pre-asymptotic estimates can drive omega past the optimum of open scenes,
// where the rate omega - 1 gets close to 1.
double sor_omega_cap(int nx, int ny) {
    const double pi = 3.14159265358979323846;
    const double mu = 0.5 * (cos(pi / (nx - 1)) + cos(pi / (ny - 1)));
    return 2.0 / (1.0 + sqrt(1.0 - mu * mu));
}

int read_max_f32(unsigned int *dmax, cudaStream_t s, float *out) {
    unsigned int h = 0;
    TW_CUDA(cudaMemcpyAsync(&h, dmax, sizeof(h), cudaMemcpyDeviceToHost, s));
    TW_CUDA(cudaStreamSynchronize(s));
    memcpy(out, &h, sizeof(h));
    return TW_OK;
}

int final_residual_full(const uint8_t *occ, int nx, int ny, int gx, int gy, const float *u,
                        RelaxScalars *scal, cudaStream_t s, double *r_inf, double *r_l2) {
    TW_CUDA(cudaMemsetAsync(&scal->max64, 0, sizeof(scal->max64) + sizeof(scal->sum64), s));
    dim3 b(32, 8), gr(ceil_div(nx, 32), ceil_div(ny, 8 * kResRows));
    TW_LAUNCH(full_residual_f64_kernel, gr, b, 0, s, occ, nx, ny, gx, gy, u, &scal->max64, &scal->sum64);
    TW_CHECK_LAUNCH();
    unsigned long long m = 0;
    double sum = 0.0;
    TW_CUDA(cudaMemcpyAsync(&m, &scal->max64, sizeof(m), cudaMemcpyDeviceToHost, s));
    TW_CUDA(cudaMemcpyAsync(&sum, &scal->sum64, sizeof(sum), cudaMemcpyDeviceToHost, s));
    TW_CUDA(cudaStreamSynchronize(s));
    memcpy(r_inf, &m, sizeof(double));
    *r_l2 = sqrt(sum);
    return TW_OK;
}

static int relax_jacobi(const uint8_t *occ, int nx, int ny, int gx, int gy, float *u,
                        const hp_params *p, hp_stats *st, RelaxLayout &R, cudaStream_t s) {
    dim3 b(16, 16), gr(ceil_div(nx, 16), ceil_div(ny, 16));
    TW_LAUNCH(jacobi_init_kernel, gr, b, 0, s, occ, nx, ny, gx, gy, u, (p->flags & HP_WARM_START) ? 1 : 0);
    TW_CHECK_LAUNCH();
    TW_CUDA(cudaMemcpyAsync(R.tmp, u, sizeof(float) * (size_t)nx * ny, cudaMemcpyDeviceToDevice, s));
    int K = p->check_every > 0 ? p->check_every : 64;
    float *src = u, *dst = R.tmp;
    int sweeps = 0, checks = 0;
    SweepTimer timer;
    if (timer.open((p->flags & HP_TIMING) != 0)) return TW_ECUDA;
    st->status = TW_NOT_CONVERGED;
    while (sweeps < p->max_sweeps) {
        int n = p->max_sweeps - sweeps < K ? p->max_sweeps - sweeps : K;
        timer.start(s);
        for (int i = 0; i < n; i++) {
            TW_LAUNCH(jacobi_sweep_kernel, gr, b, 0, s, occ, nx, ny, gx, gy, src, dst);
            float *t = src; src = dst; dst = t;
        }
        timer.stop(s);
        TW_CHECK_LAUNCH();
        timer.accumulate();
        sweeps += n;
        if (p->tol > 0.0) {
            TW_CUDA(cudaMemsetAsync(&R.scal->max32, 0, sizeof(unsigned int), s));
            TW_LAUNCH(full_residual_kernel, dim3(ceil_div(nx, 32), ceil_div(ny, 8)), dim3(32, 8), 0, s,
                      occ, nx, ny, gx, gy, src, &R.scal->max32);
            TW_CHECK_LAUNCH();
            float r;
            int e = read_max_f32(&R.scal->max32, s, &r);
            if (e) return e;
            checks++;
            if (r <= p->tol) { st->status = TW_OK; break; }
        }
    }
    if (src != u)
        TW_CUDA(cudaMemcpyAsync(u, src, sizeof(float) * (size_t)nx * ny, cudaMemcpyDeviceToDevice, s));
    st->sweeps = sweeps;
    st->checks = checks;
    st->omega = 1.0;
    st->sweep_launches = sweeps;
    st->sweep_ms = timer.ms;
    st->tblock = 1;
    return TW_OK;
}

// Red-black SOR driver on the split layout (pack -> sweeps -> unpack).
dim3 rb_residual_grid(const RBLayout &L, int ny) { return dim3(ceil_div(L.W4, 64), ceil_div(ny, 4 * kResidRows)); }

int rb_residual_blocks(const RBLayout &L, int ny) {
    const dim3 g = rb_residual_grid(L, ny);
    return (int)(g.x * g.y);
}

void *rb_residual_kernel_ptr() { return (void *)rb_residual_kernel; }

void rb_residual_launch(RBLayout &L, int ny, unsigned int *out, float *l2part, cudaStream_t s, int snap,
                        unsigned int *dmax) {
    TW_LAUNCH(rb_residual_kernel, rb_residual_grid(L, ny), dim3(64, 4), 0, s, L, ny, out, l2part, snap,
              (const int *)nullptr, dmax);
}

// Red-black SOR driver on the split layout.  By default the check intervals
// run inside one CUDA graph (a conditional while-node re-runs "K sweeps,
// residual, control" on the device); the host loop below finishes any
// remainder and serves HP_TIMING / HP_HOST_LOOP.
int rb_solve(RBLayout &L, int nx, int ny, const hp_params *p, RelaxScalars *scal, float *l2part, hp_stats *st,
             cudaStream_t s, int *ctl_on_device) {
    *ctl_on_device = 0;
    // Blocking depth: the deep tiles when they fill most of a GB300 (152 SMs)
    // in one launch, else the small tiles.
    int T = p->tblock > 0 ? p->tblock : (tb_tiles(kDeepTBlock, nx, ny) >= 96 ? kDeepTBlock : kDefaultTBlock);
    if (T > kMaxTBlock) T = kMaxTBlock;
    // Check interval: check_every rounded up to whole launches; by default the
    // largest even number of launches within 32 sweeps (the graph body needs
    // an even count to end on the same ping-pong planes).
    int K;
    if (p->check_every > 0) {
        K = p->check_every;
        if (T > 1 && K % T) K += T - K % T;
    } else {
        K = T > 1 ? 2 * T * (32 / (2 * T) > 0 ? 32 / (2 * T) : 1) : 32;
    }
    const bool checks = p->tol > 0.0 || p->omega == 0.0;
    RelaxCtl c;
    memset(&c, 0, sizeof(c));
    c.adapt = p->omega == 0.0;
    c.omega = c.adapt ? sor_initial_omega(nx, ny) : p->omega;
    c.omega_f = (float)c.omega;
    c.r_prev = -1.0;
    c.tol = p->tol;
    c.K = K;
    c.max_sweeps = p->max_sweeps;
    c.status = TW_NOT_CONVERGED;
    c.omega_max = sor_omega_cap(nx, ny);
    c.T = T;
    // the error estimate needs the snapshot planes (carved with etol > 0); the polish it may end
    // with needs T-fused launches (ping-pong planes)
    c.etol = (T > 1 && L.R2 && L.R3) ? p->etol : 0.0;
    c.Tl = K;
    c.err_raw = DBL_MAX;
    // HP_POLISH, or an error tolerance (its polish only clears the rounding noise at the end)
    c.polish_ok = (T > 1 && L.R2 && ((p->flags & HP_POLISH) || c.etol > 0.0)) ? 1 : 0;
    c.one_f = 1.0f;
    int launches = 0;
    bool done = false;
    const bool host_loop = (p->flags & (HP_TIMING | HP_HOST_LOOP)) != 0;
    if (checks && !host_loop && T > 1 && (K / T) % 2 == 0 && p->max_sweeps >= K) {
        TW_CUDA(cudaMemcpyAsync(&scal->ctl, &c, sizeof(c), cudaMemcpyHostToDevice, s));
        TW_CUDA(cudaMemsetAsync(&scal->max32, 0, sizeof(unsigned int), s));
        TW_CUDA(cudaMemsetAsync(&scal->dmax32, 0, sizeof(unsigned int), s));
        int e = rb_solve_graph(L, nx, ny, T, K, p->max_sweeps / K, c.polish_ok, c.etol > 0.0, scal, l2part, s,
                               &launches);
        if (e < 0) return e;
        if (e == TW_OK) st->loop = HP_LOOP_GRAPH;
        if (e == TW_OK && p->max_sweeps % K == 0) {
            // the graph runs every interval the cap allows: no remainder can follow, so the
            // loop state is read back later together with the final residual (one sync)
            *ctl_on_device = 1;
            st->tblock = T;
            return TW_OK;
        }
        if (e == TW_OK) {
            TW_CUDA(cudaMemcpyAsync(&c, &scal->ctl, sizeof(c), cudaMemcpyDeviceToHost, s));
            TW_CUDA(cudaStreamSynchronize(s));
            done = c.status == TW_OK;
            if (c.in_alt) {   // a polished copy was accepted: it is in the second pair
                float *t = L.R; L.R = L.R2; L.R2 = t;
                t = L.B; L.B = L.B2; L.B2 = t;
            }
            // every interval ran K/T sweep launches, the residual and the control kernel (and with
            // HP_POLISH the polish-result kernel); every polish one sweep launch and a residual
            launches += c.checks * (K / T) + c.polishes;
            count_launches((unsigned long long)c.checks * (K / T + 2 + c.polish_ok) + 2ull * c.polishes);
        }
    }
    SweepTimer timer;
    if (timer.open((p->flags & HP_TIMING) != 0)) return TW_ECUDA;
    while (!done && c.sweeps < p->max_sweeps) {
        int n = p->max_sweeps - c.sweeps < K ? p->max_sweeps - c.sweeps : K;
        int e;
        if (timer.on && T > 1) {
            // timed as the graph-driven loop runs them: one graph of the interval's launches
            const float om = (float)c.omega;
            TW_CUDA(cudaMemcpyAsync(&scal->ctl.omega_f, &om, sizeof(om), cudaMemcpyHostToDevice, s));
            TW_CUDA(cudaStreamSynchronize(s));
            timer.start(s);
            e = rb_sweeps_graph(L, nx, ny, n, T, &scal->ctl.omega_f, s, &launches);
            timer.stop(s);
        } else {
            timer.start(s);
            e = rb_sweeps(L, nx, ny, n, T, (float)c.omega, s, &launches);
            timer.stop(s);
        }
        if (e) return e;
        timer.accumulate();
        c.sweeps += n;
        if (checks) {
            // error estimate: the change since the previous check's snapshot, n sweeps ago
            const int snap = c.etol > 0.0 ? c.snap : 0;
            c.Tl = n;
            TW_CUDA(cudaMemsetAsync(&scal->max32, 0, sizeof(unsigned int), s));
            if (snap == 2) TW_CUDA(cudaMemsetAsync(&scal->dmax32, 0, sizeof(unsigned int), s));
            rb_residual_launch(L, ny, &scal->max32, l2part, s, snap, snap == 2 ? &scal->dmax32 : nullptr);
            if (l2part)
                TW_LAUNCH(l2_finalize_kernel, 1, kPartThreads, 0, s, l2part, rb_residual_blocks(L, ny), &scal->l2);
            TW_CHECK_LAUNCH();
            RelaxScalars hs;
            TW_CUDA(cudaMemcpyAsync(&hs, scal, sizeof(hs), cudaMemcpyDeviceToHost, s));
            TW_CUDA(cudaStreamSynchronize(s));
            float rf, df;
            memcpy(&rf, &hs.max32, sizeof(rf));
            memcpy(&df, &hs.dmax32, sizeof(df));
            const int cont = relax_control(c, (double)rf, l2part ? hs.l2 : -1.0, n, snap == 2 ? (double)df : -1.0);
            if (!cont) {
                done = true;
            } else if (relax_polish_decide(c, cont)) {
                // T sweeps at omega = 1 into the second pair; L keeps the SOR planes
                RBLayout Lp = L;
                timer.start(s);
                e = rb_sweeps(Lp, nx, ny, T, T, 1.0f, s, &launches);
                timer.stop(s);
                if (e) return e;
                timer.accumulate();
                TW_CUDA(cudaMemsetAsync(&scal->max32, 0, sizeof(unsigned int), s));
                rb_residual_launch(Lp, ny, &scal->max32, nullptr, s, 0, nullptr);
                TW_CHECK_LAUNCH();
                float r2;
                e = read_max_f32(&scal->max32, s, &r2);
                if (e) return e;
                if (!relax_polish_result(c, (double)r2)) {
                    done = true;
                    L = Lp;
                }
            }
        }
    }
    st->status = c.status;
    st->sweeps = c.sweeps + c.psweeps;
    st->polishes = c.polishes;
    st->polished = c.in_alt;
    st->resid_check = c.checks ? c.r_last : 0.0;
    st->err_est = c.etol > 0.0 ? c.err_est : 0.0;
    st->checks = c.checks;
    st->omega = c.omega;
    st->sweep_launches = launches;
    st->sweep_ms = timer.ms;
    st->tblock = T;
    return TW_OK;
}

static int relax_rbsor(const uint8_t *occ, int nx, int ny, int gx, int gy, float *u, int mode,
                       const hp_params *p, hp_stats *st, RelaxLayout &R, cudaStream_t s, int *ctl_dev) {
    RBLayout &L = R.rb;
    TW_CUDA(cudaMemsetAsync(L.R, 0, sizeof(float) * (size_t)ny * L.S, s));
    TW_CUDA(cudaMemsetAsync(L.B, 0, sizeof(float) * (size_t)ny * L.S, s));
    if (L.R2) {
        TW_CUDA(cudaMemsetAsync(L.R2, 0, sizeof(float) * (size_t)ny * L.S, s));
        TW_CUDA(cudaMemsetAsync(L.B2, 0, sizeof(float) * (size_t)ny * L.S, s));
    }
    TW_LAUNCH(rb_pack_kernel, dim3(ceil_div(L.W2 + 31, 128), ny), 128, 0, s,
              occ, u, nx, ny, gx, gy, mode, (p->flags & HP_WARM_START) ? 1 : 0, L);
    TW_CHECK_LAUNCH();
    int e = rb_solve(L, nx, ny, p, R.scal, R.l2part, st, s, ctl_dev);
    if (e) return e;
    TW_LAUNCH(rb_unpack_kernel, dim3(ceil_div(nx, 256), ny), 256, 0, s, L, nx, ny, u, 0,
              *ctl_dev ? (const int *)&R.scal->ctl.in_alt : (const int *)nullptr);
    TW_CHECK_LAUNCH();
    return TW_OK;
}

static int relax_common(const uint8_t *occ, int nx, int ny, int gx, int gy, float *u, int mode,
                        const hp_params *p, hp_stats *st, void *ws, size_t ws_bytes, cudaStream_t s) {
    if (!ws || !ws_aligned(ws)) return TW_EWORKSPACE;
    Carver cv(ws, ws_bytes);
    RelaxLayout R;
    carve_relax(cv, nx, ny, p, &R);
    if (!cv.ok()) return TW_EWORKSPACE;
    hp_stats local;
    memset(&local, 0, sizeof(local));
    // goal check on the device: read back with the final results (no extra sync)
    TW_CUDA(cudaMemsetAsync(&R.scal->goal_blocked, 0, sizeof(int), s));
    if (mode == 0) TW_LAUNCH(goal_check_kernel, 1, 32, 0, s, occ, nx, gx, gy, &R.scal->goal_blocked);
    int e, ctl_dev = 0;
    if (p->method == HP_JACOBI) {
        if (mode == 1) {
            // the general Dirichlet form keeps the caller's fixed values
            hp_params q = *p;
            q.flags |= HP_WARM_START;
            e = relax_jacobi(occ, nx, ny, -1, -1, u, &q, &local, R, s);
        } else {
            e = relax_jacobi(occ, nx, ny, gx, gy, u, p, &local, R, s);
        }
    } else if (p->method == HP_RBSOR) {
        e = relax_rbsor(occ, nx, ny, gx, gy, u, mode, p, &local, R, s, &ctl_dev);
    } else {
        e = relax_mixed(occ, nx, ny, gx, gy, u, mode, p, &local, R, s);
    }
    if (e) return e;
    if (p->method != HP_MIXED) {   // HP_MIXED reports the residual of its FP64 master
        TW_CUDA(cudaMemsetAsync(&R.scal->max64, 0, sizeof(R.scal->max64) + sizeof(R.scal->sum64), s));
        dim3 b(32, 8), gr(ceil_div(nx, 32), ceil_div(ny, 8 * kResRows));
        TW_LAUNCH(full_residual_f64_kernel, gr, b, 0, s, occ, nx, ny, mode == 1 ? -1 : gx, mode == 1 ? -1 : gy, u,
                  &R.scal->max64, &R.scal->sum64);
        TW_CHECK_LAUNCH();
    }
    if (mode == 0 && (p->flags & HP_OUT_PHI)) {
        size_t n = (size_t)nx * ny;
        TW_LAUNCH(to_phi_kernel, ceil_div(n, 256), 256, 0, s, u, n);
        TW_CHECK_LAUNCH();
    }
    // the one synchronisation of the call: loop state, goal flag and final residual
    RelaxScalars hs;
    TW_CUDA(cudaMemcpyAsync(&hs, R.scal, sizeof(hs), cudaMemcpyDeviceToHost, s));
    TW_CUDA(cudaStreamSynchronize(s));
    if (hs.goal_blocked) return TW_EGOAL_BLOCKED;
    if (ctl_dev) {
        const RelaxCtl &c = hs.ctl;
        const int KT = local.tblock > 1 ? c.K / local.tblock : c.K;
        local.status = c.status;
        local.sweeps = c.sweeps + c.psweeps;
        local.polishes = c.polishes;
        local.polished = c.in_alt;
        local.resid_check = c.checks ? c.r_last : 0.0;
        local.err_est = c.etol > 0.0 ? c.err_est : 0.0;
        local.checks = c.checks;
        local.omega = c.omega;
        local.sweep_launches = c.checks * KT + c.polishes;
        count_launches((unsigned long long)c.checks * (KT + 2 + c.polish_ok) + 2ull * c.polishes);
    }
    if (p->method != HP_MIXED) {
        memcpy(&local.resid_inf, &hs.max64, sizeof(double));
        local.resid_l2 = sqrt(hs.sum64);
    }
    // the FP64 residual of the output decides the residual test; with an error tolerance the
    // loop's error test must have passed as well
    const bool err_ok = !(p->method != HP_JACOBI && p->etol > 0.0 && local.err_est > 0.0) || local.status == TW_OK;
    if (p->tol > 0.0 && local.resid_inf <= p->tol && err_ok) local.status = TW_OK;
    if (st) *st = local;
    return local.status;
}

}  // namespace tw

using namespace tw;

extern "C" double hp_omega_update(double omega, double lambda, int nx, int ny) {
    if (nx < 3 || ny < 3) return omega;
    return sor_adapt(omega, lambda, sor_omega_cap(nx, ny));
}

extern "C" double hp_omega_cap(int nx, int ny) { return (nx < 3 || ny < 3) ? 0.0 : sor_omega_cap(nx, ny); }

extern "C" double hp_omega_initial(int nx, int ny) {
    return (nx < 3 || ny < 3) ? 0.0 : sor_initial_omega(nx, ny);
}

extern "C" size_t hp_relax_workspace_size(int nx, int ny, const hp_params *p) {
    if (nx < 3 || ny < 3) return 0;
    Carver cv;
    return carve_relax(cv, nx, ny, p, nullptr);
}

extern "C" int hp_relax(const tw_grid *g, const uint8_t *occ_dev, int gx, int gy, float *field_dev,
                        const hp_params *p, hp_stats *stats, void *workspace, size_t workspace_bytes,
                        void *stream) {
    if (!g || g->nx < 3 || g->ny < 3 || g->nx > 65535 || g->ny > 65535 || !occ_dev || !field_dev ||
        !valid_params(p))
        return TW_EINVAL;
    int nx = g->nx, ny = g->ny;
    if (gx < 1 || gy < 1 || gx > nx - 2 || gy > ny - 2) return TW_EGOAL_BLOCKED;
    cudaStream_t s = (cudaStream_t)stream;
    if ((p->flags & HP_WARM_START) && (p->flags & HP_OUT_PHI)) {
        // warm start given as phi: convert to u in place first
        size_t n = (size_t)nx * ny;
        TW_LAUNCH(to_phi_kernel, ceil_div(n, 256), 256, 0, s, field_dev, n);
        TW_CHECK_LAUNCH();
    }
    return relax_common(occ_dev, nx, ny, gx, gy, field_dev, 0, p, stats, workspace, workspace_bytes, s);
}

extern "C" int hp_relax_dirichlet(int nx, int ny, const uint8_t *fixed_dev, float *u_dev,
                                  const hp_params *p, hp_stats *stats, void *workspace,
                                  size_t workspace_bytes, void *stream) {
    if (nx < 3 || ny < 3 || nx > 65535 || ny > 65535 || !fixed_dev || !u_dev || !valid_params(p))
        return TW_EINVAL;
    return relax_common(fixed_dev, nx, ny, -1, -1, u_dev, 1, p, stats, workspace, workspace_bytes,
                        (cudaStream_t)stream);
}

extern "C" int hp_residual(int nx, int ny, const uint8_t *fixed_dev, const float *u_dev, double *r_inf,
                           double *r_l2, void *workspace, size_t workspace_bytes, void *stream) {
    if (nx < 3 || ny < 3 || !fixed_dev || !u_dev || !r_inf || !r_l2) return TW_EINVAL;
    if (!workspace || !ws_aligned(workspace) || workspace_bytes < sizeof(RelaxScalars)) return TW_EWORKSPACE;
    return final_residual_full(fixed_dev, nx, ny, -1, -1, u_dev, (RelaxScalars *)workspace,
                               (cudaStream_t)stream, r_inf, r_l2);
}
