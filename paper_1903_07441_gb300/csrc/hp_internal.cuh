// Internal declarations shared by the relaxation translation units.
#pragma once
#include <float.h>

#include "common.cuh"

namespace tw {

constexpr int kDefaultTBlock = 4;   // blocking depth of small fields
constexpr int kDeepTBlock = 7;      // blocking depth of fields that fill the GPU with deep tiles
constexpr int kMaxTBlock = 7;

// Colour-split layout: red cells (x + y even) and black cells in two arrays
// of ny rows; row y of colour c holds cells x = 2k + ((y + c) & 1), k < W2.
// Each row has 4 padding floats on both sides (zero, never written) so the
// +-1 neighbour of a float4 never leaves the row allocation.  Bit k of the
// mask row is 1 for a free (updatable) cell.
struct RBLayout {
    int W2;            // entries per colour row (multiple of 4)
    int W4;            // float4 per colour row
    int S;             // row stride in floats (W2 + 8)
    int MW;            // mask words per row
    float *R, *B;      // current red / black planes
    uint32_t *MR, *MB; // free-cell bits
    float *R2, *B2;    // ping-pong planes for temporal blocking
    float *R3, *B3;    // snapshot of the planes at the last residual check (error estimate; may be null)
};

// Convergence-loop state, shared by the host-driven loop and the device
// control kernel of the graph-driven loop (lives in the workspace).
struct RelaxCtl {
    float omega_f;         // omega as read by the sweep kernels
    unsigned int rmax;     // FP32 residual max accumulator (bits); reset after each check
    int sweeps, checks, status, adapt, same_iv, K, max_sweeps, pad;
    double omega, r_prev, tol, r_last;
    double e_prev;         // residual 2-norm at the previous check (<= 0: not measured)
    double omega_max;      // cap on the adapted omega (<= 1: 1.9995)
    int polish;            // 1: this check tries a polish launch
    int in_alt;            // 1: the solution is the polished copy in the other ping-pong planes
    int polishes, psweeps; // polish launches tried, and their sweeps
    int go, T;             // continue flag of the last check; sweeps per launch
    int polish_ok;         // polish enabled (HP_RBSOR with HP_POLISH and T > 1)
    int maxnorm_adapt;     // 1: adapt omega on the residual max even when the 2-norm is given (the
                           // 2-norm then only serves the error estimate's decay rate)
    float one_f;           // 1.0f, the omega the polish launches read
    int Tl;                // sweeps since the snapshot the change d is measured against
    int snap;              // snapshot state of the next check: 0 none, 1 take it, 2 compare with it and retake
    double etol;           // error tolerance (0: off; see relax_error_estimate)
    double lam;            // last clear decay rate of the residual 2-norm per sweep (0: none yet)
    double err_est;        // last error estimate (the larger of the last two checks' raw estimates)
    double err_prev;       // the estimate of the check before
    double err_raw;        // the last check's raw estimate (DBL_MAX: none)
    int r_met;             // 1 once the residual test has been met (omega frozen from then on)
    int stall;             // consecutive checks whose estimate did not fall clearly
};


struct RelaxScalars {
    unsigned int max32;
    int goal_blocked;      // set on the device when the goal cell is occupied
    unsigned int dmax32;   // FP32 max change of a free cell over the last launch (bits); reset after each check
    unsigned int pad0;
    unsigned long long max64;
    double sum64;
    double l2;             // residual 2-norm of the last check (host-driven loop)
    double pad1[4];
    RelaxCtl ctl;
};

struct MixedLayout {
    double *x;         // FP64 master field, full layout [ny][nx]
    void *e_r, *e_b;   // correction planes (colour-split, low precision)
    void *e_r2, *e_b2; // ping-pong correction planes
    void *q_r, *q_b;   // scaled right-hand side planes (colour-split, low precision)
    float *f_r, *f_b;  // FP32 colour-split scratch for the right-hand side
};

struct RelaxLayout {
    RelaxScalars *scal;
    float *tmp;        // Jacobi ping-pong buffer
    RBLayout rb;
    MixedLayout mx;
    float *l2part;     // per-CTA sums of squared residuals of rb_residual_kernel
};

RBLayout rb_layout(int nx, int ny);
size_t carve_rb(Carver &cv, int nx, int ny, RBLayout *out, bool pingpong, bool snapshot = false);
size_t carve_mixed(Carver &cv, int nx, int ny, int storage, RelaxLayout *R);
int relax_mixed(const uint8_t *occ, int nx, int ny, int gx, int gy, float *u, int mode,
                const hp_params *p, hp_stats *st, RelaxLayout &R, cudaStream_t s);
// n full red-black SOR sweeps, T fused per launch; *launches += launches made
// omega_dev (optional): the sweep kernels read omega there instead of `omega`
int rb_sweeps(RBLayout &L, int nx, int ny, int n, int T, float omega, cudaStream_t s, int *launches,
              const float *omega_dev = nullptr);
// The same n sweeps as one captured CUDA graph (cached per planes, n and T; the
// kernels read omega from omega_dev), launched on s: the sweep launches run
// back to back as in the graph-driven loop (HP_TIMING times them this way).
int rb_sweeps_graph(RBLayout &L, int nx, int ny, int n, int T, const float *omega_dev, cudaStream_t s,
                    int *launches);
// Number of tiles (CTAs) of one T-fused launch over an nx x ny field.
int tb_tiles(int T, int nx, int ny);
// Graph-driven loop: up to max_intervals check intervals of K sweeps (K/T even)
// run on the device; ctl_dev must hold the initial state.  Returns TW_OK, or
// a positive value when graphs are unavailable (the caller uses the host loop).
int rb_solve_graph(RBLayout &L, int nx, int ny, int T, int K, int max_intervals, int polish, int est,
                   RelaxScalars *scal, float *l2part, cudaStream_t s, int *launches);
// FP32 residual max (atomicMax into *out) and, if l2part is given, the sum of
// squared residuals of every CTA in l2part[rb_residual_blocks(L, ny)].
// snap: snapshot state (see RelaxCtl::snap) of this check; dmax receives the change when snap == 2.
void rb_residual_launch(RBLayout &L, int ny, unsigned int *out, float *l2part, cudaStream_t s, int snap,
                        unsigned int *dmax);
int rb_residual_blocks(const RBLayout &L, int ny);
dim3 rb_residual_grid(const RBLayout &L, int ny);   // launch grid of rb_residual_kernel (64 x 4 threads)

// Optional CUDA-event timing of the sweep kernels (HP_TIMING).
// Keep `s` busy for about 30 us (one thread polling %globaltimer, bounded).
void timing_gate(cudaStream_t s);
struct SweepTimer {
    cudaEvent_t a = nullptr, b = nullptr;
    bool on = false;
    double ms = 0.0;
    int open(bool enable) {
        on = enable;
        if (!on) return TW_OK;
        if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) return TW_ECUDA;
        return TW_OK;
    }
    // the start event follows a short device-side delay (timing_gate), so that
    // it is stamped after the host has queued the launches it brackets: the
    // measured time is the launches' run on the device, not their submission
    void start(cudaStream_t s) {
        if (!on) return;
        timing_gate(s);
        cudaEventRecord(a, s);
    }
    void stop(cudaStream_t s) { if (on) cudaEventRecord(b, s); }
    // after the stream has passed the stop event
    void accumulate() {
        if (!on) return;
        float t = 0.0f;
        cudaEventSynchronize(b);
        if (cudaEventElapsedTime(&t, a, b) == cudaSuccess) ms += t;
    }
    ~SweepTimer() {
        if (a) cudaEventDestroy(a);
        if (b) cudaEventDestroy(b);
    }
};
// *ctl_on_device = 1 when the final loop state is only on the device (in scal->ctl)
int rb_solve(RBLayout &L, int nx, int ny, const hp_params *p, RelaxScalars *scal, float *l2part, hp_stats *st,
             cudaStream_t s, int *ctl_on_device);
double sor_initial_omega(int nx, int ny);
double sor_omega_cap(int nx, int ny);
int read_max_f32(unsigned int *dmax, cudaStream_t s, float *out);
int final_residual_full(const uint8_t *occ, int nx, int ny, int gx, int gy, const float *u,
                        RelaxScalars *scal, cudaStream_t s, double *r_inf, double *r_l2);

// Adaptive SOR factor.  For a consistently ordered matrix (red-black is one)
// the SOR convergence factor lambda at omega <= omega_opt and the Jacobi
// spectral radius mu satisfy (lambda + omega - 1)^2 = lambda omega^2 mu^2
// (Young).  The observed residual decay over a check interval gives lambda,
// hence mu and omega_opt = 2 / (1 + sqrt(1 - mu^2)).  Pre-asymptotic decay
// underestimates mu, so omega approaches omega_opt from below.
//
// At or past omega_opt every eigenvalue has modulus omega - 1 and lambda says
// nothing about mu, so omega is kept while lambda <= (omega - 1)^F, F = 3/4
// (the form of test used by the adaptive SOR procedure of Hageman & Young,
// Applied Iterative Methods, 1981).  The margin scales with 2 - omega, the
// distance of omega - 1 from 1: a margin proportional to omega - 1 itself
// would exceed 1 - lambda for every omega close to 2 and freeze omega below
// its optimum (on a 2048^2 field with 30 % obstacles: 1.957 instead of about
// 1.965, 532 sweeps instead of 420).
__host__ __device__ inline double sor_adapt(double omega, double lambda, double omega_max) {
    if (!(lambda > 0.0) || lambda >= 1.0) return omega;
    if (lambda <= pow(omega > 1.0 ? omega - 1.0 : 0.0, 0.75)) return omega;
    double mu = (lambda + omega - 1.0) / (omega * sqrt(lambda));
    if (!(mu > 0.0)) return omega;
    if (mu >= 0.999999999) mu = 0.999999999;
    double w = 2.0 / (1.0 + sqrt(1.0 - mu * mu));
    // Pre-asymptotic decay underestimates mu, and the SOR rate degrades much
    // faster below omega_opt than above it: move 10 % of the way towards 2.
    w = 2.0 - (2.0 - w) * 0.9;
    const double cap = omega_max > 1.0 ? omega_max : 1.9995;
    if (w > cap) w = cap;
    return (w > omega) ? w : omega;
}

// Deterministic sum of per-CTA partials by one CTA of kPartThreads threads:
// each thread sums its strided partials in index order, then a fixed-shape
// tree in shared memory; every thread returns the same value.
// t is the thread's linear index in its CTA.  Partials are read through L2, so
// values other CTAs of the same grid have just written are seen.
constexpr int kPartThreads = 256;
__device__ inline double block_sum_partials(const float *part, int n, int t) {
    __shared__ double sm[kPartThreads];
    double s = 0.0;
    for (int i = t; i < n; i += kPartThreads) s += (double)__ldcg(part + i);
    sm[t] = s;
    __syncthreads();
    for (int w = kPartThreads / 2; w > 0; w >>= 1) {
        if (t < w) sm[t] += sm[t + w];
        __syncthreads();
    }
    return sm[0];
}

// Error estimate of the current field from d, the largest change of a free
// cell since the snapshot taken at the previous check (Tl sweeps ago).  If the
// error decays by a factor rho per sweep, |e| <= d / (1 - rho^Tl); for SOR at
// or past the optimal omega every eigenvalue has modulus omega - 1, and below
// it the slowest mode decays at the rate the residual 2-norm shows, so
// rho = max(omega - 1, lam).  This is the form of the error test of Hageman &
// Young's adaptive SOR procedure (Applied Iterative Methods, 1981, ch. 9),
// with the change over a whole check interval in place of a single sweep's:
// near omega = 2 the FP32 rounding noise in the change is amplified by
// 1 / (1 - rho^Tl), far less over an interval than over one sweep.  d < 0
// means no change was measured.  Past the optimal omega the eigenvalues are
// complex and the error turns as well as shrinks, so over one interval a
// cell can come back close to where it was: relax_control keeps the larger of
// the last two checks' estimates (on 48 seeded scenes of 256-512 cells a side
// with 5-35 % obstacles that larger one was never below 0.98 times the true
// error after the residual test had been met; a single check's estimate went
// down to 0.36 times).
__host__ __device__ inline double relax_error_estimate(const RelaxCtl &c, double d) {
    if (!(d >= 0.0)) return DBL_MAX;
    double rho = c.omega - 1.0 > c.lam ? c.omega - 1.0 : c.lam;
    if (rho < 0.0) rho = 0.0;
    if (rho > 0.9999) rho = 0.9999;
    return d / (1.0 - pow(rho, (double)(c.Tl > 0 ? c.Tl : 1)));
}

// One residual check: stop test, over-relaxation back-off at the rounding
// floor, adaptive omega.  r is the residual max (the stopping quantity); e,
// when positive, its 2-norm, from which the decay rate that drives omega is
// estimated (smoother than the max, whose location jumps between cells).
// d is the largest change of a free cell since the previous check's snapshot
// (< 0: not measured), used only with an error tolerance (c.etol > 0).  Then
// the solve waits for both r <= tol and relax_error_estimate <= etol; the
// over-relaxation back-off below is not used (it meets the residual test by
// slowing the smooth error's decay, which leaves that error behind), omega is
// frozen from the first check that meets the residual test on, so that the
// rate the estimate assumes is the iteration's own, and a check whose
// estimate is met while the FP32 rounding noise of SOR at omega near 2 keeps
// r above tol tries the polish (relax_polish_decide).  If the estimate and the
// residual both stop falling for kErrStall checks, the error target cannot be
// shown in FP32 and the solve ends unconverged instead of running to the cap
// (counted only once r < kStallFactor * tol: far from the tolerance the
// residual of an open field can hover for many intervals while it converges).
// The snapshot the change is measured against is taken from the first check
// with r < kSnapFactor * tol on (with tol = 0: from the first check).
// Returns 1 to continue, 0 when converged.
constexpr int kErrStall = 4;
constexpr double kStallFactor = 16.0;
constexpr double kSnapFactor = 100.0;
__host__ __device__ inline int relax_control(RelaxCtl &c, double r, double e, int n, double d) {
    c.checks++;
    c.r_last = r;
    if (c.etol > 0.0) {
        // the 2-norm's decay rate, kept from the last interval over which it still fell clearly
        if (e > 0.0 && c.e_prev > 0.0 && n == c.K && e <= 0.8 * c.e_prev) c.lam = pow(e / c.e_prev, 1.0 / n);
        const bool r_ok = c.tol > 0.0 ? r <= c.tol : true;
        if (r_ok) c.r_met = 1;
        const double raw = relax_error_estimate(c, d);
        c.err_est = raw > c.err_raw ? raw : c.err_raw;
        c.err_raw = raw;
        if (r_ok && c.err_est <= c.etol) {
            c.status = TW_OK;
            return 0;
        }
        if (c.snap || c.tol <= 0.0 || r < kSnapFactor * c.tol) c.snap = c.snap ? 2 : 1;
        const bool stalled = c.err_prev > 0.0 && c.err_est > 0.9 * c.err_prev && c.r_prev > 0.0 &&
                             r > 0.8 * c.r_prev && (c.tol <= 0.0 || r < kStallFactor * c.tol);
        c.stall = stalled ? c.stall + 1 : 0;
        c.err_prev = c.err_est;
        if (c.stall >= kErrStall) {
            c.status = TW_NOT_CONVERGED;
            return 0;
        }
        if (c.r_met) {
            c.r_prev = r;
            c.e_prev = e;
            return 1;
        }
    } else if (c.tol > 0.0 && r <= c.tol) {
        c.status = TW_OK;
        return 0;
    }
    // Stagnation over a whole interval close to the tolerance means the FP32
    // rounding floor, which over-relaxation amplifies by about
    // omega / (2 - omega): halve the over-relaxation and stop adapting
    // upwards.  (Far from the tolerance the max-norm can plateau while the
    // iteration still converges, so it is left alone there.)
    if (c.etol <= 0.0 && c.r_prev > 0.0 && n == c.K && r > 0.8 * c.r_prev && r < 16.0 * c.tol && c.omega > 1.0) {
        c.omega = 1.0 + 0.5 * (c.omega - 1.0);
        if (c.omega < 1.05) c.omega = 1.0;
        c.adapt = 0;
        c.same_iv = 0;
    } else if (c.adapt) {
        if (c.r_prev > 0.0 && c.same_iv >= 1 && n == c.K) {
            const bool l2 = !c.maxnorm_adapt && e > 0.0 && c.e_prev > 0.0;
            double lambda = pow(l2 ? e / c.e_prev : r / c.r_prev, 1.0 / n);
            double w = sor_adapt(c.omega, lambda, c.omega_max);
            if (w > c.omega + 1e-4) { c.omega = w; c.same_iv = -1; }
        }
        c.same_iv++;
    }
    c.r_prev = r;
    c.e_prev = e;
    c.omega_f = (float)c.omega;
    return 1;
}

// Polish (HP_POLISH): a stopping-test device beside the SOR iteration, not
// part of it.  Near convergence at omega close to 2 the residual max is
// dominated by oscillatory error that SOR damps only at the rate omega - 1
// while Gauss-Seidel (omega = 1) removes it in a few sweeps.  When a check
// finds r < kPolishFactor * tol, one launch of T sweeps at omega = 1 runs from
// the current ping-pong planes into the other pair and its residual is
// checked: at or below tol that copy is the solution; otherwise it is dropped
// and SOR continues from the unpolished planes, whose sequence it leaves
// untouched.  The smooth error stays, so at the same tol the polished field is
// less accurate than the one SOR would reach.
constexpr double kPolishFactor = 100.0;

// After relax_control returned cont: decide whether this check polishes.
// With an error tolerance the polish removes the rounding noise that keeps r
// above tol once the error estimate is met (the estimate, not the residual,
// then says the smooth error is small enough).
__host__ __device__ inline int relax_polish_decide(RelaxCtl &c, int cont) {
    if (c.etol > 0.0)
        c.polish = (cont && c.polish_ok && c.tol > 0.0 && c.r_last > c.tol && c.err_est <= c.etol) ? 1 : 0;
    else
        c.polish = (cont && c.polish_ok && c.tol > 0.0 && c.r_last < kPolishFactor * c.tol && c.omega >= 1.5) ? 1 : 0;
    return c.polish;
}

// The polished copy's residual r2: returns 0 when it meets the tolerance.
__host__ __device__ inline int relax_polish_result(RelaxCtl &c, double r2) {
    c.polishes++;
    c.psweeps += c.T;
    if (r2 <= c.tol) {
        c.status = TW_OK;
        c.in_alt = 1;
        c.r_last = r2;
        return 0;
    }
    return 1;
}

// NaN or overflow must never look converged: map them to +inf before a max.
__device__ __forceinline__ float sane(float r) { return (r <= FLT_MAX) ? r : __int_as_float(0x7f800000); }
__device__ __forceinline__ double sane(double r) { return (r <= DBL_MAX) ? r : __longlong_as_double(0x7ff0000000000000LL); }

// Block-wide max of a non-negative float, one atomicMax per CTA on its bits.
__device__ __forceinline__ void block_max_atomic(float r, unsigned int *out) {
    __shared__ float sm[32];
    r = sane(r);
    for (int o = 16; o > 0; o >>= 1) r = fmaxf(r, __shfl_xor_sync(0xffffffffu, r, o));
    int t = threadIdx.y * blockDim.x + threadIdx.x;
    int nt = blockDim.x * blockDim.y;
    if ((t & 31) == 0) sm[t >> 5] = r;
    __syncthreads();
    if (t < 32) {
        r = (t < (nt + 31) / 32) ? sm[t] : 0.0f;
        for (int o = 16; o > 0; o >>= 1) r = fmaxf(r, __shfl_xor_sync(0xffffffffu, r, o));
        if (t == 0 && r > 0.0f) atomicMax(out, __float_as_uint(r));
    }
}

// Knuth's TwoSum: s + e == a + b exactly (s = fl(a + b)).
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// |(1/4)(l + r + u + d) - c| for FP32 inputs in compensated FP32: TwoSum on
// every addition (the scaling by 1/4 is exact), the result kept as an
// unevaluated pair hi + lo of floats (hi >= 0, |lo| <= ulp(hi) / 2, so pairs
// order lexicographically as their exact values do).  hi + lo is the FP64
// evaluation of the residual to about 2^-45 relative to the inputs' magnitude,
// at FP32 cost (FP64 throughput is a small fraction of FP32 on this GPU);
// only the CTA's maximum is converted to FP64.
__device__ __forceinline__ void resid_pair(float l, float r, float u, float d, float c, float &hi, float &lo) {
    float s1, e1, s2, e2, s3, e3, dd, e4;
    two_sum(l, r, s1, e1);
    two_sum(u, d, s2, e2);
    two_sum(s1, s2, s3, e3);
    const float low = __fadd_rn(__fadd_rn(e1, e2), e3);
    two_sum(__fmul_rn(0.25f, s3), -c, dd, e4);
    two_sum(dd, __fadd_rn(__fmul_rn(0.25f, low), e4), hi, lo);
    if (hi < 0.0f || (hi == 0.0f && lo < 0.0f)) {
        hi = -hi;
        lo = -lo;
    }
    if (!(hi <= FLT_MAX)) {   // NaN or overflow must never look converged
        hi = __int_as_float(0x7f800000);
        lo = 0.0f;
    }
}

__device__ __forceinline__ void pair_max(float &hi, float &lo, float h2, float l2) {
    if (h2 > hi || (h2 == hi && l2 > lo)) {
        hi = h2;
        lo = l2;
    }
}

// Block-wide max of residual pairs and sum of squares: FP32 shuffles, then one
// FP64 atomicMax (bits of a non-negative double) and one FP64 atomicAdd per CTA.
__device__ __forceinline__ void block_max_sum_pair(float hi, float lo, float q, unsigned long long *out_max,
                                                   double *out_sum) {
    __shared__ float sh[32], sl[32], sq[32];
    for (int o = 16; o > 0; o >>= 1) {
        pair_max(hi, lo, __shfl_xor_sync(0xffffffffu, hi, o), __shfl_xor_sync(0xffffffffu, lo, o));
        q += __shfl_xor_sync(0xffffffffu, q, o);
    }
    const int t = threadIdx.y * blockDim.x + threadIdx.x;
    const int nt = blockDim.x * blockDim.y;
    if ((t & 31) == 0) {
        sh[t >> 5] = hi;
        sl[t >> 5] = lo;
        sq[t >> 5] = q;
    }
    __syncthreads();
    if (t < 32) {
        const bool in = t < (nt + 31) / 32;
        hi = in ? sh[t] : 0.0f;
        lo = in ? sl[t] : 0.0f;
        q = in ? sq[t] : 0.0f;
        for (int o = 16; o > 0; o >>= 1) {
            pair_max(hi, lo, __shfl_xor_sync(0xffffffffu, hi, o), __shfl_xor_sync(0xffffffffu, lo, o));
            q += __shfl_xor_sync(0xffffffffu, q, o);
        }
        if (t == 0) {
            const double r = (double)hi + (double)lo;
            if (r > 0.0) atomicMax(out_max, (unsigned long long)__double_as_longlong(r));
            if (q != 0.0f) atomicAdd(out_sum, (double)q);
        }
    }
}

// Block-wide FP64 max (atomicMax on the bits of a non-negative double) and sum.
__device__ __forceinline__ void block_max_sum_f64(double r, unsigned long long *out_max, double *out_sum) {
    __shared__ double smx[32], sms[32];
    r = sane(r);
    double s = r * r;
    for (int o = 16; o > 0; o >>= 1) {
        r = fmax(r, __shfl_xor_sync(0xffffffffu, r, o));
        s += __shfl_xor_sync(0xffffffffu, s, o);
    }
    int t = threadIdx.y * blockDim.x + threadIdx.x;
    int nt = blockDim.x * blockDim.y;
    if ((t & 31) == 0) { smx[t >> 5] = r; sms[t >> 5] = s; }
    __syncthreads();
    if (t < 32) {
        bool in = t < (nt + 31) / 32;
        r = in ? smx[t] : 0.0;
        s = in ? sms[t] : 0.0;
        for (int o = 16; o > 0; o >>= 1) {
            r = fmax(r, __shfl_xor_sync(0xffffffffu, r, o));
            s += __shfl_xor_sync(0xffffffffu, s, o);
        }
        if (t == 0) {
            if (r > 0.0) atomicMax(out_max, (unsigned long long)__double_as_longlong(r));
            if (s != 0.0) atomicAdd(out_sum, s);
        }
    }
}

// Neighbours of the 4 cells k..k+3 of one colour in row y: other-colour
// values left/right (same row, k+s-1 and k+s) and up/down (rows y-1, y+1, k).
// nb[0] = left, nb[1] = right, nb[2] = up, nb[3] = down (component = cell).
__device__ __forceinline__ void rb_load_neighbours(const float *V, int S, int y, int k, int s, float4 nb[4]) {
    const float *row = V + (size_t)y * S + 4;
    float4 mid = *reinterpret_cast<const float4 *>(row + k);
    float extra = s ? row[k + 4] : row[k - 1];
    nb[2] = *reinterpret_cast<const float4 *>(row - S + k);
    nb[3] = *reinterpret_cast<const float4 *>(row + S + k);
    if (s) {
        nb[0] = mid;
        nb[1] = make_float4(mid.y, mid.z, mid.w, extra);
    } else {
        nb[0] = make_float4(extra, mid.x, mid.y, mid.z);
        nb[1] = mid;
    }
}

}  // namespace tw
