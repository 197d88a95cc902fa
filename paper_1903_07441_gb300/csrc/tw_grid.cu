// Time-warped occupancy grid (Sec. 3.4-3.5, Alg. 1 "Map Update").
//
// Three launches, all stream-ordered:
//   tw_ring_table_kernel  1 thread: ring radii R_j, arrival times t_j and their
//                         fixed-point forms (the recurrence is serial and tiny)
//   tw_predict_kernel     1 thread per (track, ring) [per-cell marking] or per
//                         track [per-obstacle marking]: Eqs. 9-10 at t_j and the
//                         inflated disk, in correctly rounded FP64 (explicit
//                         _rn intrinsics, so no contraction can change a bit)
//   tw_raster_kernel      1 CTA per 32x32 tile: ring of every cell, candidate
//                         disks binned in shared memory per tile, exact integer
//                         predicates, occupancy codes written once.
// The raster is integer/ALU work (a few bytes of HBM per cell).
#include <math.h>
#include <string.h>

#include <mutex>
#include <vector>

#include "common.cuh"

namespace tw {

constexpr int kMaxRings = 64;
constexpr int kMaxGridJobs = 1 << 16;
constexpr long long kCoordClamp = 1LL << 30;
constexpr long long kRadiusClamp = 1LL << 29;

struct RingTab {
    int J, kind, mark, pad;
    long long rxq, ryq, hxq, hyq;
    double t[kMaxRings];
    long long Rq[kMaxRings];   // ring radius, 1/256 cell
    long long Aq[kMaxRings];   // elliptic semi-major axis, 2^-28 cell
    long long Cq[kMaxRings];   // elliptic centre offset 0.9 R, 2^-28 cell
};

struct Disk {
    int px, py;      // predicted centre, 1/256 cell (clamped to +-2^30)
    int j, pad;      // ring the disk belongs to; -1: every ring (per-obstacle marking)
    long long r2;    // squared inflated radius, (1/256 cell)^2
};

struct Params {
    int nx, ny, n, mark, kind, n_rings, time_outer, pad;
    double cell, ox, oy;
    double rx, ry, hx, hy, speed;
    double r0, growth, q, kappa, d_safe;
    double alpha;    // probability-threshold factor of the marking (0: every prediction is marked)
};

__device__ __forceinline__ long long qclamp(double v, long long lo, long long hi) {
    double r = rint(v);
    if (r < (double)lo) return lo;
    if (r > (double)hi) return hi;
    return (long long)r;
}

__device__ __forceinline__ long long qpos(double v, double origin, double cell) {
    return qclamp(__dmul_rn(__ddiv_rn(__dsub_rn(v, origin), cell), 256.0), -kCoordClamp, kCoordClamp);
}

// One thread per ring: thread j repeats the recurrence R_j = growth * R_{j-1}
// from r0 (the same rounded products as a serial loop), so the whole table
// costs one ring's latency.  The ring count J is the number of rings below
// the reach plus one (the radii increase).
__device__ __forceinline__ void ring_table_body(const Params &p, RingTab *tab) {
    const int j = threadIdx.x;   // blockDim.x == kMaxRings
    double w = __dmul_rn((double)p.nx, p.cell), h = __dmul_rn((double)p.ny, p.cell);
    double reach = __dsqrt_rn(__dadd_rn(__dmul_rn(w, w), __dmul_rn(h, h)));
    if (p.kind == TW_RING_ELLIPTIC) reach = __dmul_rn(reach, 10.0);
    double r = p.r0, rprev = 0.0;
    for (int i = 0; i < j; i++) {
        rprev = r;
        r = __dmul_rn(r, p.growth);
    }
    const int below = __syncthreads_count(r < reach);
    int J = (p.n_rings > 0) ? p.n_rings : below + 1;
    if (J > kMaxRings) J = -1;
    if (j == 0) {
        tab->J = J;
        tab->kind = p.kind;
        tab->mark = p.mark;
        tab->rxq = qpos(p.rx, p.ox, p.cell);
        tab->ryq = qpos(p.ry, p.oy, p.cell);
        tab->hxq = qclamp(__dmul_rn(p.hx, 1048576.0), -1048576, 1048576);
        tab->hyq = qclamp(__dmul_rn(p.hy, 1048576.0), -1048576, 1048576);
    }
    if (J < 0 || j >= J) return;
    double t;
    if (p.time_outer) t = __ddiv_rn(r, p.speed);
    else t = (j == 0) ? 0.0 : __ddiv_rn(rprev, p.speed);
    tab->t[j] = t;
    tab->Rq[j] = qclamp(__dmul_rn(__ddiv_rn(r, p.cell), 256.0), 0, kRadiusClamp);
    tab->Aq[j] = qclamp(__dmul_rn(__ddiv_rn(r, p.cell), 268435456.0), 0, 1LL << 52);
    tab->Cq[j] = qclamp(__dmul_rn(__ddiv_rn(__dmul_rn(0.9, r), p.cell), 268435456.0), 0, 1LL << 52);
}

__global__ void tw_ring_table_kernel(Params p, RingTab *tab) { ring_table_body(p, tab); }

// Smallest ring containing the fixed-point offset (dx, dy); the last ring otherwise.
__device__ __forceinline__ int ring_index(int kind, int J, long long dx, long long dy,
                                          const long long *Rq, const long long *Aq,
                                          const long long *Cq, long long hxq, long long hyq) {
    if (kind == TW_RING_CIRCULAR) {
        // the radii increase: binary search for the first ring with d2 <= Rq_j^2
        const long long d2 = dx * dx + dy * dy;
        if (d2 > Rq[J - 1] * Rq[J - 1]) return J - 1;
        int lo = 0, hi = J - 1;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (d2 <= Rq[mid] * Rq[mid]) hi = mid;
            else lo = mid + 1;
        }
        return lo;
    } else {
        __int128 u = (__int128)(hxq * dx + hyq * dy);
        __int128 v = (__int128)(hxq * dy - hyq * dx);
        __int128 v16 = 16 * v * v;
        for (int j = 0; j < J; j++) {
            __int128 a = u - (__int128)Cq[j];
            if (a * a + v16 <= (__int128)Aq[j] * (__int128)Aq[j]) return j;
        }
    }
    return J - 1;
}

// Constant-velocity prediction at time t and the inflated, quantised disk.
__device__ Disk predict_disk(const tw_track &T, double t, const Params &p, int j) {
    const double *P = T.P;
    double px = __dadd_rn(T.x[0], __dmul_rn(t, T.x[2]));
    double py = __dadd_rn(T.x[1], __dmul_rn(t, T.x[3]));
    double qt3 = __ddiv_rn(__dmul_rn(__dmul_rn(__dmul_rn(p.q, t), t), t), 3.0);
    double two_t = __dmul_rn(2.0, t), tt = __dmul_rn(t, t);
    double pxx = __dadd_rn(__dadd_rn(__dadd_rn(P[0], __dmul_rn(two_t, P[2])), __dmul_rn(tt, P[10])), qt3);
    double pyy = __dadd_rn(__dadd_rn(__dadd_rn(P[5], __dmul_rn(two_t, P[7])), __dmul_rn(tt, P[15])), qt3);
    double s2 = __dmul_rn(0.5, __dadd_rn(pxx, pyy));
    double sigma = (s2 > 0.0) ? __dsqrt_rn(s2) : 0.0;
    double rho = __dadd_rn(__dadd_rn(T.radius, p.d_safe), __dmul_rn(p.kappa, sigma));
    long long rq = qclamp(__dmul_rn(__ddiv_rn(rho, p.cell), 256.0), 0, kRadiusClamp);
    Disk d;
    d.px = (int)qpos(px, p.ox, p.cell);
    d.py = (int)qpos(py, p.oy, p.cell);
    d.j = j;
    d.pad = 0;
    d.r2 = rq * rq;
    if (p.alpha > 0.0) {   // too uncertain to place: below the marking probability, no disk (r2 < 0)
        const double a = __dmul_rn(p.alpha, __dadd_rn(T.radius, p.d_safe));
        if (s2 > __dmul_rn(a, a)) d.r2 = -1;
    }
    return d;
}

// Disk idx of one planner: per-cell marking, idx = track * J + ring over the
// first n * J slots; per-obstacle marking, one disk per track.
__device__ __forceinline__ void predict_body(const Params &p, const RingTab *tab, const tw_track *tracks,
                                             Disk *disks, long long idx) {
    int J = tab->J;
    if (J <= 0) return;
    if (p.mark == TW_MARK_PER_CELL) {
        if (idx >= (long long)p.n * J) return;
        int o = (int)(idx / J), j = (int)(idx % J);
        disks[idx] = predict_disk(tracks[o], tab->t[j], p, j);
    } else {
        if (idx >= p.n) return;
        const tw_track &T = tracks[idx];
        long long dx = qpos(T.x[0], p.ox, p.cell) - tab->rxq;
        long long dy = qpos(T.x[1], p.oy, p.cell) - tab->ryq;
        int own = ring_index(tab->kind, J, dx, dy, tab->Rq, tab->Aq, tab->Cq, tab->hxq, tab->hyq);
        Disk d = predict_disk(T, tab->t[own], p, -1);
        disks[idx] = d;
    }
}

__global__ void tw_predict_kernel(Params p, const RingTab *tab, const tw_track *tracks, Disk *disks) {
    predict_body(p, tab, tracks, disks, (long long)blockIdx.x * blockDim.x + threadIdx.x);
}

constexpr int kTile = 32;            // 32x32 cells per CTA
constexpr int kRasterThreads = 256;  // 4 cells per thread
constexpr int kChunk = 1024;         // disks examined per binning round

// Tile (bx, by) of one planner's raster (one CTA of kRasterThreads threads).
__device__ __forceinline__ void raster_body(const Params &p, const RingTab *tab, const Disk *disks,
                                            const uint8_t *static_occ, uint8_t *occ, int16_t *ring_out, int bx,
                                            int by) {
    __shared__ long long sRq[kMaxRings], sAq[kMaxRings], sCq[kMaxRings];
    __shared__ Disk sList[kChunk];
    __shared__ int sCount, sJmin, sJmax;
    __shared__ unsigned int sCover[2];   // rings whose cells in this tile a disk covers entirely
    const int tid = threadIdx.x;
    const int J = tab->J;
    const int kind = tab->kind;
    if (J <= 0) return;
    // disk count from the device-side ring table (the predict kernel used the same J)
    const int n_disks = (p.mark == TW_MARK_PER_CELL) ? p.n * J : p.n;
    for (int j = tid; j < J; j += kRasterThreads) {
        sRq[j] = tab->Rq[j];
        sAq[j] = tab->Aq[j];
        sCq[j] = tab->Cq[j];
    }
    if (tid == 0) { sJmin = 1 << 30; sJmax = -1; sCount = 0; sCover[0] = 0u; sCover[1] = 0u; }
    __syncthreads();
    const long long rxq = tab->rxq, ryq = tab->ryq, hxq = tab->hxq, hyq = tab->hyq;
    const int x0 = bx * kTile, y0 = by * kTile;
    const int lx = tid % kTile;
    const int x = x0 + lx;
    int rj[4];
    uint8_t code[4];
    int jmin = 1 << 30, jmax = -1;
#pragma unroll
    for (int r = 0; r < 4; r++) {
        int y = y0 + tid / kTile + 8 * r;
        rj[r] = -1;
        code[r] = TW_FREE;
        if (x < p.nx && y < p.ny) {
            long long cx = 256LL * x + 128, cy = 256LL * y + 128;
            rj[r] = ring_index(kind, J, cx - rxq, cy - ryq, sRq, sAq, sCq, hxq, hyq);
            size_t c = (size_t)y * p.nx + x;
            if (x == 0 || y == 0 || x == p.nx - 1 || y == p.ny - 1) code[r] = TW_BORDER;
            else if (static_occ && static_occ[c]) code[r] = TW_STATIC;
            if (code[r] == TW_FREE) { jmin = min(jmin, rj[r]); jmax = max(jmax, rj[r]); }
        }
    }
    atomicMin(&sJmin, jmin);
    atomicMax(&sJmax, jmax);
    __syncthreads();
    const int tjmin = sJmin, tjmax = sJmax;
    // tile bounds in fixed point (cell centres)
    const long long bx0 = 256LL * x0 + 128, by0 = 256LL * y0 + 128;
    const long long bx1 = 256LL * min(x0 + kTile - 1, p.nx - 1) + 128;
    const long long by1 = 256LL * min(y0 + kTile - 1, p.ny - 1) + 128;
    if (tjmax >= 0) {
        // candidates: per-cell marking, only the disks of the tile's rings
        // [tjmin, tjmax] (disk o * J + j), in index order; per obstacle, all
        const bool per_cell = p.mark == TW_MARK_PER_CELL;
        const int w = per_cell ? tjmax - tjmin + 1 : 1;
        const int n_cand = per_cell ? p.n * w : n_disks;
        for (int base = 0; base < n_cand; base += kChunk) {
            int lim = min(kChunk, n_cand - base);
            for (int k = tid; k < lim; k += kRasterThreads) {
                const int c = base + k;
                Disk d = disks[per_cell ? (c / w) * J + tjmin + c % w : c];
                if (d.j >= 0 && (d.j < tjmin || d.j > tjmax)) continue;
                long long ex = max(0LL, max(bx0 - (long long)d.px, (long long)d.px - bx1));
                long long ey = max(0LL, max(by0 - (long long)d.py, (long long)d.py - by1));
                if (ex * ex + ey * ey <= d.r2) {
                    // the farthest corner of the tile's cell-centre box inside the disk: the (convex)
                    // disk holds every cell centre of the tile, so its ring is covered outright
                    long long fx = max((long long)d.px - bx0, bx1 - (long long)d.px);
                    long long fy = max((long long)d.py - by0, by1 - (long long)d.py);
                    if (fx * fx + fy * fy <= d.r2) {
                        if (d.j >= 0) {
                            atomicOr(&sCover[d.j >> 5], 1u << (d.j & 31));
                        } else {
                            atomicOr(&sCover[0], ~0u);
                            atomicOr(&sCover[1], ~0u);
                        }
                    } else {
                        int slot = atomicAdd(&sCount, 1);
                        sList[slot] = d;
                    }
                }
            }
            __syncthreads();
            const int cnt = sCount;
            const unsigned int cov0 = sCover[0], cov1 = sCover[1];
#pragma unroll
            for (int r = 0; r < 4; r++) {
                if (code[r] != TW_FREE || rj[r] < 0) continue;
                if (((rj[r] < 32 ? cov0 : cov1) >> (rj[r] & 31)) & 1u) { code[r] = TW_DYNAMIC; continue; }
                int y = y0 + tid / kTile + 8 * r;
                long long cx = 256LL * x + 128, cy = 256LL * y + 128;
                for (int k = 0; k < cnt; k++) {
                    const Disk &d = sList[k];
                    if (d.j >= 0 && d.j != rj[r]) continue;
                    long long dx = cx - d.px, dy = cy - d.py;
                    if (dx * dx + dy * dy <= d.r2) { code[r] = TW_DYNAMIC; break; }
                }
            }
            __syncthreads();
            if (tid == 0) sCount = 0;
            __syncthreads();
        }
    }
#pragma unroll
    for (int r = 0; r < 4; r++) {
        int y = y0 + tid / kTile + 8 * r;
        if (x < p.nx && y < p.ny) {
            size_t c = (size_t)y * p.nx + x;
            occ[c] = code[r];
            if (ring_out) ring_out[c] = (int16_t)rj[r];
        }
    }
}

__global__ void __launch_bounds__(kRasterThreads)
tw_raster_kernel(Params p, const RingTab *tab, const Disk *disks, const uint8_t *static_occ, uint8_t *occ,
                 int16_t *ring_out) {
    raster_body(p, tab, disks, static_occ, occ, ring_out, (int)blockIdx.x, (int)blockIdx.y);
}

// ---- many planners in three launches ----------------------------------------
// Per planner: its parameters, ring table, output pointers and its ranges in
// the concatenated tracks, disk slots (n_tracks * kMaxRings each) and tiles.
struct JobPtrs {
    const uint8_t *static_occ;
    uint8_t *occ;
    int16_t *ring;
    long long track_off, slot_off;
    int tile_off, tiles_x;
};

// Largest i in [0, n) with off[i] <= v (off non-decreasing, off[0] = 0 <= v).
template <class I>
__device__ __forceinline__ int job_of(const I *off, int n, long long v) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if ((long long)off[mid] <= v) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__global__ void tw_ring_table_batch_kernel(const Params *P, RingTab *tabs) {
    const Params p = P[blockIdx.x];
    ring_table_body(p, tabs + blockIdx.x);
}

__global__ void tw_predict_batch_kernel(const Params *P, const RingTab *tabs, const tw_track *tracks, Disk *disks,
                                        const long long *slot_off, const JobPtrs *jobs, int n) {
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= slot_off[n]) return;
    // the planner whose slot range holds g (planners without tracks have empty ranges)
    const int i = job_of(slot_off, n + 1, g);
    const Params p = P[i];
    predict_body(p, tabs + i, tracks + jobs[i].track_off, disks + slot_off[i], g - slot_off[i]);
}

__global__ void __launch_bounds__(kRasterThreads)
tw_raster_batch_kernel(const Params *P, const RingTab *tabs, const Disk *disks, const int *tile_off,
                       const JobPtrs *jobs, int n) {
    const int t = (int)blockIdx.x;
    const int i = job_of(tile_off, n + 1, t);
    const Params p = P[i];
    const JobPtrs J = jobs[i];
    const int lt = t - J.tile_off;
    raster_body(p, tabs + i, disks + J.slot_off, J.static_occ, J.occ, J.ring, lt % J.tiles_x, lt / J.tiles_x);
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

static bool finite(double v) { return isfinite(v) != 0; }

static bool valid_grid(const tw_grid *g) {
    return g && g->nx >= 3 && g->ny >= 3 && g->nx <= 65535 && g->ny <= 65535 && finite(g->cell) &&
           g->cell > 0.0 && finite(g->ox) && finite(g->oy);
}

static bool valid_law(const tw_ring_law *L) {
    return L && (L->kind == TW_RING_CIRCULAR || L->kind == TW_RING_ELLIPTIC) &&
           (L->mark == TW_MARK_PER_CELL || L->mark == TW_MARK_PER_OBSTACLE) && finite(L->r0) &&
           L->r0 > 0.0 && finite(L->growth) && L->growth > 1.0 && L->n_rings >= 0 &&
           L->n_rings <= kMaxRings && finite(L->q_accel) && L->q_accel >= 0.0 &&
           finite(L->kappa) && L->kappa >= 0.0 && finite(L->d_safe) && L->d_safe >= 0.0 &&
           (L->time_outer == 0 || L->time_outer == 1) && finite(L->p_mark) && L->p_mark >= 0.0 &&
           L->p_mark < 1.0;
}

static bool valid_pose(const tw_pose *r) {
    if (!r || !finite(r->x) || !finite(r->y) || !finite(r->hx) || !finite(r->hy) || !finite(r->speed))
        return false;
    double h2 = r->hx * r->hx + r->hy * r->hy;
    return r->speed > 0.0 && h2 > 0.98 && h2 < 1.02;
}

static bool psd2(double a, double b, double c) {  // [[a, b], [b, c]]
    return a >= 0.0 && c >= 0.0 && b * b <= a * c * (1.0 + 1e-9) + 1e-300;
}

static bool valid_track(const tw_track &T) {
    for (int i = 0; i < 4; i++)
        if (!finite(T.x[i])) return false;
    for (int i = 0; i < 16; i++)
        if (!finite(T.P[i])) return false;
    if (!finite(T.radius) || T.radius < 0.0) return false;
    return psd2(T.P[0], T.P[2], T.P[10]) && psd2(T.P[5], T.P[7], T.P[15]);
}

// Ring count by the same recurrence the device runs (IEEE-exact ops on both).
static int ring_count(const tw_grid *g, const tw_pose *robot, const tw_ring_law *L) {
    if (!valid_grid(g) || !valid_law(L) || !valid_pose(robot)) return TW_EINVAL;
    volatile double w = (double)g->nx * g->cell, h = (double)g->ny * g->cell;
    volatile double ww = w * w, hh = h * h;
    volatile double s = ww + hh;
    double reach = sqrt((double)s);
    if (L->kind == TW_RING_ELLIPTIC) reach = reach * 10.0;
    int J = 0;
    volatile double r = L->r0;
    for (;;) {
        if (J >= kMaxRings) return TW_EINVAL;
        J++;
        if (L->n_rings > 0) { if (J == L->n_rings) break; }
        else if (r >= reach) break;
        r = r * L->growth;
    }
    return J;
}

static Params make_params(const tw_grid *g, const tw_pose *robot, const tw_ring_law *law, int n_tracks) {
    Params p;
    memset(&p, 0, sizeof(p));
    p.nx = g->nx; p.ny = g->ny; p.n = n_tracks; p.mark = law->mark; p.kind = law->kind;
    p.n_rings = law->n_rings; p.time_outer = law->time_outer;
    p.cell = g->cell; p.ox = g->ox; p.oy = g->oy;
    p.rx = robot->x; p.ry = robot->y; p.hx = robot->hx; p.hy = robot->hy; p.speed = robot->speed;
    p.r0 = law->r0; p.growth = law->growth; p.q = law->q_accel; p.kappa = law->kappa;
    p.d_safe = law->d_safe;
    // P(|X - p| <= rho0) for X ~ N(p, sigma^2 I2) is 1 - exp(-rho0^2 / (2 sigma^2)) >= p_mark
    // exactly when sigma <= alpha rho0
    p.alpha = law->p_mark > 0.0 ? 1.0 / sqrt(-2.0 * log(1.0 - law->p_mark)) : 0.0;
    return p;
}

// Workspace of tw_build_grids: a head the host fills and copies in one transfer
// (parameters, output pointers, range offsets, all tracks), then the ring
// tables and the disk slots the kernels write.
struct JobsLayout {
    Params *P;
    JobPtrs *jobs;
    int *tile_off;
    long long *slot_off;
    tw_track *tracks;
    size_t head_bytes;
    RingTab *tabs;
    Disk *disks;
};

static size_t carve_jobs(Carver &cv, int n, long long n_tracks, long long n_slots, JobsLayout *out) {
    JobsLayout l;
    l.P = cv.take<Params>(n);
    l.jobs = cv.take<JobPtrs>(n);
    l.tile_off = cv.take<int>(n + 1);
    l.slot_off = cv.take<long long>(n + 1);
    l.tracks = cv.take<tw_track>(n_tracks > 0 ? n_tracks : 1);
    l.head_bytes = cv.need;
    l.tabs = cv.take<RingTab>(n);
    l.disks = cv.take<Disk>(n_slots > 0 ? n_slots : 1);
    if (out) *out = l;
    return cv.need;
}

static bool valid_job(const tw_grid_job &j) {
    if (!valid_grid(&j.grid) || !valid_law(&j.law) || !valid_pose(&j.robot) || !j.occ_dev || j.n_tracks < 0 ||
        (j.n_tracks > 0 && !j.tracks))
        return false;
    for (int o = 0; o < j.n_tracks; o++)
        if (!valid_track(j.tracks[o])) return false;
    return ring_count(&j.grid, &j.robot, &j.law) > 0;
}

struct GridLayout {
    RingTab *tab;
    tw_track *tracks;
    Disk *disks;
};

static size_t carve_grid(Carver &cv, int n_tracks, int J, GridLayout *out) {
    GridLayout l;
    l.tab = cv.take<RingTab>(1);
    l.tracks = cv.take<tw_track>(n_tracks > 0 ? n_tracks : 1);
    l.disks = cv.take<Disk>((size_t)(n_tracks > 0 ? n_tracks : 1) * (size_t)(J > 0 ? J : 1));
    if (out) *out = l;
    return cv.need;
}

}  // namespace tw

namespace tw {

// Nearest free, non-border cell to (x, y): one block scans the grid and keeps
// the minimum of (squared distance << 32 | linear index) -- ties go to the
// lowest index, so the answer is deterministic.
__global__ void __launch_bounds__(1024) nearest_free_kernel(const uint8_t *__restrict__ occ, int nx, int ny, int x,
                                                            int y, unsigned long long *out) {
    __shared__ unsigned long long sm[32];
    unsigned long long best = ~0ull;
    const long long n = (long long)nx * ny;
    for (long long i = threadIdx.x; i < n; i += blockDim.x) {
        const int cx = (int)(i % nx), cy = (int)(i / nx);
        if (cx == 0 || cy == 0 || cx == nx - 1 || cy == ny - 1 || occ[i] != 0) continue;
        const unsigned long long d2 = (unsigned long long)((long long)(cx - x) * (cx - x) + (long long)(cy - y) * (cy - y));
        const unsigned long long key = (d2 << 32) | (unsigned long long)i;
        if (key < best) best = key;
    }
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long v = __shfl_xor_sync(0xffffffffu, best, o);
        if (v < best) best = v;
    }
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = best;
    __syncthreads();
    if (threadIdx.x < 32) {
        best = sm[threadIdx.x];
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long v = __shfl_xor_sync(0xffffffffu, best, o);
            if (v < best) best = v;
        }
        if (threadIdx.x == 0) *out = best;
    }
}

}  // namespace tw

using namespace tw;

extern "C" int tw_nearest_free(const tw_grid *g, const uint8_t *occ_dev, int x, int y, int *xy_host, void *workspace,
                               size_t workspace_bytes, void *stream) {
    // the (squared distance, index) key packs both in 32 bits each
    if (!valid_grid(g) || !occ_dev || !xy_host || x < 0 || y < 0 || x >= g->nx || y >= g->ny ||
        (double)g->nx * g->nx + (double)g->ny * g->ny >= 4294967296.0)
        return TW_EINVAL;
    if (!workspace || !ws_aligned(workspace) || workspace_bytes < sizeof(unsigned long long)) return TW_EWORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    unsigned long long *dkey = (unsigned long long *)workspace;
    TW_LAUNCH(nearest_free_kernel, 1, 1024, 0, s, occ_dev, g->nx, g->ny, x, y, dkey);
    TW_CHECK_LAUNCH();
    unsigned long long key = 0;
    TW_CUDA(cudaMemcpyAsync(&key, dkey, sizeof(key), cudaMemcpyDeviceToHost, s));
    TW_CUDA(cudaStreamSynchronize(s));
    if (key == ~0ull) return TW_NO_PATH;
    const unsigned long long idx = key & 0xffffffffull;
    xy_host[0] = (int)(idx % (unsigned long long)g->nx);
    xy_host[1] = (int)(idx / (unsigned long long)g->nx);
    return TW_OK;
}

extern "C" int tw_ring_count(const tw_grid *g, const tw_pose *robot, const tw_ring_law *law) {
    return ring_count(g, robot, law);
}

extern "C" size_t tw_build_grid_workspace_size(const tw_grid *g, int n_tracks, const tw_ring_law *law) {
    (void)g;
    (void)law;
    Carver cv;
    return carve_grid(cv, n_tracks < 0 ? 0 : n_tracks, kMaxRings, nullptr);
}

extern "C" int tw_build_grid(const tw_grid *g, const tw_pose *robot, const tw_track *tracks,
                             int n_tracks, const tw_ring_law *law, const uint8_t *static_occ_dev,
                             uint8_t *occ_dev, int16_t *ring_dev, void *workspace,
                             size_t workspace_bytes, void *stream) {
    if (!valid_grid(g) || !valid_law(law) || !valid_pose(robot) || !occ_dev || n_tracks < 0 ||
        (n_tracks > 0 && !tracks))
        return TW_EINVAL;
    for (int o = 0; o < n_tracks; o++)
        if (!valid_track(tracks[o])) return TW_EINVAL;
    int J = ring_count(g, robot, law);
    if (J <= 0) return TW_EINVAL;
    if (!workspace || !ws_aligned(workspace)) return TW_EWORKSPACE;
    Carver cv(workspace, workspace_bytes);
    GridLayout L;
    carve_grid(cv, n_tracks, kMaxRings, &L);
    if (!cv.ok()) return TW_EWORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    const Params p = make_params(g, robot, law, n_tracks);

    if (n_tracks > 0)
        TW_CUDA(cudaMemcpyAsync(L.tracks, tracks, sizeof(tw_track) * (size_t)n_tracks,
                                cudaMemcpyHostToDevice, s));
    TW_LAUNCH(tw_ring_table_kernel, 1, kMaxRings, 0, s, p, L.tab);
    TW_CHECK_LAUNCH();
    if (n_tracks > 0) {
        TW_LAUNCH(tw_predict_kernel, ceil_div((size_t)n_tracks * kMaxRings, 128), 128, 0, s, p, L.tab,
                  L.tracks, L.disks);
        TW_CHECK_LAUNCH();
    }
    dim3 grid(ceil_div(g->nx, kTile), ceil_div(g->ny, kTile));
    TW_LAUNCH(tw_raster_kernel, grid, kRasterThreads, 0, s, p, L.tab, L.disks, static_occ_dev, occ_dev,
              ring_dev);
    TW_CHECK_LAUNCH();
    return TW_OK;
}

// Pinned host staging for the head of tw_build_grids, one buffer per device,
// reused across calls and held under a lock from filling to the copy: before
// it is refilled, the copy that last read it has completed (an event recorded
// after that copy).  Pinned memory lets the copy run asynchronously at full
// link speed, where a pageable source would first be staged by the driver.
namespace {
struct PinnedStage {
    int dev;
    char *p;
    size_t cap;
    cudaEvent_t ev;
    bool used;
};
std::mutex g_stage_mutex;
std::vector<PinnedStage> g_stages;
}  // namespace

// Under the lock: a pinned buffer of `bytes` (contents undefined), fill(buf),
// then one asynchronous copy to dst on s.
template <class F>
static int staged_copy(void *dst, size_t bytes, cudaStream_t s, F fill) {
    int dev = 0;
    TW_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lock(g_stage_mutex);
    PinnedStage *st = nullptr;
    for (auto &x : g_stages)
        if (x.dev == dev) st = &x;
    if (!st) {
        PinnedStage ns = {dev, nullptr, 0, nullptr, false};
        TW_CUDA(cudaEventCreateWithFlags(&ns.ev, cudaEventDisableTiming));
        g_stages.push_back(ns);
        st = &g_stages.back();
    }
    if (st->used) TW_CUDA(cudaEventSynchronize(st->ev));   // the last copy out of the buffer is done
    if (st->cap < bytes) {
        if (st->p) cudaFreeHost(st->p);
        st->p = nullptr;
        st->cap = 0;
        const size_t cap = bytes + bytes / 2 + 4096;
        TW_CUDA(cudaMallocHost((void **)&st->p, cap));
        st->cap = cap;
    }
    fill(st->p);
    TW_CUDA(cudaMemcpyAsync(dst, st->p, bytes, cudaMemcpyHostToDevice, s));
    TW_CUDA(cudaEventRecord(st->ev, s));
    st->used = true;
    return TW_OK;
}

extern "C" size_t tw_build_grids_workspace_size(int n, const tw_grid_job *jobs) {
    if (n < 1 || !jobs) return 0;
    long long nt = 0;
    for (int i = 0; i < n; i++) nt += jobs[i].n_tracks > 0 ? jobs[i].n_tracks : 0;
    Carver cv;
    return carve_jobs(cv, n, nt, nt * kMaxRings, nullptr);
}

extern "C" int tw_build_grids(int n, const tw_grid_job *jobs, void *workspace, size_t workspace_bytes,
                              void *stream) {
    if (n < 1 || n > kMaxGridJobs || !jobs) return TW_EINVAL;
    long long nt = 0, tiles = 0;
    for (int i = 0; i < n; i++) {
        if (!valid_job(jobs[i])) return TW_EINVAL;
        nt += jobs[i].n_tracks;
        tiles += (long long)ceil_div(jobs[i].grid.nx, kTile) * ceil_div(jobs[i].grid.ny, kTile);
    }
    if (tiles >= (1LL << 31)) return TW_EINVAL;
    if (!workspace || !ws_aligned(workspace)) return TW_EWORKSPACE;
    Carver cv(workspace, workspace_bytes);
    JobsLayout D;
    carve_jobs(cv, n, nt, nt * kMaxRings, &D);
    if (!cv.ok()) return TW_EWORKSPACE;
    // the head, laid out as on the device, filled in pinned host memory and copied once
    cudaStream_t s = (cudaStream_t)stream;
    int tf = 0;
    long long so = 0;
    int e = staged_copy(workspace, D.head_bytes, s, [&](char *head) {
        Carver hc(head, D.head_bytes);
        JobsLayout H;
        carve_jobs(hc, n, nt, nt * kMaxRings, &H);   // the head part of H lies in `head`
        long long to = 0;
        for (int i = 0; i < n; i++) {
            const tw_grid_job &j = jobs[i];
            H.P[i] = make_params(&j.grid, &j.robot, &j.law, j.n_tracks);
            JobPtrs q;
            q.static_occ = j.static_occ_dev;
            q.occ = j.occ_dev;
            q.ring = j.ring_dev;
            q.track_off = to;
            q.slot_off = so;
            q.tile_off = tf;
            q.tiles_x = (int)ceil_div(j.grid.nx, kTile);
            H.jobs[i] = q;
            H.tile_off[i] = tf;
            H.slot_off[i] = so;
            if (j.n_tracks > 0) memcpy(H.tracks + to, j.tracks, sizeof(tw_track) * (size_t)j.n_tracks);
            to += j.n_tracks;
            so += (long long)j.n_tracks * kMaxRings;
            tf += (int)(ceil_div(j.grid.nx, kTile) * ceil_div(j.grid.ny, kTile));
        }
        H.tile_off[n] = tf;
        H.slot_off[n] = so;
    });
    if (e) return e;
    TW_LAUNCH(tw_ring_table_batch_kernel, n, kMaxRings, 0, s, D.P, D.tabs);
    TW_CHECK_LAUNCH();
    if (so > 0) {
        TW_LAUNCH(tw_predict_batch_kernel, ceil_div((size_t)so, 128), 128, 0, s, D.P, D.tabs, D.tracks, D.disks,
                  D.slot_off, D.jobs, n);
        TW_CHECK_LAUNCH();
    }
    TW_LAUNCH(tw_raster_batch_kernel, (unsigned)tf, kRasterThreads, 0, s, D.P, D.tabs, D.disks, D.tile_off, D.jobs,
              n);
    TW_CHECK_LAUNCH();
    return TW_OK;
}
