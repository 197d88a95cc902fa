/*
 * twgrid.h -- C ABI of the GB300 time-warped-grid planner library (libtwgrid.so).
 *
 * The library implements the data-parallel hot path of Farzan & DeSouza,
 * "Path Planning in Dynamic Environments Using Time-Warped Grids and a
 * Parallel Implementation": rasterising the time-warped occupancy grid
 * (Sec. 3.4-3.5, Alg. 1 "Map Update") and relaxing the harmonic potential
 * field (Sec. 3.1, Eqs. 1-2, Alg. 1 "Path Planning"), with the Eq. 3 path
 * and the rubber band of Sec. 3.2 as consumers.  All compute runs in CUDA
 * kernels for sm_103a; the host code validates arguments, sizes launches and
 * reads back small results.
 *
 * Conventions for every call:
 *  - Grids are row-major [ny][nx]; cell (i, j) is column i, row j.  World
 *    coordinates are metres; cell (i, j) spans [ox + i*cell, ox + (i+1)*cell).
 *  - "_dev" pointers are CUDA device pointers on the current device, owned by
 *    the caller; the library never frees or retains them after a call returns.
 *  - `workspace`/`workspace_bytes` is caller-owned device scratch of at least
 *    the size the matching *_workspace_size() call returns, 256-byte aligned.
 *    It may be reused between calls on the same stream.
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).  Work is
 *    enqueued on it; calls that return host-visible results synchronise it.
 *  - Return value: TW_OK (0), a positive warning, or a negative error.  On an
 *    error nothing is guaranteed about outputs.  TW_ECUDA keeps the CUDA
 *    error, readable through tw_last_cuda_error().
 */
#ifndef TWGRID_H
#define TWGRID_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define TW_OK 0
#define TW_NOT_CONVERGED 1     /* max_sweeps reached before tol; stats hold the residual */
#define TW_NO_PATH 2           /* the Eq. 3 descent stalled or exceeded max_len */
#define TW_EINVAL (-1)         /* bad argument (sizes, NaN, non-PSD covariance, ...) */
#define TW_EGOAL_BLOCKED (-2)  /* goal cell occupied, on the border or out of range */
#define TW_ESTART_BLOCKED (-3) /* start cell occupied */
#define TW_ECUDA (-4)          /* a CUDA call failed */
#define TW_EWORKSPACE (-5)     /* workspace missing, too small or misaligned */

/* ---- enums --------------------------------------------------------------- */
#define TW_RING_CIRCULAR 0     /* rings are circles about the robot (geometric radii) */
#define TW_RING_ELLIPTIC 1     /* Eqs. 14-15: ellipses r_x = 4 r_y, centre 0.9 r_x ahead */
#define TW_MARK_PER_CELL 0     /* a cell in ring j is tested against every obstacle at t_j */
#define TW_MARK_PER_OBSTACLE 1 /* Alg. 1: each obstacle takes its own ring's time, one disk */

/* occupancy codes written by tw_build_grid (priority border > static > dynamic) */
#define TW_FREE 0
#define TW_STATIC 1
#define TW_DYNAMIC 2
#define TW_BORDER 3

/* ---- plain-data argument structs ----------------------------------------- */
typedef struct {
    int nx, ny;        /* cells; 3 <= nx, ny <= 65535 (a launch dimension per row) */
    double cell;       /* cell side (m), > 0 */
    double ox, oy;     /* world position of the corner of cell (0, 0) (m) */
} tw_grid;

typedef struct {
    double x, y;       /* robot position (m) */
    double hx, hy;     /* heading as a unit vector (no trigonometry on the exact path) */
    double speed;      /* robot speed (m/s), > 0: ring arrival time = ring radius / speed */
} tw_pose;

/* Kalman track of one moving obstacle (Sec. 3.5): state [x, y, vx, vy] (m, m/s),
 * covariance P (4x4 row-major), body radius (m). */
typedef struct {
    double x[4];
    double P[16];
    double radius;
} tw_track;

typedef struct {
    int kind;          /* TW_RING_CIRCULAR or TW_RING_ELLIPTIC */
    int mark;          /* TW_MARK_PER_CELL or TW_MARK_PER_OBSTACLE */
    double r0;         /* first ring radius (m), > 0 */
    double growth;     /* geometric ring growth, > 1 */
    int n_rings;       /* 0: first J with R_{J-1} >= reach (grid diagonal; 10 x for elliptic) */
    double q_accel;    /* white-noise acceleration PSD of Q(t) (m^2/s^3), >= 0 */
    double kappa;      /* inflation in standard deviations, >= 0 */
    double d_safe;     /* safety distance added to the body radius (m), >= 0 */
    int time_outer;    /* 0: t_j = R_{j-1}/v (t_0 = 0); 1: t_j = R_j/v */
    double p_mark;     /* in [0, 1); 0 = off.  Gaussian marking with a probability threshold: with the
                          obstacle centre distributed N(p, sigma^2 I), the chance that it lies within
                          rho0 = radius + d_safe of its predicted position is 1 - exp(-rho0^2 / (2 sigma^2));
                          a prediction whose chance is below p_mark -- sigma > alpha rho0 with
                          alpha = 1 / sqrt(-2 ln(1 - p_mark)) -- marks no cell (too uncertain to place). */
} tw_ring_law;

/* ---- time-warped grid ------------------------------------------------------
 * tw_build_grid: Alg. 1 "Map Update" as one raster (Sec. 3.4-3.5).
 *  1. Ring table: R_0 = r0, R_j = growth * R_{j-1}; arrival t_j (see tw_ring_law).
 *  2. For every track and ring: constant-velocity prediction at t_j (Eqs. 9-10)
 *     p = x + t v, P(t) = A P A^T + Q(t); sigma^2 = (Pxx(t) + Pyy(t)) / 2;
 *     disk radius rho = (radius + d_safe) + kappa * sigma (the Gaussian marking
 *     of Sec. 3.4 made binary; with law.p_mark > 0 no disk where
 *     sigma^2 > (alpha (radius + d_safe))^2).  All of it in correctly rounded FP64, then
 *     quantised to 1/256 cell (round half to even).
 *  3. For every cell: its ring j (smallest ring whose closed boundary contains
 *     the cell centre; beyond the last ring: the last ring) and its code:
 *     TW_BORDER on the outermost rows/columns, else TW_STATIC where
 *     static_occ_dev != 0, else TW_DYNAMIC if the centre lies in a disk of its
 *     ring (per cell) or in any obstacle's own-ring disk (per obstacle), else
 *     TW_FREE.  The predicates are exact integer arithmetic.
 * tracks: HOST array of n_tracks (0 allowed; copied into the workspace).
 * static_occ_dev: device uint8 [ny][nx] or NULL.  occ_dev: device uint8
 * [ny][nx] output.  ring_dev: device int16 [ny][nx] output or NULL.
 * Asynchronous on `stream` (the host track array may be reused on return).
 * Errors: TW_EINVAL (bad grid/law/pose, non-finite track, negative radius,
 * non-PSD position-velocity block), TW_EWORKSPACE, TW_ECUDA.
 */
size_t tw_build_grid_workspace_size(const tw_grid *g, int n_tracks, const tw_ring_law *law);
int tw_build_grid(const tw_grid *g, const tw_pose *robot, const tw_track *tracks, int n_tracks,
                  const tw_ring_law *law, const uint8_t *static_occ_dev, uint8_t *occ_dev,
                  int16_t *ring_dev, void *workspace, size_t workspace_bytes, void *stream);

/* tw_build_grids: tw_build_grid for n planners at once (the batched form of
 * Alg. 1 "Map Update", Sec. 3.4-3.5): every job gets exactly the occupancy
 * and ring codes tw_build_grid gives it, from three launches in all (ring
 * tables, predictions, raster over the concatenated tiles of every grid) and
 * one host-to-device copy of all parameters and tracks.
 * jobs: HOST array of n (1..65536) job descriptions; each tracks array is a
 * HOST array of n_tracks (0 allowed).  The output buffers of different jobs
 * must not overlap.  Asynchronous on `stream`; the host arrays may be reused
 * on return.  Errors: TW_EINVAL (any job invalid as for tw_build_grid, or
 * 2^31 tiles of 32 x 32 cells or more in total), TW_EWORKSPACE, TW_ECUDA.
 * Nothing is launched when an argument is invalid. */
typedef struct {
    tw_grid grid;
    tw_pose robot;
    tw_ring_law law;
    const tw_track *tracks;         /* HOST array of n_tracks */
    int n_tracks;
    const uint8_t *static_occ_dev;  /* device uint8 [ny][nx] or NULL */
    uint8_t *occ_dev;               /* device uint8 [ny][nx] output */
    int16_t *ring_dev;              /* device int16 [ny][nx] output or NULL */
} tw_grid_job;
size_t tw_build_grids_workspace_size(int n, const tw_grid_job *jobs);
int tw_build_grids(int n, const tw_grid_job *jobs, void *workspace, size_t workspace_bytes, void *stream);

/* tw_nearest_free: the free (occ == 0), non-border cell nearest to (x, y)
 * (squared Euclidean distance in cells; ties go to the lowest row-major index),
 * written to host xy_host[0..1].  A replanning loop uses it as the goal when
 * predicted obstacles cover the nominal goal.  workspace: >= 8 bytes of
 * device scratch.  Synchronises `stream`.  (x, y) must lie in the grid and
 * nx^2 + ny^2 < 2^32.  TW_OK, TW_NO_PATH (no free cell), TW_EINVAL,
 * TW_EWORKSPACE, TW_ECUDA. */
int tw_nearest_free(const tw_grid *g, const uint8_t *occ_dev, int x, int y, int *xy_host, void *workspace,
                    size_t workspace_bytes, void *stream);

/* Number of rings tw_build_grid uses for this grid, pose and law (> 0), or TW_EINVAL. */
int tw_ring_count(const tw_grid *g, const tw_pose *robot, const tw_ring_law *law);

/* ---- harmonic potential field ----------------------------------------------- */
#define HP_JACOBI 0        /* Eq. 1, one FP32 sweep per launch: the plain comparison form */
#define HP_RBSOR 1         /* red-black SOR, FP32, temporally blocked (same fixed point) */
#define HP_MIXED 2         /* defect correction: FP64 residual, low-precision correction sweeps */

#define HP_STORE_F32 0
#define HP_STORE_F16 1
#define HP_STORE_BF16 2

#define HP_WARM_START 1    /* field_dev holds the initial guess (same representation as output) */
#define HP_OUT_PHI 2       /* write phi instead of u = 1 - phi */
#define HP_TIMING 4        /* time the sweep kernels with CUDA events on `stream` (stats.sweep_ms);
                              implies HP_HOST_LOOP */
#define HP_HOST_LOOP 8     /* drive the convergence loop from the host (one stream synchronisation per
                              residual check) instead of the default CUDA graph whose conditional
                              while-node runs the check intervals on the device */
#define HP_POLISH 16       /* HP_RBSOR, T > 1: when a check finds r_inf < 100 tol at omega >= 1.5, one
                              launch of T Gauss-Seidel sweeps (omega = 1) runs on a copy of the field;
                              if the copy meets tol it is the result, otherwise it is dropped and SOR
                              goes on unchanged.  At omega near 2 the residual max is dominated by
                              oscillatory error that Gauss-Seidel removes in a few sweeps, so the
                              tolerance is met one or more check intervals earlier -- but the smooth
                              error SOR would have removed in those intervals stays: at the same tol
                              the field is less accurate (still within tau_max * r_inf).  Off by
                              default.  max_sweeps caps the SOR sweeps; polish sweeps are counted in
                              hp_stats.sweeps on top. */

typedef struct {
    int method;        /* HP_JACOBI, HP_RBSOR or HP_MIXED */
    int storage;       /* HP_MIXED only: storage of the correction sweeps (HP_STORE_*) */
    double omega;      /* SOR factor in (0, 2); 0 = adaptive estimate (HP_RBSOR, HP_MIXED) */
    double tol;        /* stop when the residual r_inf <= tol (0: run max_sweeps) */
    int max_sweeps;    /* hard cap on full sweeps, >= 1 */
    int check_every;   /* residual check period in sweeps, rounded up to whole launches (0 = library
                          default: the largest even number of T-sweep launches within 32 sweeps) */
    int tblock;        /* temporal-blocking depth T, sweeps fused per launch (0 = library default):
                          HP_RBSOR takes 1..7 (default 7 on deep tiles when the field has at least
                          96 of them -- about 2048 x 1400 cells and up -- else 4); hp_relax_batched
                          takes 2, 4, 6 or 7 (anything else: autotuned) */
    int flags;         /* HP_WARM_START | HP_OUT_PHI | HP_TIMING | HP_HOST_LOOP | HP_POLISH */
    double etol;       /* HP_RBSOR with T >= 2 (and hp_relax_batched): also require the estimated field
                          error max |u - u*| to be
                          <= etol (0 = off).  The residual test alone does not bound the error well: the
                          slowest mode of a cluttered field has a tiny residual and a large error.  From
                          the first check with r_inf < 100 tol on, each check copies the field into
                          snapshot planes (workspace grows by one plane pair) and measures d, the largest
                          change of a free cell since the previous check's snapshot (Tl sweeps ago); its
                          estimate is d / (1 - rho^Tl), rho = max(omega - 1, the last clear decay rate of
                          the residual 2-norm) -- the error test of Hageman & Young's adaptive SOR
                          (Applied Iterative Methods, 1981, ch. 9) over a check interval -- and the larger
                          of the last two such estimates is the one compared with etol (past the optimal
                          omega the error also turns, and one interval's change can be small).  The solve
                          stops when r_inf <= tol and that estimate <= etol.  With etol > 0 the over-
                          relaxation back-off is not used, omega is frozen once r_inf <= tol, and when the
                          estimate is met while the FP32 rounding noise of SOR at omega near 2 keeps
                          r_inf above tol, one launch of T Gauss-Seidel sweeps on a copy (the polish of
                          HP_POLISH) is accepted if it meets tol.  If the estimate and the residual both
                          stop falling for four checks (once r_inf < 16 tol) the solve ends with
                          TW_NOT_CONVERGED.  HP_MIXED: the outer loop also stops only once its
                          estimate, the last FP64 update's size c divided by 1 - q with q = its ratio
                          to the update before (undefined while q >= 0.9), is <= etol.  HP_JACOBI
                          ignores etol. */
} hp_params;

typedef struct {
    int sweeps;        /* full sweeps performed (HP_RBSOR: SOR sweeps plus polish sweeps) */
    int status;        /* TW_OK or TW_NOT_CONVERGED */
    double resid_inf;  /* FP64 residual max |(1/4) sum nbr - u| over free cells of the output
                          (HP_MIXED: of its FP64 master field, which the FP32 output rounds) */
    double resid_l2;   /* sqrt(sum of squared residuals) over the same cells, to about 1e-6 relative:
                          each residual is evaluated FP64-accurately (as for resid_inf), its leading
                          FP32 part is squared and summed in FP32 over a thread's cells, and the
                          per-CTA sums are added in FP64 (HP_MIXED: the FP64 master's residuals,
                          squared and summed in FP64) */
    double omega;      /* SOR factor used last */
    int checks;        /* residual checks performed */
    int sweep_launches;/* launches of the sweep kernel */
    double sweep_ms;   /* HP_TIMING: summed CUDA-event time of the sweep launches (ms) */
    int tblock;        /* temporal-blocking depth used (sweeps fused per launch) */
    int loop;          /* how the convergence loop ran: HP_LOOP_HOST or HP_LOOP_GRAPH */
    int polishes;      /* polish launches tried (HP_POLISH) */
    int polished;      /* 1: the output is the accepted polished copy */
    double resid_check;/* the FP32 residual max of the loop's last check (0 if it made none) */
    double err_est;    /* etol > 0: the last error estimate (see hp_params.etol; DBL_MAX until two
                          checks have measured a change), else 0 */
} hp_stats;

#define HP_LOOP_HOST 0     /* host-driven: HP_HOST_LOOP, HP_TIMING, HP_JACOBI, or a cap below one
                              check interval */
#define HP_LOOP_GRAPH 1    /* CUDA graph whose conditional while-node runs the check intervals
                              (the host finishes a cap that is not a whole number of intervals;
                              HP_MIXED: each correction solve is one such graph launch, the outer
                              FP64 steps are driven by the host) */

/* hp_relax: the harmonic field of the occupancy grid (Sec. 3.1).  Cells with
 * occ != 0 and the border are Dirichlet cells at phi = 1, the goal cell is
 * fixed at phi = 0, free cells start at phi = 0.5 (or the warm start) and
 * converge to the discrete Laplace solution (the fixed point of Eq. 1; Eq. 2
 * and red-black SOR share it).  The field is kept and written as
 * u = 1 - phi (goal 1, obstacles 0), which keeps relative precision where phi
 * is close to 1; HP_OUT_PHI writes phi instead.
 * The residual is the 1/4-scaled infinity norm max |(1/4) sum_nbr u - u| over
 * free cells (the size of one Eq. 1 update); stats report it recomputed in
 * FP64 on the stored output.
 * occ_dev: device uint8 [ny][nx].  field_dev: device float [ny][nx] (in: warm
 * start if HP_WARM_START; out: the field).  stats: host, written on return.
 * Synchronises `stream` (residual checks are read on the host).
 * Errors: TW_EINVAL, TW_EGOAL_BLOCKED (goal on the border, occupied or out of
 * range), TW_EWORKSPACE, TW_ECUDA.  Warning: TW_NOT_CONVERGED. */
size_t hp_relax_workspace_size(int nx, int ny, const hp_params *p);
int hp_relax(const tw_grid *g, const uint8_t *occ_dev, int gx, int gy, float *field_dev,
             const hp_params *p, hp_stats *stats, void *workspace, size_t workspace_bytes,
             void *stream);

/* hp_relax_noalloc: hp_relax without a caller workspace, for callers that
 * cannot allocate device memory -- e.g. a real-time control loop that may not
 * allocate after start-up (cudaMalloc can synchronise the device and take
 * unbounded time) or a plug-in inside a host application that owns every
 * device allocation.  The paper has no counterpart; this is a library
 * convenience.  Its scratch is one file-scope device array of
 * HP_RELAX_NOALLOC_SCRATCH_BYTES (9 MiB), held by every GPU that loads the
 * library until the process exits; the call itself allocates nothing.
 * Same arguments and results as hp_relax (occ_dev and field_dev are still the
 * caller's), for method HP_RBSOR or HP_JACOBI without HP_TIMING; the
 * convergence loop is always host-driven (HP_HOST_LOOP).
 * Limits: grids whose hp_relax_workspace_size() exceeds the array (for
 * HP_RBSOR anything above about 1024 x 1024 cells, or 870 x 870 with
 * etol > 0, which adds the snapshot planes) return TW_EWORKSPACE
 * before any GPU work; other methods or HP_TIMING return TW_EINVAL.
 * Set-up: the first call on a device, with that device current, looks up the
 * array's device address once and caches it; make that first call before any
 * stream capture.  All calls on a device share the array and it keeps the
 * previous call's contents (each call clears what must start at zero), so
 * calls whose GPU work overlaps -- on different streams or host threads --
 * race and must be serialised by the caller.  The array is the one of the
 * device current at the call, so make the device that holds occ_dev and
 * field_dev current first.  Its address is looked up once per device and kept:
 * after cudaDeviceReset on a device, do not call hp_relax_noalloc there again
 * in the same process (the kept address belonged to the destroyed context). */
#define HP_RELAX_NOALLOC_SCRATCH_BYTES ((size_t)9 << 20)
int hp_relax_noalloc(const tw_grid *g, const uint8_t *occ_dev, int gx, int gy, float *field_dev,
                     const hp_params *p, hp_stats *stats, void *stream);

/* hp_relax_batched: many planners solved together (uneven grids).  Each
 * instance is the hp_relax problem of its own occupancy and goal; all of them
 * are relaxed by red-black SOR inside one CUDA graph whose sweep kernel is a
 * persistent, grid-stride kernel over the tiles of every still-active
 * instance, with per-instance omega, residual and convergence (converged
 * instances drop out).  The tile configuration is autotuned once per batch
 * shape (device, workspace, n, total cells) among five: depth T = 2 or 4 on
 * shallow tiles (8 x 8 rows), T = 4, 6 or 7 on deep tiles (12 x 2T rows);
 * each is timed on two launches of Gauss-Seidel sweeps (which count towards
 * the solve) and the fastest per sweep wins.  Unless p->check_every is set,
 * the check interval is tuned too, from the measured cost of a check and of a
 * sweep and the slowest instance's sweeps at the previous call of the same
 * shape (256 at the first).  p->tblock 2 or 4 forces shallow tiles at that
 * depth, 6 or 7 deep tiles; stats[i].tblock reports the depth used.
 * n: 1..1024 instances.  p: method HP_RBSOR, FP32; tol, max_sweeps, omega
 * (0 = adaptive), check_every and etol apply to every instance (with etol > 0
 * each instance gets the error estimate of hp_relax -- snapshot planes, which
 * the workspace size includes, and the residual 2-norm from per-tile sums
 * added in tile order -- while omega keeps adapting on the residual max; an
 * instance is TW_OK once r_inf <= tol and its estimate <= etol, reported in
 * stats[i].err_est); HP_WARM_START reads u from field_dev, HP_OUT_PHI writes
 * phi (not both).  stats: host array of n,
 * latency_ms: host array of n or NULL -- the time from the start of the
 * relaxation to each instance's convergence, measured on the device
 * (%globaltimer).  Returns TW_OK, TW_NOT_CONVERGED if any instance hit the
 * cap, or the first error (per-instance status in stats[i].status, e.g.
 * TW_EGOAL_BLOCKED).  Synchronises `stream`. */
typedef struct {
    int nx, ny;              /* grid of this instance (3..65535) */
    const uint8_t *occ_dev;  /* device uint8 [ny][nx] occupancy (nonzero = obstacle) */
    int gx, gy;              /* goal cell */
    float *field_dev;        /* device float [ny][nx]: the field (u unless HP_OUT_PHI) */
} hp_instance;
size_t hp_relax_batched_workspace_size(int n, const hp_instance *inst, const hp_params *p);
int hp_relax_batched(int n, const hp_instance *inst, const hp_params *p, hp_stats *stats,
                     double *latency_ms, void *workspace, size_t workspace_bytes, void *stream);

/* hp_relax_dirichlet: the same solver on a general Dirichlet problem: cells
 * with fixed_dev != 0 keep their value of u_dev, the others satisfy the
 * discrete Laplace equation.  Every border cell must be fixed.  u_dev is read
 * as the initial guess and overwritten with the solution (no phi/u mapping). */
int hp_relax_dirichlet(int nx, int ny, const uint8_t *fixed_dev, float *u_dev,
                       const hp_params *p, hp_stats *stats, void *workspace,
                       size_t workspace_bytes, void *stream);

/* hp_residual: FP64 residual of a stored field against a fixed mask (device
 * uint8, nonzero = fixed).  Results written to host r_inf / r_l2. */
int hp_residual(int nx, int ny, const uint8_t *fixed_dev, const float *u_dev,
                double *r_inf, double *r_l2, void *workspace, size_t workspace_bytes,
                void *stream);

/* ---- path ------------------------------------------------------------------
 * plan_path: Eq. 3 steepest descent on u from the start cell (neighbour order
 * +x, -x, +y, -y; the first largest u wins; a move needs a strictly larger u)
 * until the goal, then `rubber_iters` rubber-band sweeps (Eqs. 4-6) with
 * node energy w/u(q) + (k/2)(|q - p_prev|^2 + |q - p_next|^2): odd nodes then
 * even nodes move to the lowest-energy free cell of their 3x3 neighbourhood
 * that stays 8-adjacent to both path neighbours; consecutive duplicates are
 * dropped at the end.  w = 1e-3, k = 1 unless set through plan_path_ex.
 * u_dev: device float [ny][nx] (u = 1 - phi as written by hp_relax).
 * occ_dev: device uint8 occupancy (nonzero = blocked, the goal is allowed).
 * path_xy_host: host int32 [2 * max_len] output (x0, y0, x1, y1, ...).
 * len_out: host, number of nodes written.  Synchronises `stream`.
 * Returns TW_OK, TW_NO_PATH, TW_ESTART_BLOCKED, TW_EINVAL, TW_EWORKSPACE, TW_ECUDA. */
size_t plan_path_workspace_size(int max_len);
int plan_path(const tw_grid *g, const float *u_dev, const uint8_t *occ_dev, int sx, int sy,
              int gx, int gy, int rubber_iters, int max_len, int32_t *path_xy_host,
              int *len_out, void *workspace, size_t workspace_bytes, void *stream);
int plan_path_ex(const tw_grid *g, const float *u_dev, const uint8_t *occ_dev, int sx, int sy,
                 int gx, int gy, int rubber_iters, double w, double k, int max_len,
                 int32_t *path_xy_host, int *len_out, void *workspace, size_t workspace_bytes,
                 void *stream);

/* ---- learned warm start --------------------------------------------------------
 * A fully convolutional encoder-decoder (4 levels, 32/64/128/128 channels,
 * 3x3 convolutions, 2x2 average pooling, nearest upsampling, additive skips,
 * ReLU; 15 convolutions) predicts p = log(u) / 30 from two input maps: the
 * occupancy (1 where occ != 0) and the distance to the goal over the grid
 * diagonal.  Activations and gradients are stored in BF16, weights in FP32
 * (rounded to BF16 when used), all products accumulate in FP32.  The network
 * is not in the paper: the field it predicts is only a starting point for
 * hp_relax (HP_WARM_START), which finishes the solve to its tolerance.
 * H and W: multiples of 8 in [16, 8192].  params/grads/adam_m/adam_v: device
 * FP32 arrays of ws_unet_param_count() values.  occ: device uint8 [H][W];
 * (gx, gy) the goal.  workspace: ws_unet_workspace_size(H, W) bytes. */
size_t ws_unet_param_count(void);
size_t ws_unet_workspace_size(int H, int W);
/* He-normal weights from a counter-based generator seeded with `seed`, zero biases. */
int ws_unet_init(float *params, unsigned long long seed, void *stream);
/* target[i] = max(log(max(u[i], 1e-30)), log(1e-30)) / 30 for a relaxed field u (device, n values). */
int ws_make_target(const float *u, size_t n, float *target, void *stream);
/* Forward pass.  u_out (nullable): the warm start u = exp(30 p) clipped to <= 1,
 * 0 on occupied cells, 1 at the goal.  pred_out (nullable): p itself. */
int ws_unet_forward(const float *params, const uint8_t *occ, int H, int W, int gx, int gy, float *u_out,
                    float *pred_out, void *workspace, size_t workspace_bytes, void *stream);
/* The warm start for hp_relax (HP_WARM_START) from the network run at a coarser
 * resolution: stride s in {1, 2, 4}; H/s and W/s must satisfy the network's
 * size rule.  The occupancy is max-pooled by s (a coarse cell is occupied when
 * any of its cells is, except the one holding the goal), the network predicts
 * p on the H/s x W/s grid, and u_out (device FP32 [H][W]) receives
 * exp(min(30 p, 0)) with p bilinearly interpolated at every cell centre, 0 on
 * occupied cells and 1 at the goal.  s = 1 equals ws_unet_forward's u_out.
 * The network is fully convolutional and trained at one size; a coarse run
 * costs about s^2 times less and the relaxation restores the detail.
 * workspace: ws_unet_warm_start_workspace_size(H, W, s) bytes.
 * Errors: TW_EINVAL, TW_EWORKSPACE, TW_ECUDA. */
size_t ws_unet_warm_start_workspace_size(int H, int W, int stride);
int ws_unet_warm_start(const float *params, const uint8_t *occ, int H, int W, int gx, int gy, int stride,
                       float *u_out, void *workspace, size_t workspace_bytes, void *stream);
/* One training step on one field: masked mean-squared error between p and
 * target over free cells (occ == 0, not the goal), gradients into `grads`,
 * then Adam (beta 0.9 / 0.999, eps 1e-8, bias-corrected with `step` >= 1,
 * learning rate lr) when adam_m != NULL.  loss_host (nullable) receives the loss. */
int ws_unet_train_step(float *params, float *grads, float *adam_m, float *adam_v, int step, float lr,
                       const uint8_t *occ, int H, int W, int gx, int gy, const float *target, float *loss_host,
                       void *workspace, size_t workspace_bytes, void *stream);

/* ws_conv3x3: one convolution layer of the network, Y = act(conv3x3(X, Wt) + b + S)
 * with zero padding (stride 1).  X: device BF16 [cin][H][W]; Wt: device FP32
 * [cout][cin][3][3], rounded to BF16 when used; b: device FP32 [cout] or NULL;
 * S: device BF16 [cout][H][W] added before the activation, or NULL; Y: device
 * BF16 [cout][H][W]; relu: 1 for ReLU, 0 for none.  impl: WS_CONV_AUTO (BF16
 * tensor cores where cin % 16 == 0 and cout % 32 == 0, else CUDA cores),
 * WS_CONV_SIMT (direct convolution on CUDA cores), WS_CONV_MMA (tensor cores,
 * mma.sync m16n8k16, FP32 accumulation) or WS_CONV_TC (5th-generation tensor
 * cores: tcgen05.mma implicit GEMM with the accumulators in tensor memory, for
 * cin % 16 == 0, cout in {32, 64, 128}, and either W % 128 == 0 and H a
 * multiple of 4 (of 2 for cout 128), or W in {16, 32, 64} and H a multiple of
 * 256 / W (the narrow form: 128-pixel blocks spanning 128 / W rows, split K over
 * the 16-channel chunks with the partial sums added in split order); it needs
 * ws_conv3x3_workspace_size() bytes of 256-byte-aligned device workspace for
 * the weights re-arranged in BF16 (and the narrow form's partial sums), and is
 * what WS_CONV_AUTO uses inside the network wherever those conditions hold).  Every form accumulates each
 * product in FP32; they differ only in the order of the sums.  TW_EINVAL when
 * the channel counts or sizes do not allow the form asked for; TW_EWORKSPACE
 * for a missing or short workspace.  Enqueued on `stream`.  The implicit
 * GEMM's waits on its own tensor-core work are bounded (one second): a wait
 * that gives up sets a flag that ws_conv_check reads. */
#define WS_CONV_AUTO 0
#define WS_CONV_SIMT 1
#define WS_CONV_MMA 2
#define WS_CONV_TC 3
size_t ws_conv3x3_workspace_size(int cin, int cout, int H, int W, int impl);
int ws_conv3x3(const void *X, const float *Wt, const float *b, const void *S, void *Y, int cin, int cout, int H, int W,
               int relu, int impl, void *workspace, size_t workspace_bytes, void *stream);
/* ws_conv3x3_wgrad: the parameter gradients of one such layer (the backward pass
 * of Sec. 3.4's network): dW[co][ci][ky][kx] += sum_p dY[co][p] X[ci][p + (ky-1,
 * kx-1)] (zero padding) and db[co] += sum_p dY[co][p], accumulated into what dW
 * and db hold.  X: device BF16 [cin][H][W] (the layer's input); dY: device BF16
 * [cout][H][W] (the gradient of its pre-activation output); dW: device FP32
 * [cout][cin][3][3]; db: device FP32 [cout] or NULL.  impl: WS_CONV_TC (5th-
 * generation tensor cores: per tap a GEMM over the pixels issued with
 * tcgen05.mma, accumulators in tensor memory; cin and cout at most 128 (other
 * counts than 32, 64 and 128 padded), W % 16 == 0, X and dY 16-byte aligned),
 * WS_CONV_SIMT (CUDA cores) or
 * WS_CONV_AUTO (WS_CONV_TC where it applies, else CUDA cores); WS_CONV_MMA is
 * TW_EINVAL.  Both forms add BF16 x BF16 products exactly in FP32 and the
 * partial sums of their pixel chunks in a fixed order, so repeated calls give
 * identical results; they differ from each other only in the order of the sums.
 * workspace: ws_conv3x3_wgrad_workspace_size() bytes (256-byte aligned), else
 * TW_EWORKSPACE.  Enqueued on `stream`; bounded waits as for ws_conv3x3. */
size_t ws_conv3x3_wgrad_workspace_size(int cin, int cout, int H, int W, int impl);
int ws_conv3x3_wgrad(const void *X, const void *dY, float *dW, float *db, int cin, int cout, int H, int W, int impl,
                     void *workspace, size_t workspace_bytes, void *stream);
/* ws_conv_check: *timed_out = 1 if a WS_CONV_TC convolution on the current
 * device gave up a bounded wait since the last call (its output is then
 * invalid), else 0; clears the flag.  Synchronises the device. */
int ws_conv_check(int *timed_out);

/* ---- Kalman filter (host) ----------------------------------------------------
 * kf_update: one step of the constant-velocity filter of Sec. 3.5 for n host
 * tracks: predict by dt (Eqs. 9-10, A(dt), Q(dt) = q_accel x white-noise
 * acceleration block), then update with the position measurement z[2o..2o+1]
 * (Eqs. 11-13, H = [I2 0], R = r_meas^2 I2).  In place.  TW_EINVAL on bad input. */
int kf_update(tw_track *tracks, int n, const double *z, double dt, double q_accel,
              double r_meas);
/* kf_init: x = [z, 0, 0], P = diag(r^2, r^2, p_vel, p_vel), radius from `radius`. */
int kf_init(tw_track *tracks, int n, const double *z, const double *radius, double r_meas,
            double p_vel);

/* hp_omega_update: one step of the adaptive SOR factor hp_relax uses
 * (omega = 0 in hp_params), exposed for callers that drive their own
 * red-black SOR and for tests.  omega: the factor of the last check interval;
 * lambda: the observed decay rate of the residual per sweep over it (0..1);
 * nx, ny: the grid.  Young's relation for consistently ordered matrices,
 * (lambda + omega - 1)^2 = lambda omega^2 mu^2, gives the Jacobi spectral
 * radius mu and omega_opt = 2 / (1 + sqrt(1 - mu^2)), moved 10 % of the way
 * towards 2 (pre-asymptotic decay underestimates mu).  Returns the new factor:
 * never below omega, never above the empty-box optimum for nx x ny (no
 * occupancy has a larger one), and omega itself while lambda <= (omega - 1)^(3/4)
 * (at or past the optimum, where lambda says nothing about mu) or lambda is
 * outside (0, 1).  hp_omega_cap returns that upper bound;
 * hp_omega_initial the first factor of an adaptive solve. */
double hp_omega_update(double omega, double lambda, int nx, int ny);
double hp_omega_cap(int nx, int ny);
double hp_omega_initial(int nx, int ny);

/* ---- diagnostics -------------------------------------------------------------- */
const char *tw_status_string(int status);
int tw_last_cuda_error(void);          /* last cudaError_t seen by the library */
/* Number of CUDA kernels the library has launched in this process (host
 * counter, incremented at every launch; for benchmarks and tests). */
unsigned long long tw_launch_count(void);
const char *tw_version(void);

#ifdef __cplusplus
}
#endif
#endif /* TWGRID_H */
