/*
 * twgrid_oracle.c -- plain, slow, obviously correct FP64 CPU oracle for the
 * time-warped grid planner (Farzan & DeSouza, "Path Planning in Dynamic
 * Environments Using Time-Warped Grids and a Parallel Implementation").
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, table or constant generator with the CUDA library; the two are
 * written independently from the paper and from the readings recorded with
 * the project design notes.
 *
 * Build: cc -O2 -std=c11 -ffp-contract=off -fno-fast-math -shared -fPIC.
 * -ffp-contract=off matters: every floating-point operation on the raster's
 * pre-stage must round on its own (no fused multiply-add) so that the integer
 * predicates are reproducible bit for bit.
 *
 * Threads.  The same source is also built with -fopenmp, for timing the
 * oracle on every host core (the benchmark's CPU baseline).  Threads share
 * only work whose result does not depend on its order -- independent cells,
 * maxima -- and every sum keeps its serial order, so both builds return the
 * same bits; without -fopenmp the pragmas are ignored.
 *
 * Conventions.  Grids are row-major [ny][nx]; cell (i, j) is column i, row j.
 * Fixed-point coordinates are in 1/256 of a cell relative to the grid origin;
 * the centre of cell (i, j) is (256 i + 128, 256 j + 128).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_OK 0
#define OR_NOT_CONVERGED 1
#define OR_NO_PATH 2
#define OR_EINVAL (-1)
#define OR_EGOAL (-2)
#define OR_ESTART (-3)

#define OR_MAX_RINGS 64
#define OR_COORD_CLAMP 1073741824LL  /* 2^30 */
#define OR_RADIUS_CLAMP 536870912LL  /* 2^29 */

/* Threads of the OpenMP build (n > 0 sets them); returns the count in use
 * (1 in the plain build). */
int or_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

/* ------------------------------------------------------------------------
 * a1. Ring table.
 * Rings grow geometrically from r0 by `growth` (the time-warped grid's
 * "progressively wider orbits", Sec. 3.4; geometric law of the benchmark
 * configuration).  R_0 = r0, R_j = R_{j-1} * growth.  With n_rings == 0 the
 * count is the first J with R_{J-1} >= reach (reach = grid diagonal for the
 * circular law, 10 x the diagonal for the elliptic law, whose rings extend
 * only 0.1 R behind the robot).  Arrival time of ring j (Sec. 3.4: the filter
 * predicts j steps ahead for warp number j) is its inner radius over the
 * robot speed: t_0 = 0, t_j = R_{j-1} / v; with time_outer, t_j = R_j / v.
 * ---------------------------------------------------------------------- */
int or_ring_table(int kind, double r0, double growth, int n_rings, double speed,
                  int time_outer, double nx_cells, double ny_cells, double cell,
                  double *R, double *t)
{
    if (!(r0 > 0.0) || !(growth > 1.0) || !(speed > 0.0) || !(cell > 0.0)) return OR_EINVAL;
    if (n_rings < 0 || n_rings > OR_MAX_RINGS) return OR_EINVAL;
    double w = nx_cells * cell, h = ny_cells * cell;
    double reach = sqrt(w * w + h * h);
    if (kind == 1) reach = reach * 10.0;
    int J = 0;
    double r = r0;
    for (;;) {
        if (J >= OR_MAX_RINGS) return OR_EINVAL;
        R[J] = r;
        J++;
        if (n_rings > 0) { if (J == n_rings) break; }
        else if (r >= reach) break;
        r = r * growth;
    }
    for (int j = 0; j < J; j++) {
        if (time_outer) t[j] = R[j] / speed;
        else t[j] = (j == 0) ? 0.0 : R[j - 1] / speed;
    }
    return J;
}

static int64_t q_clamp(double v, int64_t lo, int64_t hi)
{
    /* v is finite by validation; rint rounds half to even. */
    double r = rint(v);
    if (r < (double)lo) return lo;
    if (r > (double)hi) return hi;
    return (int64_t)r;
}

/* Fixed-point position along one axis: rint(((v - origin) / cell) * 256). */
static int64_t q_pos(double v, double origin, double cell)
{
    return q_clamp(((v - origin) / cell) * 256.0, -OR_COORD_CLAMP, OR_COORD_CLAMP);
}

/* ------------------------------------------------------------------------
 * a2. Track prediction at ring time t (Eqs. 9-10 with the constant-velocity
 * matrix A(t) of Sec. 3.5, no input, white-noise acceleration Q(t)).
 * Track layout: x[4] = [x, y, vx, vy], P[16] row-major, radius.
 *   px = x + t*vx ; py = y + t*vy
 *   Pxx(t) = ((Pxx + (2t)*P[0][2]) + (t*t)*P[2][2]) + ((q*t)*t)*t/3   (same for y)
 *   s2 = 0.5*(Pxx(t) + Pyy(t)); sigma = s2 > 0 ? sqrt(s2) : 0
 *   rho = (radius + d_safe) + kappa*sigma        (Sec. 3.4 Gaussian marking,
 *                                                  made binary at kappa sigma)
 * ---------------------------------------------------------------------- */
void or_predict_one(const double *trk, double t, double q, double kappa, double d_safe, double alpha,
                    double ox, double oy, double cell,
                    int64_t *pxq, int64_t *pyq, int64_t *rhoq)
{
    const double *x = trk;
    const double *P = trk + 4;
    double radius = trk[20];
    double px = x[0] + t * x[2];
    double py = x[1] + t * x[3];
    double pxx = ((P[0] + (2.0 * t) * P[2]) + (t * t) * P[10]) + ((q * t) * t) * t / 3.0;
    double pyy = ((P[5] + (2.0 * t) * P[7]) + (t * t) * P[15]) + ((q * t) * t) * t / 3.0;
    double s2 = 0.5 * (pxx + pyy);
    double sigma = (s2 > 0.0) ? sqrt(s2) : 0.0;
    double rho = (radius + d_safe) + kappa * sigma;
    *pxq = q_pos(px, ox, cell);
    *pyq = q_pos(py, oy, cell);
    *rhoq = q_clamp((rho / cell) * 256.0, 0, OR_RADIUS_CLAMP);
    /* probability-threshold marking: a prediction whose centre is too uncertain to
     * lie within radius + d_safe of its mean with the threshold probability marks
     * nothing (radius -1) */
    if (alpha > 0.0) {
        double a = alpha * (radius + d_safe);
        if (s2 > a * a) *rhoq = -1;
    }
}

/* Ring of a fixed-point offset (dx, dy) from the robot: the smallest j whose
 * closed ring contains the point, else the last ring. */
static int ring_of(int kind, int64_t dx, int64_t dy, int J, const int64_t *Rq,
                   const int64_t *Aq, const int64_t *Cq, int64_t hxq, int64_t hyq)
{
    for (int j = 0; j < J; j++) {
        if (kind == 0) {
            if (dx * dx + dy * dy <= Rq[j] * Rq[j]) return j;
        } else {
            /* Eq. 14 with r_x = 4 r_y and centre 0.9 r_x ahead (Eq. 15):
             * inside ellipse j iff (u - 0.9 R_j)^2 + 16 v^2 <= R_j^2,
             * u, v the offset along / across the heading, in 2^-20 units. */
            __int128 u = (__int128)(hxq * dx + hyq * dy);
            __int128 v = (__int128)(hxq * dy - hyq * dx);
            __int128 a = u - (__int128)Cq[j];
            if (a * a + 16 * v * v <= (__int128)Aq[j] * (__int128)Aq[j]) return j;
        }
    }
    return J - 1;
}

/* ------------------------------------------------------------------------
 * a1-a3. Build the time-warped occupancy grid by brute force.
 * occ codes: 0 free, 1 static obstacle, 2 predicted dynamic obstacle,
 * 3 grid border (priority border > static > dynamic).
 * mark == 0 (per cell): cell c in ring j(c) is dynamic iff some obstacle's
 *   disk predicted at t_{j(c)} contains c's centre.
 * mark == 1 (per obstacle, Alg. 1): each obstacle takes the ring of its own
 *   current estimate and its disk at that ring's time marks every cell.
 * robot: [x, y, hx, hy, speed]; tracks: n x 21 doubles.
 * Returns J (>0) or a negative status.
 * ---------------------------------------------------------------------- */
int or_build_grid(int nx, int ny, double cell, double ox, double oy,
                  const double *robot, const double *tracks, int n,
                  int kind, int mark, double r0, double growth, int n_rings,
                  double q, double kappa, double d_safe, int time_outer, double p_mark,
                  const uint8_t *static_occ, uint8_t *occ, int16_t *ring)
{
    /* the probability that an N(p, sigma^2 I) centre lies within rho0 of p is
     * 1 - exp(-rho0^2 / (2 sigma^2)); it reaches p_mark while sigma <= alpha rho0 */
    double alpha = (p_mark > 0.0) ? 1.0 / sqrt(-2.0 * log(1.0 - p_mark)) : 0.0;
    double R[OR_MAX_RINGS], t[OR_MAX_RINGS];
    int64_t Rq[OR_MAX_RINGS], Aq[OR_MAX_RINGS], Cq[OR_MAX_RINGS];
    if (nx < 1 || ny < 1 || nx > 65536 || ny > 65536) return OR_EINVAL;
    int J = or_ring_table(kind, r0, growth, n_rings, robot[4], time_outer,
                          (double)nx, (double)ny, cell, R, t);
    if (J <= 0) return OR_EINVAL;
    for (int j = 0; j < J; j++) {
        Rq[j] = q_clamp((R[j] / cell) * 256.0, 0, OR_RADIUS_CLAMP);
        Aq[j] = q_clamp((R[j] / cell) * 268435456.0, 0, INT64_C(1) << 52);
        Cq[j] = q_clamp(((0.9 * R[j]) / cell) * 268435456.0, 0, INT64_C(1) << 52);
    }
    int64_t rxq = q_pos(robot[0], ox, cell);
    int64_t ryq = q_pos(robot[1], oy, cell);
    int64_t hxq = q_clamp(robot[2] * 1048576.0, -1048576, 1048576);
    int64_t hyq = q_clamp(robot[3] * 1048576.0, -1048576, 1048576);

    size_t nd = (size_t)(n > 0 ? n : 1) * (size_t)J;
    int64_t *PX = (int64_t *)malloc(nd * sizeof(int64_t));
    int64_t *PY = (int64_t *)malloc(nd * sizeof(int64_t));
    int64_t *RH = (int64_t *)malloc(nd * sizeof(int64_t));
    int *own = (int *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int));
    for (int o = 0; o < n; o++) {
        for (int j = 0; j < J; j++)
            or_predict_one(tracks + 21 * (size_t)o, t[j], q, kappa, d_safe, alpha, ox, oy, cell,
                           &PX[(size_t)o * J + j], &PY[(size_t)o * J + j], &RH[(size_t)o * J + j]);
        int64_t exq = q_pos(tracks[21 * (size_t)o + 0], ox, cell);
        int64_t eyq = q_pos(tracks[21 * (size_t)o + 1], oy, cell);
        own[o] = ring_of(kind, exq - rxq, eyq - ryq, J, Rq, Aq, Cq, hxq, hyq);
    }

#pragma omp parallel for schedule(dynamic, 8)
    for (int jy = 0; jy < ny; jy++) {
        for (int ix = 0; ix < nx; ix++) {
            size_t c = (size_t)jy * nx + ix;
            int64_t cx = 256 * (int64_t)ix + 128;
            int64_t cy = 256 * (int64_t)jy + 128;
            int jr = ring_of(kind, cx - rxq, cy - ryq, J, Rq, Aq, Cq, hxq, hyq);
            if (ring) ring[c] = (int16_t)jr;
            uint8_t code = 0;
            if (ix == 0 || jy == 0 || ix == nx - 1 || jy == ny - 1) code = 3;
            else if (static_occ && static_occ[c]) code = 1;
            else {
                for (int o = 0; o < n && code == 0; o++) {
                    int jj = (mark == 0) ? jr : own[o];
                    size_t d = (size_t)o * J + jj;
                    int64_t dx = cx - PX[d], dy = cy - PY[d];
                    if (RH[d] >= 0 && dx * dx + dy * dy <= RH[d] * RH[d]) code = 2;
                }
            }
            occ[c] = code;
        }
    }
    free(PX); free(PY); free(RH); free(own);
    return J;
}

/* ------------------------------------------------------------------------
 * Harmonic field.  General Dirichlet problem on a grid: cells with fixed[c]
 * keep u[c]; every other cell satisfies u[c] = (1/4) sum of its 4 neighbours
 * (Eq. 1's fixed point, the discrete Laplace equation).  Every border cell
 * must be fixed, so free cells have four in-grid neighbours.
 * ---------------------------------------------------------------------- */
static int check_border_fixed(const uint8_t *fixed, int nx, int ny)
{
    for (int i = 0; i < nx; i++)
        if (!fixed[i] || !fixed[(size_t)(ny - 1) * nx + i]) return 0;
    for (int j = 0; j < ny; j++)
        if (!fixed[(size_t)j * nx] || !fixed[(size_t)j * nx + nx - 1]) return 0;
    return 1;
}

static double nbr_avg(const double *u, int nx, size_t c)
{
    return 0.25 * (((u[c + 1] + u[c - 1]) + u[c + nx]) + u[c - nx]);
}

/* Residual (1/4-scaled): r_inf = max over free cells |avg - u|, r_l2 = sqrt(sum r^2). */
void or_residual(const double *u, const uint8_t *fixed, int nx, int ny,
                 double *r_inf, double *r_l2)
{
    double m = 0.0, s = 0.0;
    for (int j = 1; j < ny - 1; j++)
        for (int i = 1; i < nx - 1; i++) {
            size_t c = (size_t)j * nx + i;
            if (fixed[c]) continue;
            double r = fabs(nbr_avg(u, nx, c) - u[c]);
            if (r > m) m = r;
            s += r * r;
        }
    *r_inf = m;
    *r_l2 = sqrt(s);
}

/* r_inf of or_residual alone (a maximum: the same whatever the order). */
static double residual_max(const double *u, const uint8_t *fixed, int nx, int ny)
{
    double m = 0.0;
#pragma omp parallel for reduction(max : m)
    for (int j = 1; j < ny - 1; j++)
        for (int i = 1; i < nx - 1; i++) {
            size_t c = (size_t)j * nx + i;
            if (fixed[c]) continue;
            double r = fabs(nbr_avg(u, nx, c) - u[c]);
            if (r > m) m = r;
        }
    return m;
}

/* Eq. 1: Jacobi sweeps until the residual of the current iterate <= tol. */
int or_jacobi(double *u, const uint8_t *fixed, int nx, int ny, double tol,
              int max_sweeps, int *sweeps_out, double *res_out)
{
    if (!check_border_fixed(fixed, nx, ny)) return OR_EINVAL;
    size_t N = (size_t)nx * ny;
    double *v = (double *)malloc(N * sizeof(double));
    memcpy(v, u, N * sizeof(double));
    int k = 0;
    double r = residual_max(u, fixed, nx, ny);
    while (r > tol && k < max_sweeps) {
#pragma omp parallel for
        for (int j = 1; j < ny - 1; j++)
            for (int i = 1; i < nx - 1; i++) {
                size_t c = (size_t)j * nx + i;
                if (!fixed[c]) v[c] = nbr_avg(u, nx, c);
            }
        memcpy(u, v, N * sizeof(double));
        k++;
        r = residual_max(u, fixed, nx, ny);
    }
    free(v);
    *sweeps_out = k;
    *res_out = r;
    return (r <= tol) ? OR_OK : OR_NOT_CONVERGED;
}

/* Eq. 2: lexicographic Gauss-Seidel (already-updated left and upper
 * neighbours are used), in place. */
int or_gauss_seidel(double *u, const uint8_t *fixed, int nx, int ny, double tol,
                    int max_sweeps, int *sweeps_out, double *res_out)
{
    if (!check_border_fixed(fixed, nx, ny)) return OR_EINVAL;
    int k = 0;
    double r, l2;
    or_residual(u, fixed, nx, ny, &r, &l2);
    while (r > tol && k < max_sweeps) {
        for (int j = 1; j < ny - 1; j++)
            for (int i = 1; i < nx - 1; i++) {
                size_t c = (size_t)j * nx + i;
                if (!fixed[c]) u[c] = nbr_avg(u, nx, c);
            }
        k++;
        or_residual(u, fixed, nx, ny, &r, &l2);
    }
    *sweeps_out = k;
    *res_out = r;
    return (r <= tol) ? OR_OK : OR_NOT_CONVERGED;
}

/* y = A x for the free-cell operator A = I - J (J = 1/4 x free-neighbour sum);
 * entries of x on fixed cells are ignored and y is zero there. */
static void apply_A(const double *x, double *y, const uint8_t *fixed, int nx, int ny)
{
    size_t N = (size_t)nx * ny;
    memset(y, 0, N * sizeof(double));
#pragma omp parallel for
    for (int j = 1; j < ny - 1; j++)
        for (int i = 1; i < nx - 1; i++) {
            size_t c = (size_t)j * nx + i;
            if (fixed[c]) continue;
            double s = 0.0;
            if (!fixed[c + 1]) s += x[c + 1];
            if (!fixed[c - 1]) s += x[c - 1];
            if (!fixed[c + nx]) s += x[c + nx];
            if (!fixed[c - nx]) s += x[c - nx];
            y[c] = x[c] - 0.25 * s;
        }
}

/* Sum over free cells of a[c] b[c], in fixed chunks of OR_DOT_CHUNK cells:
 * each chunk summed in index order, then the chunk sums in chunk order -- the
 * same association whatever the thread count (chunks are independent). */
#define OR_DOT_CHUNK 65536
static double dot_free(const double *a, const double *b, const uint8_t *fixed, size_t N)
{
    size_t nc = (N + OR_DOT_CHUNK - 1) / OR_DOT_CHUNK;
    double *part = (double *)malloc((nc ? nc : 1) * sizeof(double));
#pragma omp parallel for
    for (size_t k = 0; k < nc; k++) {
        size_t lo = k * OR_DOT_CHUNK, hi = lo + OR_DOT_CHUNK < N ? lo + OR_DOT_CHUNK : N;
        double s = 0.0;
        for (size_t c = lo; c < hi; c++)
            if (!fixed[c]) s += a[c] * b[c];
        part[k] = s;
    }
    double s = 0.0;
    for (size_t k = 0; k < nc; k++) s += part[k];
    free(part);
    return s;
}

/* Conjugate gradients on the SPD system A u_free = b, where b holds the
 * fixed neighbours' contribution (1/4 sum of fixed neighbour values) plus
 * `source` (0 for the Laplace problem, 1 for the exit-time problem).
 * Stops when max |b - A u| <= tol (for source 0 this is the 1/4-scaled
 * residual of or_residual). */
int or_cg(double *u, const uint8_t *fixed, int nx, int ny, double source, double tol,
          int max_iters, int *iters_out, double *res_out)
{
    if (!check_border_fixed(fixed, nx, ny)) return OR_EINVAL;
    size_t N = (size_t)nx * ny;
    double *b = (double *)calloc(N, sizeof(double));
    double *r = (double *)calloc(N, sizeof(double));
    double *p = (double *)calloc(N, sizeof(double));
    double *Ap = (double *)calloc(N, sizeof(double));
    for (int j = 1; j < ny - 1; j++)
        for (int i = 1; i < nx - 1; i++) {
            size_t c = (size_t)j * nx + i;
            if (fixed[c]) continue;
            double s = 0.0;
            if (fixed[c + 1]) s += u[c + 1];
            if (fixed[c - 1]) s += u[c - 1];
            if (fixed[c + nx]) s += u[c + nx];
            if (fixed[c - nx]) s += u[c - nx];
            b[c] = 0.25 * s + source;
        }
    apply_A(u, Ap, fixed, nx, ny);
    double rmax = 0.0;
    for (size_t c = 0; c < N; c++) {
        r[c] = fixed[c] ? 0.0 : b[c] - Ap[c];
        p[c] = r[c];
        if (fabs(r[c]) > rmax) rmax = fabs(r[c]);
    }
    double rr = dot_free(r, r, fixed, N);
    int k = 0;
    while (rmax > tol && k < max_iters && rr > 0.0) {
        apply_A(p, Ap, fixed, nx, ny);
        double alpha = rr / dot_free(p, Ap, fixed, N);
#pragma omp parallel for
        for (size_t c = 0; c < N; c++)
            if (!fixed[c]) { u[c] += alpha * p[c]; r[c] -= alpha * Ap[c]; }
        k++;
        /* every 50 iterations replace the recursive residual by the true one */
        if (k % 50 == 0) {
            apply_A(u, Ap, fixed, nx, ny);
#pragma omp parallel for
            for (size_t c = 0; c < N; c++) r[c] = fixed[c] ? 0.0 : b[c] - Ap[c];
        }
        double rr_new = dot_free(r, r, fixed, N);
        double beta = rr_new / rr;
        rr = rr_new;
        rmax = 0.0;
#pragma omp parallel for reduction(max : rmax)
        for (size_t c = 0; c < N; c++) {
            if (fixed[c]) continue;
            p[c] = r[c] + beta * p[c];
            if (fabs(r[c]) > rmax) rmax = fabs(r[c]);
        }
    }
    /* final true residual */
    apply_A(u, Ap, fixed, nx, ny);
    rmax = 0.0;
    for (size_t c = 0; c < N; c++)
        if (!fixed[c] && fabs(b[c] - Ap[c]) > rmax) rmax = fabs(b[c] - Ap[c]);
    free(b); free(r); free(p); free(Ap);
    *iters_out = k;
    *res_out = rmax;
    return (rmax <= tol) ? OR_OK : OR_NOT_CONVERGED;
}

/* ------------------------------------------------------------------------
 * Path extraction on the stored quantity u = 1 - phi (largest u = lowest
 * potential).  Eq. 3's index matrix picks, among the neighbours in the order
 * +x, -x, +y, -y, the first one with the lowest potential; the path follows
 * it from the start while the potential strictly drops, until the goal.
 * Returns OR_OK and the length, OR_NO_PATH, or OR_ESTART.
 * ---------------------------------------------------------------------- */
int or_descent(const double *u, const uint8_t *fixed, int nx, int ny,
               int sx, int sy, int gx, int gy, int max_len, int32_t *path, int *len)
{
    static const int DX[4] = {1, -1, 0, 0};
    static const int DY[4] = {0, 0, 1, -1};
    *len = 0;
    if (sx < 0 || sy < 0 || sx >= nx || sy >= ny || gx < 0 || gy < 0 || gx >= nx || gy >= ny)
        return OR_EINVAL;
    if (max_len < 1) return OR_EINVAL;
    int x = sx, y = sy;
    if (fixed[(size_t)y * nx + x] && !(x == gx && y == gy)) return OR_ESTART;
    path[0] = x; path[1] = y;
    int L = 1;
    while (!(x == gx && y == gy)) {
        double cur = u[(size_t)y * nx + x];
        int best = -1;
        double bu = cur;
        for (int k = 0; k < 4; k++) {
            int xx = x + DX[k], yy = y + DY[k];
            if (xx < 0 || yy < 0 || xx >= nx || yy >= ny) continue;
            double v = u[(size_t)yy * nx + xx];
            if (v > bu) { bu = v; best = k; }
        }
        if (best < 0 || L >= max_len) { *len = L; return OR_NO_PATH; }
        x += DX[best]; y += DY[best];
        path[2 * L] = x; path[2 * L + 1] = y;
        L++;
    }
    *len = L;
    return OR_OK;
}

/* ------------------------------------------------------------------------
 * Rubber band (Sec. 3.2, Eqs. 4-6) -- parity unpinned: the paper gives no
 * tension law, so this is a reading checked only by invariants.  Node energy
 *   E_i(q) = w / u(q) + (k/2) (|q - p_{i-1}|^2 + |q - p_{i+1}|^2)
 * (w/u is the potential term of Eq. 6 in the u = 1 - phi form, the
 * quadratic terms the tensions of the two adjacent nodes).  A sweep moves
 * the odd interior nodes, then the even ones; each goes to the lowest-energy
 * candidate of its 3x3 neighbourhood (staying is the first candidate, then
 * dy = -1..1, dx = -1..1; a move needs a strictly lower energy) among cells
 * that are free (or the goal), have u > 0, and lie within Chebyshev distance 1
 * of both path neighbours.  Endpoints stay.  Stops when no node moves or
 * after `iters` sweeps; consecutive duplicate nodes are then removed.
 * Returns the number of sweeps run; *len is updated.
 * ---------------------------------------------------------------------- */
static double band_energy(const double *u, int nx, int qx, int qy, const int32_t *path,
                          int i, double w, double k)
{
    double uq = u[(size_t)qy * nx + qx];
    double ax = qx - path[2 * (i - 1)], ay = qy - path[2 * (i - 1) + 1];
    double bx = qx - path[2 * (i + 1)], by = qy - path[2 * (i + 1) + 1];
    return w / uq + 0.5 * k * ((ax * ax + ay * ay) + (bx * bx + by * by));
}

int or_rubber_band(const double *u, const uint8_t *fixed, int nx, int ny, int gx, int gy,
                   int32_t *path, int *len, int iters, double w, double k)
{
    int L = *len;
    int s = 0;
    for (; s < iters; s++) {
        int moved = 0;
        for (int parity = 1; parity >= 0; parity--) {
            for (int i = 1; i < L - 1; i++) {
                if ((i & 1) != parity) continue;
                int px = path[2 * i], py = path[2 * i + 1];
                double best = band_energy(u, nx, px, py, path, i, w, k);
                int bx = px, by = py;
                for (int dy = -1; dy <= 1; dy++)
                    for (int dx = -1; dx <= 1; dx++) {
                        if (dx == 0 && dy == 0) continue;
                        int qx = px + dx, qy = py + dy;
                        if (qx < 0 || qy < 0 || qx >= nx || qy >= ny) continue;
                        size_t c = (size_t)qy * nx + qx;
                        if (fixed[c] && !(qx == gx && qy == gy)) continue;
                        if (!(u[c] > 0.0)) continue;
                        if (abs(qx - path[2 * (i - 1)]) > 1 || abs(qy - path[2 * (i - 1) + 1]) > 1) continue;
                        if (abs(qx - path[2 * (i + 1)]) > 1 || abs(qy - path[2 * (i + 1) + 1]) > 1) continue;
                        double e = band_energy(u, nx, qx, qy, path, i, w, k);
                        if (e < best) { best = e; bx = qx; by = qy; }
                    }
                if (bx != px || by != py) { path[2 * i] = bx; path[2 * i + 1] = by; moved = 1; }
            }
        }
        if (!moved) { s++; break; }
    }
    /* drop consecutive duplicates */
    int o = 1;
    for (int i = 1; i < L; i++) {
        if (path[2 * i] == path[2 * (o - 1)] && path[2 * i + 1] == path[2 * (o - 1) + 1]) continue;
        path[2 * o] = path[2 * i]; path[2 * o + 1] = path[2 * i + 1];
        o++;
    }
    *len = o;
    return s;
}

/* ------------------------------------------------------------------------
 * Kalman filter, constant-velocity model (Sec. 3.5): state [x, y, vx, vy],
 * A = [[1,0,dt,0],[0,1,0,dt],[0,0,1,0],[0,0,0,1]], B = 0, H = [I2 0],
 * Q(dt) = q * [[dt^3/3,0,dt^2/2,0],[0,dt^3/3,0,dt^2/2],[dt^2/2,0,dt,0],[0,dt^2/2,0,dt]],
 * R = r^2 I2.  Predict (Eqs. 9-10), then update (Eqs. 11-13).
 * ---------------------------------------------------------------------- */
static void mat4_mul(const double *a, const double *b, double *c)
{
    for (int i = 0; i < 4; i++)
        for (int j = 0; j < 4; j++) {
            double s = 0.0;
            for (int k = 0; k < 4; k++) s += a[4 * i + k] * b[4 * k + j];
            c[4 * i + j] = s;
        }
}

void or_kf_predict(double *x, double *P, double dt, double q)
{
    double A[16] = {1, 0, dt, 0, 0, 1, 0, dt, 0, 0, 1, 0, 0, 0, 0, 1};
    double At[16], T[16], Pn[16];
    for (int i = 0; i < 4; i++)
        for (int j = 0; j < 4; j++) At[4 * i + j] = A[4 * j + i];
    double xn[4];
    for (int i = 0; i < 4; i++) {
        double s = 0.0;
        for (int k = 0; k < 4; k++) s += A[4 * i + k] * x[k];
        xn[i] = s;
    }
    memcpy(x, xn, sizeof(xn));
    mat4_mul(A, P, T);
    mat4_mul(T, At, Pn);
    double d3 = dt * dt * dt / 3.0, d2 = dt * dt / 2.0;
    double Q[16] = {d3, 0, d2, 0, 0, d3, 0, d2, d2, 0, dt, 0, 0, d2, 0, dt};
    for (int i = 0; i < 16; i++) P[i] = Pn[i] + q * Q[i];
}

void or_kf_update(double *x, double *P, const double *z, double r)
{
    /* S = H P H^T + R (2x2), K = P H^T S^{-1} (4x2) */
    double S00 = P[0] + r * r, S01 = P[1], S10 = P[4], S11 = P[5] + r * r;
    double det = S00 * S11 - S01 * S10;
    double I00 = S11 / det, I01 = -S01 / det, I10 = -S10 / det, I11 = S00 / det;
    double K[8];
    for (int i = 0; i < 4; i++) {
        double ph0 = P[4 * i + 0], ph1 = P[4 * i + 1];
        K[2 * i + 0] = ph0 * I00 + ph1 * I10;
        K[2 * i + 1] = ph0 * I01 + ph1 * I11;
    }
    double y0 = z[0] - x[0], y1 = z[1] - x[1];
    for (int i = 0; i < 4; i++) x[i] += K[2 * i] * y0 + K[2 * i + 1] * y1;
    /* P = (I - K H) P */
    double IKH[16];
    for (int i = 0; i < 4; i++)
        for (int j = 0; j < 4; j++) {
            double kh = (j == 0) ? K[2 * i] : (j == 1) ? K[2 * i + 1] : 0.0;
            IKH[4 * i + j] = ((i == j) ? 1.0 : 0.0) - kh;
        }
    double Pn[16];
    mat4_mul(IKH, P, Pn);
    memcpy(P, Pn, sizeof(Pn));
}

/* One filter step for n tracks (n x 21 layout): predict by dt, update with z. */
void or_kf_step(double *tracks, int n, const double *z, double dt, double q, double r)
{
    for (int o = 0; o < n; o++) {
        double *T = tracks + 21 * (size_t)o;
        or_kf_predict(T, T + 4, dt, q);
        or_kf_update(T, T + 4, z + 2 * (size_t)o, r);
    }
}
