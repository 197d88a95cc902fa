"""Pins for the FP64 oracle: checks against what the paper and the mathematics fix,
not against the oracle itself.

Field: exact discrete harmonics (polynomials and the separable discrete
sine-sinh), the annulus log-radial solution at second order, brute-force dense
solves on small grids, the maximum principle, the random-walk reading by Monte
Carlo, symmetry, goal-free components, and the a-posteriori bound through the
exit time.  Raster: hand cases with counts of lattice points, the closed ring
boundary, the ring count of the 512x512 benchmark scene, and the closed forms
of the elliptic law (Eqs. 14-15).  Kalman filter: ordinary least squares under
a diffuse prior with Q = 0 (Eqs. 9-13) and the steady state of the discrete
algebraic Riccati equation.  Path: Eq. 3 descent invariants and rubber-band
energy monotonicity.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
import scenes

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------------------
# field: exact discrete harmonic functions
# ---------------------------------------------------------------------------

def _rect_problem(nx, ny, f):
    """Dirichlet problem on a rectangle: border fixed at f, interior free."""
    jj, ii = np.mgrid[0:ny, 0:nx].astype(np.float64)
    exact = f(ii, jj)
    fixed = np.zeros((ny, nx), np.uint8)
    fixed[0, :] = fixed[-1, :] = fixed[:, 0] = fixed[:, -1] = 1
    u0 = np.where(fixed == 1, exact, 0.0)
    return u0, fixed, exact


POLYS = {
    "linear": lambda x, y: 0.3 + 0.02 * x - 0.05 * y,
    "xy": lambda x, y: (x - 9.0) * (y - 7.0) / 100.0,
    "x2-y2": lambda x, y: ((x - 9.0) ** 2 - (y - 7.0) ** 2) / 100.0,
    "x3-3xy2": lambda x, y: ((x - 9.0) ** 3 - 3.0 * (x - 9.0) * (y - 7.0) ** 2) / 1000.0,
}


@pytest.mark.parametrize("name", sorted(POLYS))
def test_polynomials_are_fixed_points_of_all_solvers(name):
    u0, fixed, exact = _rect_problem(21, 17, POLYS[name])
    scale = np.abs(exact).max()
    u, _, r, st = oracle.cg(u0, fixed, tol=1e-15 * scale)
    assert st == oracle.OK
    assert np.abs(u - exact).max() <= 1e-12 * scale
    uj, _, _, st = oracle.jacobi(u0, fixed, tol=1e-13 * scale)
    assert st == oracle.OK and np.abs(uj - exact).max() <= 1e-10 * scale
    ug, _, _, st = oracle.gauss_seidel(u0, fixed, tol=1e-13 * scale)
    assert st == oracle.OK and np.abs(ug - exact).max() <= 1e-10 * scale


@pytest.mark.parametrize("k", [1, 2, 3])
def test_discrete_sine_sinh(k):
    N, M = 24, 30   # i = 0..N, j = 0..M
    mu = math.acosh(2.0 - math.cos(k * math.pi / N))

    def f(i, j):
        return np.sin(k * np.pi * i / N) * np.sinh(mu * j) / math.sinh(mu * M)

    u0, fixed, exact = _rect_problem(N + 1, M + 1, f)
    u, _, _, st = oracle.cg(u0, fixed, tol=1e-15)
    assert st == oracle.OK
    assert np.abs(u - exact).max() <= 1e-13


def test_continuous_sine_matches_to_second_order():
    errs = []
    for n in (17, 33, 65):
        h = 1.0 / (n - 1)

        def f(i, j):
            x, y = i * h, j * h
            return np.sin(np.pi * x) * np.sinh(np.pi * y) / math.sinh(math.pi)

        u0, fixed, exact = _rect_problem(n, n, f)
        u, _, _, _ = oracle.cg(u0, fixed, tol=1e-14)
        errs.append(np.abs(u - exact).max())
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(1.8 < o < 2.2 for o in orders), (errs, orders)


def _annulus(n, a=0.25, b=0.9):
    h = 2.0 / (n - 1)
    jj, ii = np.mgrid[0:n, 0:n].astype(np.float64)
    x, y = -1.0 + ii * h, -1.0 + jj * h
    r = np.hypot(x, y)
    exact = np.log(np.maximum(r, 1e-300) / a) / math.log(b / a)
    fixed = ((r <= a) | (r >= b)).astype(np.uint8)
    fixed[0, :] = fixed[-1, :] = fixed[:, 0] = fixed[:, -1] = 1
    u0 = np.where(fixed == 1, exact, 0.5)
    return u0, fixed, exact


def test_annulus_log_radial_second_order():
    errs = []
    for n in (32, 64, 128, 256):
        u0, fixed, exact = _annulus(n)
        u, _, _, st = oracle.cg(u0, fixed, tol=1e-13)
        assert st == oracle.OK
        free = fixed == 0
        errs.append(np.abs(u - exact)[free].max())
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
    # staircase boundary: the order fluctuates around 2 but the error must fall ~4x
    assert np.mean(orders) > 1.6, (errs, orders)
    assert errs[-1] < 2e-3


# ---------------------------------------------------------------------------
# field: brute-force dense solve and invariants
# ---------------------------------------------------------------------------

def _random_small(seed, nx=16, ny=16, p=0.2):
    rng = np.random.default_rng(seed)
    occ = (rng.random((ny, nx)) < p).astype(np.uint8)
    occ[0, :] = occ[-1, :] = occ[:, 0] = occ[:, -1] = 3
    free = np.argwhere(occ == 0)
    gy, gx = free[rng.integers(len(free))]
    return occ, (int(gx), int(gy))


def _dense_solve(occ, goal):
    """Assemble (I - J) on free cells with numpy and solve it directly."""
    u0, fixed = oracle.dirichlet_from_occ(occ, goal)
    ny, nx = occ.shape
    idx = -np.ones((ny, nx), np.int64)
    free = np.argwhere(fixed == 0)
    for n, (j, i) in enumerate(free):
        idx[j, i] = n
    A = np.eye(len(free))
    b = np.zeros(len(free))
    for n, (j, i) in enumerate(free):
        for dj, di in ((0, 1), (0, -1), (1, 0), (-1, 0)):
            jj, ii = j + dj, i + di
            if fixed[jj, ii]:
                b[n] += 0.25 * u0[jj, ii]
            else:
                A[n, idx[jj, ii]] -= 0.25
    x = np.linalg.solve(A, b)
    u = u0.copy()
    u[fixed == 0] = x
    return u, fixed


@pytest.mark.parametrize("seed", [1, 2, 3, 4, 5])
def test_brute_force_dense_solve(seed):
    occ, goal = _random_small(seed, 16, 13 + seed % 3)
    ref, fixed = _dense_solve(occ, goal)
    u0, _ = oracle.dirichlet_from_occ(occ, goal)
    u, _, _, st = oracle.cg(u0, fixed, tol=1e-15)
    assert st == oracle.OK and np.abs(u - ref).max() <= 1e-14
    uj, _, _, st = oracle.jacobi(u0, fixed, tol=1e-15)
    assert st == oracle.OK and np.abs(uj - ref).max() <= 1e-12
    ug, _, _, st = oracle.gauss_seidel(u0, fixed, tol=1e-15)
    assert st == oracle.OK and np.abs(ug - ref).max() <= 1e-12


def test_maximum_principle_and_no_interior_extrema():
    sc = scenes.static_occupancy(77, 48, 6, 0.15, start=(3, 3), goal=(44, 44))
    occ, _, _ = oracle.build_grid(sc)
    u, fixed = oracle.solve_field(occ, sc.goal, tol=1e-15)
    assert u.min() >= 0.0 and u.max() <= 1.0
    from scipy import ndimage
    lab, _ = ndimage.label(fixed == 0)
    gx, gy = sc.goal
    # the goal's component: free cells adjacent to the goal
    comp = {lab[gy + dy, gx + dx] for dx, dy in ((1, 0), (-1, 0), (0, 1), (0, -1))} - {0}
    ny, nx = u.shape
    checked = 0
    for j in range(1, ny - 1):
        for i in range(1, nx - 1):
            if fixed[j, i] or lab[j, i] not in comp or u[j, i] < 1e-9:
                continue
            nb = max(u[j, i + 1], u[j, i - 1], u[j + 1, i], u[j - 1, i])
            assert nb > u[j, i]
            checked += 1
    assert checked > 500


def test_component_without_goal_is_zero():
    n = 32
    occ = np.zeros((n, n), np.uint8)
    occ[0, :] = occ[-1, :] = occ[:, 0] = occ[:, -1] = 3
    occ[8:20, 8] = occ[8:20, 19] = occ[8, 8:20] = occ[19, 8:20] = 1   # closed box
    u, fixed = oracle.solve_field(occ, (26, 26), tol=1e-15)
    assert np.abs(u[9:19, 9:19]).max() <= 1e-14
    assert u[25, 25] > 0.1


def test_transpose_and_mirror_symmetry():
    occ, goal = _random_small(11, 24, 24, 0.15)
    u, _ = oracle.solve_field(occ, goal, tol=1e-15)
    ut, _ = oracle.solve_field(np.ascontiguousarray(occ.T), (goal[1], goal[0]), tol=1e-15)
    assert np.abs(u.T - ut).max() <= 1e-13
    um, _ = oracle.solve_field(np.ascontiguousarray(occ[:, ::-1]), (23 - goal[0], goal[1]), tol=1e-15)
    assert np.abs(u[:, ::-1] - um).max() <= 1e-13


def test_random_walk_monte_carlo():
    """u(c) = P(a simple random walk from c reaches the goal before any obstacle)."""
    occ, goal = _random_small(3, 8, 8, 0.1)
    u, fixed = oracle.solve_field(occ, goal, tol=1e-15)
    rng = np.random.default_rng(12345)
    free = np.argwhere(fixed == 0)
    steps = np.array([(1, 0), (-1, 0), (0, 1), (0, -1)])
    W = 40000
    for (j, i) in free[:: max(1, len(free) // 6)]:
        pos = np.tile([i, j], (W, 1))
        alive = np.ones(W, bool)
        hit = np.zeros(W, bool)
        for _ in range(4000):
            if not alive.any():
                break
            pos[alive] += steps[rng.integers(0, 4, alive.sum())]
            at_fixed = fixed[pos[:, 1], pos[:, 0]] == 1
            newly = alive & at_fixed
            hit |= newly & (pos[:, 0] == goal[0]) & (pos[:, 1] == goal[1])
            alive &= ~at_fixed
        p = hit.mean()
        sd = math.sqrt(max(u[j, i] * (1 - u[j, i]), 1e-12) / W)
        assert abs(p - u[j, i]) <= 3.5 * sd + 1e-4, (i, j, p, u[j, i])


def test_a_posteriori_bound_through_exit_time():
    sc = scenes.static128()
    occ, _, _ = oracle.build_grid(sc)
    ustar, fixed = oracle.solve_field(occ, sc.goal, tol=1e-14)
    tau = oracle.exit_time(fixed)
    assert tau.min() >= 0.0
    u0, _ = oracle.dirichlet_from_occ(occ, sc.goal)
    for sweeps in (50, 400, 2000):
        uj, _, r, _ = oracle.jacobi(u0, fixed, tol=0.0, max_sweeps=sweeps)
        err = np.abs(uj - ustar).max()
        assert err <= tau.max() * r * (1 + 1e-9) + 1e-13
        assert err >= r          # an error of at least one update size remains


def test_jacobi_gs_cg_share_the_fixed_point():
    sc = scenes.static128()
    occ, _, _ = oracle.build_grid(sc)
    ustar, fixed = oracle.solve_field(occ, sc.goal, tol=1e-14)
    u0, _ = oracle.dirichlet_from_occ(occ, sc.goal)
    tau_max = oracle.exit_time(fixed).max()
    uj, _, rj, _ = oracle.jacobi(u0, fixed, tol=1e-8)
    ug, _, rg, _ = oracle.gauss_seidel(u0, fixed, tol=1e-11)
    assert np.abs(uj - ustar).max() <= tau_max * rj
    assert np.abs(ug - ustar).max() <= tau_max * rg


# ---------------------------------------------------------------------------
# raster: hand cases
# ---------------------------------------------------------------------------

def _lattice_count(r2):
    """Number of integer points (a, b) with a^2 + b^2 <= r2."""
    r = int(math.isqrt(int(r2)))
    return sum(1 for a in range(-r, r + 1) for b in range(-r, r + 1) if a * a + b * b <= r2)


def _one_track(x, y, vx, vy, radius, P=None):
    T = np.zeros((1, 21))
    T[0, :4] = (x, y, vx, vy)
    if P is not None:
        T[0, 4:20] = np.asarray(P, float).reshape(16)
    T[0, 20] = radius
    return T


def test_raster_stationary_disk_is_gauss_circle():
    # 0.1 m cells; obstacle centred on cell (30, 30) with rho = 0.2 m = 2 cells
    sc = scenes.Scene("hand", 0, 64, 64, 0.1, static_occ=np.zeros((64, 64), np.uint8))
    sc.robot = np.array([0.55, 0.55, 1.0, 0.0, 1.0])
    law = scenes.RingLaw(r0=0.5, growth=1.5, q_accel=0.0, kappa=2.0, d_safe=0.05)
    T = _one_track(3.05, 3.05, 0.0, 0.0, 0.15)
    occ, ring, J = oracle.build_grid(sc, law=law, tracks=T)
    dyn = np.argwhere(occ == 2)
    assert len(dyn) == _lattice_count(4) == 13
    assert set(map(tuple, dyn - [30, 30])) == {(a, b) for a in range(-2, 3) for b in range(-2, 3)
                                                if a * a + b * b <= 4}


def test_raster_border_and_static_priority():
    sc = scenes.Scene("hand", 0, 20, 10, 0.1, static_occ=np.zeros((10, 20), np.uint8))
    sc.static_occ[4, 5] = 1
    sc.static_occ[0, 3] = 1          # static on the border stays border
    sc.robot = np.array([0.55, 0.55, 1.0, 0.0, 1.0])
    T = _one_track(0.55, 0.45, 0.0, 0.0, 0.3)   # disk over the border corner and cell (5, 4)?
    occ, _, _ = oracle.build_grid(sc, law=scenes.RingLaw(kappa=0.0, d_safe=0.0, q_accel=0.0), tracks=T)
    assert (occ[0, :] == 3).all() and (occ[-1, :] == 3).all()
    assert (occ[:, 0] == 3).all() and (occ[:, -1] == 3).all()
    assert occ[4, 5] == 1
    assert set(np.unique(occ)) <= {0, 1, 2, 3}


def test_ring_boundary_is_closed_and_rings_nest():
    # robot at the centre of cell (50, 50); 0.1 m cells; R = 1, 2, 4, 8 m (10, 20, 40, 80 cells)
    sc = scenes.Scene("hand", 0, 101, 101, 0.1, static_occ=np.zeros((101, 101), np.uint8))
    sc.robot = np.array([5.05, 5.05, 1.0, 0.0, 1.0])
    law = scenes.RingLaw(r0=1.0, growth=2.0, n_rings=4)
    _, ring, J = oracle.build_grid(sc, law=law, tracks=np.zeros((0, 21)))
    assert J == 4
    assert ring[50, 60] == 0 and ring[50, 61] == 1      # exactly 10 cells: inner ring
    assert ring[50, 70] == 1 and ring[50, 71] == 2
    assert ring[56, 58] == 0                            # 6^2 + 8^2 = 10^2, on the boundary
    assert ring[50, 100] == 3 and ring[0, 0] == 3       # beyond the last ring: last ring


def test_ring_count_of_512_scene():
    R, t = oracle.ring_table(scenes.RingLaw(), 512, 512, 0.05, 0.75)
    with open(os.path.join(GOLDEN, "ring_table_512.json")) as f:
        g = json.load(f)
    assert len(R) == g["J"]
    assert R[-1] >= g["diagonal_m"] > R[-2]
    assert abs(R[-1] - g["R_last_m"]) < 0.05
    assert t[0] == 0.0 and abs(t[1] - 0.5 / 0.75) < 1e-15


def test_arrival_time_moves_the_disk_into_the_right_ring():
    # robot at cell (50,50) centre, v = 1 m/s, rings 1, 2, 4, 8 m -> t = 0, 1, 2, 4 s.
    # An obstacle 6 m ahead closing at 1 m/s is predicted 4 m ahead at t_2 = 2 s: the
    # disk (rho = 0.25 m = 2.5 cells) is marked only where it overlaps ring 2.
    sc = scenes.Scene("hand", 0, 161, 101, 0.1, static_occ=np.zeros((101, 161), np.uint8))
    sc.robot = np.array([5.05, 5.05, 1.0, 0.0, 1.0])
    law = scenes.RingLaw(r0=1.0, growth=2.0, n_rings=4, q_accel=0.0, kappa=0.0, d_safe=0.05)
    T = _one_track(5.05 + 6.0, 5.05, -1.0, 0.0, 0.2)
    occ, ring, _ = oracle.build_grid(sc, law=law, tracks=T)
    got = {(int(i) - 50, int(j) - 50) for j, i in np.argwhere(occ == 2)}
    want = {(40 + a, b) for a in range(-3, 4) for b in range(-3, 4)
            if a * a + b * b <= 6.25 and (40 + a) ** 2 + b * b <= 1600}
    assert got == want and len(want) == 9


def _elliptic_ring_radius(d_ahead, d_side):
    """Closed form of Eqs. 14-15 with r_x = 4 r_y and centre 0.9 r_x ahead."""
    u, v = d_ahead, d_side
    return (-1.8 * u + math.sqrt(4 * u * u + 12.16 * v * v)) / 0.38


def test_elliptic_closed_forms():
    with open(os.path.join(GOLDEN, "elliptic_ring.json")) as f:
        g = json.load(f)
    assert abs(_elliptic_ring_radius(1.0, 0.0) - g["ahead_factor"]) < 1e-12
    assert abs(_elliptic_ring_radius(-1.0, 0.0) - g["behind_factor"]) < 1e-12
    assert abs(_elliptic_ring_radius(0.0, 1.0) - g["abeam_factor"]) < 1e-9
    # oracle's elliptic rings against the closed form, for cells straight ahead,
    # behind and abeam of a robot heading +x (rings 1, 2, 4, ... cells x 0.1 m)
    sc = scenes.Scene("hand", 0, 301, 301, 0.1, static_occ=np.zeros((301, 301), np.uint8))
    sc.robot = np.array([15.05, 15.05, 1.0, 0.0, 1.0])
    law = scenes.RingLaw(kind=scenes.RING_ELLIPTIC, r0=0.1, growth=2.0, n_rings=12)
    R, _ = oracle.ring_table(law, 301, 301, 0.1, 1.0)
    _, ring, _ = oracle.build_grid(sc, law=law, tracks=np.zeros((0, 21)))
    for dx, dy in ((37, 0), (-3, 0), (-11, 0), (0, 2), (0, 5), (123, 0), (0, 13)):
        r_needed = _elliptic_ring_radius(dx * 0.1, dy * 0.1)
        want = next((j for j in range(len(R)) if R[j] >= r_needed * (1 + 1e-12)), len(R) - 1)
        assert ring[150 + dy, 150 + dx] == want, (dx, dy, r_needed)


def test_per_obstacle_marking_uses_own_ring():
    sc = scenes.Scene("hand", 0, 161, 101, 0.1, static_occ=np.zeros((101, 161), np.uint8))
    sc.robot = np.array([5.05, 5.05, 1.0, 0.0, 1.0])
    law = scenes.RingLaw(r0=1.0, growth=2.0, n_rings=4, q_accel=0.0, kappa=0.0, d_safe=0.05,
                         mark=scenes.MARK_PER_OBSTACLE)
    # 6 m ahead: own ring 3 (4, 8] -> t_3 = 4 s -> predicted 2 m ahead, marked in full
    T = _one_track(5.05 + 6.0, 5.05, -1.0, 0.0, 0.2)
    occ, _, _ = oracle.build_grid(sc, law=law, tracks=T)
    got = {(int(i) - 50, int(j) - 50) for j, i in np.argwhere(occ == 2)}
    want = {(20 + a, b) for a in range(-3, 4) for b in range(-3, 4) if a * a + b * b <= 6.25}
    assert got == want and len(want) == 21


def test_inflation_grows_with_covariance_and_time():
    sc = scenes.Scene("hand", 0, 161, 161, 0.1, static_occ=np.zeros((161, 161), np.uint8))
    law = scenes.RingLaw(q_accel=0.0, kappa=2.0, d_safe=0.0)
    P = np.diag([0.01, 0.01, 0.04, 0.04])
    _, _, r0q = oracle.predict_disk(_one_track(0, 0, 0, 0, 0.2, P)[0], 0.0, law, 0.1)
    _, _, r1q = oracle.predict_disk(_one_track(0, 0, 0, 0, 0.2, P)[0], 1.0, law, 0.1)
    # sigma(0) = 0.1 -> rho = 0.4 m = 4 cells; sigma(1) = sqrt(0.01 + 0.04) -> rho = 0.2 + 2 sqrt(0.05)
    assert r0q == 4 * 256
    assert r1q == round((0.2 + 2 * math.sqrt(0.05)) / 0.1 * 256)


def _cv_prediction(x, P, t, q):
    """Mean and covariance of the constant-velocity model (Eqs. 9-10) after t
    seconds, built from the model's definition rather than from any closed-form
    entry: the transition A(t) as a 4x4 matrix, the propagated covariance
    A P A^T by matrix products, and the white-noise-acceleration term
    Q(t) = q * integral_0^t A(s) L L^T A(s)^T ds (L maps the two accelerations
    onto the velocities), integrated with Simpson's rule, which is exact here
    because the integrand is a polynomial of degree 2 in s."""
    def A(s):
        a = np.eye(4)
        a[0, 2] = a[1, 3] = s
        return a
    L = np.zeros((4, 2))
    L[2, 0] = L[3, 1] = 1.0
    f = lambda s: A(s) @ L @ L.T @ A(s).T
    Q = q * (t / 6.0) * (f(0.0) + 4.0 * f(t / 2.0) + f(t))
    return A(t) @ x, A(t) @ P @ A(t).T + Q


def test_prediction_matches_the_constant_velocity_model_with_process_noise():
    # a non-diagonal covariance (position-velocity cross terms of both axes, an x-y
    # coupling that must not matter) and q > 0: every term of the prediction counts
    rng = np.random.default_rng(11)
    cell, ox, oy = 0.05, -1.3, 2.1
    law = scenes.RingLaw(q_accel=0.02, kappa=2.0, d_safe=0.25)
    G = rng.normal(size=(4, 4)) * np.array([0.15, 0.15, 0.3, 0.3])[:, None]
    P = G @ G.T + np.diag([0.01, 0.02, 0.05, 0.04])
    P[0, 2] = P[2, 0] = 0.03     # Pxv
    P[1, 3] = P[3, 1] = -0.02    # Pyv
    x = np.array([3.7, -0.4, 0.6, -0.9])
    radius = 0.3
    trk = _one_track(*x, radius, P)[0]
    for t in (0.0, 0.4, 1.3, 3.0, 7.5):
        mean, S = _cv_prediction(x, P, t, law.q_accel)
        sigma = math.sqrt(0.5 * (S[0, 0] + S[1, 1]))
        rho = radius + law.d_safe + law.kappa * sigma
        pxq, pyq, rhoq = oracle.predict_disk(trk, t, law, cell, ox, oy)
        # one quantum (cell / 256) of slack for the different rounding order
        assert abs(pxq - round((mean[0] - ox) / cell * 256)) <= 1, t
        assert abs(pyq - round((mean[1] - oy) / cell * 256)) <= 1, t
        assert abs(rhoq - round(rho / cell * 256)) <= 1, (t, rhoq, rho / cell * 256)
        if t < 1.0:
            continue
        # the pin separates the plausible misreadings of Eqs. 9-10 by many quanta
        def q_rho(s2):
            return round((radius + law.d_safe + law.kappa * math.sqrt(s2)) / cell * 256)
        pxx, pyy = S[0, 0], S[1, 1]
        q3 = law.q_accel * t ** 3 / 3.0
        wrong = {
            "no 1/3 on the process noise": 0.5 * (pxx + pyy) + 2.0 * q3,
            "no process noise": 0.5 * (pxx + pyy) - q3,
            "no position-velocity cross terms": 0.5 * (pxx + pyy) - 2.0 * t * (P[0, 2] + P[1, 3]) / 2.0,
            "cross terms once, not twice": 0.5 * (pxx + pyy) - t * (P[0, 2] + P[1, 3]) / 2.0,
            "velocity variance times t, not t^2": 0.5 * (pxx + pyy) - (t * t - t) * (P[2, 2] + P[3, 3]) / 2.0,
            "x axis only": pxx,
        }
        for name, s2 in wrong.items():
            assert abs(q_rho(s2) - rhoq) >= 5, (t, name)


# ---------------------------------------------------------------------------
# Kalman filter
# ---------------------------------------------------------------------------

def test_kf_matches_least_squares_under_diffuse_prior():
    rng = np.random.default_rng(5)
    n, dt = 12, 0.1
    times = dt * np.arange(n)
    truth = np.stack([1.0 + 0.7 * times, -2.0 + 0.3 * times], 1)
    z = truth + 0.05 * rng.standard_normal((n, 2))
    # diffuse prior P0 = 1e6 I: its pull on the posterior is O(r^2 / 1e6) ~ 1e-9,
    # while the (I - KH) P form of Eq. 12 loses ~6 digits of P to cancellation
    T = oracle.kf_init(z[0:1], np.array([0.2]), r_meas=0.05, p_vel=1e6)
    T[0, 4:20] = np.diag([1e6, 1e6, 1e6, 1e6]).reshape(16)
    T[0, 0:2] = 0.0
    T = oracle.kf_step(T, z[0:1], dt=0.0, q=0.0, r=0.05)
    for k in range(1, n):
        T = oracle.kf_step(T, z[k:k + 1], dt=dt, q=0.0, r=0.05)
    for ax in range(2):
        X = np.stack([np.ones(n), times - times[-1]], 1)
        coef, *_ = np.linalg.lstsq(X, z[:, ax], rcond=None)
        assert abs(T[0, ax] - coef[0]) < 1e-6
        assert abs(T[0, 2 + ax] - coef[1]) < 1e-5


def test_kf_covariance_reaches_riccati_steady_state():
    from scipy.linalg import solve_discrete_are
    dt, q, r = 0.1, 0.01, 0.05
    T = oracle.kf_init(np.zeros((1, 2)), np.array([0.2]), r_meas=r, p_vel=1.0)
    for _ in range(2000):
        T = oracle.kf_step(T, np.zeros((1, 2)), dt=dt, q=q, r=r)
    P_post = T[0, 4:20].reshape(4, 4)
    assert np.allclose(P_post, P_post.T, atol=1e-15)
    assert np.linalg.eigvalsh(P_post).min() > 0
    A = np.array([[1, 0, dt, 0], [0, 1, 0, dt], [0, 0, 1, 0], [0, 0, 0, 1.0]])
    H = np.hstack([np.eye(2), np.zeros((2, 2))])
    d3, d2 = dt ** 3 / 3, dt ** 2 / 2
    Q = q * np.array([[d3, 0, d2, 0], [0, d3, 0, d2], [d2, 0, dt, 0], [0, d2, 0, dt]])
    P_prior = solve_discrete_are(A.T, H.T, Q, r * r * np.eye(2))
    # the filter's prior for the next step is A P_post A^T + Q
    assert np.allclose(A @ P_post @ A.T + Q, P_prior, rtol=1e-8, atol=1e-14)


# ---------------------------------------------------------------------------
# path
# ---------------------------------------------------------------------------

def test_descent_invariants_on_static_scene():
    sc = scenes.static128()
    occ, _, _ = oracle.build_grid(sc)
    u, fixed = oracle.solve_field(occ, sc.goal, tol=1e-14)
    st, path = oracle.descent(u, fixed, sc.start, sc.goal)
    assert st == oracle.OK
    assert tuple(path[0]) == sc.start and tuple(path[-1]) == sc.goal
    steps = np.abs(np.diff(path, axis=0)).sum(1)
    assert (steps == 1).all()
    vals = u[path[:, 1], path[:, 0]]
    assert (np.diff(vals) > 0).all()
    assert (occ[path[:-1, 1], path[:-1, 0]] == 0).all()


def test_rubber_band_energy_non_increasing_and_valid():
    sc = scenes.static128()
    occ, _, _ = oracle.build_grid(sc)
    u, fixed = oracle.solve_field(occ, sc.goal, tol=1e-14)
    st, path = oracle.descent(u, fixed, sc.start, sc.goal)
    # total energy E = sum_i w/u(p_i) + (k/2) sum_i |p_{i+1} - p_i|^2 over the chain
    def E(p):
        pot = (1e-3 / u[p[1:-1, 1], p[1:-1, 0]]).sum()
        d = np.diff(p.astype(np.float64), axis=0)
        return pot + 0.5 * (d * d).sum()
    e_prev = E(path)
    for _ in range(30):
        path, _ = oracle.rubber_band(u, fixed, sc.goal, path, iters=1)
        e = E(path)
        assert e <= e_prev * (1 + 1e-12)
        e_prev = e
        assert (np.abs(np.diff(path, axis=0)).max(1) == 1).all()    # 8-connected, no repeats
        inner = path[:-1]
        assert (fixed[inner[:, 1], inner[:, 0]] == 0).all()
    assert tuple(path[0]) == sc.start and tuple(path[-1]) == sc.goal


def test_enclosed_goal_has_no_path_and_blocked_start():
    n = 40
    occ = np.zeros((n, n), np.uint8)
    occ[0, :] = occ[-1, :] = occ[:, 0] = occ[:, -1] = 3
    occ[10:20, 10] = occ[10:20, 19] = occ[10, 10:20] = occ[19, 10:20] = 1
    u, fixed = oracle.solve_field(occ, (15, 15), tol=1e-15)
    st, _ = oracle.descent(u, fixed, (30, 30), (15, 15))
    assert st == oracle.NO_PATH
    st, _ = oracle.descent(u, fixed, (10, 12), (15, 15))
    assert st == oracle.ESTART


# ---------------------------------------------------------------------------
# warm-start network reference
# ---------------------------------------------------------------------------

def test_nn_oracle_gradients_match_finite_differences():
    from oracle import nn_oracle as nn
    rng = np.random.default_rng(3)
    H = W = 16
    occ = (rng.random((H, W)) < 0.2).astype(np.uint8)
    goal = (9, 6)
    occ[goal[1], goal[0]] = 0
    p = np.zeros(nn.param_count())
    o = 0
    for ci, co in nn.LAYERS:   # He-scaled weights, small biases: every ReLU sees both signs
        p[o:o + co * ci * 9] = rng.standard_normal(co * ci * 9) * np.sqrt(2.0 / (9 * ci))
        o += co * ci * 9
        p[o:o + co] = 0.05 * rng.standard_normal(co)
        o += co
    target = rng.standard_normal((H, W)) * 0.3
    loss, g = nn.loss_and_grads(p, occ, goal, target)
    assert loss > 0
    idx = rng.choice(len(p), 40, replace=False)
    h = 1e-6
    for i in idx:
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        num = (nn.loss_and_grads(pp, occ, goal, target)[0] - nn.loss_and_grads(pm, occ, goal, target)[0]) / (2 * h)
        assert abs(num - g[i]) <= 1e-5 * max(1.0, abs(num)) + 1e-8, (i, num, g[i])


def test_nn_oracle_conv_delta_reproduces_kernel():
    from oracle import nn_oracle as nn
    rng = np.random.default_rng(4)
    Wt = rng.standard_normal((3, 2, 3, 3))
    b = rng.standard_normal(3)
    X = np.zeros((2, 7, 7))
    X[1, 3, 3] = 1.0
    Y = nn.conv(X, Wt, b)
    # a unit impulse at (3, 3) of channel 1 leaves the flipped kernel around (3, 3)
    for ky in range(3):
        for kx in range(3):
            assert np.allclose(Y[:, 3 + 1 - ky, 3 + 1 - kx], Wt[:, 1, ky, kx] + b)


def test_stored_static2048_reference_matches_the_scene():
    """The stored FP64 reference of the measured workload (written by
    tests/golden/make_static2048_field.py from the oracle) belongs to the scene
    the generator makes today, and is self-consistent: the sampled u* lie in
    (0, 1], the start cell is among them, and tau_max is at least the exit time
    of a free cell next to the goal (1) and below the square of the grid side.
    The sampled u* obey the maximum principle up to the reference's own error
    bound tau_max * r* (most of this cluttered field is below 1e-8: the
    potential decays exponentially away from the goal)."""
    import hashlib
    import json
    import os
    ref = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "static2048_field.json")))
    sc = scenes.static2048()
    occ, _, _ = oracle.build_grid(sc)
    assert hashlib.sha256(np.ascontiguousarray(occ).tobytes()).hexdigest() == ref["occupancy_sha256"]
    assert (ref["nx"], ref["ny"]) == (sc.nx, sc.ny) and tuple(ref["goal"]) == tuple(sc.goal)
    u = np.array([float(v) for v in ref["u_star"]])
    noise = ref["tau_max"] * ref["reference_resid_inf"]
    assert np.all((u >= -noise) & (u <= 1.0)) and ref["cells"][0] == list(sc.start)
    cells = np.asarray(ref["cells"])
    assert np.all(occ[cells[:, 1], cells[:, 0]] == 0)
    assert 1.0 <= ref["tau_max"] < float(sc.nx) ** 2 and ref["reference_resid_inf"] <= 1e-12


def test_threaded_oracle_build_returns_the_same_bits():
    """The OpenMP build (the CPU baseline's multi-core timing) shares only order-independent work
    among threads: raster, Jacobi and CG results equal the plain build's bit for bit."""
    if oracle.build_threads() is None:
        pytest.skip("no OpenMP in this compiler")
    sc = scenes.dynamic(seed=1041, side=96, n_obs=16, frames=1, static_shapes=8)
    try:
        oracle.use_threads(1)
        occ1, ring1, _ = oracle.build_grid(sc)
        u0, fixed = oracle.dirichlet_from_occ(occ1, sc.goal)
        j1 = oracle.jacobi(u0.copy(), fixed, tol=0.0, max_sweeps=200)[0]
        c1 = oracle.cg(u0.copy(), fixed, tol=1e-12)[0]
        assert oracle.use_threads(4) >= 1
        occ4, ring4, _ = oracle.build_grid(sc)
        j4 = oracle.jacobi(u0.copy(), fixed, tol=0.0, max_sweeps=200)[0]
        c4 = oracle.cg(u0.copy(), fixed, tol=1e-12)[0]
    finally:
        oracle.use_threads(1)
    assert np.array_equal(occ1, occ4) and np.array_equal(ring1, ring4)
    assert np.array_equal(j1, j4) and np.array_equal(c1, c4)


def test_marking_threshold_is_the_coverage_probability():
    """Probability-threshold marking (tw_ring_law.p_mark): a prediction marks cells only while the
    chance that the obstacle centre, distributed N(p, sigma^2 I2), lies within rho0 = radius + d_safe
    of p is at least p_mark.  That chance is the Rayleigh distribution function of |X - p| at rho0;
    here it comes from scipy's Rayleigh law (and a Monte Carlo check), not from the oracle's formula,
    and the oracle's disk appears exactly on the right side of the threshold."""
    from scipy.stats import rayleigh
    radius, d_safe, cell = 0.3, 0.25, 0.05
    rho0 = radius + d_safe
    for p_mark in (0.2, 0.5, 0.9):
        law = scenes.RingLaw(q_accel=0.0, kappa=2.0, d_safe=d_safe, p_mark=p_mark)
        # sigma at which the coverage probability equals p_mark, by bisection on scipy's CDF
        lo, hi = 1e-3, 10.0
        for _ in range(200):
            mid = 0.5 * (lo + hi)
            lo, hi = (mid, hi) if rayleigh.cdf(rho0, scale=mid) > p_mark else (lo, mid)
        s_star = 0.5 * (lo + hi)
        for f, marked in ((0.98, True), (1.02, False)):
            s = f * s_star
            P = np.diag([s * s, s * s, 0.0, 0.0])
            _, _, rq = oracle.predict_disk(_one_track(1.0, 1.0, 0.0, 0.0, radius, P)[0], 0.0, law, cell)
            assert (rq >= 0) == marked, (p_mark, f, rq)
        # Monte Carlo: the coverage at 0.98 s* is above p_mark, at 1.02 s* below
        rng = np.random.default_rng(int(p_mark * 100))
        for f, above in ((0.95, True), (1.05, False)):
            r = np.hypot(*rng.normal(0.0, f * s_star, (2, 400000)))
            assert ((r <= rho0).mean() > p_mark) == above
    # in the raster: one uncertain obstacle vanishes, a certain one stays
    sc = scenes.Scene("hand", 0, 64, 64, cell, static_occ=np.zeros((64, 64), np.uint8))
    sc.robot = np.array([0.5, 0.5, 1.0, 0.0, 1.0])
    T = np.vstack([_one_track(1.6, 1.6, 0.0, 0.0, radius, np.diag([1e-4, 1e-4, 0.0, 0.0])),
                   _one_track(2.4, 2.4, 0.0, 0.0, radius, np.diag([1.0, 1.0, 0.0, 0.0]))])
    law = scenes.RingLaw(q_accel=0.0, kappa=2.0, d_safe=d_safe, p_mark=0.5)
    occ, _, _ = oracle.build_grid(sc, law=law, tracks=T)
    dyn = np.argwhere(occ == 2)
    assert len(dyn) > 0 and np.all(np.hypot(dyn[:, 1] - 31.5, dyn[:, 0] - 31.5) <= 20)
    occ0, _, _ = oracle.build_grid(sc, law=scenes.RingLaw(q_accel=0.0, kappa=2.0, d_safe=d_safe), tracks=T)
    assert (occ0 == 2).sum() > (occ == 2).sum()
