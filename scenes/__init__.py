"""Seeded synthetic scenes shaped like the paper's workloads.

The paper's experiments (Sec. 4) run MobileSim on four unpublished indoor maps
with 1-16 moving obstacles; none of that is available, so these generators
stand in for them: a square arena, a Pioneer-class robot, static rectangles and
disks, and constant-velocity disk obstacles observed with Gaussian position
noise.  Everything here is an *input*: cell masks, world poses, track states
and noisy measurements.  No step of the planner (ring law, prediction, raster,
relaxation, path) is computed here, so the oracle and the CUDA path can both
consume these scenes without sharing any of the method's arithmetic.

Scene kinds (sizes follow the planner's benchmark configurations):

* ``static128``  -- 128x128 grid, 5 cm cells, 20 shapes, robot (10,10), goal (118,118).
* ``dynamic512`` -- 512x512 grid, 5 cm cells, 200 moving disks with noisy tracks.
* ``static2048`` -- 2048x2048 grid, 2000 shapes bisected to 30 % occupancy.
* ``batch``      -- one instance of the batched form: side U{64..1024}, 5-35 % occupancy,
                    10-300 tracks, per-instance ring law.
* ``dynamic1024``-- 1024x1024 grid drawn like ``dynamic512`` scaled to the arena.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Optional

import numpy as np

from .rng import Stream

# Ring-law kinds and marking modes (values match the C header's enums).
RING_CIRCULAR = 0
RING_ELLIPTIC = 1
MARK_PER_CELL = 0
MARK_PER_OBSTACLE = 1


@dataclass
class RingLaw:
    kind: int = RING_CIRCULAR
    mark: int = MARK_PER_CELL
    r0: float = 0.5          # m, first ring radius
    growth: float = 1.3      # geometric ring growth
    n_rings: int = 0         # 0: first J with R_{J-1} >= grid diagonal
    q_accel: float = 1e-4    # m^2/s^3 white-noise acceleration PSD ("very small" Q)
    kappa: float = 2.0       # inflation in standard deviations
    d_safe: float = 0.25     # m, safety distance
    time_outer: int = 0      # 0: arrival time from inner ring radius; 1: outer
    p_mark: float = 0.0      # probability threshold of the marking (0: every prediction marked)


@dataclass
class Scene:
    name: str
    seed: int
    nx: int
    ny: int
    cell: float                       # m
    ox: float = 0.0                   # world x of the corner of cell (0,0)
    oy: float = 0.0
    static_occ: Optional[np.ndarray] = None   # uint8 [ny][nx], 1 = static obstacle
    start: tuple = (0, 0)             # robot cell (i, j)
    goal: tuple = (0, 0)              # goal cell (i, j)
    robot: Optional[np.ndarray] = None        # [x, y, hx, hy, speed] (m, unit heading, m/s)
    tracks: Optional[np.ndarray] = None       # [n, 21] float64: x[4], P[16] row-major, radius
    law: RingLaw = field(default_factory=RingLaw)
    truth_pos: Optional[np.ndarray] = None    # [frames, n, 2] true obstacle centres
    truth_vel: Optional[np.ndarray] = None    # [frames, n, 2]
    meas: Optional[np.ndarray] = None         # [frames, n, 2] noisy position observations
    radius: Optional[np.ndarray] = None       # [n] obstacle body radius (m)
    dt: float = 0.1
    sigma_meas: float = 0.05

    @property
    def n_tracks(self) -> int:
        return 0 if self.tracks is None else int(self.tracks.shape[0])


# ----------------------------------------------------------------------------
# static shapes
# ----------------------------------------------------------------------------

def _paint_rect(occ, i0, j0, w, h):
    ny, nx = occ.shape
    a, b = max(i0, 0), min(i0 + w, nx)
    c, d = max(j0, 0), min(j0 + h, ny)
    if a < b and c < d:
        occ[c:d, a:b] = 1


def _paint_disk(occ, ci, cj, r):
    ny, nx = occ.shape
    r = int(r)
    a, b = max(ci - r, 0), min(ci + r + 1, nx)
    c, d = max(cj - r, 0), min(cj + r + 1, ny)
    if a >= b or c >= d:
        return
    ii = np.arange(a, b)[None, :] - ci
    jj = np.arange(c, d)[:, None] - cj
    occ[c:d, a:b] |= ((ii * ii + jj * jj) <= r * r).astype(np.uint8)


def _covers(kind, p, cell_ij):
    i, j = cell_ij
    if kind == 0:
        i0, j0, w, h = p
        return i0 <= i < i0 + w and j0 <= j < j0 + h
    ci, cj, r = p
    return (i - ci) ** 2 + (j - cj) ** 2 <= r * r


def _shapes(st: Stream, n, nx, ny, scale, keep_free, rect_frac=0.5, half_exact=False):
    """Draw n shapes (rect side U{4..20}, disk radius U{3..10}, scaled)."""
    kinds = (np.arange(n) % 2) if half_exact else (st.uniform(n) >= rect_frac).astype(np.int64)
    side_w = st.integers(4, 20, n)
    side_h = st.integers(4, 20, n)
    rad = st.integers(3, 10, n)
    px = st.uniform(n)
    py = st.uniform(n)
    out = []
    for k in range(n):
        if kinds[k] == 0:
            w = max(1, int(round(side_w[k] * scale)))
            h = max(1, int(round(side_h[k] * scale)))
            i0 = int(px[k] * (nx - w + 1))
            j0 = int(py[k] * (ny - h + 1))
            p = (i0, j0, w, h)
        else:
            r = max(1, int(round(rad[k] * scale)))
            ci = int(px[k] * nx)
            cj = int(py[k] * ny)
            p = (ci, cj, r)
        if any(_covers(int(kinds[k]), p, c) for c in keep_free):
            continue
        out.append((int(kinds[k]), p))
    return out


def _paint(nx, ny, shapes):
    occ = np.zeros((ny, nx), dtype=np.uint8)
    for kind, p in shapes:
        if kind == 0:
            _paint_rect(occ, *p)
        else:
            _paint_disk(occ, *p)
    return occ


def _connected(occ, a, b):
    """True if cells a and b lie in one 4-connected free component (border excluded)."""
    from scipy import ndimage
    free = occ == 0
    free[0, :] = free[-1, :] = False
    free[:, 0] = free[:, -1] = False
    lab, _ = ndimage.label(free)
    la = lab[a[1], a[0]]
    return la != 0 and la == lab[b[1], b[0]]


def _static_at_occupancy(seed, nx, ny, n_shapes, target, tol, keep_free, half_exact=True):
    """Bisect one global size scale until the painted occupancy hits target +- tol."""
    lo, hi = 0.05, 40.0
    best = None
    for _ in range(60):
        s = 0.5 * (lo + hi)
        occ = _paint(nx, ny, _shapes(Stream(seed), n_shapes, nx, ny, s, keep_free,
                                     half_exact=half_exact))
        frac = float(occ.mean())
        best = (occ, frac, s)
        if abs(frac - target) <= tol:
            return best
        if frac < target:
            lo = s
        else:
            hi = s
    return best


# ----------------------------------------------------------------------------
# moving obstacles
# ----------------------------------------------------------------------------

def _simulate_tracks(st: Stream, n, arena, frames, dt, sigma, avoid, clearance,
                     r_lo=0.15, r_hi=0.5, v_hi=1.0):
    """Constant-velocity disks with specular reflection at the arena walls."""
    x0, y0, x1, y1 = arena
    radius = st.uniform(n, r_lo, r_hi)
    speed = st.uniform(n, 0.0, v_hi)
    head = st.uniform(n, 0.0, 2.0 * np.pi)
    pos = np.zeros((n, 2))
    for k in range(n):
        for _ in range(1000):
            p = np.array([st.scalar() * (x1 - x0 - 2 * radius[k]) + x0 + radius[k],
                          st.scalar() * (y1 - y0 - 2 * radius[k]) + y0 + radius[k]])
            if all(np.hypot(*(p - a)) >= clearance + radius[k] for a in avoid):
                break
        pos[k] = p
    vel = np.stack([speed * np.cos(head), speed * np.sin(head)], axis=1)
    tp = np.zeros((frames, n, 2))
    tv = np.zeros((frames, n, 2))
    for f in range(frames):
        tp[f] = pos
        tv[f] = vel
        pos = pos + vel * dt
        for ax, lo_, hi_ in ((0, x0, x1), (1, y0, y1)):
            lo_b = lo_ + radius
            hi_b = hi_ - radius
            under = pos[:, ax] < lo_b
            over = pos[:, ax] > hi_b
            pos[under, ax] = 2 * lo_b[under] - pos[under, ax]
            pos[over, ax] = 2 * hi_b[over] - pos[over, ax]
            vel[under | over, ax] *= -1.0
    meas = tp + sigma * st.normal(frames * n * 2).reshape(frames, n, 2)
    return radius, tp, tv, meas


def synth_tracks(st: Stream, pos, vel, radius, sigma=0.05):
    """Plausible track states (estimate + SPD covariance) drawn around the truth.

    Used where a test needs a track state without running a filter: the
    estimate is the truth plus noise and the covariance is a random SPD matrix
    with the constant-velocity block structure (x-vx and y-vy coupled).
    """
    n = pos.shape[0]
    T = np.zeros((n, 21))
    T[:, 0:2] = pos + 0.4 * sigma * st.normal(2 * n).reshape(n, 2)
    T[:, 2:4] = vel + 0.05 * st.normal(2 * n).reshape(n, 2)
    # magnitudes around the steady state of a 10 Hz filter with sigma = 5 cm
    # measurements and a very small process noise (Pxx ~ 3e-4 m^2, Pvv ~ 2e-4 m^2/s^2)
    a = st.uniform(n, 0.4, 2.0) * 2.5e-4 * (sigma / 0.05) ** 2
    b = st.uniform(n, 0.3, 3.0) * 1.7e-4
    c = st.uniform(n, 0.2, 0.9) * np.sqrt(a * b)
    a2 = a * st.uniform(n, 0.7, 1.3)
    b2 = b * st.uniform(n, 0.7, 1.3)
    c2 = st.uniform(n, 0.2, 0.9) * np.sqrt(a2 * b2)
    P = np.zeros((n, 4, 4))
    P[:, 0, 0], P[:, 0, 2], P[:, 2, 0], P[:, 2, 2] = a, c, c, b
    P[:, 1, 1], P[:, 1, 3], P[:, 3, 1], P[:, 3, 3] = a2, c2, c2, b2
    T[:, 4:20] = P.reshape(n, 16)
    T[:, 20] = radius
    return T


def _robot_pose(scene_start_xy, goal_xy, speed):
    d = np.asarray(goal_xy, float) - np.asarray(scene_start_xy, float)
    h = d / np.hypot(*d)
    return np.array([scene_start_xy[0], scene_start_xy[1], h[0], h[1], speed])


# ----------------------------------------------------------------------------
# public constructors
# ----------------------------------------------------------------------------

def static128(seed: int = 1000) -> Scene:
    nx = ny = 128
    start, goal = (10, 10), (118, 118)
    st = Stream(seed)
    shapes = _shapes(st, 20, nx, ny, 1.0, keep_free=(start, goal))
    occ = _paint(nx, ny, shapes)
    cell = 0.05
    rx, ry = (start[0] + 0.5) * cell, (start[1] + 0.5) * cell
    gxw, gyw = (goal[0] + 0.5) * cell, (goal[1] + 0.5) * cell
    return Scene("static128", seed, nx, ny, cell, static_occ=occ, start=start, goal=goal,
                 robot=_robot_pose((rx, ry), (gxw, gyw), 0.75),
                 tracks=np.zeros((0, 21)))


def dynamic(seed: int = 1001, side: int = 512, n_obs: int = 200, frames: int = 100,
            frame: int = 0, static_shapes: int = 0) -> Scene:
    """Arena of side*5 cm with n_obs moving disks; track state synthesised at `frame`."""
    cell = 0.05 * 512.0 / side if side != 512 else 0.05
    L = side * cell
    nx = ny = side
    rxy = (1.0 * L / 25.6, 1.0 * L / 25.6)
    gxy = (L - 1.0 * L / 25.6, L - 1.0 * L / 25.6)
    st = Stream(seed)
    radius, tp, tv, meas = _simulate_tracks(st, n_obs, (0.0, 0.0, L, L), frames, 0.1, 0.05,
                                            avoid=(np.array(rxy), np.array(gxy)), clearance=1.0)
    start = (int(rxy[0] / cell), int(rxy[1] / cell))
    goal = (int(gxy[0] / cell), int(gxy[1] / cell))
    if static_shapes:
        occ = _paint(nx, ny, _shapes(st, static_shapes, nx, ny, side / 128.0, (start, goal)))
    else:
        occ = np.zeros((ny, nx), np.uint8)
    tracks = synth_tracks(st, tp[frame], tv[frame], radius)
    return Scene(f"dynamic{side}", seed, nx, ny, cell, static_occ=occ, start=start, goal=goal,
                 robot=_robot_pose(rxy, gxy, 0.75), tracks=tracks, truth_pos=tp, truth_vel=tv,
                 meas=meas, radius=radius)


def dynamic512(seed: int = 1001, frame: int = 0) -> Scene:
    return dynamic(seed, 512, 200, 100, frame)


def dynamic1024(seed: int = 1004, frame: int = 0) -> Scene:
    return dynamic(seed, 1024, 200, 100, frame)


def static_occupancy(seed: int, side: int, n_shapes: int, occupancy: float,
                     start=None, goal=None, tol: float = 0.005, name="static") -> Scene:
    """Square static scene whose shapes are scaled until `occupancy` +- tol is reached."""
    nx = ny = side
    start = start or (max(1, side // 100 + 1), max(1, side // 100 + 1))
    goal = goal or (side - 1 - start[0], side - 1 - start[1])
    s = seed
    for _ in range(64):
        occ, frac, _scale = _static_at_occupancy(s, nx, ny, n_shapes, occupancy, tol, (start, goal))
        if _connected(occ, start, goal):
            break
        s += 7919
    cell = 0.05
    rxy = ((start[0] + 0.5) * cell, (start[1] + 0.5) * cell)
    gxy = ((goal[0] + 0.5) * cell, (goal[1] + 0.5) * cell)
    sc = Scene(name, s, nx, ny, cell, static_occ=occ, start=start, goal=goal,
               robot=_robot_pose(rxy, gxy, 0.75), tracks=np.zeros((0, 21)))
    return sc


def static2048(seed: int = 1002) -> Scene:
    return static_occupancy(seed, 2048, 2000, 0.30, start=(20, 20), goal=(2027, 2027),
                            name="static2048")


def batch_instance(seed: int) -> Scene:
    """One planner of the batched form: its own size, occupancy, tracks and ring law."""
    st = Stream(seed)
    side = int(st.integers(64, 1024, 1)[0])
    occupancy = float(st.uniform(1, 0.05, 0.35)[0])
    n_obs = int(st.integers(10, 300, 1)[0])
    growth = float(st.uniform(1, 1.2, 1.4)[0])
    r0 = float(st.uniform(1, 0.3, 0.7)[0])
    n_shapes = max(4, int(round(2000 * side * side / 2048.0 ** 2)))
    sc = static_occupancy(seed + 17, side, n_shapes, occupancy, tol=0.01, name="batch")
    L = side * sc.cell
    radius, tp, tv, meas = _simulate_tracks(st, n_obs, (0.0, 0.0, L, L), 1, 0.1, 0.05,
                                            avoid=(sc.robot[:2], np.array([(sc.goal[0] + 0.5) * sc.cell,
                                                                          (sc.goal[1] + 0.5) * sc.cell])),
                                            clearance=1.0)
    sc.tracks = synth_tracks(st, tp[0], tv[0], radius)
    sc.radius = radius
    sc.law = RingLaw(r0=r0, growth=growth)
    sc.seed = seed
    return sc


def batch_fast(seed: int, side_lo: int = 64, side_hi: int = 1024) -> Scene:
    """One planner of the batched form drawn in a single painting pass: side
    U{side_lo..side_hi}, target occupancy U[5 %, 35 %] reached by adding
    shapes (rectangles sides U{4..20}, disks radius U{3..10}) until the
    painted fraction reaches it; 10-300 tracks and its own ring law.  The
    robot (5 %, 5 %) and goal (95 %, 95 %) cells are kept free; connectivity is
    not enforced (an enclosed goal is still a valid relaxation)."""
    st = Stream(seed)
    side = int(st.integers(side_lo, side_hi, 1)[0])
    target = float(st.uniform(1, 0.05, 0.35)[0])
    n_obs = int(st.integers(10, 300, 1)[0])
    growth = float(st.uniform(1, 1.2, 1.4)[0])
    r0 = float(st.uniform(1, 0.3, 0.7)[0])
    start = (max(1, side // 20), max(1, side // 20))
    goal = (side - 1 - start[0], side - 1 - start[1])
    occ = np.zeros((side, side), np.uint8)
    cells = float(side * side)
    painted = 0
    while painted < target * cells:
        batch = _shapes(st, 16, side, side, 1.0, keep_free=(start, goal))
        for kind, p in batch:
            (_paint_rect if kind == 0 else _paint_disk)(occ, *p)
        painted = int(occ.sum())
    cell = 0.05
    rxy = ((start[0] + 0.5) * cell, (start[1] + 0.5) * cell)
    gxy = ((goal[0] + 0.5) * cell, (goal[1] + 0.5) * cell)
    L = side * cell
    radius, tp, tv, meas = _simulate_tracks(st, n_obs, (0.0, 0.0, L, L), 1, 0.1, 0.05,
                                            avoid=(np.array(rxy), np.array(gxy)), clearance=1.0)
    sc = Scene("batch", seed, side, side, cell, static_occ=occ, start=start, goal=goal,
               robot=_robot_pose(rxy, gxy, 0.75), tracks=synth_tracks(st, tp[0], tv[0], radius),
               law=RingLaw(r0=r0, growth=growth), radius=radius)
    return sc


def by_name(name: str, seed: Optional[int] = None) -> Scene:
    table = {"static128": (static128, 1000), "dynamic512": (dynamic512, 1001),
             "static2048": (static2048, 1002), "dynamic1024": (dynamic1024, 1004)}
    fn, default = table[name]
    return fn(default if seed is None else seed)
