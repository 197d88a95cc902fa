"""Replanning loop of Alg. 1 driven through the C ABI.

Per frame (10 Hz): the Kalman filter takes the frame's position measurements
(kf_update, Eqs. 7-13), the time-warped occupancy is rebuilt around the
robot's current pose (tw_build_grid, Sec. 3.4-3.5), the harmonic field is
relaxed from the previous frame's field (hp_relax with HP_WARM_START: the
occupancy is rebuilt, the field persists), and the path is extracted and
smoothed (plan_path, Eq. 3 and Eqs. 4-6).  The robot then moves along the path
by one frame's travel (Alg. 1: move to the next cell of the current path).

If predicted obstacles cover the goal cell, the frame aims at the nearest cell
that is free in this frame's raster (the robot keeps heading towards the goal
region instead of stopping).  If the robot's own cell is covered, or no path
exists, it holds its position for the frame.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

from . import (HP_WARM_START, TW_NO_PATH, TW_OK, Params, hp_relax, kf_init, kf_update, make_grid, plan_path,
               tw_build_grid, tw_nearest_free)


@dataclass
class FrameLog:
    frame: int
    robot: np.ndarray                  # pose used for the raster [x, y, hx, hy, v]
    tracks: np.ndarray                 # track states used for the raster [n, 21]
    goal: tuple
    relax: dict
    path_status: int
    path_len: int
    moved: float                       # metres travelled this frame


@dataclass
class RunResult:
    frames: List[FrameLog] = field(default_factory=list)
    trajectory: List[tuple] = field(default_factory=list)   # robot positions (m)
    reached: bool = False
    collision_frame: Optional[int] = None
    min_clearance: float = math.inf    # min over frames of (distance to a true obstacle - radii)

    @property
    def collision_free(self) -> bool:
        return self.collision_frame is None

    def path_length(self) -> float:
        t = np.asarray(self.trajectory)
        return float(np.hypot(*np.diff(t, axis=0).T).sum()) if len(t) > 1 else 0.0

    def turning_angles(self) -> np.ndarray:
        """Heading changes (degrees) between consecutive moves of the traversed path."""
        t = np.asarray(self.trajectory)
        if len(t) < 3:
            return np.zeros(0)
        d = np.diff(t, axis=0)
        d = d[np.hypot(*d.T) > 1e-9]
        a = np.arctan2(d[:, 1], d[:, 0])
        da = np.angle(np.exp(1j * np.diff(a)))
        return np.degrees(np.abs(da))


def _goal_candidates(static_occ: np.ndarray, goal, max_r: int = 40, count: int = 64):
    """Statically free cells around the goal, nearest first (the goal itself first)."""
    gx, gy = goal
    ny, nx = static_occ.shape
    cand = []
    for r in range(0, max_r + 1):
        ring = []
        for dy in range(-r, r + 1):
            for dx in range(-r, r + 1):
                if max(abs(dx), abs(dy)) != r:
                    continue
                x, y = gx + dx, gy + dy
                if 1 <= x < nx - 1 and 1 <= y < ny - 1 and static_occ[y, x] == 0:
                    ring.append((dx * dx + dy * dy, x, y))
        cand += [(x, y) for _, x, y in sorted(ring)]
        if len(cand) >= count:
            break
    return cand[:count]


def _advance(path_m: np.ndarray, dist: float):
    """Point at arc length `dist` along a polyline (metres) and the heading there."""
    seg = np.diff(path_m, axis=0)
    ln = np.hypot(*seg.T)
    acc = 0.0
    for i, L in enumerate(ln):
        if L <= 0:
            continue
        if acc + L >= dist:
            f = (dist - acc) / L
            p = path_m[i] + f * seg[i]
            return p, seg[i] / L, dist
        acc += L
    if len(ln) and ln.sum() > 0:
        j = int(np.nonzero(ln > 0)[0][-1])
        return path_m[-1].copy(), seg[j] / ln[j], acc
    return path_m[0].copy(), None, 0.0


def run(scene, frames: int, law=None, params: Optional[Params] = None, rubber_iters: int = 50,
        robot_radius: float = 0.25, speed: float = 0.75, dt: float = 0.1, r_meas: float = 0.05,
        q_accel: Optional[float] = None, device="cuda", log_fields: bool = False) -> RunResult:
    """Simulate `frames` replanning frames of `scene` (which carries true obstacle
    positions and noisy measurements per frame)."""
    import torch
    law = law or scene.law
    q_accel = law.q_accel if q_accel is None else q_accel
    params = params or Params(tol=1e-6)
    grid = make_grid(scene.nx, scene.ny, scene.cell, scene.ox, scene.oy)
    static = torch.from_numpy(np.ascontiguousarray(scene.static_occ)).to(device)
    occ = torch.empty((scene.ny, scene.nx), dtype=torch.uint8, device=device)
    u = torch.zeros((scene.ny, scene.nx), dtype=torch.float32, device=device)
    cands = _goal_candidates(scene.static_occ, scene.goal)
    cand_idx = torch.tensor([y * scene.nx + x for x, y in cands], dtype=torch.long, device=device)
    tracks = kf_init(scene.meas[0], scene.radius, r_meas=r_meas, p_vel=1.0)
    robot = np.array(scene.robot, dtype=np.float64)
    res = RunResult(trajectory=[(robot[0], robot[1])])
    warm = False
    gxm, gym = (scene.goal[0] + 0.5) * scene.cell + scene.ox, (scene.goal[1] + 0.5) * scene.cell + scene.oy
    for f in range(frames):
        if f > 0:
            kf_update(tracks, scene.meas[f], dt=dt, q_accel=q_accel, r_meas=r_meas)
        pose = robot.copy()
        tw_build_grid(grid, pose, tracks, law, static_occ=static, occ=occ)
        free = (occ.view(-1)[cand_idx] == 0).nonzero()
        if len(free):
            goal = cands[int(free[0].item())]
        else:
            goal = tw_nearest_free(grid, occ, scene.goal[0], scene.goal[1])
        sx = min(max(int((robot[0] - scene.ox) / scene.cell), 0), scene.nx - 1)
        sy = min(max(int((robot[1] - scene.oy) / scene.cell), 0), scene.ny - 1)
        moved = 0.0
        relax = {}
        pst, plen = TW_NO_PATH, 0
        if goal is not None:
            p = Params(**{**params.__dict__})
            p.flags = params.flags | (HP_WARM_START if warm else 0)
            _, relax = hp_relax(grid, occ, goal, field=u, params=p)
            warm = True
            pst, path = plan_path(grid, u, occ, (sx, sy), goal, rubber_iters=rubber_iters)
            plen = len(path)
            if pst == TW_OK and plen > 1:
                pm = (path.astype(np.float64) + 0.5) * scene.cell + np.array([scene.ox, scene.oy])
                pm[0] = robot[:2]
                pos, head, moved = _advance(pm, speed * dt)
                if head is not None:
                    robot[0:2] = pos
                    robot[2:4] = head
        res.frames.append(FrameLog(f, pose, tracks.copy(), goal or scene.goal, relax, pst, plen, moved))
        res.trajectory.append((robot[0], robot[1]))
        # collision with the true obstacles at the next frame's time
        tf = min(f + 1, scene.truth_pos.shape[0] - 1)
        d = np.hypot(*(scene.truth_pos[tf] - robot[:2]).T) - scene.radius - robot_radius
        res.min_clearance = min(res.min_clearance, float(d.min()) if len(d) else math.inf)
        if res.collision_frame is None and len(d) and d.min() < 0:
            res.collision_frame = f
        if math.hypot(robot[0] - gxm, robot[1] - gym) <= 2 * scene.cell:
            res.reached = True
            break
    return res
