"""FP64 CPU oracle for the time-warped grid planner -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library never does, and
the oracle shares no code with it: the C source here (``twgrid_oracle.c``) is
an independent, plain restatement of the paper's method (Farzan & DeSouza,
Sec. 3, Eqs. 1-15, Alg. 1) and of the readings recorded in the design notes.

Functions and the passage each follows:

* ``ring_table``      -- time-warped rings and arrival times (Sec. 3.4, Eq. 15 for the elliptic law)
* ``predict_disk``    -- constant-velocity prediction and inflation (Eqs. 9-10, Sec. 3.4-3.5)
* ``build_grid``      -- brute-force raster: every cell x every obstacle (Alg. 1 map update)
* ``jacobi``          -- Eq. 1; ``gauss_seidel`` -- Eq. 2; ``cg`` -- the Eq. 1 fixed point by conjugate gradients
* ``residual``        -- 1/4-scaled residual, max and l2 over free cells
* ``exit_time``       -- expected exit time tau, giving the bound |u - u*| <= tau_max * r_inf
* ``descent``         -- Eq. 3 index-matrix path; ``rubber_band`` -- Eqs. 4-6 reading
* ``kf_step``         -- Kalman predict + update (Eqs. 7-13)

The field is handled as u = 1 - phi (goal 1, obstacles and border 0), the
same linear equation, which keeps relative precision where phi is near 1.

Parity unpinned: ``rubber_band``.  The paper gives the rubber band only
qualitatively (Eqs. 4-5 and a figure); the energy and move rule here are a
reading, checked by invariants (the path stays an 8-connected chain of free
cells, the energy never increases) but not by any value the paper fixes.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "twgrid_oracle.c")
_LIB = os.path.join(_HERE, "liboracle_twgrid.so")
_LIB_OMP = os.path.join(_HERE, "liboracle_twgrid_omp.so")

OK, NOT_CONVERGED, NO_PATH, EINVAL, EGOAL, ESTART = 0, 1, 2, -1, -2, -3

_lib = None
_libs = {}


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction, no fast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["cc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math",
               "-shared", "-fPIC", "-o", _LIB + ".tmp", _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(_LIB + ".tmp", _LIB)
    return _LIB


def build_threads(force: bool = False):
    """The same source built with OpenMP (the CPU baseline's multi-core timing); None if the
    compiler has no OpenMP.  Threads share only order-independent work, so results are the
    plain build's bit for bit."""
    if force or not os.path.exists(_LIB_OMP) or os.path.getmtime(_LIB_OMP) < os.path.getmtime(_SRC):
        cmd = ["cc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
               "-shared", "-fPIC", "-o", _LIB_OMP + ".tmp", _SRC, "-lm"]
        try:
            subprocess.check_call(cmd, stderr=subprocess.DEVNULL)
        except (subprocess.CalledProcessError, OSError):
            return None
        os.replace(_LIB_OMP + ".tmp", _LIB_OMP)
    return _LIB_OMP


def use_threads(n: int) -> int:
    """Run the following oracle calls on n threads (the OpenMP build) or, for n <= 1, on the
    plain build.  Returns the thread count in use."""
    global _lib
    if n <= 1:
        _lib = _open(build())
        return 1
    path = build_threads()
    if path is None:
        _lib = _open(build())
        return 1
    _lib = _open(path)
    return int(_lib.or_set_threads(int(n)))


def _load():
    global _lib
    if _lib is None:
        _lib = _open(build())
    return _lib


def _open(path):
    if path not in _libs:
        lib = ctypes.CDLL(path)
        P = ctypes.c_void_p
        i32, f64 = ctypes.c_int, ctypes.c_double
        lib.or_ring_table.argtypes = [i32, f64, f64, i32, f64, i32, f64, f64, f64, P, P]
        lib.or_ring_table.restype = i32
        lib.or_predict_one.argtypes = [P, f64, f64, f64, f64, f64, f64, f64, f64, P, P, P]
        lib.or_predict_one.restype = None
        lib.or_build_grid.argtypes = [i32, i32, f64, f64, f64, P, P, i32, i32, i32, f64, f64,
                                      i32, f64, f64, f64, i32, f64, P, P, P]
        lib.or_build_grid.restype = i32
        lib.or_residual.argtypes = [P, P, i32, i32, P, P]
        lib.or_residual.restype = None
        for name in ("or_jacobi", "or_gauss_seidel"):
            getattr(lib, name).argtypes = [P, P, i32, i32, f64, i32, P, P]
            getattr(lib, name).restype = i32
        lib.or_cg.argtypes = [P, P, i32, i32, f64, f64, i32, P, P]
        lib.or_cg.restype = i32
        lib.or_descent.argtypes = [P, P, i32, i32, i32, i32, i32, i32, i32, P, P]
        lib.or_descent.restype = i32
        lib.or_rubber_band.argtypes = [P, P, i32, i32, i32, i32, P, P, i32, f64, f64]
        lib.or_rubber_band.restype = i32
        lib.or_kf_predict.argtypes = [P, P, f64, f64]
        lib.or_kf_update.argtypes = [P, P, P, f64]
        lib.or_kf_step.argtypes = [P, i32, P, f64, f64, f64]
        lib.or_set_threads.argtypes = [i32]
        lib.or_set_threads.restype = i32
        _libs[path] = lib
    return _libs[path]


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


# ---------------------------------------------------------------------------
# time-warped grid
# ---------------------------------------------------------------------------

def ring_table(law, nx, ny, cell, speed):
    R = np.zeros(64)
    t = np.zeros(64)
    J = _load().or_ring_table(int(law.kind), float(law.r0), float(law.growth), int(law.n_rings),
                              float(speed), int(law.time_outer), float(nx), float(ny), float(cell),
                              _p(R), _p(t))
    if J <= 0:
        raise ValueError("invalid ring law")
    return R[:J].copy(), t[:J].copy()


def predict_disk(track, t, law, cell, ox=0.0, oy=0.0):
    """Fixed-point predicted centre and inflated radius of one track at time t."""
    trk = np.ascontiguousarray(track, dtype=np.float64)
    out = [ctypes.c_int64() for _ in range(3)]
    p_mark = float(getattr(law, "p_mark", 0.0))
    alpha = 1.0 / math.sqrt(-2.0 * math.log(1.0 - p_mark)) if p_mark > 0.0 else 0.0   # as or_build_grid
    _load().or_predict_one(_p(trk), float(t), float(law.q_accel), float(law.kappa),
                           float(law.d_safe), float(alpha), float(ox), float(oy), float(cell),
                           *[ctypes.byref(o) for o in out])
    return tuple(int(o.value) for o in out)


def build_grid(scene, law=None, robot=None, tracks=None, static_occ="scene"):
    """Brute-force time-warped occupancy raster; returns (occ uint8, ring int16, J)."""
    law = law or scene.law
    robot = np.ascontiguousarray(scene.robot if robot is None else robot, dtype=np.float64)
    tracks = scene.tracks if tracks is None else tracks
    tracks = np.ascontiguousarray(tracks if tracks is not None else np.zeros((0, 21)),
                                  dtype=np.float64).reshape(-1, 21)
    st = scene.static_occ if isinstance(static_occ, str) else static_occ
    occ = np.zeros((scene.ny, scene.nx), np.uint8)
    ring = np.zeros((scene.ny, scene.nx), np.int16)
    st_p = None
    if st is not None:
        st = np.ascontiguousarray(st, dtype=np.uint8)
        st_p = _p(st)
    J = _load().or_build_grid(scene.nx, scene.ny, scene.cell, scene.ox, scene.oy, _p(robot),
                              _p(tracks), tracks.shape[0], int(law.kind), int(law.mark),
                              float(law.r0), float(law.growth), int(law.n_rings),
                              float(law.q_accel), float(law.kappa), float(law.d_safe),
                              int(law.time_outer), float(getattr(law, "p_mark", 0.0)), st_p, _p(occ), _p(ring))
    if J <= 0:
        raise ValueError(f"or_build_grid failed: {J}")
    return occ, ring, J


# ---------------------------------------------------------------------------
# harmonic field (u = 1 - phi)
# ---------------------------------------------------------------------------

def dirichlet_from_occ(occ, goal, init=0.5):
    """Initial u and fixed mask of the planner's problem (Sec. 3.1): obstacles and
    border fixed at u = 0 (phi = 1), the goal fixed at u = 1 (phi = 0), free
    cells start at u = 0.5."""
    fixed = occ != 0
    u = np.where(fixed, 0.0, init).astype(np.float64)
    gx, gy = goal
    u[gy, gx] = 1.0
    fixed = fixed.copy()
    fixed[gy, gx] = True
    return np.ascontiguousarray(u), np.ascontiguousarray(fixed.astype(np.uint8))


def residual(u, fixed):
    u = np.ascontiguousarray(u, dtype=np.float64)
    fixed = np.ascontiguousarray(fixed, dtype=np.uint8)
    a, b = ctypes.c_double(), ctypes.c_double()
    _load().or_residual(_p(u), _p(fixed), u.shape[1], u.shape[0], ctypes.byref(a), ctypes.byref(b))
    return a.value, b.value


def _iterate(name, u, fixed, tol, max_sweeps):
    u = np.array(u, dtype=np.float64, order="C", copy=True)
    fixed = np.ascontiguousarray(fixed, dtype=np.uint8)
    k, r = ctypes.c_int(), ctypes.c_double()
    st = getattr(_load(), name)(_p(u), _p(fixed), u.shape[1], u.shape[0], float(tol),
                                int(max_sweeps), ctypes.byref(k), ctypes.byref(r))
    if st < 0:
        raise ValueError(f"{name}: invalid problem (border must be fixed)")
    return u, k.value, r.value, st


def jacobi(u, fixed, tol, max_sweeps=10_000_000):
    """Eq. 1 sweeps to residual <= tol; returns (u, sweeps, residual, status)."""
    return _iterate("or_jacobi", u, fixed, tol, max_sweeps)


def gauss_seidel(u, fixed, tol, max_sweeps=10_000_000):
    """Eq. 2 (lexicographic) sweeps to residual <= tol."""
    return _iterate("or_gauss_seidel", u, fixed, tol, max_sweeps)


def cg(u, fixed, tol=1e-13, source=0.0, max_iters=1_000_000):
    u = np.array(u, dtype=np.float64, order="C", copy=True)
    fixed = np.ascontiguousarray(fixed, dtype=np.uint8)
    k, r = ctypes.c_int(), ctypes.c_double()
    st = _load().or_cg(_p(u), _p(fixed), u.shape[1], u.shape[0], float(source), float(tol),
                       int(max_iters), ctypes.byref(k), ctypes.byref(r))
    if st < 0:
        raise ValueError("or_cg: invalid problem (border must be fixed)")
    return u, k.value, r.value, st


def solve_field(occ, goal, tol=1e-13):
    """Tightly converged u* of the planner's Dirichlet problem (CG from the 0.5 init)."""
    u0, fixed = dirichlet_from_occ(occ, goal)
    u, _, r, st = cg(u0, fixed, tol=tol)
    if st != OK:
        raise RuntimeError(f"oracle CG did not reach {tol} (r={r})")
    return u, fixed


def exit_time(fixed, tol=1e-10):
    """tau with tau_c = 1 + (1/4) sum tau_n on free cells, 0 on fixed cells."""
    u0 = np.zeros(fixed.shape)
    tau, _, _, st = cg(u0, fixed, tol=tol, source=1.0)
    return tau


# ---------------------------------------------------------------------------
# path
# ---------------------------------------------------------------------------

def descent(u, fixed, start, goal, max_len=None):
    u = np.ascontiguousarray(u, dtype=np.float64)
    fixed = np.ascontiguousarray(fixed, dtype=np.uint8)
    ny, nx = u.shape
    max_len = max_len or 4 * nx * ny
    path = np.zeros((max_len, 2), np.int32)
    L = ctypes.c_int()
    st = _load().or_descent(_p(u), _p(fixed), nx, ny, int(start[0]), int(start[1]),
                            int(goal[0]), int(goal[1]), int(max_len), _p(path), ctypes.byref(L))
    return st, path[:L.value].copy()


def rubber_band(u, fixed, goal, path, iters=100, w=1e-3, k=1.0):
    u = np.ascontiguousarray(u, dtype=np.float64)
    fixed = np.ascontiguousarray(fixed, dtype=np.uint8)
    p = np.ascontiguousarray(path, dtype=np.int32).copy()
    L = ctypes.c_int(p.shape[0])
    s = _load().or_rubber_band(_p(u), _p(fixed), u.shape[1], u.shape[0], int(goal[0]),
                               int(goal[1]), _p(p), ctypes.byref(L), int(iters), float(w), float(k))
    return p[:L.value].copy(), s


def plan_path(u, fixed, start, goal, rubber_iters=100, max_len=None, w=1e-3, k=1.0):
    st, path = descent(u, fixed, start, goal, max_len)
    if st != OK:
        return st, path
    if rubber_iters > 0 and path.shape[0] > 2:
        path, _ = rubber_band(u, fixed, goal, path, rubber_iters, w, k)
    return st, path


# ---------------------------------------------------------------------------
# Kalman filter
# ---------------------------------------------------------------------------

def kf_init(z, radius, r_meas=0.05, p_vel=1.0):
    """x0 = [z, 0, 0], P0 = diag(r^2, r^2, p_vel, p_vel)."""
    n = z.shape[0]
    T = np.zeros((n, 21))
    T[:, 0:2] = z
    P = np.zeros((n, 4, 4))
    P[:, 0, 0] = P[:, 1, 1] = r_meas ** 2
    P[:, 2, 2] = P[:, 3, 3] = p_vel
    T[:, 4:20] = P.reshape(n, 16)
    T[:, 20] = radius
    return T


def kf_step(tracks, z, dt=0.1, q=0.01, r=0.05):
    T = np.array(tracks, dtype=np.float64, order="C", copy=True).reshape(-1, 21)
    zz = np.ascontiguousarray(z, dtype=np.float64).reshape(-1, 2)
    _load().or_kf_step(_p(T), T.shape[0], _p(zz), float(dt), float(q), float(r))
    return T
