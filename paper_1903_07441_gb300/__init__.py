"""GB300-native time-warped grid planner (Farzan & DeSouza, arXiv 1903.07441).

Thin Python binding over ``libtwgrid.so`` (C ABI in ``include/twgrid.h``).
The functions carry the C names and only marshal arguments: every step of the
planner -- ring table, track prediction, raster, relaxation, residuals, path
descent and rubber band -- runs in the library's CUDA kernels.  PyTorch
supplies device memory and the current stream.  There is no CPU fallback: if
the library is missing or no GPU is present, the calls raise.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtwgrid.so")

# status codes (include/twgrid.h)
TW_OK, TW_NOT_CONVERGED, TW_NO_PATH = 0, 1, 2
TW_EINVAL, TW_EGOAL_BLOCKED, TW_ESTART_BLOCKED, TW_ECUDA, TW_EWORKSPACE = -1, -2, -3, -4, -5
TW_RING_CIRCULAR, TW_RING_ELLIPTIC = 0, 1
TW_MARK_PER_CELL, TW_MARK_PER_OBSTACLE = 0, 1
TW_FREE, TW_STATIC, TW_DYNAMIC, TW_BORDER = 0, 1, 2, 3
HP_JACOBI, HP_RBSOR, HP_MIXED = 0, 1, 2
HP_STORE_F32, HP_STORE_F16, HP_STORE_BF16 = 0, 1, 2
HP_WARM_START, HP_OUT_PHI, HP_TIMING, HP_HOST_LOOP, HP_POLISH = 1, 2, 4, 8, 16
HP_LOOP_HOST, HP_LOOP_GRAPH = 0, 1
WS_CONV_AUTO, WS_CONV_SIMT, WS_CONV_MMA, WS_CONV_TC = 0, 1, 2, 3

EXPORTS = (
    "tw_build_grid_workspace_size", "tw_build_grid", "tw_build_grids_workspace_size", "tw_build_grids",
    "tw_ring_count", "tw_nearest_free", "hp_omega_update", "hp_omega_cap", "hp_omega_initial",
    "hp_relax_workspace_size", "hp_relax", "hp_relax_noalloc", "hp_relax_dirichlet", "hp_residual",
    "hp_relax_batched_workspace_size", "hp_relax_batched",
    "plan_path_workspace_size", "plan_path", "plan_path_ex",
    "kf_update", "kf_init", "ws_unet_param_count", "ws_unet_workspace_size", "ws_unet_init", "ws_make_target",
    "ws_unet_forward", "ws_unet_train_step", "ws_unet_warm_start_workspace_size", "ws_unet_warm_start",
    "ws_conv3x3_workspace_size", "ws_conv3x3", "ws_conv3x3_wgrad_workspace_size", "ws_conv3x3_wgrad",
    "ws_conv_check",
    "tw_status_string", "tw_last_cuda_error", "tw_launch_count", "tw_version",
)


class TwError(RuntimeError):
    def __init__(self, fn, status):
        self.status = status
        super().__init__(f"{fn}: {status_string(status)} ({status})")


# ---------------------------------------------------------------------------
# C structs
# ---------------------------------------------------------------------------

class tw_grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("cell", ctypes.c_double),
                ("ox", ctypes.c_double), ("oy", ctypes.c_double)]


class tw_pose(ctypes.Structure):
    _fields_ = [("x", ctypes.c_double), ("y", ctypes.c_double), ("hx", ctypes.c_double),
                ("hy", ctypes.c_double), ("speed", ctypes.c_double)]


class tw_ring_law(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("mark", ctypes.c_int), ("r0", ctypes.c_double),
                ("growth", ctypes.c_double), ("n_rings", ctypes.c_int), ("q_accel", ctypes.c_double),
                ("kappa", ctypes.c_double), ("d_safe", ctypes.c_double), ("time_outer", ctypes.c_int),
                ("p_mark", ctypes.c_double)]


class tw_grid_job(ctypes.Structure):
    _fields_ = [("grid", tw_grid), ("robot", tw_pose), ("law", tw_ring_law), ("tracks", ctypes.c_void_p),
                ("n_tracks", ctypes.c_int), ("static_occ_dev", ctypes.c_void_p), ("occ_dev", ctypes.c_void_p),
                ("ring_dev", ctypes.c_void_p)]


class hp_params(ctypes.Structure):
    _fields_ = [("method", ctypes.c_int), ("storage", ctypes.c_int), ("omega", ctypes.c_double),
                ("tol", ctypes.c_double), ("max_sweeps", ctypes.c_int), ("check_every", ctypes.c_int),
                ("tblock", ctypes.c_int), ("flags", ctypes.c_int), ("etol", ctypes.c_double)]


class hp_instance(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("occ_dev", ctypes.c_void_p),
                ("gx", ctypes.c_int), ("gy", ctypes.c_int), ("field_dev", ctypes.c_void_p)]


class hp_stats(ctypes.Structure):
    _fields_ = [("sweeps", ctypes.c_int), ("status", ctypes.c_int), ("resid_inf", ctypes.c_double),
                ("resid_l2", ctypes.c_double), ("omega", ctypes.c_double), ("checks", ctypes.c_int),
                ("sweep_launches", ctypes.c_int), ("sweep_ms", ctypes.c_double), ("tblock", ctypes.c_int),
                ("loop", ctypes.c_int), ("polishes", ctypes.c_int),
                ("polished", ctypes.c_int), ("resid_check", ctypes.c_double), ("err_est", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


TRACK_DOUBLES = 21  # tw_track: x[4], P[16], radius


@dataclass
class Params:
    method: int = HP_RBSOR
    storage: int = HP_STORE_F32
    omega: float = 0.0
    tol: float = 1e-6
    max_sweeps: int = 1_000_000
    check_every: int = 0
    tblock: int = 0
    flags: int = 0
    etol: float = 0.0

    def c(self) -> hp_params:
        return hp_params(self.method, self.storage, self.omega, self.tol, self.max_sweeps,
                         self.check_every, self.tblock, self.flags, self.etol)


# ---------------------------------------------------------------------------
# library loading
# ---------------------------------------------------------------------------

_lib = None


def load() -> ctypes.CDLL:
    """Load libtwgrid.so; raises if it has not been built (no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libtwgrid.so not built at {LIB_PATH}: run paper_1903_07441_gb300/build.py "
                          "(or __graft_entry__.build())")
    lib = ctypes.CDLL(LIB_PATH)
    P, I, D, Z = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_size_t
    lib.tw_build_grid_workspace_size.argtypes = [P, I, P]
    lib.tw_build_grid_workspace_size.restype = Z
    lib.tw_build_grid.argtypes = [P, P, P, I, P, P, P, P, P, Z, P]
    lib.tw_build_grid.restype = I
    lib.hp_omega_update.argtypes = [ctypes.c_double, ctypes.c_double, I, I]
    lib.hp_omega_update.restype = ctypes.c_double
    lib.hp_omega_cap.argtypes = [I, I]
    lib.hp_omega_cap.restype = ctypes.c_double
    lib.hp_omega_initial.argtypes = [I, I]
    lib.hp_omega_initial.restype = ctypes.c_double
    lib.tw_build_grids_workspace_size.argtypes = [I, P]
    lib.tw_build_grids_workspace_size.restype = Z
    lib.tw_build_grids.argtypes = [I, P, P, Z, P]
    lib.tw_build_grids.restype = I
    lib.tw_nearest_free.argtypes = [P, P, I, I, P, P, Z, P]
    lib.tw_nearest_free.restype = I
    lib.tw_ring_count.argtypes = [P, P, P]
    lib.tw_ring_count.restype = I
    lib.hp_relax_workspace_size.argtypes = [I, I, P]
    lib.hp_relax_workspace_size.restype = Z
    lib.hp_relax.argtypes = [P, P, I, I, P, P, P, P, Z, P]
    lib.hp_relax.restype = I
    lib.hp_relax_noalloc.argtypes = [P, P, I, I, P, P, P, P]
    lib.hp_relax_noalloc.restype = I
    lib.hp_relax_batched_workspace_size.argtypes = [I, P, P]
    lib.hp_relax_batched_workspace_size.restype = Z
    lib.hp_relax_batched.argtypes = [I, P, P, P, P, P, Z, P]
    lib.hp_relax_batched.restype = I
    lib.hp_relax_dirichlet.argtypes = [I, I, P, P, P, P, P, Z, P]
    lib.hp_relax_dirichlet.restype = I
    lib.hp_residual.argtypes = [I, I, P, P, P, P, P, Z, P]
    lib.hp_residual.restype = I
    lib.plan_path_workspace_size.argtypes = [I]
    lib.plan_path_workspace_size.restype = Z
    lib.plan_path.argtypes = [P, P, P, I, I, I, I, I, I, P, P, P, Z, P]
    lib.plan_path.restype = I
    lib.plan_path_ex.argtypes = [P, P, P, I, I, I, I, I, D, D, I, P, P, P, Z, P]
    lib.plan_path_ex.restype = I
    lib.kf_update.argtypes = [P, I, P, D, D, D]
    lib.kf_update.restype = I
    lib.kf_init.argtypes = [P, I, P, P, D, D]
    lib.kf_init.restype = I
    lib.ws_unet_param_count.restype = Z
    lib.ws_unet_workspace_size.argtypes = [I, I]
    lib.ws_unet_workspace_size.restype = Z
    lib.ws_unet_init.argtypes = [P, ctypes.c_ulonglong, P]
    lib.ws_unet_init.restype = I
    lib.ws_make_target.argtypes = [P, Z, P, P]
    lib.ws_make_target.restype = I
    lib.ws_unet_forward.argtypes = [P, P, I, I, I, I, P, P, P, Z, P]
    lib.ws_unet_forward.restype = I
    lib.ws_unet_train_step.argtypes = [P, P, P, P, I, ctypes.c_float, P, I, I, I, I, P, P, P, Z, P]
    lib.ws_unet_train_step.restype = I
    lib.ws_unet_warm_start_workspace_size.argtypes = [I, I, I]
    lib.ws_unet_warm_start_workspace_size.restype = Z
    lib.ws_unet_warm_start.argtypes = [P, P, I, I, I, I, I, P, P, Z, P]
    lib.ws_unet_warm_start.restype = I
    lib.ws_conv3x3.argtypes = [P, P, P, P, P, I, I, I, I, I, I, P, Z, P]
    lib.ws_conv3x3.restype = I
    lib.ws_conv3x3_workspace_size.argtypes = [I, I, I, I, I]
    lib.ws_conv3x3_workspace_size.restype = Z
    lib.ws_conv3x3_wgrad.argtypes = [P, P, P, P, I, I, I, I, I, P, Z, P]
    lib.ws_conv3x3_wgrad.restype = I
    lib.ws_conv3x3_wgrad_workspace_size.argtypes = [I, I, I, I, I]
    lib.ws_conv3x3_wgrad_workspace_size.restype = Z
    lib.ws_conv_check.argtypes = [P]
    lib.ws_conv_check.restype = I
    lib.tw_status_string.argtypes = [I]
    lib.tw_status_string.restype = ctypes.c_char_p
    lib.tw_last_cuda_error.restype = I
    lib.tw_launch_count.restype = ctypes.c_ulonglong
    lib.tw_version.restype = ctypes.c_char_p
    _lib = lib
    return lib


def launch_count() -> int:
    """Kernels the library has launched in this process."""
    return int(load().tw_launch_count())


def status_string(status: int) -> str:
    return load().tw_status_string(int(status)).decode()


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("twgrid needs a CUDA GPU; there is no CPU fallback")
    return torch


def _ptr(t) -> ctypes.c_void_p:
    return ctypes.c_void_p(t.data_ptr())


def _stream(device):
    torch = _torch()
    return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)


_ws_cache: dict = {}


def workspace(nbytes: int, device, tag: str = "default"):
    """Cached device scratch (torch-allocated, 256-byte aligned)."""
    torch = _torch()
    key = (str(device), tag)
    buf = _ws_cache.get(key)
    if buf is None or buf.numel() < nbytes:
        buf = torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)
        _ws_cache[key] = buf
    assert buf.data_ptr() % 256 == 0
    return buf


def make_grid(nx, ny, cell, ox=0.0, oy=0.0) -> tw_grid:
    return tw_grid(int(nx), int(ny), float(cell), float(ox), float(oy))


def make_pose(robot) -> tw_pose:
    r = [float(v) for v in robot]
    return tw_pose(*r)


def make_law(law) -> tw_ring_law:
    return tw_ring_law(int(law.kind), int(law.mark), float(law.r0), float(law.growth), int(law.n_rings),
                       float(law.q_accel), float(law.kappa), float(law.d_safe), int(law.time_outer),
                       float(getattr(law, "p_mark", 0.0)))


def _check(fn, st, ok=(TW_OK,)):
    if st not in ok:
        raise TwError(fn, st)
    return st


# ---------------------------------------------------------------------------
# entry points (same names as the C ABI)
# ---------------------------------------------------------------------------

def tw_ring_count(grid: tw_grid, robot, law) -> int:
    """Ring count J of the time-warped grid (host computation, no GPU needed)."""
    J = load().tw_ring_count(ctypes.byref(grid), ctypes.byref(make_pose(robot)), ctypes.byref(make_law(law)))
    if J <= 0:
        raise TwError("tw_ring_count", J)
    return J


def tw_build_grid(grid: tw_grid, robot, tracks: np.ndarray, law, static_occ=None, occ=None, ring=None,
                  device="cuda"):
    """Time-warped occupancy raster.  tracks: host float64 [n, 21].  Returns (occ, ring)."""
    torch = _torch()
    lib = load()
    tracks = np.ascontiguousarray(tracks if tracks is not None else np.zeros((0, 21)),
                                  dtype=np.float64).reshape(-1, TRACK_DOUBLES)
    n = tracks.shape[0]
    if occ is None:
        occ = torch.empty((grid.ny, grid.nx), dtype=torch.uint8, device=device)
    c_law = make_law(law)
    ws_n = lib.tw_build_grid_workspace_size(ctypes.byref(grid), n, ctypes.byref(c_law))
    ws = workspace(ws_n, occ.device, "grid")
    st = lib.tw_build_grid(ctypes.byref(grid), ctypes.byref(make_pose(robot)),
                           tracks.ctypes.data_as(ctypes.c_void_p) if n else None, n, ctypes.byref(c_law),
                           _ptr(static_occ) if static_occ is not None else None, _ptr(occ),
                           _ptr(ring) if ring is not None else None, _ptr(ws), ws.numel(),
                           _stream(occ.device))
    _check("tw_build_grid", st)
    return occ, ring


class GridBatch:
    """A prepared tw_build_grids call: the job table (grids, poses, laws, track
    and buffer pointers) is built once and run() rasters every job.  The track
    arrays are read at each run(), so a replanning loop updates them in place.
    jobs: list of dicts with keys grid, robot, tracks (host float64 [n, 21]),
    law, and optionally static_occ, occ, ring (device tensors)."""

    def __init__(self, jobs, device="cuda"):
        torch = _torch()
        self._lib = load()
        n = len(jobs)
        self._arr = (tw_grid_job * n)()
        self._keep, self.outputs = [], []
        for i, j in enumerate(jobs):
            g = j["grid"]
            tr = np.ascontiguousarray(j.get("tracks") if j.get("tracks") is not None else np.zeros((0, 21)),
                                      dtype=np.float64).reshape(-1, TRACK_DOUBLES)
            occ = j.get("occ")
            if occ is None:
                occ = torch.empty((g.ny, g.nx), dtype=torch.uint8, device=device)
            ring, st_ = j.get("ring"), j.get("static_occ")
            self._keep.append((tr, st_))
            self._arr[i] = tw_grid_job(g, make_pose(j["robot"]), make_law(j["law"]),
                                       tr.ctypes.data if len(tr) else None, len(tr),
                                       _ptr(st_) if st_ is not None else None, _ptr(occ),
                                       _ptr(ring) if ring is not None else None)
            self.outputs.append((occ, ring))
        self.tracks = [k[0] for k in self._keep]
        self._dev = self.outputs[0][0].device
        self._ws = workspace(self._lib.tw_build_grids_workspace_size(n, self._arr), self._dev, "grids")

    def run(self):
        st = self._lib.tw_build_grids(len(self._arr), self._arr, _ptr(self._ws), self._ws.numel(),
                                      _stream(self._dev))
        _check("tw_build_grids", st)
        return self.outputs


def tw_build_grids(jobs, device="cuda"):
    """Many time-warped rasters in one call (see GridBatch).  Returns the list of (occ, ring)."""
    return GridBatch(jobs, device).run()


def tw_nearest_free(grid: tw_grid, occ, x, y):
    """Nearest free non-border cell to (x, y), or None if there is none."""
    ws = workspace(256, occ.device, "nearest")
    xy = (ctypes.c_int * 2)()
    st = load().tw_nearest_free(ctypes.byref(grid), _ptr(occ), int(x), int(y), xy, _ptr(ws), ws.numel(),
                                _stream(occ.device))
    _check("tw_nearest_free", st, ok=(TW_OK, TW_NO_PATH))
    return (int(xy[0]), int(xy[1])) if st == TW_OK else None


def hp_relax(grid: tw_grid, occ, goal, field=None, params: Optional[Params] = None):
    """Harmonic field (u = 1 - phi unless HP_OUT_PHI).  Returns (field, stats dict)."""
    torch = _torch()
    lib = load()
    params = params or Params()
    if field is None:
        field = torch.empty((grid.ny, grid.nx), dtype=torch.float32, device=occ.device)
    cp = params.c()
    ws = workspace(lib.hp_relax_workspace_size(grid.nx, grid.ny, ctypes.byref(cp)), occ.device, "relax")
    stats = hp_stats()
    st = lib.hp_relax(ctypes.byref(grid), _ptr(occ), int(goal[0]), int(goal[1]), _ptr(field),
                      ctypes.byref(cp), ctypes.byref(stats), _ptr(ws), ws.numel(), _stream(occ.device))
    _check("hp_relax", st, ok=(TW_OK, TW_NOT_CONVERGED))
    return field, stats.as_dict()


def hp_relax_noalloc(grid: tw_grid, occ, goal, field=None, params: Optional[Params] = None):
    """hp_relax on the library's static scratch array (no workspace; see the C header)."""
    torch = _torch()
    params = params or Params()
    if field is None:
        field = torch.empty((grid.ny, grid.nx), dtype=torch.float32, device=occ.device)
    cp = params.c()
    stats = hp_stats()
    # the library takes the scratch array of the current device: make it the tensors' device
    with torch.cuda.device(occ.device):
        st = load().hp_relax_noalloc(ctypes.byref(grid), _ptr(occ), int(goal[0]), int(goal[1]), _ptr(field),
                                     ctypes.byref(cp), ctypes.byref(stats), _stream(occ.device))
    _check("hp_relax_noalloc", st, ok=(TW_OK, TW_NOT_CONVERGED))
    return field, stats.as_dict()


def hp_relax_batched(occs, goals, fields=None, params: Optional[Params] = None):
    """Relax many planners together.  occs: list of device uint8 [ny][nx];
    goals: list of (gx, gy).  Returns (fields, list of stats dicts, latency_ms array)."""
    torch = _torch()
    lib = load()
    params = params or Params()
    n = len(occs)
    if fields is None:
        fields = [torch.empty(o.shape, dtype=torch.float32, device=o.device) for o in occs]
    arr = (hp_instance * n)()
    for i, (o, g, f) in enumerate(zip(occs, goals, fields)):
        arr[i] = hp_instance(int(o.shape[1]), int(o.shape[0]), o.data_ptr(), int(g[0]), int(g[1]), f.data_ptr())
    cp = params.c()
    ws = workspace(lib.hp_relax_batched_workspace_size(n, arr, ctypes.byref(cp)), occs[0].device, "batch")
    stats = (hp_stats * n)()
    lat = np.zeros(n, np.float64)
    st = lib.hp_relax_batched(n, arr, ctypes.byref(cp), stats, lat.ctypes.data_as(ctypes.c_void_p), _ptr(ws),
                              ws.numel(), _stream(occs[0].device))
    if st < 0 and all(s_.status < 0 for s_ in stats):
        raise TwError("hp_relax_batched", st)
    return fields, [s_.as_dict() for s_ in stats], lat


def hp_relax_dirichlet(fixed, u, params: Optional[Params] = None):
    """General Dirichlet solve in place on u (fixed != 0 keeps its value)."""
    lib = load()
    params = params or Params()
    ny, nx = u.shape
    cp = params.c()
    ws = workspace(lib.hp_relax_workspace_size(nx, ny, ctypes.byref(cp)), u.device, "relax")
    stats = hp_stats()
    st = lib.hp_relax_dirichlet(nx, ny, _ptr(fixed), _ptr(u), ctypes.byref(cp), ctypes.byref(stats),
                                _ptr(ws), ws.numel(), _stream(u.device))
    _check("hp_relax_dirichlet", st, ok=(TW_OK, TW_NOT_CONVERGED))
    return u, stats.as_dict()


def hp_residual(fixed, u):
    lib = load()
    ny, nx = u.shape
    ws = workspace(4096, u.device, "resid")
    a, b = ctypes.c_double(), ctypes.c_double()
    _check("hp_residual", lib.hp_residual(nx, ny, _ptr(fixed), _ptr(u), ctypes.byref(a), ctypes.byref(b),
                                          _ptr(ws), ws.numel(), _stream(u.device)))
    return a.value, b.value


def plan_path(grid: tw_grid, u, occ, start, goal, rubber_iters=100, max_len=None, w=1e-3, k=1.0):
    """Eq. 3 descent + rubber band.  Returns (status, path int32 [L, 2])."""
    lib = load()
    max_len = int(max_len or 4 * grid.nx * grid.ny)
    ws = workspace(lib.plan_path_workspace_size(max_len), u.device, "path")
    out = np.zeros((max_len, 2), np.int32)
    L = ctypes.c_int()
    st = lib.plan_path_ex(ctypes.byref(grid), _ptr(u), _ptr(occ), int(start[0]), int(start[1]), int(goal[0]),
                          int(goal[1]), int(rubber_iters), float(w), float(k), max_len,
                          out.ctypes.data_as(ctypes.c_void_p), ctypes.byref(L), _ptr(ws), ws.numel(),
                          _stream(u.device))
    _check("plan_path", st, ok=(TW_OK, TW_NO_PATH, TW_ESTART_BLOCKED))
    return st, out[:L.value].copy()


def kf_update(tracks: np.ndarray, z: np.ndarray, dt=0.1, q_accel=0.01, r_meas=0.05) -> np.ndarray:
    """One predict + update step for host tracks [n, 21] (in place, also returned)."""
    assert tracks.dtype == np.float64 and tracks.flags.c_contiguous
    zz = np.ascontiguousarray(z, dtype=np.float64).reshape(-1, 2)
    n = tracks.reshape(-1, TRACK_DOUBLES).shape[0]
    _check("kf_update", load().kf_update(tracks.ctypes.data_as(ctypes.c_void_p), n,
                                         zz.ctypes.data_as(ctypes.c_void_p), float(dt), float(q_accel),
                                         float(r_meas)))
    return tracks


def kf_init(z: np.ndarray, radius: np.ndarray, r_meas=0.05, p_vel=1.0) -> np.ndarray:
    zz = np.ascontiguousarray(z, dtype=np.float64).reshape(-1, 2)
    rr = np.ascontiguousarray(radius, dtype=np.float64).reshape(-1)
    T = np.zeros((zz.shape[0], TRACK_DOUBLES))
    _check("kf_init", load().kf_init(T.ctypes.data_as(ctypes.c_void_p), zz.shape[0],
                                     zz.ctypes.data_as(ctypes.c_void_p), rr.ctypes.data_as(ctypes.c_void_p),
                                     float(r_meas), float(p_vel)))
    return T


# ---------------------------------------------------------------------------
# learned warm start
# ---------------------------------------------------------------------------

def ws_conv3x3(x, w, b=None, skip=None, relu=False, impl=WS_CONV_AUTO):
    """One convolution layer of the warm-start network: x bf16 [cin, H, W] (device),
    w fp32 [cout, cin, 3, 3], b fp32 [cout] or None, skip bf16 [cout, H, W] or None.
    Returns y bf16 [cout, H, W]."""
    torch = _torch()
    cin, H, W = x.shape
    cout = w.shape[0]
    y = torch.empty((cout, H, W), dtype=torch.bfloat16, device=x.device)
    lib = load()
    nws = lib.ws_conv3x3_workspace_size(cin, cout, H, W, int(impl))
    ws = workspace(nws, x.device, "conv") if nws else None
    _check("ws_conv3x3", lib.ws_conv3x3(_ptr(x), _ptr(w), _ptr(b) if b is not None else None,
                                        _ptr(skip) if skip is not None else None, _ptr(y), cin, cout, H, W,
                                        1 if relu else 0, int(impl), _ptr(ws) if ws is not None else None,
                                        ws.numel() if ws is not None else 0, _stream(x.device)))
    return y


def ws_conv3x3_wgrad(x, dy, impl=WS_CONV_AUTO):
    """Parameter gradients of one convolution layer from its input x bf16 [cin, H, W] and output
    gradient dy bf16 [cout, H, W] (device).  Returns (dW fp32 [cout, cin, 3, 3], db fp32 [cout])."""
    torch = _torch()
    cin, H, W = x.shape
    cout = dy.shape[0]
    dw = torch.zeros((cout, cin, 3, 3), dtype=torch.float32, device=x.device)
    db = torch.zeros((cout,), dtype=torch.float32, device=x.device)
    lib = load()
    nws = lib.ws_conv3x3_wgrad_workspace_size(cin, cout, H, W, int(impl))
    ws = workspace(nws, x.device, "wgrad") if nws else None
    _check("ws_conv3x3_wgrad", lib.ws_conv3x3_wgrad(_ptr(x), _ptr(dy), _ptr(dw), _ptr(db), cin, cout, H, W, int(impl),
                                                    _ptr(ws) if ws is not None else None,
                                                    ws.numel() if ws is not None else 0, _stream(x.device)))
    return dw, db


def ws_conv_check() -> bool:
    """True if a WS_CONV_TC convolution on the current device gave up a bounded wait since the last
    call (its output is then invalid); clears the flag."""
    flag = ctypes.c_int()
    _check("ws_conv_check", load().ws_conv_check(ctypes.byref(flag)))
    return bool(flag.value)


class WarmStartNet:
    """Parameters and Adam state of the warm-start network, on one device."""

    def __init__(self, device="cuda", seed=1):
        torch = _torch()
        lib = load()
        self.n = int(lib.ws_unet_param_count())
        self.device = torch.device(device)
        self.params = torch.empty(self.n, dtype=torch.float32, device=self.device)
        self.grads = torch.zeros_like(self.params)
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        self.step_count = 0
        _check("ws_unet_init", lib.ws_unet_init(_ptr(self.params), int(seed), _stream(self.device)))

    def _ws(self, H, W):
        return workspace(load().ws_unet_workspace_size(int(H), int(W)), self.device, "unet")

    def target(self, u):
        torch = _torch()
        t = torch.empty(u.shape, dtype=torch.float32, device=u.device)
        _check("ws_make_target", load().ws_make_target(_ptr(u), u.numel(), _ptr(t), _stream(u.device)))
        return t

    def forward(self, occ, goal, u_out=True):
        """Returns (u warm start or None, prediction p = log(u) / 30)."""
        torch = _torch()
        H, W = occ.shape
        u = torch.empty((H, W), dtype=torch.float32, device=occ.device) if u_out else None
        p = torch.empty((H, W), dtype=torch.float32, device=occ.device)
        ws = self._ws(H, W)
        _check("ws_unet_forward", load().ws_unet_forward(_ptr(self.params), _ptr(occ), H, W, int(goal[0]),
                                                          int(goal[1]), _ptr(u) if u is not None else None, _ptr(p),
                                                          _ptr(ws), ws.numel(), _stream(occ.device)))
        return u, p

    def warm_start(self, occ, goal, stride=1, u=None):
        """The warm start u for hp_relax from the network run at 1/stride of the
        resolution (stride 1, 2 or 4), upsampled to the grid of `occ`."""
        torch = _torch()
        lib = load()
        H, W = occ.shape
        if u is None:
            u = torch.empty((H, W), dtype=torch.float32, device=occ.device)
        ws = workspace(lib.ws_unet_warm_start_workspace_size(int(H), int(W), int(stride)), self.device, "unet")
        _check("ws_unet_warm_start", lib.ws_unet_warm_start(_ptr(self.params), _ptr(occ), H, W, int(goal[0]),
                                                            int(goal[1]), int(stride), _ptr(u), _ptr(ws),
                                                            ws.numel(), _stream(occ.device)))
        return u

    def gradients(self, occ, goal, target):
        """Loss and gradients for one field (no parameter update)."""
        H, W = occ.shape
        ws = self._ws(H, W)
        loss = ctypes.c_float()
        _check("ws_unet_train_step", load().ws_unet_train_step(
            _ptr(self.params), _ptr(self.grads), None, None, 0, 0.0, _ptr(occ), H, W, int(goal[0]), int(goal[1]),
            _ptr(target), ctypes.byref(loss), _ptr(ws), ws.numel(), _stream(occ.device)))
        return loss.value, self.grads

    def train_step(self, occ, goal, target, lr=1e-3):
        H, W = occ.shape
        ws = self._ws(H, W)
        self.step_count += 1
        loss = ctypes.c_float()
        _check("ws_unet_train_step", load().ws_unet_train_step(
            _ptr(self.params), _ptr(self.grads), _ptr(self.m), _ptr(self.v), self.step_count, float(lr), _ptr(occ),
            H, W, int(goal[0]), int(goal[1]), _ptr(target), ctypes.byref(loss), _ptr(ws), ws.numel(),
            _stream(occ.device)))
        return loss.value
