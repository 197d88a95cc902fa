"""C-ABI boundary checks that need no GPU: the library loads, exports every
function include/twgrid.h declares, validates arguments on the host before
any CUDA call, and its host-only parts (ring count, Kalman filter) agree with
the oracle."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
import paper_1903_07441_gb300 as tw
import scenes

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1903_07441_gb300 import build
    build.build()
    return tw.load()


def _declared_functions():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if not h.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", h)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w \*]*?\b([a-z_][a-z0-9_]*)\s*\(", text, flags=re.M):
            if not m.group(0).lstrip().startswith(("#", "typedef", "return")):
                names.add(m.group(1))
    return names


def test_header_declares_the_boundary():
    names = _declared_functions()
    for fn in ("tw_build_grid", "hp_relax", "plan_path", "kf_update", "tw_status_string"):
        assert fn in names


def test_library_exports_every_declared_symbol(lib):
    for name in sorted(_declared_functions()):
        assert hasattr(lib, name), name
        assert ctypes.cast(getattr(lib, name), ctypes.c_void_p).value


def test_binding_lists_the_exports(lib):
    assert set(tw.EXPORTS) == _declared_functions()


def test_status_strings(lib):
    for st in (0, 1, 2, -1, -2, -3, -4, -5):
        assert tw.status_string(st) and tw.status_string(st) != "unknown status"
    assert tw.status_string(12345) == "unknown status"


def test_ring_count_matches_oracle(lib):
    for name, side in (("static128", 128), ("dynamic512", 512)):
        sc = scenes.by_name(name) if name != "dynamic512" else scenes.dynamic(side=512, n_obs=3, frames=1)
        for law in (scenes.RingLaw(), scenes.RingLaw(kind=scenes.RING_ELLIPTIC),
                    scenes.RingLaw(r0=0.3, growth=1.2), scenes.RingLaw(n_rings=7)):
            R, _ = oracle.ring_table(law, sc.nx, sc.ny, sc.cell, sc.robot[4])
            assert tw.tw_ring_count(tw.make_grid(sc.nx, sc.ny, sc.cell), sc.robot, law) == len(R)


def test_kf_host_matches_oracle(lib):
    sc = scenes.dynamic512()
    n = 50
    z0 = sc.meas[0, :n]
    T = tw.kf_init(z0, sc.radius[:n], r_meas=0.05, p_vel=1.0)
    R = oracle.kf_init(z0, sc.radius[:n], r_meas=0.05, p_vel=1.0)
    assert np.array_equal(T, R)
    for f in range(1, 40):
        tw.kf_update(T, sc.meas[f, :n], dt=0.1, q_accel=1e-4, r_meas=0.05)
        R = oracle.kf_step(R, sc.meas[f, :n], dt=0.1, q=1e-4, r=0.05)
    # same equations, different operation order: agreement to rounding
    assert np.abs(T - R).max() <= 1e-12 * max(1.0, np.abs(R).max())
    # the filter tracks the truth
    err = np.hypot(*(T[:, :2] - sc.truth_pos[39, :n]).T)
    assert np.median(err) < 0.05


def _bad_grid_call(lib, **kw):
    g = tw.make_grid(kw.get("nx", 64), kw.get("ny", 64), kw.get("cell", 0.05))
    robot = tw.make_pose(kw.get("robot", [0.5, 0.5, 1.0, 0.0, 0.75]))
    law = tw.make_law(kw.get("law", scenes.RingLaw()))
    tracks = np.ascontiguousarray(kw.get("tracks", np.zeros((0, 21))), dtype=np.float64)
    n = tracks.shape[0]
    return lib.tw_build_grid(ctypes.byref(g), ctypes.byref(robot),
                             tracks.ctypes.data_as(ctypes.c_void_p) if n else None, n, ctypes.byref(law),
                             None, ctypes.c_void_p(256), None, ctypes.c_void_p(256), 1 << 20, None)


def test_build_grid_rejects_bad_input_on_host(lib):
    good = scenes.synth_tracks(scenes.rng.Stream(1), np.array([[1.0, 1.0]]), np.array([[0.1, 0.0]]),
                               np.array([0.3]))
    assert _bad_grid_call(lib, nx=2) == tw.TW_EINVAL
    assert _bad_grid_call(lib, cell=0.0) == tw.TW_EINVAL
    assert _bad_grid_call(lib, robot=[0.5, 0.5, 0.5, 0.0, 0.75]) == tw.TW_EINVAL   # heading not unit
    assert _bad_grid_call(lib, robot=[0.5, 0.5, 1.0, 0.0, 0.0]) == tw.TW_EINVAL    # zero speed
    assert _bad_grid_call(lib, law=scenes.RingLaw(growth=1.0)) == tw.TW_EINVAL
    assert _bad_grid_call(lib, law=scenes.RingLaw(r0=0.001, growth=1.01)) == tw.TW_EINVAL  # > 64 rings
    bad = good.copy(); bad[0, 2] = np.nan
    assert _bad_grid_call(lib, tracks=bad) == tw.TW_EINVAL
    bad = good.copy(); bad[0, 20] = -0.1
    assert _bad_grid_call(lib, tracks=bad) == tw.TW_EINVAL
    bad = good.copy(); bad[0, 4 + 2] = bad[0, 4 + 8] = 1.0    # |Pxv| > sqrt(Pxx Pvv): not PSD
    assert _bad_grid_call(lib, tracks=bad) == tw.TW_EINVAL
    bad = good.copy(); bad[0, 4 + 0] = -1e-3
    assert _bad_grid_call(lib, tracks=bad) == tw.TW_EINVAL


def test_build_grids_rejects_bad_input_on_host(lib):
    """The batched raster validates every job (as tw_build_grid does) before it
    launches anything, so these calls never touch the (fake) device pointers."""
    good = scenes.synth_tracks(scenes.rng.Stream(1), np.array([[1.0, 1.0]]), np.array([[0.1, 0.0]]),
                               np.array([0.3]))
    keep = []

    def job(nx=64, cell=0.05, robot=(0.5, 0.5, 1.0, 0.0, 0.75), law=None, tracks=None, occ=256):
        tr = np.ascontiguousarray(good if tracks is None else tracks, dtype=np.float64)
        keep.append(tr)
        return tw.tw_grid_job(tw.make_grid(nx, 64, cell), tw.make_pose(robot), tw.make_law(law or scenes.RingLaw()),
                              tr.ctypes.data if len(tr) else None, len(tr), None, occ, None)

    def call(*jobs, ws=256, nbytes=1 << 24):
        arr = (tw.tw_grid_job * len(jobs))(*jobs)
        return lib.tw_build_grids(len(jobs), arr, ctypes.c_void_p(ws), nbytes, None)

    arr = (tw.tw_grid_job * 2)(job(), job(nx=100))
    need = lib.tw_build_grids_workspace_size(2, arr)
    assert need > lib.tw_build_grids_workspace_size(1, arr) > 0
    assert lib.tw_build_grids(0, arr, ctypes.c_void_p(256), 1 << 20, None) == tw.TW_EINVAL
    assert call(job(), job(nx=2)) == tw.TW_EINVAL
    assert call(job(cell=0.0), job()) == tw.TW_EINVAL
    assert call(job(), job(robot=(0.5, 0.5, 0.5, 0.0, 0.75))) == tw.TW_EINVAL
    assert call(job(law=scenes.RingLaw(growth=1.0))) == tw.TW_EINVAL
    bad = good.copy(); bad[0, 2] = np.nan
    assert call(job(), job(tracks=bad)) == tw.TW_EINVAL
    bad = good.copy(); bad[0, 4 + 2] = bad[0, 4 + 8] = 1.0    # not PSD
    assert call(job(tracks=bad)) == tw.TW_EINVAL
    assert call(job(occ=None)) == tw.TW_EINVAL
    assert call(job(), job(), nbytes=need - 1) == tw.TW_EWORKSPACE
    assert call(job(), ws=4096 + 8) == tw.TW_EWORKSPACE


def test_workspace_errors_and_sizes(lib):
    g = tw.make_grid(64, 64, 0.05)
    robot = tw.make_pose([0.5, 0.5, 1.0, 0.0, 0.75])
    law = tw.make_law(scenes.RingLaw())
    assert lib.tw_build_grid_workspace_size(ctypes.byref(g), 10, ctypes.byref(law)) > 0
    st = lib.tw_build_grid(ctypes.byref(g), ctypes.byref(robot), None, 0, ctypes.byref(law), None,
                           ctypes.c_void_p(256), None, None, 0, None)
    assert st == tw.TW_EWORKSPACE
    st = lib.tw_build_grid(ctypes.byref(g), ctypes.byref(robot), None, 0, ctypes.byref(law), None,
                           ctypes.c_void_p(256), None, ctypes.c_void_p(4096 + 8), 1 << 20, None)
    assert st == tw.TW_EWORKSPACE  # misaligned
    for m in (tw.HP_JACOBI, tw.HP_RBSOR):
        p = tw.Params(method=m).c()
        a = lib.hp_relax_workspace_size(2048, 2048, ctypes.byref(p))
        b = lib.hp_relax_workspace_size(128, 128, ctypes.byref(p))
        assert a > b > 0
    assert lib.plan_path_workspace_size(1000) >= 8000


def test_relax_rejects_bad_params_and_goal_on_host(lib):
    g = tw.make_grid(64, 64, 0.05)
    st = tw.hp_stats()

    def call(params, gx=30, gy=30):
        cp = params.c()
        return lib.hp_relax(ctypes.byref(g), ctypes.c_void_p(256), gx, gy, ctypes.c_void_p(256),
                            ctypes.byref(cp), ctypes.byref(st), ctypes.c_void_p(256), 1 << 30, None)

    assert call(tw.Params(omega=2.0)) == tw.TW_EINVAL
    assert call(tw.Params(omega=float("nan"))) == tw.TW_EINVAL
    assert call(tw.Params(max_sweeps=0)) == tw.TW_EINVAL
    assert call(tw.Params(tol=-1.0)) == tw.TW_EINVAL
    assert call(tw.Params(method=7)) == tw.TW_EINVAL
    assert call(tw.Params(), gx=0, gy=30) == tw.TW_EGOAL_BLOCKED     # on the border
    assert call(tw.Params(), gx=64, gy=30) == tw.TW_EGOAL_BLOCKED    # out of range
    big = tw.make_grid(64, 65536, 0.05)   # one launch row per grid row: at most 65535 rows
    cp = tw.Params().c()
    assert lib.hp_relax(ctypes.byref(big), ctypes.c_void_p(256), 30, 30, ctypes.c_void_p(256), ctypes.byref(cp),
                        ctypes.byref(st), ctypes.c_void_p(256), 1 << 30, None) == tw.TW_EINVAL


def test_warm_start_entry_points_reject_bad_input_on_host(lib):
    """The network's entry points validate sizes and choices before any GPU work."""
    P = ctypes.c_void_p(256)
    # ws_conv3x3: unknown implementation, non-positive sizes, missing pointers
    assert lib.ws_conv3x3(P, P, None, None, P, 32, 32, 16, 16, 1, 7, None, 0, None) == tw.TW_EINVAL
    assert lib.ws_conv3x3(P, P, None, None, P, 0, 32, 16, 16, 1, tw.WS_CONV_AUTO, None, 0, None) == tw.TW_EINVAL
    assert lib.ws_conv3x3(P, P, None, None, P, 32, 32, 0, 16, 1, tw.WS_CONV_AUTO, None, 0, None) == tw.TW_EINVAL
    assert lib.ws_conv3x3(None, P, None, None, P, 32, 32, 16, 16, 1, tw.WS_CONV_AUTO, None, 0, None) == tw.TW_EINVAL
    # the tensor-core form needs cin % 16 == 0 and cout % 32 == 0
    assert lib.ws_conv3x3(P, P, None, None, P, 8, 32, 16, 16, 1, tw.WS_CONV_MMA, None, 0, None) == tw.TW_EINVAL
    assert lib.ws_conv3x3(P, P, None, None, P, 32, 16, 16, 16, 1, tw.WS_CONV_MMA, None, 0, None) == tw.TW_EINVAL
    # the tensor-memory form: cin % 16 == 0, cout in {32, 64, 128}, W % 128 == 0, H even, and a workspace
    assert lib.ws_conv3x3_workspace_size(64, 128, 16, 256, tw.WS_CONV_TC) >= 64 * 128 * 9 * 2
    assert lib.ws_conv3x3_workspace_size(64, 128, 16, 256, tw.WS_CONV_MMA) == 0
    for cin, cout, H, W in ((64, 96, 16, 256), (8, 64, 16, 256), (64, 64, 16, 200), (64, 64, 15, 256),
                            (64, 64, 6, 256), (64, 128, 7, 256)):
        assert lib.ws_conv3x3_workspace_size(cin, cout, H, W, tw.WS_CONV_TC) == 0
        assert lib.ws_conv3x3(P, P, None, None, P, cin, cout, H, W, 1, tw.WS_CONV_TC, P, 1 << 20, None) == tw.TW_EINVAL
    # the narrow form: W in {16, 32, 64}, H a multiple of 256 / W; its workspace adds split-K partial sums
    assert lib.ws_conv3x3_workspace_size(128, 128, 64, 64, tw.WS_CONV_TC) > 128 * 128 * 9 * 2 + 128 * 64 * 64 * 4
    assert lib.ws_conv3x3_workspace_size(16, 32, 16, 16, tw.WS_CONV_TC) >= 16 * 32 * 9 * 2
    for cin, cout, H, W in ((64, 64, 6, 64), (64, 64, 12, 32), (64, 64, 8, 48), (8, 64, 16, 64)):
        assert lib.ws_conv3x3_workspace_size(cin, cout, H, W, tw.WS_CONV_TC) == 0
        assert lib.ws_conv3x3(P, P, None, None, P, cin, cout, H, W, 1, tw.WS_CONV_TC, P, 1 << 20, None) == tw.TW_EINVAL
    assert lib.ws_conv3x3(P, P, None, None, P, 64, 64, 16, 64, 1, tw.WS_CONV_TC, P, 100, None) == tw.TW_EWORKSPACE
    assert lib.ws_conv3x3(P, P, None, None, P, 64, 64, 16, 256, 1, tw.WS_CONV_TC, None, 0, None) == tw.TW_EWORKSPACE
    assert lib.ws_conv3x3(P, P, None, None, P, 64, 64, 16, 256, 1, tw.WS_CONV_TC, P, 100, None) == tw.TW_EWORKSPACE
    # ws_conv3x3_wgrad: the tensor-memory form needs cin, cout <= 128 and W % 16 == 0; no mma.sync
    # form; the workspace holds the partial sums of the pixel chunks
    per = 9 * 64 * 128 + 128
    # 4096 pixels: about 50 chunks, rounded up to whole 64-pixel stages of 128 pixels -> 32 chunks
    assert lib.ws_conv3x3_wgrad_workspace_size(64, 128, 16, 256, tw.WS_CONV_TC) >= 32 * per * 4
    assert lib.ws_conv3x3_wgrad_workspace_size(64, 128, 1, 16, tw.WS_CONV_TC) >= per * 4
    assert lib.ws_conv3x3_wgrad_workspace_size(2, 32, 16, 16, tw.WS_CONV_AUTO) >= (9 * 2 * 32 + 32) * 4
    assert lib.ws_conv3x3_wgrad_workspace_size(64, 64, 16, 256, tw.WS_CONV_MMA) == 0
    assert lib.ws_conv3x3_wgrad_workspace_size(2, 32, 16, 256, tw.WS_CONV_TC) > 0
    assert lib.ws_conv3x3_wgrad_workspace_size(32, 1, 16, 256, tw.WS_CONV_TC) > 0
    for cin, cout, H, W in ((256, 64, 16, 256), (64, 160, 16, 256), (64, 64, 16, 200), (64, 64, 16, 8)):
        assert lib.ws_conv3x3_wgrad_workspace_size(cin, cout, H, W, tw.WS_CONV_TC) == 0
        assert lib.ws_conv3x3_wgrad(P, P, P, None, cin, cout, H, W, tw.WS_CONV_TC, P, 1 << 30, None) == tw.TW_EINVAL
    assert lib.ws_conv3x3_wgrad(P, P, P, None, 64, 64, 16, 256, tw.WS_CONV_MMA, P, 1 << 30, None) == tw.TW_EINVAL
    assert lib.ws_conv3x3_wgrad(P, P, P, None, 64, 64, 16, 256, 9, P, 1 << 30, None) == tw.TW_EINVAL
    assert lib.ws_conv3x3_wgrad(None, P, P, None, 64, 64, 16, 256, tw.WS_CONV_AUTO, P, 1 << 30, None) == tw.TW_EINVAL
    assert lib.ws_conv3x3_wgrad(P, P, None, None, 64, 64, 16, 256, tw.WS_CONV_AUTO, P, 1 << 30, None) == tw.TW_EINVAL
    assert lib.ws_conv3x3_wgrad(P, P, P, None, 64, 64, 0, 256, tw.WS_CONV_AUTO, P, 1 << 30, None) == tw.TW_EINVAL
    assert lib.ws_conv3x3_wgrad(P, P, P, None, 64, 64, 16, 256, tw.WS_CONV_TC, None, 0, None) == tw.TW_EWORKSPACE
    assert lib.ws_conv3x3_wgrad(P, P, P, None, 64, 64, 16, 256, tw.WS_CONV_TC, P, 1024, None) == tw.TW_EWORKSPACE
    assert lib.ws_conv3x3_wgrad(P, P, P, None, 64, 64, 16, 256, tw.WS_CONV_SIMT, P, 1024, None) == tw.TW_EWORKSPACE
    # the network: H and W multiples of 8, goal inside, workspace present
    assert lib.ws_unet_workspace_size(64, 64) > lib.ws_unet_workspace_size(16, 16) > 0
    assert lib.ws_unet_forward(P, P, 60, 64, 1, 1, None, None, P, 1 << 30, None) == tw.TW_EINVAL
    assert lib.ws_unet_forward(P, P, 64, 64, 64, 1, None, None, P, 1 << 30, None) == tw.TW_EINVAL
    assert lib.ws_unet_forward(P, P, 64, 64, 1, 1, None, None, None, 1 << 30, None) == tw.TW_EWORKSPACE


def test_product_path_has_no_cpu_fallback():
    """The binding imports no oracle code and fails loudly without a GPU."""
    src = open(os.path.join(ROOT, "paper_1903_07441_gb300", "__init__.py")).read()
    assert "oracle" not in src.replace("no CPU fallback", "")
    import torch
    if not torch.cuda.is_available():
        with pytest.raises(RuntimeError):
            tw.hp_relax(tw.make_grid(8, 8, 0.1), torch.zeros((8, 8), dtype=torch.uint8), (3, 3))


# ---------------------------------------------------------------------------
# the adaptive SOR factor (host logic, pinned by brute-force linear algebra)
# ---------------------------------------------------------------------------

def _jacobi_and_sor(free):
    """Dense Jacobi matrix of the free cells (1/4 of the free 4-neighbours; the
    rest are Dirichlet cells) and the red-black SOR iteration matrix builder."""
    idx = -np.ones(free.shape, int)
    cells = np.argwhere(free)
    idx[free] = np.arange(len(cells))
    n = len(cells)
    Jm = np.zeros((n, n))
    for k, (y, x) in enumerate(cells):
        for dy, dx in ((0, 1), (0, -1), (1, 0), (-1, 0)):
            j = idx[y + dy, x + dx]
            if j >= 0:
                Jm[k, j] = 0.25
    red = ((cells[:, 0] + cells[:, 1]) % 2) == 0

    def sor(omega):
        # red half-sweep then black: u <- u + omega (J u - u) colour by colour
        n_ = len(cells)
        M = np.eye(n_)
        for colour in (red, ~red):
            S = np.eye(n_)
            S[colour] = (1 - omega) * np.eye(n_)[colour] + omega * Jm[colour]
            M = S @ M
        return M
    return Jm, sor


def test_omega_cap_is_the_empty_box_optimum_and_bounds_every_occupancy(lib):
    for nx, ny in ((9, 7), (12, 12), (5, 16)):
        free = np.zeros((ny, nx), bool)
        free[1:-1, 1:-1] = True
        Jm, _ = _jacobi_and_sor(free)
        mu = np.abs(np.linalg.eigvals(Jm)).max()
        assert abs(lib.hp_omega_cap(nx, ny) - 2.0 / (1.0 + np.sqrt(1.0 - mu * mu))) < 1e-12
        rng = np.random.default_rng(nx * ny)
        for _ in range(5):   # obstacles only lower the Jacobi spectral radius (Perron-Frobenius)
            f = free & (rng.random(free.shape) > 0.25)
            if f.sum() < 2:
                continue
            Jf, _ = _jacobi_and_sor(f)
            assert np.abs(np.linalg.eigvals(Jf)).max() <= mu + 1e-12
    # the first factor of an adaptive solve never exceeds the cap
    for n in (3, 5, 9, 64, 255, 256, 1023, 1024, 4096):
        w0 = lib.hp_omega_initial(n, n)
        assert 0.0 < w0 <= lib.hp_omega_cap(n, n) + 1e-15
        assert w0 == min({True: 1.9, False: 1.85 if n >= 256 else 1.75}[n >= 1024], lib.hp_omega_cap(n, n))


def test_omega_update_recovers_mu_through_youngs_relation(lib):
    """On a red-black ordered box the spectral radius of the SOR matrix at
    omega < omega_opt, computed by brute force, gives back the Jacobi spectral
    radius: the update lands 10 % of the way from omega_opt to 2 (capped)."""
    nx, ny = 14, 12
    free = np.zeros((ny, nx), bool)
    free[1:-1, 1:-1] = True
    free[5:8, 4:9] = False   # an obstacle block keeps the matrix consistently ordered
    Jm, sor = _jacobi_and_sor(free)
    mu = np.abs(np.linalg.eigvals(Jm)).max()
    w_opt = 2.0 / (1.0 + np.sqrt(1.0 - mu * mu))
    cap = lib.hp_omega_cap(nx, ny)
    adapted = 0
    for omega in (1.0, 1.1, 1.2, 1.3, 0.5 * (1.0 + w_opt), w_opt - 0.01):
        lam = np.abs(np.linalg.eigvals(sor(omega))).max()   # decay rate per full red + black sweep
        got = lib.hp_omega_update(omega, lam, nx, ny)
        if lam <= (omega - 1.0) ** 0.75:   # too close to omega - 1 to tell mu: omega is kept
            assert got == omega
            continue
        want = min(cap, 2.0 - 0.9 * (2.0 - w_opt))
        assert abs(got - max(omega, want)) < 1e-9, (omega, lam, got, want)
        adapted += 1
    assert adapted >= 3
    # past the optimum every eigenvalue has modulus omega - 1: omega is kept
    for omega in (w_opt + 0.01, w_opt + 0.05):
        lam = np.abs(np.linalg.eigvals(sor(omega))).max()
        assert abs(lam - (omega - 1.0)) < 1e-6
        assert lib.hp_omega_update(omega, lam, nx, ny) == omega


def test_omega_update_edge_cases(lib):
    for lam in (0.0, -0.1, 1.0, 1.5, float("nan")):
        assert lib.hp_omega_update(1.7, lam, 512, 512) == 1.7
    # never below the current factor, never above the cap
    rng = np.random.default_rng(5)
    for _ in range(200):
        n = int(rng.integers(3, 3000))
        w = 1.0 + 0.99 * rng.random()
        lam = rng.random()
        got = lib.hp_omega_update(w, lam, n, n)
        assert got >= w
        assert got <= max(w, lib.hp_omega_cap(n, n)) + 1e-15
    assert lib.hp_omega_update(1.5, 0.5, 2, 10) == 1.5   # not a grid


# ---------------------------------------------------------------------------
# temporal-blocking halo (host-side check of the tile geometry)
# ---------------------------------------------------------------------------

def _contaminated_after(T, rows, xcells):
    """Grid-level red-black sweeps on a tile whose outside is unknown (NaN):
    which cells of the tile depend on the outside after T full sweeps."""
    u = np.zeros((rows + 2, xcells + 2))
    u[0, :] = u[-1, :] = u[:, 0] = u[:, -1] = np.nan
    yy, xx = np.mgrid[0:rows, 0:xcells]
    red = ((xx + yy) & 1) == 0
    for _ in range(T):
        for colour in (red, ~red):
            c = u[1:-1, 1:-1]
            nb = 0.25 * (u[1:-1, :-2] + u[1:-1, 2:] + u[:-2, 1:-1] + u[2:, 1:-1])
            c[colour] = nb[colour]
    return np.isnan(u[1:-1, 1:-1])


@pytest.mark.parametrize("T", [1, 2, 3, 4, 5, 6, 7])
def test_tile_halo_is_enough_for_T_fused_sweeps(T):
    """The fused sweep kernels keep a halo of 2T rows and ceil((T + 1) / 4)
    float4 columns of each colour (8 cells of the row per float4 column) around
    the tile interior they store; after T red-black sweeps no interior cell may
    depend on values outside the tile.  Outside values reach exactly 2T rows and
    2T cells of a row deep: the row halo is the least that works, the column
    halo that rounded up to whole float4 columns."""
    hy = 2 * T
    hx = 8 * ((T + 1 + 3) // 4)
    rows, xcells = 4 * hy + 16, 2 * hx + 64
    bad = _contaminated_after(T, rows, xcells)
    assert not bad[hy:rows - hy, hx:xcells - hx].any()
    depth_rows = max(i for i in range(rows // 2) if bad[i, hx:xcells - hx].any()) + 1
    depth_cols = max(j for j in range(xcells // 2) if bad[hy:rows - hy, j].any()) + 1
    assert depth_rows == 2 * T == hy
    assert depth_cols == 2 * T <= hx


def test_header_is_plain_c_and_links(lib, tmp_path):
    """include/twgrid.h is a C header: a C program that takes the address of
    every declared function compiles with gcc (-std=c99, warnings as errors),
    links against libtwgrid.so and calls the entry points that need no GPU."""
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("no gcc")
    names = sorted(_declared_functions())
    cuda_inc = "/usr/local/cuda/include"
    src = ["#include <stdio.h>", "#include \"twgrid.h\"", "int main(void) {", "    void *f[] = {"]
    src += [f"        (void *){n}," for n in names]
    src += ["    };",
            "    int n = 0;",
            "    for (unsigned i = 0; i < sizeof f / sizeof f[0]; i++) n += f[i] != 0;",
            "    tw_grid g = {64, 48, 0.05, 0.0, 0.0};",
            "    tw_pose r = {1.0, 1.0, 1.0, 0.0, 0.75};",
            "    tw_ring_law law = {TW_RING_CIRCULAR, TW_MARK_PER_CELL, 0.5, 1.3, 0, 1e-4, 2.0, 0.25, 0};",
            "    printf(\"%d %s|%s|%d|%.6f\\n\", n, tw_version(), tw_status_string(TW_EINVAL),",
            "           tw_ring_count(&g, &r, &law), hp_omega_cap(64, 48));",
            "    return 0;", "}"]
    c = tmp_path / "abi.c"
    c.write_text("\n".join(src) + "\n")
    exe = tmp_path / "abi"
    libdir = os.path.dirname(tw.LIB_PATH)
    cmd = ["gcc", "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(c), "-o", str(exe),
           "-L", libdir, "-ltwgrid", f"-Wl,-rpath,{libdir}"]
    if os.path.isdir(cuda_inc):
        cmd[4:4] = ["-I", cuda_inc]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert out.returncode == 0, out.stderr
    count, rest = out.stdout.split(" ", 1)
    version, status, rings, cap = rest.strip().split("|")
    assert int(count) == len(names)
    assert version == lib.tw_version().decode()
    assert status == tw.status_string(tw.TW_EINVAL)
    assert int(rings) == lib.tw_ring_count(ctypes.byref(tw.make_grid(64, 48, 0.05)),
                                           ctypes.byref(tw.make_pose([1.0, 1.0, 1.0, 0.0, 0.75])),
                                           ctypes.byref(tw.make_law(scenes.RingLaw(q_accel=1e-4))))
    assert abs(float(cap) - lib.hp_omega_cap(64, 48)) < 1e-6
