"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

* raster: bit-exact occupancy and ring index, every ring law / marking mode,
  several seeds and frames, ragged and odd grid sizes, the full 2048x2048 size;
* field: max |u - u*| against the oracle's tightly converged solution, bounded
  by the a-posteriori bound tau_max * r_inf (exit time tau); <= 1e-5 over the
  whole field with the error tolerance (etol = 1e-5) at r_inf <= 1e-6, from
  300 x 300 to the full 2048 x 2048 size, and once the FP32 iteration has
  converged to its floor; closed-form Dirichlet data;
* path: valid (collision-free, reaches the goal) and within Hausdorff 2 cells
  of the oracle path.
"""
import numpy as np
import pytest

import oracle
import paper_1903_07441_gb300 as tw
import scenes

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1903_07441_gb300 import build
    build.build()
    return torch.device("cuda:0")


def _gpu_grid(sc, dev, law=None, tracks=None, with_ring=True):
    grid = tw.make_grid(sc.nx, sc.ny, sc.cell, sc.ox, sc.oy)
    static = torch.from_numpy(np.ascontiguousarray(sc.static_occ)).to(dev) if sc.static_occ is not None else None
    ring = torch.empty((sc.ny, sc.nx), dtype=torch.int16, device=dev) if with_ring else None
    occ, ring = tw.tw_build_grid(grid, sc.robot, sc.tracks if tracks is None else tracks, law or sc.law,
                                 static_occ=static, ring=ring)
    torch.cuda.synchronize()
    return occ, ring


def _assert_raster_equal(sc, dev, law=None, tracks=None):
    occ, ring = _gpu_grid(sc, dev, law, tracks)
    occ_ref, ring_ref, _ = oracle.build_grid(sc, law=law, tracks=tracks)
    o = occ.cpu().numpy()
    diff = np.argwhere(o != occ_ref)
    assert diff.size == 0, f"{len(diff)} cells differ, first {diff[:5]}"
    assert np.array_equal(ring.cpu().numpy(), ring_ref)
    return o


# ---------------------------------------------------------------------------
# raster
# ---------------------------------------------------------------------------

def test_raster_static128(dev):
    o = _assert_raster_equal(scenes.static128(), dev)
    assert (o == tw.TW_STATIC).sum() > 1000


@pytest.mark.parametrize("seed,frame", [(1001, 0), (1001, 50), (1011, 99), (1021, 10)])
def test_raster_dynamic512(dev, seed, frame):
    o = _assert_raster_equal(scenes.dynamic(seed=seed, side=512, n_obs=200, frames=frame + 1, frame=frame), dev)
    assert (o == tw.TW_DYNAMIC).sum() > 1000


@pytest.mark.parametrize("kind,mark,outer", [(scenes.RING_ELLIPTIC, scenes.MARK_PER_CELL, 0),
                                             (scenes.RING_CIRCULAR, scenes.MARK_PER_OBSTACLE, 0),
                                             (scenes.RING_ELLIPTIC, scenes.MARK_PER_OBSTACLE, 0),
                                             (scenes.RING_CIRCULAR, scenes.MARK_PER_CELL, 1)])
def test_raster_law_variants(dev, kind, mark, outer):
    sc = scenes.dynamic(seed=1031, side=512, n_obs=60, frames=1, static_shapes=10)
    law = scenes.RingLaw(kind=kind, mark=mark, time_outer=outer)
    _assert_raster_equal(sc, dev, law=law)


@pytest.mark.parametrize("frame,mark", [(0, scenes.MARK_PER_CELL), (50, scenes.MARK_PER_CELL),
                                        (50, scenes.MARK_PER_OBSTACLE)])
def test_raster_probability_threshold_marking(dev, frame, mark):
    """The marking threshold (p_mark = 0.5: a prediction too uncertain to place the obstacle within
    radius + d_safe of its mean with probability 1/2 marks nothing) on the 200-track scene: bit-exact
    against the oracle, and fewer predicted cells than the plain marking."""
    sc = scenes.dynamic(seed=1001, side=512, n_obs=200, frames=frame + 1, frame=frame)
    law = scenes.RingLaw(mark=mark, p_mark=0.5)
    o = _assert_raster_equal(sc, dev, law=law)
    o0 = _assert_raster_equal(sc, dev, law=scenes.RingLaw(mark=mark))
    assert 0 < (o == tw.TW_DYNAMIC).sum() < (o0 == tw.TW_DYNAMIC).sum()


@pytest.mark.parametrize("nx,ny", [(3, 3), (3, 5), (5, 3), (17, 33), (33, 17), (1023, 3), (3, 1025),
                                   (65, 1025), (97, 31)])
def test_raster_odd_sizes(dev, nx, ny):
    st = scenes.rng.Stream(nx * 1000 + ny)
    cell = 0.05
    static = (st.uniform(nx * ny).reshape(ny, nx) < 0.1).astype(np.uint8)
    sc = scenes.Scene("odd", 0, nx, ny, cell, static_occ=static)
    sc.robot = np.array([nx * cell * 0.3, ny * cell * 0.6, 0.6, 0.8, 0.75])
    n = 25
    pos = np.stack([st.uniform(n, -0.5, nx * cell + 0.5), st.uniform(n, -0.5, ny * cell + 0.5)], 1)
    vel = np.stack([st.uniform(n, -1, 1), st.uniform(n, -1, 1)], 1)
    tr = scenes.synth_tracks(st, pos, vel, st.uniform(n, 0.05, 0.3))
    for law in (scenes.RingLaw(r0=0.1, growth=1.4), scenes.RingLaw(kind=scenes.RING_ELLIPTIC, r0=0.1)):
        _assert_raster_equal(sc, dev, law=law, tracks=tr)


def test_raster_batch_instances(dev):
    for seed in (5000, 5001, 5002):
        _assert_raster_equal(scenes.batch_instance(seed), dev)


def test_raster_many_planners_in_one_call(dev):
    """tw_build_grids: uneven planners (own sizes, laws, tracks; with and
    without static map, ring output or tracks, both ring kinds and marking
    modes) rastered in one call give the oracle's codes and rings bit for bit."""
    scs = [scenes.batch_instance(5100 + i) for i in range(12)]
    laws = [sc.law for sc in scs]
    laws[1] = scenes.RingLaw(kind=scenes.RING_ELLIPTIC, r0=0.4, growth=1.25)
    laws[2] = scenes.RingLaw(mark=scenes.MARK_PER_OBSTACLE)
    laws[3] = scenes.RingLaw(kind=scenes.RING_ELLIPTIC, mark=scenes.MARK_PER_OBSTACLE, time_outer=1)
    tracks = [sc.tracks for sc in scs]
    tracks[4] = np.zeros((0, 21))
    odd = scenes.Scene("odd", 0, 37, 5, 0.05, static_occ=None)
    odd.robot = np.array([0.3, 0.1, 0.6, 0.8, 0.75])
    scs.append(odd); laws.append(scenes.RingLaw(r0=0.1, growth=1.4)); tracks.append(scs[0].tracks[:7])
    jobs = []
    for i, (sc, law, tr) in enumerate(zip(scs, laws, tracks)):
        static = None
        if sc.static_occ is not None and i != 5:
            static = torch.from_numpy(np.ascontiguousarray(sc.static_occ)).to(dev)
        ring = torch.empty((sc.ny, sc.nx), dtype=torch.int16, device=dev) if i != 6 else None
        jobs.append({"grid": tw.make_grid(sc.nx, sc.ny, sc.cell, sc.ox, sc.oy), "robot": sc.robot, "law": law,
                     "tracks": tr, "static_occ": static, "ring": ring})
    outs = tw.tw_build_grids(jobs)
    torch.cuda.synchronize()
    for i, ((occ, ring), sc, law, tr) in enumerate(zip(outs, scs, laws, tracks)):
        so = "scene" if i != 5 else None
        occ_ref, ring_ref, _ = oracle.build_grid(sc, law=law, tracks=tr, static_occ=so)
        assert np.array_equal(occ.cpu().numpy(), occ_ref), i
        if ring is not None:
            assert np.array_equal(ring.cpu().numpy(), ring_ref), i
    # a second call reusing the cached workspace, one job
    (occ0, _), = tw.tw_build_grids(jobs[:1])
    assert np.array_equal(occ0.cpu().numpy(), outs[0][0].cpu().numpy())
    # a prepared batch re-run after its tracks were updated in place (the next frame)
    gb = tw.GridBatch(jobs[:3])
    gb.run()
    for k in range(3):
        if len(gb.tracks[k]):
            gb.tracks[k][:, 0] += 0.4
            gb.tracks[k][:, 2] *= -1.0
    outs2 = gb.run()
    torch.cuda.synchronize()
    for k in range(3):
        so = "scene" if k != 5 else None
        occ_ref, ring_ref, _ = oracle.build_grid(scs[k], law=laws[k], tracks=gb.tracks[k], static_occ=so)
        assert np.array_equal(outs2[k][0].cpu().numpy(), occ_ref), k


def test_raster_full_size_2048_with_tracks(dev):
    sc = scenes.static2048()
    st = scenes.rng.Stream(42)
    n = 200
    L = sc.nx * sc.cell
    pos = np.stack([st.uniform(n, 0, L), st.uniform(n, 0, L)], 1)
    ang = st.uniform(n, 0, 2 * np.pi)
    spd = st.uniform(n, 0, 1)
    tr = scenes.synth_tracks(st, pos, np.stack([spd * np.cos(ang), spd * np.sin(ang)], 1),
                             st.uniform(n, 0.15, 0.5))
    _assert_raster_equal(sc, dev, tracks=tr)


def test_raster_empty_tracks_and_no_static(dev):
    sc = scenes.Scene("empty", 0, 40, 30, 0.05, static_occ=None)
    sc.robot = np.array([1.0, 0.7, 1.0, 0.0, 0.75])
    occ, ring = _gpu_grid(sc, dev, tracks=np.zeros((0, 21)))
    o = occ.cpu().numpy()
    assert (o[1:-1, 1:-1] == 0).all() and (o[0] == 3).all() and (o[:, -1] == 3).all()
    _, ring_ref, _ = oracle.build_grid(sc, tracks=np.zeros((0, 21)))
    assert np.array_equal(ring.cpu().numpy(), ring_ref)


# ---------------------------------------------------------------------------
# field
# ---------------------------------------------------------------------------

def _relax(sc_or_occ, goal, dev, params, grid=None):
    occ = sc_or_occ if isinstance(sc_or_occ, np.ndarray) else None
    occ_t = torch.from_numpy(np.ascontiguousarray(occ)).to(dev)
    ny, nx = occ.shape
    grid = grid or tw.make_grid(nx, ny, 0.05)
    u, stats = tw.hp_relax(grid, occ_t, goal, params=params)
    torch.cuda.synchronize()
    return u.cpu().numpy().astype(np.float64), stats


@pytest.fixture(scope="module")
def ref128():
    sc = scenes.static128()
    occ, _, _ = oracle.build_grid(sc)
    u, fixed = oracle.solve_field(occ, sc.goal, tol=1e-14)
    tau = oracle.exit_time(fixed)
    return sc, occ, u, fixed, tau.max()


def _np_residual(u, fixed):
    a = np.zeros_like(u)
    a[1:-1, 1:-1] = 0.25 * (((u[1:-1, 2:] + u[1:-1, :-2]) + u[2:, 1:-1]) + u[:-2, 1:-1])
    r = np.abs(a - u)
    r[fixed != 0] = 0
    return r.max()


@pytest.mark.parametrize("method", [tw.HP_JACOBI, tw.HP_RBSOR])
def test_field_static128_at_tolerance(dev, ref128, method):
    sc, occ, ustar, fixed, tau_max = ref128
    u, st = _relax(occ, sc.goal, dev, tw.Params(method=method, tol=1e-6))
    assert st["status"] == tw.TW_OK and st["resid_inf"] <= 1e-6
    assert abs(_np_residual(u, fixed) - st["resid_inf"]) <= 1e-12
    err = np.abs(u - ustar).max()
    assert err <= tau_max * st["resid_inf"] * 1.001 + 1e-7, (err, tau_max, st)


@pytest.mark.parametrize("method,omega", [(tw.HP_RBSOR, 0.0), (tw.HP_RBSOR, 1.0), (tw.HP_RBSOR, 1.9)])
def test_field_static128_converged_within_1e5(dev, ref128, method, omega):
    sc, occ, ustar, fixed, _ = ref128
    u, st = _relax(occ, sc.goal, dev, tw.Params(method=method, omega=omega, tol=0.0, max_sweeps=20000))
    err = np.abs(u - ustar).max()
    assert err <= 1e-5, (err, st)
    assert u.min() >= -1e-6 and u.max() <= 1.0


def test_field_jacobi_plain_converged_within_1e5(dev, ref128):
    sc, occ, ustar, fixed, _ = ref128
    u, st = _relax(occ, sc.goal, dev, tw.Params(method=tw.HP_JACOBI, tol=0.0, max_sweeps=60000))
    assert np.abs(u - ustar).max() <= 1e-5


def test_field_dynamic512(dev):
    sc = scenes.dynamic512()
    occ, _, _ = oracle.build_grid(sc)
    free = np.argwhere(occ == 0)
    d = np.hypot(free[:, 1] - sc.goal[0], free[:, 0] - sc.goal[1])
    gy, gx = free[np.argmin(d)]
    ustar, fixed = oracle.solve_field(occ, (gx, gy), tol=1e-13)
    tau_max = oracle.exit_time(fixed).max()
    u, st = _relax(occ, (int(gx), int(gy)), dev, tw.Params(method=tw.HP_RBSOR, tol=1e-6))
    assert st["resid_inf"] <= 1e-6
    assert np.abs(u - ustar).max() <= tau_max * st["resid_inf"] * 1.001 + 1e-7


@pytest.mark.parametrize("nx,ny", [(3, 3), (4, 3), (3, 5), (5, 4), (17, 33), (33, 17), (1025, 5), (6, 301)])
def test_field_odd_sizes(dev, nx, ny):
    occ = np.zeros((ny, nx), np.uint8)
    occ[0, :] = occ[-1, :] = occ[:, 0] = occ[:, -1] = 3
    rng = np.random.default_rng(nx * 7 + ny)
    inner = occ[1:-1, 1:-1]
    inner[rng.random(inner.shape) < 0.1] = 1
    goal = (1 + (nx - 2) // 2, 1 + (ny - 2) // 2)
    occ[goal[1], goal[0]] = 0
    ustar, fixed = oracle.solve_field(occ, goal, tol=1e-15)
    for method in (tw.HP_JACOBI, tw.HP_RBSOR):
        u, st = _relax(occ, goal, dev, tw.Params(method=method, tol=0.0, max_sweeps=40000))
        assert np.abs(u - ustar).max() <= 1e-5, (method, nx, ny)


def test_dirichlet_closed_form_on_gpu(dev):
    nx, ny = 61, 45
    jj, ii = np.mgrid[0:ny, 0:nx].astype(np.float64)
    exact = 0.5 + ((ii - 30) ** 2 - (jj - 22) ** 2) / 2000.0   # discrete-harmonic, in [0, 1]
    fixed = np.zeros((ny, nx), np.uint8)
    fixed[0, :] = fixed[-1, :] = fixed[:, 0] = fixed[:, -1] = 1
    fixed[20:25, 10:14] = 1                                   # an interior Dirichlet block
    u0 = np.where(fixed == 1, exact, 0.5).astype(np.float32)
    f = torch.from_numpy(fixed).to(dev)
    # converged to the FP32 floor: Jacobi and red-black Gauss-Seidel round each
    # update once (floor ~ 1 ulp); over-relaxation amplifies the rounding noise
    # by ~omega / (2 - omega), so at omega = 1.9 only the field error is checked
    for method, omega, r_max in ((tw.HP_JACOBI, 0.0, 1e-6), (tw.HP_RBSOR, 1.0, 1e-6), (tw.HP_RBSOR, 1.9, None)):
        u = torch.from_numpy(u0.copy()).to(dev)
        u, st = tw.hp_relax_dirichlet(f, u, tw.Params(method=method, omega=omega, tol=0.0, max_sweeps=30000))
        assert np.abs(u.cpu().numpy() - exact).max() <= 1e-5, (method, omega)
        r_inf, _ = tw.hp_residual(f, u)
        assert r_max is None or r_inf <= r_max, (method, omega, r_inf)
    # adaptive SOR with a tolerance below its over-relaxed floor backs off and reaches it
    u = torch.from_numpy(u0.copy()).to(dev)
    u, st = tw.hp_relax_dirichlet(f, u, tw.Params(method=tw.HP_RBSOR, tol=3e-7, max_sweeps=30000))
    assert st["status"] == tw.TW_OK and st["resid_inf"] <= 3e-7, st


@pytest.mark.parametrize("tblock", [1, 2, 3, 4, 5, 6, 7])
def test_temporal_blocking_matches_unfused_sweeps(dev, tblock):
    """T fused sweeps per launch (small tiles up to T = 4, deep tiles for 5..7)
    give exactly the field of T separate red-black half-sweep launches."""
    for nx, ny in ((128, 128), (301, 97), (1030, 67), (67, 1030)):
        occ = np.zeros((ny, nx), np.uint8)
        occ[0, :] = occ[-1, :] = occ[:, 0] = occ[:, -1] = 3
        rng = np.random.default_rng(nx + 3 * ny)
        inner = occ[1:-1, 1:-1]
        inner[rng.random(inner.shape) < 0.2] = 1
        goal = (nx // 2, ny // 2)
        occ[goal[1], goal[0]] = 0
        outs = []
        for tb in (1, tblock):
            u, st = _relax(occ, goal, dev, tw.Params(method=tw.HP_RBSOR, omega=1.7, tol=0.0, max_sweeps=37,
                                                     tblock=tb, check_every=12))
            assert st["sweeps"] == 37
            outs.append(u)
        assert np.array_equal(outs[0], outs[1]), (nx, ny, tblock)


def test_graph_loop_matches_host_loop(dev):
    """The CUDA-graph convergence loop takes the same decisions as the host loop
    and returns the same field, bit for bit."""
    for sc in (scenes.static128(), scenes.static_occupancy(5, 700, 260, 0.25)):
        occ, _, _ = oracle.build_grid(sc)
        a, sa = _relax(occ, sc.goal, dev, tw.Params(tol=1e-6))
        b, sb = _relax(occ, sc.goal, dev, tw.Params(tol=1e-6, flags=tw.HP_HOST_LOOP))
        assert sa["loop"] == tw.HP_LOOP_GRAPH and sb["loop"] == tw.HP_LOOP_HOST
        assert sa["status"] == sb["status"] == tw.TW_OK
        assert sa["sweeps"] == sb["sweeps"] and sa["checks"] == sb["checks"]
        assert sa["polishes"] == sb["polishes"] and sa["polished"] == sb["polished"]
        # omega adapts on the device (graph) or on the host: their libm may differ in the last bit
        assert abs(sa["omega"] - sb["omega"]) <= 1e-12
        assert np.array_equal(a, b)
        # a cap that is not a multiple of the check interval: graph intervals + host remainder
        c, sc_ = _relax(occ, sc.goal, dev, tw.Params(tol=1e-12, max_sweeps=100))
        d, sd = _relax(occ, sc.goal, dev, tw.Params(tol=1e-12, max_sweeps=100, flags=tw.HP_HOST_LOOP))
        assert sc_["sweeps"] == sd["sweeps"] == 100 and sc_["status"] == tw.TW_NOT_CONVERGED
        assert np.array_equal(c, d)


def test_deep_tiles_graph_matches_host_loop(dev):
    """A field large enough for the deep tiles (T = 7, 28-sweep check interval by
    default): graph and host loops agree bit for bit, including a cap that ends
    inside an interval, and the explicit T = 4 form reaches the same tolerance."""
    nx, ny = 2048, 1500
    rng = np.random.default_rng(77)
    occ = (rng.random((ny, nx)) < 0.25).astype(np.uint8)
    occ[0, :] = occ[-1, :] = occ[:, 0] = occ[:, -1] = 3
    goal = (1500, 700)
    occ[goal[1], goal[0]] = 0
    a, sa = _relax(occ, goal, dev, tw.Params(tol=1e-6))
    b, sb = _relax(occ, goal, dev, tw.Params(tol=1e-6, flags=tw.HP_HOST_LOOP))
    assert sa["tblock"] == sb["tblock"] == 7 and sa["loop"] == tw.HP_LOOP_GRAPH
    assert sa["status"] == sb["status"] == tw.TW_OK and sa["sweeps"] == sb["sweeps"]
    assert sa["polishes"] == sb["polishes"] and sa["polished"] == sb["polished"]
    assert (sa["sweeps"] - 7 * sa["polishes"]) % 28 == 0 and abs(sa["omega"] - sb["omega"]) <= 1e-12
    assert np.array_equal(a, b)
    c, sc_ = _relax(occ, goal, dev, tw.Params(tol=1e-12, max_sweeps=100))
    d, sd = _relax(occ, goal, dev, tw.Params(tol=1e-12, max_sweeps=100, flags=tw.HP_HOST_LOOP))
    assert sc_["sweeps"] == sd["sweeps"] == 100 and np.array_equal(c, d)
    # HP_TIMING runs each interval's launches as one captured graph (omega read from device memory)
    t, st_ = _relax(occ, goal, dev, tw.Params(tol=1e-6, flags=tw.HP_TIMING))
    assert st_["loop"] == tw.HP_LOOP_HOST and st_["sweeps"] == sb["sweeps"] and st_["sweep_ms"] > 0.0
    assert st_["sweep_launches"] == sb["sweep_launches"]
    assert np.array_equal(t, b)
    e, se = _relax(occ, goal, dev, tw.Params(tol=1e-6, tblock=4))
    assert se["tblock"] == 4 and se["status"] == tw.TW_OK
    assert np.abs(e - a).max() <= 1e-4   # both within their a-posteriori bounds of the same solution


@pytest.mark.parametrize("nx,ny,tb", [(2048, 1500, 7), (1800, 1403, 7), (600, 300, 4), (333, 97, 2)])
def test_loop_check_residual_is_the_fields_residual(dev, nx, ny, tb):
    """The residual the convergence loop stops on is the FP32 residual max of
    the whole output field, exactly: the loop's last check equals the max over
    the free cells of the FP32 residual of the returned field (neighbour sums
    in FP32, then one rounding of 0.25 s - c), for ragged tiles and either loop."""
    rng = np.random.default_rng(nx + ny)
    occ = (rng.random((ny, nx)) < 0.25).astype(np.uint8)
    occ[0, :] = occ[-1, :] = occ[:, 0] = occ[:, -1] = 3
    goal = (nx // 3, ny // 2)
    occ[goal[1], goal[0]] = 0
    fixed = oracle.dirichlet_from_occ(occ, goal)[1].astype(bool)
    K = 28 if tb == 7 else 32
    for flags in (0, tw.HP_HOST_LOOP):
        for n_int in (1, 3):
            u, st = _relax(occ, goal, dev, tw.Params(omega=1.93, tol=1e-30, max_sweeps=K * n_int, tblock=tb,
                                                      flags=flags))
            assert st["sweeps"] == K * n_int and st["checks"] == n_int and st["tblock"] == tb
            u32 = u.astype(np.float32)
            c = u32[1:-1, 1:-1]
            s32 = (u32[1:-1, :-2] + u32[1:-1, 2:]) + (u32[:-2, 1:-1] + u32[2:, 1:-1])
            t = (0.25 * s32.astype(np.float64) - c.astype(np.float64)).astype(np.float32)
            r = float(np.abs(t)[~fixed[1:-1, 1:-1]].max())
            assert st["resid_check"] == r, (st["resid_check"], r)


def _polish_scenes():
    rng = np.random.default_rng(77)
    occ = (rng.random((1500, 2048)) < 0.25).astype(np.uint8)
    occ[0, :] = occ[-1, :] = occ[:, 0] = occ[:, -1] = 3
    occ[700, 1500] = 0
    sc = scenes.static128()
    occ128, _, _ = oracle.build_grid(sc)
    s700 = scenes.static_occupancy(5, 700, 260, 0.25)
    occ700, _, _ = oracle.build_grid(s700)
    return [(occ128, sc.goal), (occ700, s700.goal), (occ, (1500, 700))]


@pytest.mark.parametrize("case", [0, 1, 2])
def test_polish_is_gauss_seidel_on_the_sor_planes(dev, case):
    """HP_POLISH is a side branch: an accepted polished solve returns exactly
    T Gauss-Seidel sweeps (omega = 1, same kernel) applied to the SOR field the
    plain solve reaches after the same SOR sweeps, and the SOR sequence itself
    is the plain one (same omega, same checks); graph and host loops agree."""
    occ, goal = _polish_scenes()[case]
    res = []
    for flags in (0, tw.HP_HOST_LOOP):
        a, sa = _relax(occ, goal, dev, tw.Params(tol=1e-6, flags=flags | tw.HP_POLISH))
        res.append((a, sa))
        n, sn = _relax(occ, goal, dev, tw.Params(tol=1e-6, flags=flags))
        assert sa["status"] == sn["status"] == tw.TW_OK and sn["polishes"] == 0
        assert sa["resid_inf"] <= 1e-6
        T = sa["tblock"]
        assert sa["polishes"] >= 1 and sa["polished"] == 1, sa
        s_sor = sa["sweeps"] - T * sa["polishes"]
        assert s_sor <= sn["sweeps"]
        # the unpolished SOR field after s_sor sweeps, then T sweeps at omega = 1
        b, sb = _relax(occ, goal, dev, tw.Params(tol=1e-6, max_sweeps=s_sor, flags=flags))
        assert sb["sweeps"] == s_sor and abs(sb["omega"] - sa["omega"]) <= 1e-12
        occ_t = torch.from_numpy(np.ascontiguousarray(occ)).to(dev)
        grid = tw.make_grid(occ.shape[1], occ.shape[0], 0.05)
        u = torch.from_numpy(b.astype(np.float32)).to(dev)
        g, sg = tw.hp_relax(grid, occ_t, goal, field=u,
                            params=tw.Params(omega=1.0, tol=0.0, max_sweeps=T, tblock=T, flags=tw.HP_WARM_START))
        assert sg["sweeps"] == T and sg["sweep_launches"] == 1
        assert np.array_equal(g.cpu().numpy().astype(np.float64), a)
    (a, sa), (b, sb) = res
    assert sa["loop"] == tw.HP_LOOP_GRAPH and sb["loop"] == tw.HP_LOOP_HOST
    assert sa["sweeps"] == sb["sweeps"] and sa["polishes"] == sb["polishes"] and np.array_equal(a, b)


def test_warm_start_and_phi_output(dev, ref128):
    sc, occ, ustar, fixed, tau_max = ref128
    occ_t = torch.from_numpy(occ).to(dev)
    grid = tw.make_grid(sc.nx, sc.ny, sc.cell)
    u, st1 = tw.hp_relax(grid, occ_t, sc.goal, params=tw.Params(tol=1e-4))
    u2, st2 = tw.hp_relax(grid, occ_t, sc.goal, field=u.clone(),
                          params=tw.Params(tol=1e-6, flags=tw.HP_WARM_START))
    _, st3 = tw.hp_relax(grid, occ_t, sc.goal, params=tw.Params(tol=1e-6))
    assert st2["sweeps"] < st3["sweeps"]
    phi, st4 = tw.hp_relax(grid, occ_t, sc.goal, params=tw.Params(tol=1e-6, flags=tw.HP_OUT_PHI))
    p = phi.cpu().numpy().astype(np.float64)
    assert np.abs((1.0 - p) - ustar).max() <= tau_max * st4["resid_inf"] * 1.001 + 1e-6
    assert p[sc.goal[1], sc.goal[0]] == 0.0 and p[0, 0] == 1.0


def test_goal_blocked_errors(dev, ref128):
    sc, occ, *_ = ref128
    occ_t = torch.from_numpy(occ).to(dev)
    grid = tw.make_grid(sc.nx, sc.ny, sc.cell)
    blocked = tuple(int(v) for v in np.argwhere(occ == 1)[0][::-1])
    with pytest.raises(tw.TwError) as e:
        tw.hp_relax(grid, occ_t, blocked)
    assert e.value.status == tw.TW_EGOAL_BLOCKED


def test_not_converged_status(dev, ref128):
    sc, occ, *_ = ref128
    u, st = _relax(occ, sc.goal, dev, tw.Params(tol=1e-9, max_sweeps=10))
    assert st["status"] == tw.TW_NOT_CONVERGED and st["sweeps"] == 10


@pytest.fixture(scope="module")
def ref2048():
    sc = scenes.static2048()
    occ, _, _ = oracle.build_grid(sc)
    ustar, fixed = oracle.solve_field(occ, sc.goal, tol=1e-13)
    return sc, occ, ustar, fixed


@pytest.mark.slow
def test_field_full_size_2048(dev, ref2048):
    """The residual test alone (r_inf <= 1e-6): the a-posteriori bound holds."""
    sc, occ, ustar, fixed = ref2048
    u, st = _relax(occ, sc.goal, dev, tw.Params(method=tw.HP_RBSOR, tol=1e-6))
    assert st["status"] == tw.TW_OK and st["resid_inf"] <= 1e-6
    assert _np_residual(u, fixed) <= 1e-6
    tau_max = oracle.exit_time(fixed, tol=1e-6).max()
    bound = tau_max * st["resid_inf"] * 1.01 + 1e-6
    # u* lies in [0, 1] (maximum principle), so u may leave it by the bound at most
    assert u.min() >= -bound and u.max() <= 1.0
    err = np.abs(u - ustar).max()
    assert err <= bound, (err, tau_max, st)


@pytest.mark.slow
@pytest.mark.parametrize("flags", [0, tw.HP_HOST_LOOP])
def test_field_full_size_2048_within_1e5(dev, ref2048, flags):
    """The measured form: r_inf <= 1e-6 and the error estimate <= 1e-5 (deep tiles, T = 7);
    max |u - u*| over every cell of the 2048 x 2048 field is at most 1e-5."""
    sc, occ, ustar, fixed = ref2048
    u, st = _relax(occ, sc.goal, dev, tw.Params(method=tw.HP_RBSOR, tol=1e-6, etol=1e-5, flags=flags))
    assert st["status"] == tw.TW_OK and st["resid_inf"] <= 1e-6 and st["tblock"] == 7, st
    assert _np_residual(u, fixed) <= 1e-6
    err = np.abs(u - ustar).max()
    assert err <= 1e-5 and st["err_est"] <= 1e-5, (err, st)


@pytest.mark.slow
def test_path_full_size_2048(dev, ref2048):
    """Eq. 3 descent + rubber band on the measured form's 2048 x 2048 field, from the free cell nearest
    the robot whose u* is at least 1e-3 (the robot's own cell has u* ~ 1e-12, far below what a field
    accurate to 1e-5 -- or the oracle's own CG solve -- resolves): valid and within 2 cells of the
    oracle's path."""
    sc, occ, ustar, fixed = ref2048
    yy, xx = np.nonzero((ustar >= 1e-3) & (occ == 0))
    j = int(np.argmin((xx - sc.start[0]) ** 2 + (yy - sc.start[1]) ** 2))
    start = (int(xx[j]), int(yy[j]))
    occ_t = torch.from_numpy(occ).to(dev)
    grid = tw.make_grid(sc.nx, sc.ny, sc.cell)
    u, st = tw.hp_relax(grid, occ_t, sc.goal, params=tw.Params(tol=1e-6, etol=1e-5))
    assert st["status"] == tw.TW_OK
    for rubber in (0, 100):
        status, path = tw.plan_path(grid, u, occ_t, start, sc.goal, rubber_iters=rubber)
        ost, opath = oracle.plan_path(ustar, fixed, start, sc.goal, rubber_iters=rubber)
        assert status == tw.TW_OK and ost == oracle.OK
        assert tuple(path[0]) == start and tuple(path[-1]) == tuple(sc.goal) and len(path) >= 50
        assert (occ[path[:, 1], path[:, 0]] == 0).all()
        assert (np.abs(np.diff(path, axis=0)).max(1) == 1).all()
        assert _hausdorff(path, opath) <= 2.0


def _static_case(name):
    if name == "batch7003":
        return scenes.batch_fast(7003)
    side, occf, seed = {"s300": (300, 0.2, 77), "s512": (512, 0.3, 5), "s768": (768, 0.35, 9),
                        "s384": (384, 0.25, 122)}[name]
    return scenes.static_occupancy(seed, side, 40 if name != "s384" else 30, occf, name=name)


@pytest.mark.parametrize("name", ["s300", "s512", "s768", "s384", "batch7003"])
def test_field_error_estimate_within_1e5(dev, name):
    """r_inf <= 1e-6 with the error estimate <= 1e-5 on small-tile fields (T = 4): max |u - u*| <= 1e-5
    over the whole field, and the graph-driven and host-driven loops agree bit for bit."""
    sc = _static_case(name)
    occ, _, _ = oracle.build_grid(sc)
    if occ[sc.goal[1], sc.goal[0]] != 0:
        pytest.skip("goal covered")
    ustar, fixed = oracle.solve_field(occ, sc.goal, tol=1e-13)
    u, st = _relax(occ, sc.goal, dev, tw.Params(tol=1e-6, etol=1e-5))
    uh, sth = _relax(occ, sc.goal, dev, tw.Params(tol=1e-6, etol=1e-5, flags=tw.HP_HOST_LOOP))
    assert st["status"] == tw.TW_OK and st["resid_inf"] <= 1e-6, st
    assert np.array_equal(u, uh) and st["sweeps"] == sth["sweeps"]
    err = np.abs(u - ustar).max()
    assert err <= 1e-5 and st["err_est"] <= 1e-5, (err, st)


def test_field_error_estimate_open_scene(dev):
    """An open 1024 x 1024 field (5 % obstacles), where SOR runs at omega near 2: the solve either
    certifies the estimate (and then the error is within it) or stops unconverged; the residual-only
    test on the same field ends with an error far above 1e-5 (the back-off meets r_inf by slowing
    the smooth error's decay)."""
    sc = scenes.static_occupancy(8, 1024, 40, 0.05, name="s1024")
    occ, _, _ = oracle.build_grid(sc)
    ustar, fixed = oracle.solve_field(occ, sc.goal, tol=1e-13)
    u, st = _relax(occ, sc.goal, dev, tw.Params(tol=1e-6, etol=1e-5))
    err = np.abs(u - ustar).max()
    assert st["status"] in (tw.TW_OK, tw.TW_NOT_CONVERGED)
    if st["status"] == tw.TW_OK:
        assert err <= 1e-5 and st["resid_inf"] <= 1e-6, (err, st)
    u0, st0 = _relax(occ, sc.goal, dev, tw.Params(tol=1e-6))
    assert st0["status"] == tw.TW_OK and np.abs(u0 - ustar).max() > 1e-4


# ---------------------------------------------------------------------------
# path
# ---------------------------------------------------------------------------

def _hausdorff(a, b):
    a = a.astype(np.float64)
    b = b.astype(np.float64)
    d = np.hypot(a[:, None, 0] - b[None, :, 0], a[:, None, 1] - b[None, :, 1])
    return max(d.min(1).max(), d.min(0).max())


@pytest.fixture(scope="module")
def polished128():
    sc = scenes.static128()
    occ, _, _ = oracle.build_grid(sc)
    u, fixed = oracle.solve_field(occ, sc.goal, tol=1e-14)
    u, _, _, _ = oracle.gauss_seidel(u, fixed, tol=0.0, max_sweeps=20000)
    return sc, occ, u, fixed


@pytest.mark.parametrize("rubber", [0, 100])
def test_path_static128(dev, polished128, rubber):
    sc, occ, uref, fixed = polished128
    occ_t = torch.from_numpy(occ).to(dev)
    grid = tw.make_grid(sc.nx, sc.ny, sc.cell)
    # red-black Gauss-Seidel (omega = 1) keeps tiny far-field values relatively accurate
    u, st = tw.hp_relax(grid, occ_t, sc.goal, params=tw.Params(omega=1.0, tol=0.0, max_sweeps=30000))
    status, path = tw.plan_path(grid, u, occ_t, sc.start, sc.goal, rubber_iters=rubber)
    ost, opath = oracle.plan_path(uref, fixed, sc.start, sc.goal, rubber_iters=rubber)
    assert ost == oracle.OK and status == tw.TW_OK
    assert tuple(path[0]) == sc.start and tuple(path[-1]) == sc.goal
    assert (occ[path[:, 1], path[:, 0]] == 0).all()
    step = np.abs(np.diff(path, axis=0)).max(1)
    assert (step == 1).all()
    if rubber == 0:
        uu = u.cpu().numpy()[path[:, 1], path[:, 0]]
        assert (np.diff(uu) > 0).all()
    assert _hausdorff(path, opath) <= 2.0


def test_nearest_free(dev):
    occ = np.ones((20, 30), np.uint8)
    occ[5, 7] = occ[15, 25] = occ[9, 12] = 0
    occ_t = torch.from_numpy(occ).to(dev)
    grid = tw.make_grid(30, 20, 0.05)
    assert tw.tw_nearest_free(grid, occ_t, 12, 9) == (12, 9)
    assert tw.tw_nearest_free(grid, occ_t, 24, 14) == (25, 15)
    assert tw.tw_nearest_free(grid, occ_t, 1, 1) == (7, 5)
    occ[:] = 1
    assert tw.tw_nearest_free(grid, torch.from_numpy(occ).to(dev), 3, 3) is None


def test_path_errors(dev):
    n = 40
    occ = np.zeros((n, n), np.uint8)
    occ[0, :] = occ[-1, :] = occ[:, 0] = occ[:, -1] = 3
    occ[10:20, 10] = occ[10:20, 19] = occ[10, 10:20] = occ[19, 10:20] = 1
    occ_t = torch.from_numpy(occ).to(dev)
    grid = tw.make_grid(n, n, 0.05)
    u, _ = tw.hp_relax(grid, occ_t, (15, 15), params=tw.Params(tol=1e-7))
    st, _ = tw.plan_path(grid, u, occ_t, (30, 30), (15, 15))
    assert st == tw.TW_NO_PATH
    st, _ = tw.plan_path(grid, u, occ_t, (10, 12), (15, 15))
    assert st == tw.TW_ESTART_BLOCKED
    st, p = tw.plan_path(grid, u, occ_t, (15, 15), (15, 15))
    assert st == tw.TW_OK and len(p) == 1


def test_end_to_end_planner_frame(dev):
    """Raster -> relaxation -> path on one frame, all through the C ABI."""
    sc = scenes.dynamic(seed=1041, side=256, n_obs=16, frames=1, static_shapes=12)
    occ, _ = _gpu_grid(sc, dev, with_ring=False)
    occ_ref, _, _ = oracle.build_grid(sc)
    assert np.array_equal(occ.cpu().numpy(), occ_ref)
    grid = tw.make_grid(sc.nx, sc.ny, sc.cell)
    if occ_ref[sc.goal[1], sc.goal[0]] != 0:
        pytest.skip("goal covered by a prediction in this frame")
    u, st = tw.hp_relax(grid, occ, sc.goal, params=tw.Params(omega=1.0, tol=0.0, max_sweeps=40000))
    status, path = tw.plan_path(grid, u, occ, sc.start, sc.goal, rubber_iters=50)
    uref, fixed = oracle.solve_field(occ_ref, sc.goal, tol=1e-14)
    uref, _, _, _ = oracle.gauss_seidel(uref, fixed, tol=0.0, max_sweeps=20000)
    ost, opath = oracle.plan_path(uref, fixed, sc.start, sc.goal, rubber_iters=50)
    assert status == ost
    if status == tw.TW_OK:
        assert (occ_ref[path[:, 1], path[:, 0]] == 0).all()
        assert _hausdorff(path, opath) <= 2.0


@pytest.mark.parametrize("seed,rubber", [(1041, 50), (1042, 100), (1046, 7)])
def test_path_equals_oracle_on_the_same_field(dev, seed, rubber):
    """Given the GPU's own field, the GPU descent (Eq. 3, tie order +x, -x, +y, -y) and rubber band
    (odd-then-even node sweeps, candidates in dy-then-dx order, FP64 energies) return exactly the
    oracle's path, node for node -- not just within the Hausdorff tolerance that separate fields
    need.  Starts: the scene's start, and the free cell farthest from the goal where u >= 1e-5."""
    sc = scenes.dynamic(seed=seed, side=256, n_obs=16, frames=1, static_shapes=12)
    occ, _, _ = oracle.build_grid(sc)
    goal = sc.goal
    assert occ[goal[1], goal[0]] == 0
    occ_t = torch.from_numpy(occ).to(dev)
    grid = tw.make_grid(sc.nx, sc.ny, sc.cell)
    u, _ = tw.hp_relax(grid, occ_t, goal, params=tw.Params(omega=1.0, tol=0.0, max_sweeps=40000))
    u64 = u.cpu().numpy().astype(np.float64)
    _, fixed = oracle.dirichlet_from_occ(occ, goal)
    cand = np.argwhere((occ == 0) & (u64 >= 1e-5))
    far = cand[np.argmax(np.abs(cand[:, 1] - goal[0]) + np.abs(cand[:, 0] - goal[1]))]
    long_paths = 0
    for start in (sc.start, (int(far[1]), int(far[0]))):
        status, path = tw.plan_path(grid, u, occ_t, start, goal, rubber_iters=rubber)
        ost, opath = oracle.plan_path(u64, fixed, start, goal, rubber_iters=rubber)
        assert status == ost
        if status == tw.TW_OK:
            assert np.array_equal(path, opath)
            long_paths += len(path) > 50
    assert long_paths >= 1
