"""Mixed-precision defect correction (HP_MIXED) against the FP64 oracle.

The correction sweeps store the field in FP16 / BF16 (or FP32) and compute in
FP32; the residual and the accumulated solution are FP64.  The FP64 master can
therefore go far below the FP32 rounding floor: the tests ask for residuals of
1e-9 and a field within 1e-5 of the oracle, and for the Eq. 3 index matrix
(direction of the largest u) to agree with the oracle's in the near-flat region
phi > 0.99, away from oracle near-ties."""
import numpy as np
import pytest

import oracle
import paper_1903_07441_gb300 as tw
import scenes

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

STORES = [tw.HP_STORE_F32, tw.HP_STORE_F16, tw.HP_STORE_BF16]


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1903_07441_gb300 import build
    build.build()
    return torch.device("cuda:0")


def _nearest_free(occ, g):
    free = np.argwhere(occ == 0)
    d = np.hypot(free[:, 1] - g[0], free[:, 0] - g[1])
    j = int(np.argmin(d))
    return int(free[j, 1]), int(free[j, 0])


def _solve(dev, occ, goal, **kw):
    occ_t = torch.from_numpy(occ).to(dev)
    grid = tw.make_grid(occ.shape[1], occ.shape[0], 0.05)
    u, st = tw.hp_relax(grid, occ_t, goal, params=tw.Params(method=tw.HP_MIXED, **kw))
    return u.cpu().numpy().astype(np.float64), st


def _index_matrix(u):
    """Eq. 3 direction (0..3 = +x, -x, +y, -y) of the largest neighbour, and the gap to the runner-up."""
    nb = np.stack([u[1:-1, 2:], u[1:-1, :-2], u[2:, 1:-1], u[:-2, 1:-1]])
    d = np.argmax(nb, axis=0)
    srt = np.sort(nb, axis=0)
    return d, srt[-1] - srt[-2]


@pytest.mark.parametrize("storage", STORES)
def test_mixed_static128_tight(dev, storage):
    sc = scenes.static128()
    occ, _, _ = oracle.build_grid(sc)
    ustar, fixed = oracle.solve_field(occ, sc.goal, tol=1e-14)
    u, st = _solve(dev, occ, sc.goal, storage=storage, tol=1e-9)
    assert st["status"] == tw.TW_OK and st["resid_inf"] <= 1e-9, st
    assert np.abs(u - ustar).max() <= 1e-5


@pytest.mark.parametrize("storage", STORES)
def test_mixed_dynamic512_and_flat_region_directions(dev, storage):
    sc = scenes.dynamic512()
    occ, _, _ = oracle.build_grid(sc)
    goal = _nearest_free(occ, sc.goal)
    ustar, fixed = oracle.solve_field(occ, goal, tol=1e-14)
    tol = 1e-11
    u, st = _solve(dev, occ, goal, storage=storage, tol=tol)
    assert st["status"] == tw.TW_OK and st["resid_inf"] <= tol, st
    assert np.abs(u - ustar).max() <= 1e-5
    # direction agreement where phi > 0.99 (u < 0.01) on free cells whose oracle
    # gap to the runner-up exceeds twice the a-posteriori error bound tau_max * tol
    # plus the FP32 rounding of the output (near-ties may legitimately differ)
    tau_max = oracle.exit_time(fixed).max()
    d_ref, gap = _index_matrix(ustar)
    d_gpu, _ = _index_matrix(u)
    inner = ustar[1:-1, 1:-1]
    thresh = 2.0 * (tau_max * tol + 6e-8 * inner)
    flat = (inner < 0.01) & (fixed[1:-1, 1:-1] == 0) & (gap > thresh)
    assert flat.sum() >= 200, flat.sum()
    agree = (d_ref[flat] == d_gpu[flat]).mean()
    assert agree >= 0.99, agree


def test_mixed_reaches_1e6_at_2048(dev):
    """At 2048^2 the field is checked against the stored FP64 reference of the
    scene (CG to 1e-12, with its exit time tau_max): everywhere within the
    a-posteriori bound tau_max * r_inf of [0, 1] (u* lies there by the maximum
    principle), and at the stored sample cells within that bound of u*."""
    import hashlib
    import json
    import os
    sc = scenes.static2048()
    occ, _, _ = oracle.build_grid(sc)
    ref = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "static2048_field.json")))
    assert hashlib.sha256(np.ascontiguousarray(occ).tobytes()).hexdigest() == ref["occupancy_sha256"]
    cells = np.asarray(ref["cells"], dtype=np.int64)
    ustar = np.asarray([float(v) for v in ref["u_star"]])
    for storage in (tw.HP_STORE_F16, tw.HP_STORE_BF16):
        u, st = _solve(dev, occ, sc.goal, storage=storage, tol=1e-6)
        assert st["status"] == tw.TW_OK and st["resid_inf"] <= 1e-6, st
        bound = ref["tau_max"] * st["resid_inf"] * 1.001 + 1e-7   # + the FP32 rounding of the output
        assert u.min() >= -bound and u.max() <= 1.0 + bound
        assert np.abs(u[cells[:, 1], cells[:, 0]] - ustar).max() <= bound


@pytest.mark.slow
def test_mixed_with_error_tolerance_at_2048(dev):
    """With the error tolerance (etol = 1e-5, r_inf <= 1e-6) at 2048^2, against the oracle's full
    field: the FP16-storage form and the FP32-correction form (FP64 refinement) meet max |u - u*|
    <= 1e-5 over every cell -- far below it, since the FP64 master goes under the FP32 rounding
    floor -- and the BF16-storage form, whose 8-bit mantissa makes each correction solve short,
    either meets the tolerance or reports TW_NOT_CONVERGED (it never claims an accuracy it has not
    shown)."""
    sc = scenes.static2048()
    occ, _, _ = oracle.build_grid(sc)
    ustar, fixed = oracle.solve_field(occ, sc.goal, tol=1e-13)
    for storage, bound in ((tw.HP_STORE_F16, 1e-5), (tw.HP_STORE_F32, 1e-7)):
        u, st = _solve(dev, occ, sc.goal, storage=storage, tol=1e-6, etol=1e-5)
        err = np.abs(u - ustar).max()
        assert st["status"] == tw.TW_OK and st["resid_inf"] <= 1e-6 and st["err_est"] <= 1e-5, st
        assert err <= bound, (storage, err, st)
    u, st = _solve(dev, occ, sc.goal, storage=tw.HP_STORE_BF16, tol=1e-6, etol=1e-5)
    if st["status"] == tw.TW_OK:
        assert np.abs(u - ustar).max() <= 1e-5, st
    else:
        assert st["status"] == tw.TW_NOT_CONVERGED and np.abs(u - ustar).max() > 1e-6


@pytest.mark.parametrize("storage", STORES)
def test_mixed_inner_graph_matches_host_loop(dev, storage):
    """The correction solves run as CUDA graphs (conditional while-node, control on
    the device) by default and from the host with HP_HOST_LOOP: the same decisions,
    so both converge to the same field (omega is adapted by the device's or the
    host's libm, which may differ in the last bit, so the fields are compared
    within the a-posteriori bound rather than bit for bit)."""
    sc = scenes.static128()
    occ, _, _ = oracle.build_grid(sc)
    _, fixed = oracle.solve_field(occ, sc.goal, tol=1e-12)
    tau_max = oracle.exit_time(fixed).max()
    tol = 1e-9
    a, sa = _solve(dev, occ, sc.goal, storage=storage, tol=tol)
    b, sb = _solve(dev, occ, sc.goal, storage=storage, tol=tol, flags=tw.HP_HOST_LOOP)
    assert sa["loop"] == tw.HP_LOOP_GRAPH and sb["loop"] == tw.HP_LOOP_HOST
    assert sa["status"] == sb["status"] == tw.TW_OK
    assert sa["resid_inf"] <= tol and sb["resid_inf"] <= tol
    assert np.abs(a - b).max() <= 2.0 * tau_max * tol + 1e-7
    assert abs(sa["sweeps"] - sb["sweeps"]) <= 0.1 * sb["sweeps"] + 64


@pytest.mark.parametrize("storage", STORES)
def test_mixed_error_tolerance_on_several_scenes(dev, storage):
    """The mixed form's outer error estimate (the last FP64 update's size over 1 - q) holds the
    field within etol = 1e-5 of the FP64 oracle over the whole field on scenes of different sizes
    and occupancies, for every storage (BF16 may instead report TW_NOT_CONVERGED, never a field
    outside the tolerance with TW_OK)."""
    cases = [scenes.dynamic512(), scenes.static_occupancy(31, 640, 300, 0.30),
             scenes.static_occupancy(32, 768, 150, 0.15)]
    for sc in cases:
        occ, _, _ = oracle.build_grid(sc)
        goal = _nearest_free(occ, sc.goal)
        ustar, _ = oracle.solve_field(occ, goal, tol=1e-13)
        u, st = _solve(dev, occ, goal, storage=storage, tol=1e-6, etol=1e-5)
        err = np.abs(u - ustar).max()
        if st["status"] == tw.TW_OK:
            assert st["err_est"] <= 1e-5 and err <= 1e-5, (sc.nx, sc.ny, err, st)
        else:
            assert storage == tw.HP_STORE_BF16 and st["status"] == tw.TW_NOT_CONVERGED, st
