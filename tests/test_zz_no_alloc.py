"""hp_relax_noalloc: the relaxation for callers that cannot allocate device
memory (for example a real-time loop that may not call cudaMalloc after
start-up), running on the library's static scratch array.  Called through the
C ABI and compared with hp_relax, which uses a caller workspace, on two calls
in a row (the second on a different grid, so stale contents of the shared
array would show).  This file sorts last so that a run stopping at the first
failure has run every other test first."""
import ctypes

import numpy as np
import pytest

import oracle
import paper_1903_07441_gb300 as tw
import scenes

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _scene_occ(sc):
    occ, _, _ = oracle.build_grid(sc)
    return occ


def _call_noalloc(lib, grid, occ_t, goal, out, params):
    cp = params.c()
    st = tw.hp_stats()
    rc = lib.hp_relax_noalloc(ctypes.byref(grid), ctypes.c_void_p(occ_t.data_ptr()), int(goal[0]), int(goal[1]),
                              ctypes.c_void_p(out.data_ptr()), ctypes.byref(cp), ctypes.byref(st),
                              ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    return rc, st


def test_noalloc_matches_workspace_entry_point_twice():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1903_07441_gb300 import build
    build.build()
    lib = tw.load()
    dev = torch.device("cuda:0")
    cases = [scenes.static128(), scenes.static_occupancy(77, 300, 40, 0.2, name="s300")]
    for sc in cases:   # two calls in a row on different grids
        occ = _scene_occ(sc)
        occ_t = torch.from_numpy(occ).to(dev)
        grid = tw.make_grid(sc.nx, sc.ny, sc.cell)
        params = tw.Params(method=tw.HP_RBSOR, tol=1e-6)
        ref, st_ref = tw.hp_relax(grid, occ_t, sc.goal, params=params)
        out = torch.full((sc.ny, sc.nx), -7.0, dtype=torch.float32, device=dev)
        rc, st = _call_noalloc(lib, grid, occ_t, sc.goal, out, params)
        assert rc == tw.TW_OK, tw.status_string(rc)
        assert st.status == tw.TW_OK and st.resid_inf <= 1e-6
        assert st.sweeps == st_ref["sweeps"]
        # the same kernels in the same order (host-driven loop = graph-driven loop bit for bit)
        assert torch.equal(out, ref), np.abs(out.cpu().numpy() - ref.cpu().numpy()).max()


def test_noalloc_rejects_oversized_grid_and_timing():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lib = tw.load()
    dev = torch.device("cuda:0")
    grid = tw.make_grid(2048, 2048, 0.05)
    occ_t = torch.zeros((8, 8), dtype=torch.uint8, device=dev)   # never touched: rejected on the host
    out = torch.zeros((8, 8), dtype=torch.float32, device=dev)
    rc, _ = _call_noalloc(lib, grid, occ_t, (5, 5), out, tw.Params(method=tw.HP_RBSOR))
    assert rc == tw.TW_EWORKSPACE
    rc, _ = _call_noalloc(lib, tw.make_grid(8, 8, 0.05), occ_t, (5, 5), out,
                          tw.Params(method=tw.HP_RBSOR, flags=tw.HP_TIMING))
    assert rc == tw.TW_EINVAL
