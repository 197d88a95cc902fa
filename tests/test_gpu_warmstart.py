"""Learned warm start: the library's BF16 network kernels against the FP64
reference network (forward and gradients), training on fields the method
generates, and the gain the trained network gives the relaxation (fewer sweeps
to the same tolerance, with the final field still checked against the oracle)."""
import numpy as np
import pytest

import oracle
import paper_1903_07441_gb300 as tw
import scenes
from oracle import nn_oracle as nn

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1903_07441_gb300 import build
    build.build()
    return torch.device("cuda:0")


def _scene(seed, side):
    """Dynamic-style training scene: static shapes plus time-warped predicted disks."""
    sc = scenes.dynamic(seed=seed, side=side, n_obs=12, frames=1, static_shapes=10)
    occ, _, _ = oracle.build_grid(sc)
    if occ[sc.goal[1], sc.goal[0]] != 0:
        free = np.argwhere(occ == 0)
        j = int(np.argmin(np.hypot(free[:, 1] - sc.goal[0], free[:, 0] - sc.goal[1])))
        sc.goal = (int(free[j, 1]), int(free[j, 0]))
    return sc, occ


@pytest.mark.parametrize("cin,cout", [(32, 32), (32, 64), (64, 128), (128, 128), (128, 64), (64, 32), (16, 96)])
@pytest.mark.parametrize("H,W", [(16, 16), (24, 40), (48, 72)])
def test_conv3x3_tensor_core_matches_cuda_core_and_fp64(dev, cin, cout, H, W):
    """The BF16 tensor-core convolution (mma.sync implicit GEMM) and the CUDA-core
    direct convolution compute the same layer: against the FP64 convolution of the
    same BF16-rounded inputs and weights, both stay within BF16 output rounding
    (plus FP32 summation noise), and they differ from each other by at most one
    BF16 ulp -- ragged tiles in x and y, bias, skip and ReLU included."""
    g = torch.Generator(device="cpu").manual_seed(cin * 1000 + cout * 10 + H + W)
    x = (torch.randn((cin, H, W), generator=g)).to(torch.bfloat16).to(dev)
    w = (torch.randn((cout, cin, 3, 3), generator=g) / (3.0 * cin ** 0.5)).to(dev)
    b = (0.1 * torch.randn((cout,), generator=g)).to(dev)
    skip = torch.randn((cout, H, W), generator=g).to(torch.bfloat16).to(dev)
    outs = {}
    for impl in (tw.WS_CONV_SIMT, tw.WS_CONV_MMA, tw.WS_CONV_AUTO):
        outs[impl] = tw.ws_conv3x3(x, w, b, skip, relu=True, impl=impl).float().cpu().numpy()
    xr = x.float().cpu().numpy().astype(np.float64)
    wr = w.to(torch.bfloat16).float().cpu().numpy().astype(np.float64)
    ref = nn.conv(xr, wr, b.cpu().numpy().astype(np.float64)) + skip.float().cpu().numpy()
    ref = np.maximum(ref, 0.0)
    scale = np.abs(ref) + 1e-2
    for impl, y in outs.items():
        assert np.all(np.abs(y - ref) <= 2.0 ** -7 * scale), (impl, np.abs(y - ref).max())
    # one BF16 ulp apart, except where the FP32 sums cancel to near zero (and ReLU may cut either)
    both = np.maximum(np.abs(outs[tw.WS_CONV_SIMT]), np.abs(outs[tw.WS_CONV_MMA]))
    assert np.all(np.abs(outs[tw.WS_CONV_MMA] - outs[tw.WS_CONV_SIMT]) <= 2.0 ** -7 * (both + 1e-2))
    assert np.array_equal(outs[tw.WS_CONV_AUTO], outs[tw.WS_CONV_MMA])


@pytest.mark.parametrize("cin,cout,H,W,with_skip", [(16, 32, 4, 128, False), (32, 32, 8, 256, True),
                                                    (64, 64, 12, 128, True), (128, 128, 4, 384, True),
                                                    (64, 128, 10, 128, False), (128, 64, 4, 256, True),
                                                    (32, 128, 6, 128, True), (128, 32, 8, 128, False),
                                                    (64, 128, 8, 64, True), (128, 128, 16, 32, True),
                                                    (128, 64, 16, 16, False), (32, 32, 12, 64, True),
                                                    (64, 32, 8, 32, True), (16, 128, 4, 64, False),
                                                    (128, 128, 64, 64, True)])
def test_conv3x3_tensor_memory_matches_cuda_core_and_fp64(dev, cin, cout, H, W, with_skip):
    """The tcgen05 implicit GEMM (accumulators in tensor memory, operands staged channel-last in shared
    memory) computes the same layer as the CUDA-core direct convolution: within BF16 output rounding of
    the FP64 convolution of the same BF16 inputs and weights, at most one BF16 ulp from the CUDA-core
    result, every edge pixel (zero padding) and every channel block included; its bounded waits never
    gave up.  Widths below 128 take the narrow form (M blocks spanning 128 / W rows, x taps as shifted
    copies, split K over the channel chunks with a fixed-order finalisation)."""
    g = torch.Generator(device="cpu").manual_seed(cin * 977 + cout * 13 + H * 7 + W)
    x = (torch.randn((cin, H, W), generator=g)).to(torch.bfloat16).to(dev)
    w = (torch.randn((cout, cin, 3, 3), generator=g) / (3.0 * cin ** 0.5)).to(dev)
    b = (0.1 * torch.randn((cout,), generator=g)).to(dev)
    skip = torch.randn((cout, H, W), generator=g).to(torch.bfloat16).to(dev) if with_skip else None
    tc_out = tw.ws_conv3x3(x, w, b, skip, relu=with_skip, impl=tw.WS_CONV_TC).float().cpu().numpy()
    simt = tw.ws_conv3x3(x, w, b, skip, relu=with_skip, impl=tw.WS_CONV_SIMT).float().cpu().numpy()
    torch.cuda.synchronize()
    assert not tw.ws_conv_check()
    xr = x.float().cpu().numpy().astype(np.float64)
    wr = w.to(torch.bfloat16).float().cpu().numpy().astype(np.float64)
    ref = nn.conv(xr, wr, b.cpu().numpy().astype(np.float64))
    if with_skip:
        ref = np.maximum(ref + skip.float().cpu().numpy(), 0.0)
    scale = np.abs(ref) + 1e-2
    assert np.all(np.abs(tc_out - ref) <= 2.0 ** -7 * scale), np.abs(tc_out - ref).max()
    both = np.maximum(np.abs(tc_out), np.abs(simt))
    assert np.all(np.abs(tc_out - simt) <= 2.0 ** -7 * (both + 1e-2))


@pytest.mark.parametrize("cin,cout,H,W", [(32, 32, 8, 256), (32, 64, 10, 128), (64, 64, 12, 48), (64, 128, 6, 64),
                                          (128, 128, 9, 128), (128, 64, 5, 80), (64, 32, 16, 256), (128, 32, 7, 32),
                                          (32, 128, 4, 16), (128, 128, 64, 64), (2, 32, 16, 256),
                                          (32, 1, 16, 256), (16, 96, 6, 48), (128, 48, 5, 32)])
def test_conv3x3_weight_gradient_tensor_memory_matches_fp64(dev, cin, cout, H, W):
    """The tcgen05 weight gradient (per tap a GEMM over the pixels, X staged three times shifted by one
    pixel, accumulators in tensor memory, channel counts other than 32, 64 and 128 padded, pixel chunks
    summed in a fixed order) and the CUDA-core one
    against the FP64 gradient of the same BF16 inputs: every weight and bias within 2^-12 of the sum of
    the absolute products it adds (FP32 accumulation; one pixel more or less moves a weight by about
    1 / (H W) of that sum, so a dropped, repeated or misplaced pixel, tap or channel fails), ragged
    chunks, image rows shorter than a stage, and every edge (zero padding) included.  Repeated calls
    give identical bits, the automatic choice is the tensor-memory form, and no bounded wait gave up."""
    g = torch.Generator(device="cpu").manual_seed(cin * 31 + cout * 7 + H * 5 + W)
    x = torch.randn((cin, H, W), generator=g).to(torch.bfloat16).to(dev)
    dy = torch.randn((cout, H, W), generator=g).to(torch.bfloat16).to(dev)
    tc = tw.ws_conv3x3_wgrad(x, dy, impl=tw.WS_CONV_TC)
    tc2 = tw.ws_conv3x3_wgrad(x, dy, impl=tw.WS_CONV_TC)
    auto = tw.ws_conv3x3_wgrad(x, dy, impl=tw.WS_CONV_AUTO)
    simt = tw.ws_conv3x3_wgrad(x, dy, impl=tw.WS_CONV_SIMT)
    torch.cuda.synchronize()
    assert not tw.ws_conv_check()
    xr = x.float().cpu().numpy().astype(np.float64)
    dyr = dy.float().cpu().numpy().astype(np.float64)
    w0 = np.zeros((cout, cin, 3, 3))
    _, ref_w, ref_b = nn.conv_bwd(xr, w0, dyr)
    _, abs_w, abs_b = nn.conv_bwd(np.abs(xr), w0, np.abs(dyr))
    for name, (dw, db) in (("tc", tc), ("simt", simt)):
        dw = dw.cpu().numpy()
        db = db.cpu().numpy()
        assert np.all(np.abs(dw - ref_w) <= 2.0 ** -12 * abs_w + 1e-30), (name, np.abs(dw - ref_w).max())
        assert np.all(np.abs(db - ref_b) <= 2.0 ** -12 * abs_b + 1e-30), (name, np.abs(db - ref_b).max())
    for a, b in zip(tc, tc2):
        assert torch.equal(a, b)
    for a, b in zip(tc, auto):
        assert torch.equal(a, b)


def test_conv3x3_weight_gradient_adds_to_what_it_is_given(dev):
    """dW and db are accumulated into, as the network's backward pass needs for a sum of layers."""
    g = torch.Generator(device="cpu").manual_seed(77)
    x = torch.randn((64, 8, 64), generator=g).to(torch.bfloat16).to(dev)
    dy = torch.randn((32, 8, 64), generator=g).to(torch.bfloat16).to(dev)
    dw, db = tw.ws_conv3x3_wgrad(x, dy, impl=tw.WS_CONV_TC)
    lib = tw.load()
    dw2 = torch.full_like(dw, 0.5)
    db2 = torch.full_like(db, -0.25)
    nws = lib.ws_conv3x3_wgrad_workspace_size(64, 32, 8, 64, tw.WS_CONV_TC)
    ws = torch.empty(nws, dtype=torch.uint8, device=dev)
    assert lib.ws_conv3x3_wgrad(x.data_ptr(), dy.data_ptr(), dw2.data_ptr(), db2.data_ptr(), 64, 32, 8, 64,
                                tw.WS_CONV_TC, ws.data_ptr(), nws, None) == tw.TW_OK
    torch.cuda.synchronize()
    assert torch.allclose(dw2, dw + 0.5, rtol=0, atol=1e-6 * float(dw.abs().max()) + 1e-6)
    assert torch.allclose(db2, db - 0.25, rtol=0, atol=1e-6 * float(db.abs().max()) + 1e-6)


def test_conv3x3_rejects_tensor_core_shapes_it_cannot_take(dev):
    x = torch.zeros((8, 16, 16), dtype=torch.bfloat16, device=dev)
    w = torch.zeros((32, 8, 3, 3), dtype=torch.float32, device=dev)
    with pytest.raises(tw.TwError) as e:
        tw.ws_conv3x3(x, w, impl=tw.WS_CONV_MMA)
    assert e.value.status == tw.TW_EINVAL
    # the automatic choice falls back to the CUDA-core kernel
    assert tw.ws_conv3x3(x, w, impl=tw.WS_CONV_AUTO).shape == (32, 16, 16)


# Bounds from the BF16 storage of activations and gradients (relative precision 2^-9 per rounding,
# about 30 roundings deep): measured on GB300 the forward differs by 1.8 % (32^2) and 3.5 % (128^2,
# where the level-0 layers run on the tensor-memory kernel) of its range, the layer gradients by at
# most 6.4 % and 11.3 % in norm, with cosine similarity 0.9994 and 0.9996.
@pytest.mark.parametrize("side,seed,fwd_tol,layer_tol", [(32, 9100, 0.03, 0.08), (128, 9101, 0.05, 0.15)])
def test_forward_and_gradients_match_fp64_reference(dev, side, seed, fwd_tol, layer_tol):
    net = tw.WarmStartNet(dev, seed=7)
    sc, occ = _scene(seed, side)
    occ_t = torch.from_numpy(occ).to(dev)
    p = net.params.cpu().numpy().astype(np.float64)
    rng = np.random.default_rng(1)
    _, pred = net.forward(occ_t, sc.goal)
    ref, _ = nn.forward(p, occ, sc.goal)
    g = pred.cpu().numpy()
    scale = np.abs(ref).max()
    assert scale > 0
    assert np.abs(g - ref).max() <= fwd_tol * scale + 1e-3
    target = (rng.standard_normal(occ.shape) * 0.1 - 0.3).astype(np.float32)
    tt = torch.from_numpy(target).to(dev)
    loss, grads = net.gradients(occ_t, sc.goal, tt)
    grads = grads.clone()   # the network keeps one gradient buffer
    loss2, grads2 = net.gradients(occ_t, sc.goal, tt)
    # fixed-order reductions everywhere (no floating-point atomics): the same bits twice
    assert loss == loss2 and torch.equal(grads, grads2)
    loss_ref, g_ref = nn.loss_and_grads(p, occ, sc.goal, target.astype(np.float64))
    assert abs(loss - loss_ref) <= 0.04 * loss_ref
    gg = grads.cpu().numpy().astype(np.float64)
    cos = gg @ g_ref / (np.linalg.norm(gg) * np.linalg.norm(g_ref))
    assert cos >= 0.998, cos
    o = 0
    for ci, co in nn.LAYERS:
        k = co * ci * 9 + co
        a, b = gg[o:o + k], g_ref[o:o + k]
        assert np.linalg.norm(a - b) <= layer_tol * np.linalg.norm(b) + 1e-6, (ci, co)
        o += k
    assert not tw.ws_conv_check()


def _fields(dev, seeds, side):
    out = []
    for s in seeds:
        sc, occ = _scene(s, side)
        occ_t = torch.from_numpy(occ).to(dev)
        grid = tw.make_grid(side, side, sc.cell)
        u, st = tw.hp_relax(grid, occ_t, sc.goal, params=tw.Params(omega=1.0, tol=0.0, max_sweeps=6000))
        out.append((sc, occ, occ_t, u))
    return out


def test_training_reduces_loss_and_warm_start_saves_sweeps(dev):
    side = 128
    train = _fields(dev, range(9200, 9240), side)
    net = tw.WarmStartNet(dev, seed=3)
    targets = [net.target(u) for _, _, _, u in train]
    first = np.mean([net.gradients(o, sc.goal, t)[0] for (sc, _, o, _), t in zip(train[:8], targets[:8])])
    for it in range(800):
        i = it % len(train)
        sc, _, o, _ = train[i]
        net.train_step(o, sc.goal, targets[i], lr=1e-3 if it < 600 else 3e-4)
    last = np.mean([net.gradients(o, sc.goal, t)[0] for (sc, _, o, _), t in zip(train[:8], targets[:8])])
    assert last < 0.2 * first, (first, last)
    # held-out scenes: sweeps to 1e-6 from the network's field vs the cold start
    cold, warm, coarse = [], [], []
    for sc, occ, occ_t, _ in _fields(dev, range(9300, 9306), side):
        grid = tw.make_grid(side, side, sc.cell)
        _, s0 = tw.hp_relax(grid, occ_t, sc.goal, params=tw.Params(tol=1e-6))
        u0, _ = net.forward(occ_t, sc.goal)
        u0_h = u0.cpu().numpy()   # hp_relax overwrites its field argument
        u1, s1 = tw.hp_relax(grid, occ_t, sc.goal, field=u0, params=tw.Params(tol=1e-6, flags=tw.HP_WARM_START))
        assert s1["status"] == tw.TW_OK
        ustar, fixed = oracle.solve_field(occ, sc.goal, tol=1e-13)
        tau = oracle.exit_time(fixed).max()
        assert np.abs(u1.cpu().numpy() - ustar).max() <= tau * s1["resid_inf"] * 1.001 + 1e-7
        cold.append(s0["sweeps"])
        warm.append(s1["sweeps"])
        # the warm start at stride 1 is the forward pass's own u; at stride 2 (the network on a
        # max-pooled 64 x 64 grid, its prediction interpolated back) it is a valid start too
        assert np.array_equal(net.warm_start(occ_t, sc.goal, 1).cpu().numpy(), u0_h)
        u2 = net.warm_start(occ_t, sc.goal, 2)
        h = u2.cpu().numpy()
        assert np.all((h >= 0.0) & (h <= 1.0)) and np.all(h[occ != 0] == 0.0) and h[sc.goal[1], sc.goal[0]] == 1.0
        _, s2 = tw.hp_relax(grid, occ_t, sc.goal, field=u2, params=tw.Params(tol=1e-6, flags=tw.HP_WARM_START))
        assert s2["status"] == tw.TW_OK
        coarse.append(s2["sweeps"])
    assert np.mean(warm) < np.mean(cold), (cold, warm)
    assert np.mean(coarse) < np.mean(cold), (cold, coarse)
