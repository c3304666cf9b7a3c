"""BF16 tensor-core network kernels of the learned warm start against the FP64 CPU oracle
(oracle/nn_oracle.py).  Inputs are rounded to bf16 once and the oracle gets the same rounded
values; the GPU accumulates in fp32, so fp32 outputs agree to ~1e-5 relative, bf16 outputs to bf16
rounding.  The whole encoder-decoder's parameter gradients are checked against the oracle composed
layer by layer."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2401_01672_gb300 import build
    build.build()
    from paper_2401_01672_gb300 import nn
    from oracle import nn_oracle as O
    nn._lib()
    return torch, nn, O


def bf(torch, a):
    """numpy -> bf16 device tensor, and the rounded values back as float64 numpy."""
    t = torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda().to(torch.bfloat16).contiguous()
    return t, t.float().cpu().numpy().astype(np.float64)


def relerr(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-30))


def no_failed_waits(nn):
    flag = nn.C.c_int(-1)
    st = nn._lib().pfnn_status(nn.C.byref(flag))
    assert st in (0, -7)
    return st == 0 and flag.value == 0


# grid shapes choose the three brick shapes of the tensor-core tiles (x extent 9 -> 8 x 8 x 2,
# 20 -> 16 x 8 x 1, 37 -> 32 x 4 x 1), each with ragged edges in every direction
SHAPES = [(2, 6, 5, 9), (1, 3, 9, 20), (1, 2, 5, 37)]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("cin,cout", [(16, 16), (16, 32), (32, 16), (64, 128), (128, 64), (48, 48), (32, 256)])
def test_conv_forward(env, cin, cout, shape):
    torch, nn, O = env
    L = nn._lib()
    g = np.random.default_rng(cin * 7 + cout)
    n, d, h, w = shape
    xt, x = bf(torch, g.standard_normal((n, d, h, w, cin)))
    wt, wv = bf(torch, g.standard_normal((27, cout, cin)) / math.sqrt(27 * cin))
    b = g.standard_normal(cout).astype(np.float32)
    bt = torch.from_numpy(b).cuda()
    y = torch.zeros((n * d * h * w, cout), dtype=torch.float32, device="cuda")
    st = L.pfnn_conv3d(nn._p(xt), cin, 0, nn._p(wt), cin, cout, nn._p(bt), 1, 0, None, nn._p(y), cout, 0, 0, n, d, h, w,
                       None)
    assert st == 0
    torch.cuda.synchronize()
    ref = O.conv3d(x, wv, b.astype(np.float64), relu=True).reshape(-1, cout)
    assert relerr(y.cpu().numpy(), ref) <= 2e-5
    yb = torch.zeros((n * d * h * w, cout), dtype=torch.bfloat16, device="cuda")
    assert L.pfnn_conv3d(nn._p(xt), cin, 0, nn._p(wt), cin, cout, nn._p(bt), 1, 0, nn._p(yb), None, cout, 0, 0, n, d, h,
                         w, None) == 0
    torch.cuda.synchronize()
    assert relerr(yb.float().cpu().numpy(), ref) <= 8e-3
    assert no_failed_waits(nn)


# narrow layers (16 or 32 channels in and out, grids at least 8 x 16 x 4) take the halo-tile kernel: one
# input tile per 8 x 16 x 4-or-8 brick, tap windows addressed in shared memory, one block per SM walking
# the bricks through two tile buffers and two accumulators; ragged in every direction, and one grid with
# several bricks per block (2 x 32 x 96 x 96: 576 or 1152 bricks on 152 blocks)
HALO_SHAPES = [(1, 5, 17, 12), (2, 8, 16, 8), (1, 9, 33, 21), (2, 32, 96, 96)]


@pytest.mark.parametrize("shape", HALO_SHAPES)
@pytest.mark.parametrize("cin,cout", [(16, 16), (16, 32), (32, 16), (32, 32)])
def test_conv_halo_tile_kernel(env, cin, cout, shape):
    """Forward (bias, ReLU, bf16 and fp32 outputs, channel slices of wider buffers) and backward data
    (flipped taps, transposed weights, accumulation into a non-zero fp32 gradient) against the oracle."""
    torch, nn, O = env
    L = nn._lib()
    g = np.random.default_rng(cin * 5 + cout + shape[2])
    n, d, h, w = shape
    big = g.standard_normal((n, d, h, w, cin + 16))                  # input slice [8, 8 + cin)
    bt, bv = bf(torch, big)
    x = bv[..., 8:8 + cin]
    wt, wv = bf(torch, g.standard_normal((27, cout, cin)) / math.sqrt(27 * cin))
    b = g.standard_normal(cout).astype(np.float32)
    btt = torch.from_numpy(b).cuda()
    ref = O.conv3d(x, wv, b.astype(np.float64), relu=True).reshape(-1, cout)
    yf = torch.full((n * d * h * w, cout + 24), 5.0, dtype=torch.float32, device="cuda")   # output slice [8, 8 + cout)
    assert L.pfnn_conv3d(nn._p(bt), cin + 16, 8, nn._p(wt), cin, cout, nn._p(btt), 1, 0, None, nn._p(yf), cout + 24, 8,
                         0, n, d, h, w, None) == 0
    yb = torch.zeros((n * d * h * w, cout), dtype=torch.bfloat16, device="cuda")
    assert L.pfnn_conv3d(nn._p(bt), cin + 16, 8, nn._p(wt), cin, cout, nn._p(btt), 1, 0, nn._p(yb), None, cout, 0, 0, n,
                         d, h, w, None) == 0
    torch.cuda.synchronize()
    o = yf.cpu().numpy()
    assert relerr(o[:, 8:8 + cout], ref) <= 2e-5
    assert np.all(o[:, :8] == 5.0) and np.all(o[:, 8 + cout:] == 5.0)
    assert relerr(yb.float().cpu().numpy(), ref) <= 8e-3
    # backward data into a gradient that already holds values
    dyt, dy = bf(torch, g.standard_normal((n, d, h, w, cout)))
    wtr = torch.empty((27, cin, cout), dtype=torch.bfloat16, device="cuda")
    assert L.pfnn_weight_transpose(nn._p(wt), nn._p(wtr), cout, cin, None) == 0
    base = g.standard_normal((n * d * h * w, cin)).astype(np.float32)
    dx = torch.from_numpy(base.copy()).cuda()
    assert L.pfnn_conv3d(nn._p(dyt), cout, 0, nn._p(wtr), cout, cin, None, 0, 1, None, nn._p(dx), cin, 0, 1, n, d, h, w,
                         None) == 0
    torch.cuda.synchronize()
    assert relerr(dx.cpu().numpy() - base, O.conv3d_bwd_data(dy, wv).reshape(-1, cin)) <= 2e-5
    assert no_failed_waits(nn)


def test_conv_halo_tile_gives_up_withheld_tile(env):
    """The halo-tile kernel's bounded waits: its tile loads withheld, the call stores nothing, pfnn_status
    reports PF_E_TIMEOUT once, and the next call is correct."""
    torch, nn, O = env
    L = nn._lib()
    g = np.random.default_rng(12)
    n, d, h, w, cin, cout = 1, 8, 16, 16, 16, 16
    xt, x = bf(torch, g.standard_normal((n, d, h, w, cin)))
    wt, wv = bf(torch, g.standard_normal((27, cout, cin)) / math.sqrt(27 * cin))
    y = torch.full((n * d * h * w, cout), 3.0, dtype=torch.float32, device="cuda")
    assert no_failed_waits(nn)
    assert L.pfnn_test_withhold_stage(0, 1 << 10) == 0
    assert L.pfnn_conv3d(nn._p(xt), cin, 0, nn._p(wt), cin, cout, None, 0, 0, None, nn._p(y), cout, 0, 0, n, d, h, w,
                         None) == 0
    torch.cuda.synchronize()
    flag = nn.C.c_int(0)
    assert L.pfnn_status(nn.C.byref(flag)) == -7 and flag.value == 1
    assert bool(torch.all(y == 3.0))
    assert no_failed_waits(nn)
    assert L.pfnn_conv3d(nn._p(xt), cin, 0, nn._p(wt), cin, cout, None, 0, 0, None, nn._p(y), cout, 0, 0, n, d, h, w,
                         None) == 0
    torch.cuda.synchronize()
    assert relerr(y.cpu().numpy(), O.conv3d(x, wv).reshape(-1, cout)) <= 2e-5
    assert no_failed_waits(nn)


def test_conv_rejects_unsupported(env):
    """Sizes the tensor-core tiles do not take are refused on the host, before any launch."""
    torch, nn, O = env
    L = nn._lib()
    x = torch.zeros((1, 4, 4, 8, 32), dtype=torch.bfloat16, device="cuda")
    w = torch.zeros((27, 8, 32), dtype=torch.bfloat16, device="cuda")
    y = torch.zeros((128, 16), dtype=torch.float32, device="cuda")
    assert L.pfnn_conv3d(nn._p(x), 32, 0, nn._p(w), 32, 8, None, 0, 0, None, nn._p(y), 16, 0, 0, 1, 4, 4, 8, None) == -1
    assert L.pfnn_conv3d(nn._p(x), 32, 0, nn._p(w), 32, 16, None, 0, 0, None, nn._p(y), 16, 4, 0, 1, 4, 4, 8, None) == -1
    assert L.pfnn_conv3d(nn._p(x), 32, 0, nn._p(w), 24, 16, None, 0, 0, None, nn._p(y), 16, 0, 0, 1, 4, 4, 8, None) == -1


@pytest.mark.parametrize("stage", [0, 5, 26])
def test_conv_gives_up_a_withheld_stage_and_recovers(env, stage):
    """Failure path of the bounded pipeline waits: with the loads of one stage withheld (a wait that
    nothing will complete; no bad access) and a short bound, the call finishes without storing,
    pfnn_status reports PF_E_TIMEOUT once, and the next normal call is correct."""
    torch, nn, O = env
    L = nn._lib()
    g = np.random.default_rng(11)
    n, d, h, w, cin, cout = 1, 4, 8, 32, 16, 32
    xt, x = bf(torch, g.standard_normal((n, d, h, w, cin)))
    wt, wv = bf(torch, g.standard_normal((27, cout, cin)) / math.sqrt(27 * cin))
    y = torch.full((n * d * h * w, cout), 3.0, dtype=torch.float32, device="cuda")
    assert no_failed_waits(nn)
    assert L.pfnn_test_withhold_stage(stage, 1 << 10) == 0
    assert L.pfnn_conv3d(nn._p(xt), cin, 0, nn._p(wt), cin, cout, None, 0, 0, None, nn._p(y), cout, 0, 0, n, d, h, w,
                         None) == 0
    torch.cuda.synchronize()
    flag = nn.C.c_int(0)
    assert L.pfnn_status(nn.C.byref(flag)) == -7 and flag.value == 1
    assert bool(torch.all(y == 3.0))          # nothing stored by the call that gave up
    assert no_failed_waits(nn)                # the flag was cleared
    assert L.pfnn_conv3d(nn._p(xt), cin, 0, nn._p(wt), cin, cout, None, 0, 0, None, nn._p(y), cout, 0, 0, n, d, h, w,
                         None) == 0
    torch.cuda.synchronize()
    assert relerr(y.cpu().numpy(), O.conv3d(x, wv).reshape(-1, cout)) <= 2e-5
    assert no_failed_waits(nn)
    assert L.pfnn_test_withhold_stage(-1, 10) == -1


def test_conv_channel_slices(env):
    """Input and output as channel slices of wider buffers (skip concatenation)."""
    torch, nn, O = env
    L = nn._lib()
    g = np.random.default_rng(3)
    n, d, h, w = 1, 4, 4, 8
    big = g.standard_normal((n, d, h, w, 48))
    bt, bv = bf(torch, big)
    wt, wv = bf(torch, g.standard_normal((27, 16, 32)) * 0.1)
    out = torch.full((n * d * h * w, 40), 7.0, dtype=torch.float32, device="cuda")
    assert L.pfnn_conv3d(nn._p(bt), 48, 16, nn._p(wt), 32, 16, None, 0, 0, None, nn._p(out), 40, 8, 0, n, d, h, w,
                         None) == 0
    torch.cuda.synchronize()
    ref = O.conv3d(bv[..., 16:48], wv).reshape(-1, 16)
    o = out.cpu().numpy()
    assert relerr(o[:, 8:24], ref) <= 2e-5
    assert np.all(o[:, :8] == 7.0) and np.all(o[:, 24:] == 7.0)
    assert no_failed_waits(nn)


@pytest.mark.parametrize("cin,cout", [(16, 16), (32, 64), (128, 64)])
def test_conv_backward_data_and_weight(env, cin, cout):
    torch, nn, O = env
    L = nn._lib()
    g = np.random.default_rng(11 + cin + cout)
    n, d, h, w = 2, 4, 6, 8
    xt, x = bf(torch, g.standard_normal((n, d, h, w, cin)))
    wtt, wv = bf(torch, g.standard_normal((27, cout, cin)) * 0.1)
    dyt, dy = bf(torch, g.standard_normal((n, d, h, w, cout)))
    # backward data: transposed weights, flipped taps
    wtr = torch.empty((27, cin, cout), dtype=torch.bfloat16, device="cuda")
    assert L.pfnn_weight_transpose(nn._p(wtt), nn._p(wtr), cout, cin, None) == 0
    dx = torch.zeros((n * d * h * w, cin), dtype=torch.float32, device="cuda")
    assert L.pfnn_conv3d(nn._p(dyt), cout, 0, nn._p(wtr), cout, cin, None, 0, 1, None, nn._p(dx), cin, 0, 1, n, d, h, w,
                         None) == 0
    dw = torch.zeros((27, cout, cin), dtype=torch.float32, device="cuda")
    wb = L.pfnn_conv3d_wgrad_work_bytes(cout, cin, n, d, h, w)
    work = torch.empty(wb, dtype=torch.uint8, device="cuda")
    assert L.pfnn_conv3d_wgrad(nn._p(dyt), cout, 0, cout, nn._p(xt), cin, 0, cin, nn._p(dw), n, d, h, w, nn._p(work),
                               wb, None) == 0
    torch.cuda.synchronize()
    assert relerr(dx.cpu().numpy(), O.conv3d_bwd_data(dy, wv).reshape(-1, cin)) <= 2e-5
    assert relerr(dw.cpu().numpy(), O.conv3d_bwd_weight(dy, x)) <= 2e-5
    assert no_failed_waits(nn)


@pytest.mark.parametrize("cin,cout,shape", [(16, 16, (1, 5, 3, 9)), (32, 32, (2, 4, 6, 8)), (64, 128, (1, 3, 7, 5)),
                                            (128, 64, (2, 2, 2, 2)), (16, 128, (1, 9, 4, 17)), (48, 16, (3, 3, 3, 3))])
def test_conv_weight_gradient_on_tensor_cores(env, cin, cout, shape):
    """Weight gradient (tcgen05 GEMM over packed, zero-padded voxels, rows = taps x output channels) against
    the FP64 oracle, element by element: ragged grids, channel slices of wider buffers, accumulation into
    a non-zero gradient, every tap tile (128 / cout taps per tile, the last one partial)."""
    torch, nn, O = env
    L = nn._lib()
    g = np.random.default_rng(cin * 3 + cout)
    n, d, h, w = shape
    xt, x = bf(torch, g.standard_normal((n, d, h, w, cin + 16)))      # input slice [8, 8 + cin)
    dyt, dy = bf(torch, g.standard_normal((n, d, h, w, cout + 32)))   # gradient slice [16, 16 + cout)
    base = g.standard_normal((27, cout, cin)).astype(np.float32)
    dw = torch.from_numpy(base.copy()).cuda()
    wb = L.pfnn_conv3d_wgrad_work_bytes(cout, cin, n, d, h, w)
    work = torch.full((wb,), 255, dtype=torch.uint8, device="cuda")   # stale scratch must not matter
    assert L.pfnn_conv3d_wgrad(nn._p(dyt), cout + 32, 16, cout, nn._p(xt), cin + 16, 8, cin, nn._p(dw), n, d, h, w,
                               nn._p(work), wb, None) == 0
    torch.cuda.synchronize()
    ref = O.conv3d_bwd_weight(dy[..., 16:16 + cout], x[..., 8:8 + cin])
    assert relerr(dw.cpu().numpy() - base, ref) <= 2e-5
    assert no_failed_waits(nn)
    # refused on the host: unsupported channel counts, a short scratch
    assert L.pfnn_conv3d_wgrad(nn._p(dyt), cout + 32, 16, 48, nn._p(xt), cin + 16, 8, cin, nn._p(dw), n, d, h, w,
                               nn._p(work), wb, None) == -1
    assert L.pfnn_conv3d_wgrad(nn._p(dyt), cout + 32, 16, cout, nn._p(xt), cin + 16, 8, cin, nn._p(dw), n, d, h, w,
                               nn._p(work), wb - 16, None) == -1


def test_pool_upsample_head(env):
    torch, nn, O = env
    L = nn._lib()
    g = np.random.default_rng(5)
    n, d, h, w, c = 2, 4, 6, 8, 16
    xt, x = bf(torch, g.standard_normal((n, d, h, w, c)))
    p = torch.zeros((n * d * h * w // 8, c), dtype=torch.bfloat16, device="cuda")
    assert L.pfnn_avgpool(nn._p(xt), c, 0, nn._p(p), c, 0, c, n, d, h, w, None) == 0
    u = torch.zeros((n * d * h * w, c), dtype=torch.bfloat16, device="cuda")
    assert L.pfnn_upsample(nn._p(p), c, nn._p(u), c, 0, n, d, h, w, None) == 0
    dyp = torch.from_numpy(g.standard_normal((n * d * h * w // 8, c)).astype(np.float32)).cuda()
    dx = torch.zeros((n * d * h * w, c), dtype=torch.float32, device="cuda")
    assert L.pfnn_avgpool_bwd(nn._p(dyp), c, nn._p(dx), c, 0, n, d, h, w, None) == 0
    dyu = torch.from_numpy(g.standard_normal((n * d * h * w, c)).astype(np.float32)).cuda()
    dp = torch.zeros((n * d * h * w // 8, c), dtype=torch.float32, device="cuda")
    assert L.pfnn_upsample_bwd(nn._p(dyu), c, 0, c, nn._p(dp), n, d // 2, h // 2, w // 2, None) == 0
    torch.cuda.synchronize()
    pr = O.avgpool(x)
    assert relerr(p.float().cpu().numpy(), pr.reshape(-1, c)) <= 8e-3
    assert np.array_equal(u.float().cpu().numpy(), O.upsample(p.float().cpu().numpy().reshape(n, d // 2, h // 2, w // 2, c)).reshape(-1, c))
    assert relerr(dx.cpu().numpy(), O.avgpool_bwd(dyp.cpu().numpy().astype(np.float64).reshape(n, d // 2, h // 2, w // 2, c)).reshape(-1, c)) <= 1e-6
    assert relerr(dp.cpu().numpy(), O.upsample_bwd(dyu.cpu().numpy().astype(np.float64).reshape(n, d, h, w, c)).reshape(-1, c)) <= 1e-6
    # head
    hw = g.standard_normal(c).astype(np.float32)
    tgt = g.uniform(0, 1, n * d * h * w).astype(np.float32)
    hwt, hb = torch.from_numpy(hw).cuda(), torch.tensor([0.2], dtype=torch.float32, device="cuda")
    prob = torch.zeros(n * d * h * w, device="cuda")
    dl = torch.zeros(n * d * h * w, device="cuda")
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    assert L.pfnn_head_forward(nn._p(xt), c, nn._p(hwt), nn._p(hb), nn._p(torch.from_numpy(tgt).cuda()), n * d * h * w,
                               nn._p(prob), nn._p(dl), nn._p(loss), None) == 0
    torch.cuda.synchronize()
    pr, lr, dlr = O.head(x.reshape(-1, c), hw.astype(np.float64), 0.2, tgt.astype(np.float64))
    assert relerr(prob.cpu().numpy(), pr) <= 1e-5
    assert abs(loss.item() - lr) <= 1e-5 * lr
    assert relerr(dl.cpu().numpy(), dlr) <= 1e-4


def bf16r(a):
    """Round to bfloat16 (nearest, ties to even) through binary32, as the kernels store activations."""
    x = np.asarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = ((x + 0x7FFF + ((x >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def oracle_unet_grads(nn, O, net, G, feat, target):
    """The same encoder-decoder in FP64 numpy oracle operations, with the network's BF16 storage points
    (input, weights, every stored activation, the ReLU-masked gradient fed to the weight and data
    products) rounded as the kernels round them; returns the loss and every parameter's gradient."""
    n = feat.shape[0]
    S = round((G.size // n) ** (1 / 3))
    inp = np.zeros((n, S, S, S, 16))
    inp[..., 0] = G.reshape(n, S, S, S)
    for f in range(feat.shape[1]):
        inp[..., 1 + f] = feat[:, f][:, None, None, None]
    inp = bf16r(inp)
    W = {}
    for k in net.names[:-1]:
        w, b = net.get_params(k)
        W[k] = (bf16r(w), b.astype(np.float64))
    act = {"in0": inp}
    cache = {}

    def conv(name, x):
        z = O.conv3d(x, W[name][0], W[name][1])
        y = bf16r(np.maximum(z, 0))
        cache[name] = (x, y)
        return y

    def pool(x):
        return bf16r(O.avgpool(x))

    a = act
    a["e1a"] = conv("e1a", a["in0"]); a["e1b"] = conv("e1b", a["e1a"])
    a["p1"] = pool(a["e1b"]); a["e2a"] = conv("e2a", a["p1"]); a["e2b"] = conv("e2b", a["e2a"])
    a["p2"] = pool(a["e2b"]); a["e3a"] = conv("e3a", a["p2"]); a["e3b"] = conv("e3b", a["e3a"])
    a["p3"] = pool(a["e3b"]); a["e4a"] = conv("e4a", a["p3"]); a["e4b"] = conv("e4b", a["e4a"])
    a["u3"] = conv("u3", O.upsample(a["e4b"])); c3 = np.concatenate([a["e3b"], a["u3"]], -1)
    a["d3a"] = conv("d3a", c3); a["d3b"] = conv("d3b", a["d3a"])
    a["u2"] = conv("u2", O.upsample(a["d3b"])); c2 = np.concatenate([a["e2b"], a["u2"]], -1)
    a["d2a"] = conv("d2a", c2); a["d2b"] = conv("d2b", a["d2a"])
    a["u1"] = conv("u1", O.upsample(a["d2b"])); c1 = np.concatenate([a["e1b"], a["u1"]], -1)
    a["d1a"] = conv("d1a", c1); a["d1b"] = conv("d1b", a["d1a"])
    hw, hb = net.get_params("head")
    hw = hw.astype(np.float64)
    prob, loss, dlog = O.head(a["d1b"].reshape(-1, 16), hw, float(hb[0]), target.astype(np.float64))
    grads = {"head": (a["d1b"].reshape(-1, 16).T @ dlog, np.array([np.sum(dlog)]))}
    gd = dlog[:, None] * hw[None, :]

    def back(name, gy):
        x, y = cache[name]
        dz = gy * (y > 0)
        dzb = bf16r(dz)
        grads[name] = (O.conv3d_bwd_weight(dzb, x), dz.sum(axis=(0, 1, 2, 3)))
        return O.conv3d_bwd_data(dzb, W[name][0])

    g = back("d1b", gd.reshape(a["d1b"].shape)); g = back("d1a", g)
    ge1b, gu1 = g[..., :16], g[..., 16:]
    g = O.upsample_bwd(back("u1", gu1))
    g = back("d2b", g); g = back("d2a", g)
    ge2b, gu2 = g[..., :32], g[..., 32:]
    g = O.upsample_bwd(back("u2", gu2))
    g = back("d3b", g); g = back("d3a", g)
    ge3b, gu3 = g[..., :64], g[..., 64:]
    g = O.upsample_bwd(back("u3", gu3))
    g = back("e4b", g); g = back("e4a", g)
    g = back("e3b", ge3b + O.avgpool_bwd(g)); g = back("e3a", g)
    g = back("e2b", ge2b + O.avgpool_bwd(g)); g = back("e2a", g)
    g = back("e1b", ge1b + O.avgpool_bwd(g)); back("e1a", g)
    return loss, prob, grads


# End to end (a hand-written oracle composition of the whole network): element-wise bar of every
# parameter gradient, relative to that tensor's largest entry.  The oracle rounds at the kernels' BF16
# storage points, but an activation whose BF16 rounding falls the other way (FP32 against FP64
# accumulation) changes everything downstream by a BF16 step, and 17 layers forward and back compound
# that to a few per cent at the first layers; a wrong channel, slice, tap or skip connection is an O(1)
# error.  The layer-by-layer test below checks each kernel's step element-wise at FP32 accuracy.
GRAD_BAR = 1e-1


def test_unet_gradients_against_oracle(env):
    """The library's network (pfnn_net, driven through the C ABI) against the oracle composition:
    loss, output probabilities and every parameter's weight and bias gradient, element by element."""
    torch, nn, O = env
    net = nn.UNet(seed=1)
    n, S = 1, 16
    rng = np.random.default_rng(9)
    G = rng.uniform(0, 1, n * S ** 3).astype(np.float32)
    feat = np.array([[0.3, -0.2]], dtype=np.float32)
    target = (rng.uniform(0, 1, n * S ** 3) > 0.5).astype(np.float32)
    prob = net.forward(torch.from_numpy(G).cuda(), torch.from_numpy(feat).cuda(), torch.from_numpy(target).cuda())
    net.backward()
    torch.cuda.synchronize()
    loss, ref_prob, grads = oracle_unet_grads(nn, O, net, G.astype(np.float64), feat.astype(np.float64), target)
    assert abs(net.loss_value() - loss) <= 1e-3 * loss
    assert relerr(prob.cpu().numpy(), ref_prob) <= 1e-2
    worst = {}
    for name in net.names:
        gw, gb = net.get_grads(name)
        rw, rb = grads[name]
        ew = relerr(gw.astype(np.float64).ravel(), np.asarray(rw).ravel())
        eb = relerr(gb.astype(np.float64).ravel(), np.asarray(rb).ravel())
        worst[name] = (ew, eb)
    print("\nend to end, per-parameter max|dg|/max|g| (weights, biases): " +
          ", ".join(f"{k} {v[0]:.1e}/{v[1]:.1e}" for k, v in worst.items()))
    for name, (ew, eb) in worst.items():
        assert ew <= GRAD_BAR and eb <= GRAD_BAR, (name, ew, eb)
    net.close()


def test_unet_layer_by_layer_against_oracle(env):
    """Every step of the library network's forward and backward, element by element, on the network's own
    buffers: each convolution's output from its input buffer (BF16 storage: equal up to one BF16 step where
    FP32 and FP64 accumulation round differently, on few elements), each pooling and upsampling, each
    parameter gradient from the layer's input and its ReLU-masked output gradient, and each activation
    gradient as the sum of the adjoints of its consumers (FP32 accumulation against FP64)."""
    torch, nn, O = env
    net = nn.UNet(seed=5)
    n, S = 1, 16
    rng = np.random.default_rng(13)
    G = rng.uniform(0, 1, n * S ** 3).astype(np.float32)
    feat = np.array([[0.5, 0.1]], dtype=np.float32)
    target = (rng.uniform(0, 1, n * S ** 3) > 0.5).astype(np.float32)
    prob = net.forward(torch.from_numpy(G).cuda(), torch.from_numpy(feat).cuda(), torch.from_numpy(target).cuda())
    net.backward()
    torch.cuda.synchronize()
    L = nn._lib()
    nb = L.pfnn_net_buffers()
    act, grad = zip(*[net.buffer(b) for b in range(nb)])
    ref_grad = [np.zeros_like(g) for g in grad]
    nconv = len(net.names) - 1
    report = {}
    for q in range(nconv):
        w = net.layer(q)
        name = net.names[q]
        W, bias = net.get_params(name)
        Wb = bf16r(W)
        x = act[w["src"]][..., w["soff"]:w["soff"] + w["cin"]]
        y = act[w["dst"]][..., w["doff"]:w["doff"] + w["cout"]]
        if w["pre"] == 1:
            src = act[w["pre_src"]][..., :w["pre_c"]]
            pooled = bf16r(O.avgpool(src))
            assert np.all(np.abs(act[w["pre_dst"]][..., :w["pre_c"]] - pooled) <= np.abs(pooled) * 2.0 ** -7), name
        elif w["pre"] == 2:
            assert np.array_equal(act[w["pre_dst"]][..., :w["pre_c"]], O.upsample(act[w["pre_src"]][..., :w["pre_c"]]))
        yr = bf16r(np.maximum(O.conv3d(x, Wb, bias.astype(np.float64)), 0))
        diff = np.abs(y - yr)
        # one BF16 step of the value, plus the FP32 accumulation's noise on sums that cancel to near zero
        step = np.abs(yr) * 2.0 ** -7 + np.max(np.abs(yr)) * 2.0 ** -14
        assert np.all(diff <= step), (name, float(np.max(diff / step)))
        frac = float(np.mean(diff > 0))
        assert frac <= 0.02, (name, frac)
        # backward of this layer from the network's own output gradient
        dz = grad[w["dst"]][..., w["doff"]:w["doff"] + w["cout"]] * (y > 0)
        dzb = bf16r(dz)
        gw, gb = net.get_grads(name)
        ew = relerr(gw.astype(np.float64), O.conv3d_bwd_weight(dzb, x))
        eb = relerr(gb.astype(np.float64), dz.sum(axis=(0, 1, 2, 3)))
        report[name] = (frac, ew, eb)
        assert ew <= 1e-4 and eb <= 1e-4, (name, ew, eb)
        if w["src"] != 0:
            ref_grad[w["src"]][..., w["soff"]:w["soff"] + w["cin"]] += O.conv3d_bwd_data(dzb, Wb)
        if w["pre"] == 1:
            ref_grad[w["pre_src"]][..., :w["pre_c"]] += O.avgpool_bwd(grad[w["pre_dst"]][..., :w["pre_c"]])
        elif w["pre"] == 2:
            ref_grad[w["pre_src"]][..., :w["pre_c"]] += O.upsample_bwd(grad[w["pre_dst"]][..., :w["pre_c"]])
    # the head's adjoint into the last buffer
    hw, _ = net.get_params("head")
    dlog = (prob.cpu().numpy().astype(np.float64) - target) / target.size
    last = net.layer(nconv - 1)["dst"]
    ref_grad[last] += (dlog[:, None] * hw.astype(np.float64)[None, :]).reshape(ref_grad[last].shape)
    for b in range(1, nb):
        e = relerr(grad[b], ref_grad[b])
        assert e <= 1e-4, (b, e)
    print("\nlayer by layer (BF16 steps differing, max|dgw|/max, max|dgb|/max): " +
          ", ".join(f"{k} {v[0]:.0e}/{v[1]:.0e}/{v[2]:.0e}" for k, v in report.items()))
    net.close()


def test_network_abi_trains_and_infers(env):
    """Training and inference through the network C ABI only: parameters set from the host, one forward
    with a target, backward, an Adam step that moves every parameter, inference into a caller buffer
    equal to the training forward's output on the same input."""
    torch, nn, O = env
    L = nn._lib()
    net = nn.UNet(seed=3)
    n, S = 2, 8
    rng = np.random.default_rng(5)
    G = torch.from_numpy(rng.uniform(0, 1, n * S ** 3).astype(np.float32)).cuda()
    feat = torch.from_numpy(rng.uniform(-1, 1, (n, 2)).astype(np.float32)).cuda()
    target = (G < 0.5).float().contiguous()
    before = {k: net.get_params(k) for k in net.names}
    p1 = net.forward(G, feat, target).clone()
    net.backward()
    net.adam_step(lr=1e-3)
    out = torch.empty(n * S ** 3, dtype=torch.float32, device="cuda")
    assert L.pfnn_net_infer(net.handle, nn._p(G), nn._p(feat), n, S, nn._p(out)) == 0
    torch.cuda.synchronize()
    for k in net.names:
        w0, b0 = before[k]
        w1, b1 = net.get_params(k)
        assert np.any(w1 != w0), k
    assert not torch.equal(out, p1)   # the step changed the network
    # with the parameters put back, inference reproduces the first forward exactly
    for k in net.names:
        net.set_params(k, *before[k])
    assert L.pfnn_net_infer(net.handle, nn._p(G), nn._p(feat), n, S, nn._p(out)) == 0
    torch.cuda.synchronize()
    assert torch.equal(out, p1)
    # backward without a forward that had a target is refused
    net2 = nn.UNet(seed=4)
    assert L.pfnn_net_backward(net2.handle) == -8
    net2.close()
    net.close()


def test_training_lowers_loss(env):
    """A few Adam steps of the kernels' own forward/backward on a fixed toy target (ice where the glass
    field is small) lower the cross-entropy."""
    torch, nn, O = env
    net = nn.UNet(seed=2)
    n, S = 2, 16
    rng = np.random.default_rng(4)
    G = torch.from_numpy(rng.uniform(0, 1, n * S ** 3).astype(np.float32)).cuda()
    feat = torch.zeros((n, 2), dtype=torch.float32, device="cuda")
    target = (G < 0.4).float().contiguous()
    losses = []
    for it in range(60):
        net.forward(G, feat, target)
        net.backward()
        net.adam_step(lr=3e-3)
        losses.append(net.loss_value())
    assert losses[-1] < 0.7 * losses[0]
    assert min(losses[-10:]) < min(losses[:10])
