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
    assert L.pfnn_conv3d_wgrad(nn._p(dyt), cout, 0, cout, nn._p(xt), cin, 0, cin, nn._p(dw), n, d, h, w, None) == 0
    torch.cuda.synchronize()
    assert relerr(dx.cpu().numpy(), O.conv3d_bwd_data(dy, wv).reshape(-1, cin)) <= 2e-5
    assert relerr(dw.cpu().numpy(), O.conv3d_bwd_weight(dy, x)) <= 2e-5
    assert no_failed_waits(nn)


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


def oracle_unet_grads(nn, O, net, G, feat, target):
    """The same encoder-decoder in FP64 numpy oracle operations (bf16-rounded weights and input),
    returning the loss and every parameter's gradient."""
    n = feat.shape[0]
    S = round((G.size // n) ** (1 / 3))
    inp = np.zeros((n, S, S, S, 16))
    inp[..., 0] = G.reshape(n, S, S, S)
    for f in range(feat.shape[1]):
        inp[..., 1 + f] = feat[:, f][:, None, None, None]
    inp = net.torch.from_numpy(inp.astype(np.float32)).to(net.torch.bfloat16).float().numpy().astype(np.float64)
    W = {k: (P["wb"].float().cpu().numpy().astype(np.float64), P["b"].cpu().numpy().astype(np.float64))
         for k, P in net.params.items()}
    act = {"in0": inp}
    cache = {}

    def conv(name, x):
        z = O.conv3d(x, W[name][0], W[name][1])
        cache[name] = (x, z)
        return np.maximum(z, 0)

    a = act
    a["e1a"] = conv("e1a", a["in0"]); a["e1b"] = conv("e1b", a["e1a"])
    a["p1"] = O.avgpool(a["e1b"]); a["e2a"] = conv("e2a", a["p1"]); a["e2b"] = conv("e2b", a["e2a"])
    a["p2"] = O.avgpool(a["e2b"]); a["e3a"] = conv("e3a", a["p2"]); a["e3b"] = conv("e3b", a["e3a"])
    a["p3"] = O.avgpool(a["e3b"]); a["e4a"] = conv("e4a", a["p3"]); a["e4b"] = conv("e4b", a["e4a"])
    a["u3"] = conv("u3", O.upsample(a["e4b"])); c3 = np.concatenate([a["e3b"], a["u3"]], -1)
    a["d3a"] = conv("d3a", c3); a["d3b"] = conv("d3b", a["d3a"])
    a["u2"] = conv("u2", O.upsample(a["d3b"])); c2 = np.concatenate([a["e2b"], a["u2"]], -1)
    a["d2a"] = conv("d2a", c2); a["d2b"] = conv("d2b", a["d2a"])
    a["u1"] = conv("u1", O.upsample(a["d2b"])); c1 = np.concatenate([a["e1b"], a["u1"]], -1)
    a["d1a"] = conv("d1a", c1); a["d1b"] = conv("d1b", a["d1a"])
    hw = net.head["w"].cpu().numpy().astype(np.float64)
    hb = float(net.head["b"].cpu().numpy()[0])
    prob, loss, dlog = O.head(a["d1b"].reshape(-1, 16), hw, hb, target.astype(np.float64))
    grads = {"head_w": a["d1b"].reshape(-1, 16).T @ dlog, "head_b": np.sum(dlog)}
    gd = dlog[:, None] * hw[None, :]

    def back(name, gy):
        x, z = cache[name]
        dz = gy * (z > 0)
        grads[name] = (O.conv3d_bwd_weight(dz, x), dz.sum(axis=(0, 1, 2, 3)))
        return O.conv3d_bwd_data(dz, W[name][0])

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
    return loss, grads


def test_unet_gradients_against_oracle(env):
    torch, nn, O = env
    net = nn.UNet(seed=1)
    n, S = 1, 16
    rng = np.random.default_rng(9)
    G = rng.uniform(0, 1, n * S ** 3).astype(np.float32)
    feat = np.array([[0.3, -0.2]], dtype=np.float32)
    target = (rng.uniform(0, 1, n * S ** 3) > 0.5).astype(np.float32)
    net.forward(torch.from_numpy(G).cuda(), torch.from_numpy(feat).cuda(), torch.from_numpy(target).cuda())
    net.backward()
    torch.cuda.synchronize()
    loss, grads = oracle_unet_grads(nn, O, net, G.astype(np.float64), feat.astype(np.float64), target)
    assert abs(net.loss_value() - loss) <= 1e-2 * loss
    cos_min = 1.0
    for name in net.params:
        gw = net.params[name]["gw"].cpu().numpy().ravel().astype(np.float64)
        rw = grads[name][0].ravel()
        cos = gw @ rw / (np.linalg.norm(gw) * np.linalg.norm(rw) + 1e-300)
        cos_min = min(cos_min, cos)
        assert cos > 0.99, (name, cos)
        assert abs(np.linalg.norm(gw) / np.linalg.norm(rw) - 1) < 0.05, name
    hg = net.head["gw"].cpu().numpy().astype(np.float64)
    assert relerr(hg, grads["head_w"]) <= 2e-2


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
