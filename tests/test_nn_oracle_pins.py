"""Pins of the network-operation oracle: every backward function is the adjoint of its forward
function (inner-product identities hold to rounding) and matches central finite differences; an
identity kernel reproduces its input and a one-tap kernel is a shift."""
import numpy as np

from oracle import nn_oracle as N


def rs(seed):
    return np.random.default_rng(seed)


def test_identity_and_shift_kernels():
    x = rs(0).standard_normal((1, 4, 5, 6, 3))
    w = np.zeros((27, 3, 3))
    w[13] = np.eye(3)                       # centre tap
    assert np.allclose(N.conv3d(x, w), x)
    w = np.zeros((27, 3, 3))
    w[14] = np.eye(3)                       # tap (0, 0, +1): y[v] = x[v + e_x]
    y = N.conv3d(x, w)
    assert np.allclose(y[..., :-1, :], x[..., 1:, :]) and np.allclose(y[..., -1, :], 0)


def test_conv_adjoint_identities():
    g = rs(1)
    x = g.standard_normal((2, 4, 5, 3, 4))
    w = g.standard_normal((27, 5, 4))
    dy = g.standard_normal((2, 4, 5, 3, 5))
    # <conv(x), dy> = <x, conv_bwd_data(dy)>  and  = <w, conv_bwd_weight(dy, x)>
    lhs = np.sum(N.conv3d(x, w) * dy)
    assert abs(lhs - np.sum(x * N.conv3d_bwd_data(dy, w))) <= 1e-10 * abs(lhs)
    assert abs(lhs - np.sum(w * N.conv3d_bwd_weight(dy, x))) <= 1e-10 * abs(lhs)


def test_pool_upsample_adjoints():
    g = rs(2)
    x = g.standard_normal((1, 4, 6, 2, 3))
    dy = g.standard_normal((1, 2, 3, 1, 3))
    assert abs(np.sum(N.avgpool(x) * dy) - np.sum(x * N.avgpool_bwd(dy))) < 1e-12
    u = g.standard_normal((1, 2, 3, 1, 3))
    du = g.standard_normal((1, 4, 6, 2, 3))
    assert abs(np.sum(N.upsample(u) * du) - np.sum(u * N.upsample_bwd(du))) < 1e-12


def test_head_gradient_finite_difference():
    g = rs(3)
    x = g.standard_normal((50, 4))
    w = g.standard_normal(4)
    t = g.uniform(0, 1, 50)
    p, loss, dl = N.head(x, w, 0.3, t)
    # d loss / d w = x^T dlogit, checked by central differences
    gw = x.T @ dl
    for i in range(4):
        e = np.zeros(4)
        e[i] = 1e-6
        fd = (N.head(x, w + e, 0.3, t)[1] - N.head(x, w - e, 0.3, t)[1]) / 2e-6
        assert abs(fd - gw[i]) < 1e-7


def test_conv_relu_chain_finite_difference():
    g = rs(4)
    x = g.standard_normal((1, 3, 3, 3, 2))
    w = g.standard_normal((27, 2, 2)) * 0.3
    b = g.standard_normal(2) * 0.1
    dy = g.standard_normal((1, 3, 3, 3, 2))
    f = lambda ww: np.sum(N.conv3d(x, ww, b, relu=True) * dy)
    z = N.conv3d(x, w, b)
    dz = dy * (z > 0)
    gw = N.conv3d_bwd_weight(dz, x)
    for idx in [(0, 0, 0), (13, 1, 0), (26, 1, 1), (5, 0, 1)]:
        e = np.zeros_like(w)
        e[idx] = 1e-6
        fd = (f(w + e) - f(w - e)) / 2e-6
        assert abs(fd - gw[idx]) < 1e-6
