"""FP64 CPU oracle of the learned warm start's network operations (numpy, plain definitions).

TEST INFRASTRUCTURE ONLY: the tests use it to check the GPU kernels' forward and backward results.
Layout as in the GPU code: activations (N, D, H, W, C), weights (27, Cout, Cin), tap
t = (dz+1)*9 + (dy+1)*3 + (dx+1), zero padding 1.  Each backward function is the adjoint (the
derivative) of its forward function; tests/test_nn_oracle_pins.py pins that by inner-product
identities and finite differences.
"""
import numpy as np

TAPS = [(t // 9 - 1, (t // 3) % 3 - 1, t % 3 - 1) for t in range(27)]


def _shifted(x, dz, dy, dx):
    """s[v] = x[v + (dz, dy, dx)] with zeros outside."""
    N, D, H, W, C = x.shape
    p = np.pad(x, ((0, 0), (1, 1), (1, 1), (1, 1), (0, 0)))
    return p[:, 1 + dz:1 + dz + D, 1 + dy:1 + dy + H, 1 + dx:1 + dx + W, :]


def conv3d(x, w, b=None, relu=False):
    """y[v][co] = b[co] + sum_t sum_ci x[v + off(t)][ci] w[t][co][ci], then max(0, .) if relu."""
    y = np.zeros(x.shape[:4] + (w.shape[1],))
    for t, (dz, dy, dx) in enumerate(TAPS):
        y += _shifted(x, dz, dy, dx) @ w[t].T
    if b is not None:
        y += b
    return np.maximum(y, 0.0) if relu else y


def conv3d_bwd_data(dy, w):
    """dx[v][ci] = sum_t sum_co dy[v - off(t)][co] w[t][co][ci]."""
    dx = np.zeros(dy.shape[:4] + (w.shape[2],))
    for t, (dz, ddy, ddx) in enumerate(TAPS):
        dx += _shifted(dy, -dz, -ddy, -ddx) @ w[t]
    return dx


def conv3d_bwd_weight(dy, x):
    """dw[t][co][ci] = sum_v dy[v][co] x[v + off(t)][ci]."""
    cout, cin = dy.shape[-1], x.shape[-1]
    dw = np.zeros((27, cout, cin))
    dyf = dy.reshape(-1, cout)
    for t, (dz, ddy, ddx) in enumerate(TAPS):
        dw[t] = dyf.T @ _shifted(x, dz, ddy, ddx).reshape(-1, cin)
    return dw


def avgpool(x):
    N, D, H, W, C = x.shape
    return x.reshape(N, D // 2, 2, H // 2, 2, W // 2, 2, C).mean(axis=(2, 4, 6))


def avgpool_bwd(dy):
    return np.repeat(np.repeat(np.repeat(dy, 2, 1), 2, 2), 2, 3) / 8.0


def upsample(x):
    return np.repeat(np.repeat(np.repeat(x, 2, 1), 2, 2), 2, 3)


def upsample_bwd(dy):
    N, D, H, W, C = dy.shape
    return dy.reshape(N, D // 2, 2, H // 2, 2, W // 2, 2, C).sum(axis=(2, 4, 6))


def head(x, w, b, target=None):
    """prob = sigmoid(x @ w + b); with a target: (prob, mean BCE, dlogit = (prob - target)/n)."""
    z = x @ w + b
    p = 1.0 / (1.0 + np.exp(-z))
    if target is None:
        return p
    pc = np.clip(p, 1e-7, 1 - 1e-7)
    loss = float(np.mean(-(target * np.log(pc) + (1 - target) * np.log(1 - pc))))
    return p, loss, (p - target) / p.size
