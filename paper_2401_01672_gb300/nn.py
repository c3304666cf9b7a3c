"""Learned warm start: a 3D convolutional encoder-decoder that predicts the micro-scale equilibrium
phase field from the glass field, the supercooling and the surface-tension scale.

Every forward, backward and optimiser operation runs in the library's CUDA kernels (include/pfnn.h):
BF16 tensor-core 3x3x3 convolutions with FP32 accumulation, pooling/upsampling, the sigmoid head
with binary cross-entropy, Adam on FP32 master weights.  torch only allocates the device buffers.

Architecture (4 levels, channels 16/32/64/128, two 3x3x3 convolutions + ReLU per level, 2x2x2
average-pool down, x2 nearest up + 3x3x3 convolution, skip concatenation, 1x1x1 sigmoid head):

  in(16) -> e1a(16) -> e1b(16)=cat1[0:16] -> pool -> e2a(32) -> e2b(32)=cat2[0:32] -> pool
         -> e3a(64) -> e3b(64)=cat3[0:64] -> pool -> e4a(128) -> e4b(128)
         -> up -> u3(64)=cat3[64:128] -> d3a(64) -> d3b(64) -> up -> u2(32)=cat2[32:64] -> d2a(32) -> d2b(32)
         -> up -> u1(16)=cat1[16:32] -> d1a(16) -> d1b(16) -> head(1) -> sigmoid
"""
from __future__ import annotations

import ctypes as C
import math

import numpy as np

from . import pf as _pf

# (name, input buffer, input channel offset, cin, output buffer, output offset, cout, level)
LAYERS = [
    ("e1a", "in0", 0, 16, "e1a", 0, 16, 0),
    ("e1b", "e1a", 0, 16, "cat1", 0, 16, 0),
    ("e2a", "p1", 0, 16, "e2a", 0, 32, 1),
    ("e2b", "e2a", 0, 32, "cat2", 0, 32, 1),
    ("e3a", "p2", 0, 32, "e3a", 0, 64, 2),
    ("e3b", "e3a", 0, 64, "cat3", 0, 64, 2),
    ("e4a", "p3", 0, 64, "e4a", 0, 128, 3),
    ("e4b", "e4a", 0, 128, "e4b", 0, 128, 3),
    ("u3", "up3", 0, 128, "cat3", 64, 64, 2),
    ("d3a", "cat3", 0, 128, "d3a", 0, 64, 2),
    ("d3b", "d3a", 0, 64, "d3b", 0, 64, 2),
    ("u2", "up2", 0, 64, "cat2", 32, 32, 1),
    ("d2a", "cat2", 0, 64, "d2a", 0, 32, 1),
    ("d2b", "d2a", 0, 32, "d2b", 0, 32, 1),
    ("u1", "up1", 0, 32, "cat1", 16, 16, 0),
    ("d1a", "cat1", 0, 32, "d1a", 0, 16, 0),
    ("d1b", "d1a", 0, 16, "d1b", 0, 16, 0),
]
# buffer channels and level
BUFFERS = {"in0": (16, 0), "e1a": (16, 0), "cat1": (32, 0), "p1": (16, 1), "e2a": (32, 1), "cat2": (64, 1),
           "p2": (32, 2), "e3a": (64, 2), "cat3": (128, 2), "p3": (64, 3), "e4a": (128, 3), "e4b": (128, 3),
           "up3": (128, 2), "d3a": (64, 2), "d3b": (64, 2), "up2": (64, 1), "d2a": (32, 1), "d2b": (32, 1),
           "up1": (32, 0), "d1a": (16, 0), "d1b": (16, 0)}
N_FEATURES = 2

_nn = None


def _lib():
    global _nn
    if _nn is None:
        lib = _pf.load_library()
        vp, i, ll, f, d = C.c_void_p, C.c_int, C.c_longlong, C.c_float, C.c_double
        sig = {
            "pfnn_conv3d": [vp, i, i, vp, i, i, vp, i, i, vp, vp, i, i, i, i, i, i, i, vp],
            "pfnn_conv3d_wgrad": [vp, i, i, i, vp, i, i, i, vp, i, i, i, i, vp],
            "pfnn_bias_grad": [vp, i, i, i, ll, vp, vp],
            "pfnn_relu_bwd_cast": [vp, i, i, vp, i, i, i, ll, vp, vp, vp],
            "pfnn_weight_transpose": [vp, vp, i, i, vp],
            "pfnn_avgpool": [vp, i, i, vp, i, i, i, i, i, i, i, vp],
            "pfnn_avgpool_bwd": [vp, i, vp, i, i, i, i, i, i, vp],
            "pfnn_upsample": [vp, i, vp, i, i, i, i, i, i, vp],
            "pfnn_upsample_bwd": [vp, i, i, i, vp, i, i, i, i, vp],
            "pfnn_head_forward": [vp, i, vp, vp, vp, ll, vp, vp, vp, vp],
            "pfnn_head_backward": [vp, i, vp, vp, ll, vp, vp, vp, vp],
            "pfnn_pack_input": [vp, vp, i, ll, ll, vp, vp],
            "pfnn_adam": [vp, vp, vp, vp, vp, ll, f, f, f, f, i, vp],
            "pfnn_status": [C.POINTER(i)],
            "pfnn_test_withhold_stage": [i, ll],
        }
        for name, args in sig.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = C.c_int
        _nn = lib
    return _nn


def _ck(st, what):
    if st != 0:
        raise _pf.PfError(st, what)


def _p(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def check_device():
    """Raise if a tensor-core convolution gave up a pipeline wait since the last check (synchronous)."""
    flag = C.c_int(0)
    st = _lib().pfnn_status(C.byref(flag))
    if st == _pf.PF_E_TIMEOUT or flag.value:
        raise _pf.PfError(_pf.PF_E_TIMEOUT, "a tensor-core convolution gave up waiting for its pipeline; outputs are invalid")
    _ck(st, "status")


class UNet:
    """Parameters (FP32 master + BF16 working copies), gradients, Adam moments, and the kernels' calls."""

    def __init__(self, seed=0, device="cuda"):
        import torch
        self.torch = torch
        self.dev = device
        g = np.random.default_rng(seed)
        self.params = {}
        for (name, _, _, cin, _, _, cout, _) in LAYERS:
            std = math.sqrt(2.0 / (27 * cin))      # He initialisation for ReLU layers
            w = torch.from_numpy((g.standard_normal((27, cout, cin)) * std).astype(np.float32)).to(device)
            self.params[name] = self._param(w, torch.zeros(cout, device=device))
        hw = torch.from_numpy((g.standard_normal(16) * math.sqrt(1.0 / 16)).astype(np.float32)).to(device)
        self.head = self._param(hw, torch.zeros(1, device=device))
        self.step_count = 0
        self.stream = torch.cuda.current_stream().cuda_stream

    def _param(self, w, b):
        t = self.torch
        return {"w": w.contiguous(), "b": b.contiguous(), "wb": w.to(t.bfloat16).contiguous(),
                "wt": t.empty((w.shape[0], w.shape[2], w.shape[1]) if w.dim() == 3 else w.shape, dtype=t.bfloat16,
                              device=self.dev) if w.dim() == 3 else None,
                "gw": t.zeros_like(w), "gb": t.zeros_like(b), "mw": t.zeros_like(w), "vw": t.zeros_like(w),
                "mb": t.zeros_like(b), "vb": t.zeros_like(b)}

    # ---------------------------------------------------------------- buffers
    def _buffers(self, n, S):
        t = self.torch
        key = (n, S)
        if getattr(self, "_bkey", None) == key:
            return
        self._bkey = key
        self.n, self.S = n, S
        self.act, self.grad = {}, {}
        for name, (c, lev) in BUFFERS.items():
            s = S >> lev
            self.act[name] = t.zeros((n * s ** 3, c), dtype=t.bfloat16, device=self.dev)
            self.grad[name] = t.zeros((n * s ** 3, c), dtype=t.float32, device=self.dev)
        nmax = n * S ** 3 * 128
        self.dz_f = t.empty(nmax, dtype=t.float32, device=self.dev)
        self.dz_b = t.empty(nmax, dtype=t.bfloat16, device=self.dev)
        self.logit_grad = t.empty(n * S ** 3, dtype=t.float32, device=self.dev)
        self.prob = t.empty(n * S ** 3, dtype=t.float32, device=self.dev)
        self.loss = t.zeros(1, dtype=t.float64, device=self.dev)

    def _dims(self, lev):
        s = self.S >> lev
        return self.n, s, s, s

    # ---------------------------------------------------------------- forward
    def forward(self, G, feat, target=None):
        """G: fp32 (n * S^3,) glass field; feat: fp32 (n, N_FEATURES); returns probabilities (n * S^3,)."""
        t = self.torch
        n = feat.shape[0]
        S = round((G.numel() // n) ** (1 / 3))
        assert n * S ** 3 == G.numel() and S % 8 == 0, "grid side must be a multiple of 8"
        self._buffers(n, S)
        L = _lib()
        st = self.stream
        _ck(L.pfnn_pack_input(_p(G), _p(feat), N_FEATURES, S ** 3, n * S ** 3, _p(self.act["in0"]), st), "pack")
        A = self.act
        for (name, src, soff, cin, dst, doff, cout, lev) in LAYERS:
            if name == "e2a":
                self._pool("cat1", 0, 16, "p1", 0)
            elif name == "e3a":
                self._pool("cat2", 1, 32, "p2", 0)
            elif name == "e4a":
                self._pool("cat3", 2, 64, "p3", 0)
            elif name == "u3":
                _ck(L.pfnn_upsample(_p(A["e4b"]), 128, _p(A["up3"]), 128, 0, *self._dims(2), st), "up")
            elif name == "u2":
                _ck(L.pfnn_upsample(_p(A["d3b"]), 64, _p(A["up2"]), 64, 0, *self._dims(1), st), "up")
            elif name == "u1":
                _ck(L.pfnn_upsample(_p(A["d2b"]), 32, _p(A["up1"]), 32, 0, *self._dims(0), st), "up")
            P = self.params[name]
            ldx, ldy = BUFFERS[src][0], BUFFERS[dst][0]
            _ck(L.pfnn_conv3d(_p(A[src]), ldx, soff, _p(P["wb"]), cin, cout, _p(P["b"]), 1, 0, _p(A[dst]), None, ldy,
                              doff, 0, *self._dims(lev), st), name)
        self.loss.zero_()
        _ck(L.pfnn_head_forward(_p(A["d1b"]), 16, _p(self.head["w"]), _p(self.head["b"]), _p(target), n * S ** 3,
                                _p(self.prob), _p(self.logit_grad) if target is not None else None,
                                _p(self.loss) if target is not None else None, st), "head")
        return self.prob

    def _pool(self, src, lev, c, dst, doff):
        _ck(_lib().pfnn_avgpool(_p(self.act[src]), BUFFERS[src][0], 0, _p(self.act[dst]), BUFFERS[dst][0], doff, c,
                                *self._dims(lev), self.stream), "pool")

    # ---------------------------------------------------------------- backward
    def backward(self):
        """Gradients of the mean BCE of the last forward (with a target) into every parameter."""
        L = _lib()
        st = self.stream
        A, Gr = self.act, self.grad
        for g in Gr.values():
            g.zero_()
        for P in list(self.params.values()) + [self.head]:
            P["gw"].zero_()
            P["gb"].zero_()
        nvox0 = self.n * self.S ** 3
        _ck(L.pfnn_head_backward(_p(A["d1b"]), 16, _p(self.head["w"]), _p(self.logit_grad), nvox0, _p(Gr["d1b"]),
                                 _p(self.head["gw"]), _p(self.head["gb"]), st), "head bwd")
        for (name, src, soff, cin, dst, doff, cout, lev) in reversed(LAYERS):
            P = self.params[name]
            n, d, h, w = self._dims(lev)
            nvox = n * d * h * w
            ldy = BUFFERS[dst][0]
            dzf = self.dz_f[: nvox * cout]
            dzb = self.dz_b[: nvox * cout]
            # ReLU backward on this layer's output slice
            _ck(L.pfnn_relu_bwd_cast(_p(Gr[dst]), ldy, doff, _p(A[dst]), ldy, doff, cout, nvox, _p(dzf), _p(dzb), st),
                "relu bwd")
            _ck(L.pfnn_bias_grad(_p(dzf), cout, 0, cout, nvox, _p(P["gb"]), st), "bias grad")
            _ck(L.pfnn_conv3d_wgrad(_p(dzb), cout, 0, cout, _p(A[src]), BUFFERS[src][0], soff, cin, _p(P["gw"]), n, d,
                                    h, w, st), "wgrad")
            if src != "in0":
                _ck(L.pfnn_weight_transpose(_p(P["wb"]), _p(P["wt"]), cout, cin, st), "wt")
                _ck(L.pfnn_conv3d(_p(dzb), cout, 0, _p(P["wt"]), cout, cin, None, 0, 1, None, _p(Gr[src]),
                                  BUFFERS[src][0], soff, 1, n, d, h, w, st), "dgrad")
            # adjoints of the data movement that produced this layer's input
            if name == "e2a":
                _ck(L.pfnn_avgpool_bwd(_p(Gr["p1"]), 16, _p(Gr["cat1"]), 32, 0, *self._dims(0), st), "pool bwd")
            elif name == "e3a":
                _ck(L.pfnn_avgpool_bwd(_p(Gr["p2"]), 32, _p(Gr["cat2"]), 64, 0, *self._dims(1), st), "pool bwd")
            elif name == "e4a":
                _ck(L.pfnn_avgpool_bwd(_p(Gr["p3"]), 64, _p(Gr["cat3"]), 128, 0, *self._dims(2), st), "pool bwd")
            elif name == "u3":
                _ck(L.pfnn_upsample_bwd(_p(Gr["up3"]), 128, 0, 128, _p(Gr["e4b"]), *self._dims(3), st), "up bwd")
            elif name == "u2":
                _ck(L.pfnn_upsample_bwd(_p(Gr["up2"]), 64, 0, 64, _p(Gr["d3b"]), *self._dims(2), st), "up bwd")
            elif name == "u1":
                _ck(L.pfnn_upsample_bwd(_p(Gr["up1"]), 32, 0, 32, _p(Gr["d2b"]), *self._dims(1), st), "up bwd")

    def adam_step(self, lr=2e-3, b1=0.9, b2=0.999, eps=1e-8):
        L = _lib()
        self.step_count += 1
        for P in list(self.params.values()) + [self.head]:
            _ck(L.pfnn_adam(_p(P["w"]), _p(P["gw"]), _p(P["mw"]), _p(P["vw"]), _p(P["wb"]) if P["wt"] is not None else None,
                            P["w"].numel(), lr, b1, b2, eps, self.step_count, self.stream), "adam")
            _ck(L.pfnn_adam(_p(P["b"]), _p(P["gb"]), _p(P["mb"]), _p(P["vb"]), None, P["b"].numel(), lr, b1, b2, eps,
                            self.step_count, self.stream), "adam")

    def loss_value(self):
        return float(self.loss.item())


def features(dT, sigma_scale):
    """Per-sample network features: log-supercooling and log-surface-tension scale, O(1)."""
    return [math.log10(dT) / 1.3, math.log10(sigma_scale) / 2.5]
