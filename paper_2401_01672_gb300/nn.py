"""Learned warm start: a 3D convolutional encoder-decoder that predicts the micro-scale equilibrium
phase field from the glass field, the supercooling and the surface-tension scale.

Every forward, backward and optimiser operation runs in the library's CUDA kernels (include/pfnn.h):
BF16 tensor-core 3x3x3 convolutions with FP32 accumulation, pooling/upsampling, the sigmoid head
with binary cross-entropy, Adam on FP32 master weights.  The network itself (its layer sequence,
parameters and buffers) is the library's pfnn_net; this module marshals arguments (torch allocates
the caller's input and output tensors).

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

N_FEATURES = 2

_nn = None


def _lib():
    global _nn
    if _nn is None:
        lib = _pf.load_library()
        vp, i, ll, f, d = C.c_void_p, C.c_int, C.c_longlong, C.c_float, C.c_double
        sig = {
            "pfnn_conv3d": [vp, i, i, vp, i, i, vp, i, i, vp, vp, i, i, i, i, i, i, i, vp],
            "pfnn_conv3d_wgrad": [vp, i, i, i, vp, i, i, i, vp, i, i, i, i, vp, ll, vp],
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
            "pfnn_net_create": [C.c_ulonglong, vp, C.POINTER(vp)],
            "pfnn_net_destroy": [vp],
            "pfnn_net_param_shape": [i, C.POINTER(i), C.POINTER(i)],
            "pfnn_net_set_params": [vp, i, vp, vp],
            "pfnn_net_get_params": [vp, i, vp, vp],
            "pfnn_net_get_grads": [vp, i, vp, vp],
            "pfnn_net_forward": [vp, vp, vp, i, i, vp, vp],
            "pfnn_net_infer": [vp, vp, vp, i, i, vp],
            "pfnn_net_loss": [vp, C.POINTER(d)],
            "pfnn_net_backward": [vp],
            "pfnn_net_adam_step": [vp, f, f, f, f],
            "pfnn_seed_connect": [vp, vp, vp, i, i, i, d, i, i, vp, vp, vp, C.POINTER(ll)],
            "pfnn_net_layer": [i, C.POINTER(i)],
            "pfnn_net_buffer": [i, C.POINTER(i), C.POINTER(i)],
            "pfnn_net_read_buffer": [vp, i, vp, vp],
        }
        for name, args in sig.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = C.c_int
        lib.pfnn_conv3d_wgrad_work_bytes.argtypes = [i, i, i, i, i, i]
        lib.pfnn_conv3d_wgrad_work_bytes.restype = ll
        lib.pfnn_net_params.argtypes = []
        lib.pfnn_net_params.restype = C.c_int
        lib.pfnn_net_buffers.argtypes = []
        lib.pfnn_net_buffers.restype = C.c_int
        lib.pfnn_net_param_name.argtypes = [i]
        lib.pfnn_net_param_name.restype = C.c_char_p
        lib.pfnn_net_last_error.argtypes = [vp]
        lib.pfnn_net_last_error.restype = C.c_char_p
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
    """Handle of the library's encoder-decoder (pfnn_net in include/pfnn.h): parameters, gradients, Adam
    moments and activations live in the library; this class only marshals arguments."""

    def __init__(self, seed=0, device="cuda"):
        import torch
        self.torch = torch
        self.dev = device
        self.stream = torch.cuda.current_stream().cuda_stream
        out = C.c_void_p()
        _ck(_lib().pfnn_net_create(int(seed), C.c_void_p(self.stream), C.byref(out)), "pfnn_net_create")
        self.handle = out
        self.names = [_lib().pfnn_net_param_name(q).decode() for q in range(_lib().pfnn_net_params())]
        self._prob = None

    def _ck(self, st, what):
        if st != 0:
            msg = _lib().pfnn_net_last_error(self.handle)
            raise _pf.PfError(st, f"{what}: {msg.decode() if msg else ''}")

    def close(self):
        if getattr(self, "handle", None):
            _lib().pfnn_net_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def shape(self, name):
        q = self.names.index(name)
        ci, co = C.c_int(), C.c_int()
        _ck(_lib().pfnn_net_param_shape(q, C.byref(ci), C.byref(co)), "shape")
        return (27, co.value, ci.value) if name != "head" else (16,), (co.value,)

    def get_params(self, name):
        """(weights, biases) as float32 numpy arrays ([27][cout][cin] for a convolution, [16] for the head)."""
        ws, bs = self.shape(name)
        w, b = np.empty(ws, np.float32), np.empty(bs, np.float32)
        self._ck(_lib().pfnn_net_get_params(self.handle, self.names.index(name), w.ctypes.data, b.ctypes.data), name)
        return w, b

    def set_params(self, name, w, b):
        w = np.ascontiguousarray(w, dtype=np.float32)
        b = np.ascontiguousarray(b, dtype=np.float32)
        self._ck(_lib().pfnn_net_set_params(self.handle, self.names.index(name), w.ctypes.data, b.ctypes.data), name)

    def get_grads(self, name):
        ws, bs = self.shape(name)
        w, b = np.empty(ws, np.float32), np.empty(bs, np.float32)
        self._ck(_lib().pfnn_net_get_grads(self.handle, self.names.index(name), w.ctypes.data, b.ctypes.data), name)
        return w, b

    def forward(self, G, feat, target=None):
        """G: fp32 (n * S^3,) glass field; feat: fp32 (n, N_FEATURES); returns probabilities (n * S^3,)."""
        t = self.torch
        n = feat.shape[0]
        S = round((G.numel() // n) ** (1 / 3))
        assert n * S ** 3 == G.numel() and S % 8 == 0, "grid side must be a multiple of 8"
        if self._prob is None or self._prob.numel() != G.numel():
            self._prob = t.empty(G.numel(), dtype=t.float32, device=self.dev)
        self._ck(_lib().pfnn_net_forward(self.handle, _p(G), _p(feat), n, S, _p(target), _p(self._prob)), "forward")
        self._n, self._S = n, S
        return self._prob

    def backward(self):
        """Gradients of the mean BCE of the last forward (with a target) into every parameter."""
        self._ck(_lib().pfnn_net_backward(self.handle), "backward")

    def adam_step(self, lr=2e-3, b1=0.9, b2=0.999, eps=1e-8):
        self._ck(_lib().pfnn_net_adam_step(self.handle, lr, b1, b2, eps), "adam")

    def layer(self, q):
        """Wiring of convolution q (see pfnn_net_layer)."""
        w = (C.c_int * 12)()
        _ck(_lib().pfnn_net_layer(int(q), w), "layer")
        keys = ("src", "soff", "cin", "dst", "doff", "cout", "lev", "pre", "pre_src", "pre_c", "pre_dst", "pre_lev")
        return dict(zip(keys, list(w)))

    def buffer(self, b):
        """(activations, gradients) of buffer b of the last forward / backward as float64 numpy arrays
        (n, s, s, s, channels)."""
        c, lev = C.c_int(), C.c_int()
        _ck(_lib().pfnn_net_buffer(int(b), C.byref(c), C.byref(lev)), "buffer")
        s = self._S >> lev.value
        shape = (self._n, s, s, s, c.value)
        a = np.empty(shape, dtype=np.uint16)
        g = np.empty(shape, dtype=np.float32)
        self._ck(_lib().pfnn_net_read_buffer(self.handle, int(b), a.ctypes.data, g.ctypes.data), "read_buffer")
        act = (a.astype(np.uint32) << 16).view(np.float32).astype(np.float64)
        return act, g.astype(np.float64)

    def loss_value(self):
        v = C.c_double()
        self._ck(_lib().pfnn_net_loss(self.handle, C.byref(v)), "loss")
        return v.value


def seed_connect(prob, phi_seed, G, shape, zeta, halo=3, erode=0):
    """Network output restricted to the ice region connected to the seed (device tensors; returns a
    binary64 device tensor and the flood-fill sweeps run)."""
    import torch
    n = int(shape[0]) * int(shape[1]) * int(shape[2])
    for name, t, dt in (("prob", prob, torch.float32), ("phi_seed", phi_seed, torch.float64), ("G", G, torch.float64)):
        if not t.is_cuda or t.dtype != dt or t.numel() != n or not t.is_contiguous():
            raise ValueError(f"{name}: contiguous {dt} CUDA tensor of {n} values required")
    out = torch.empty(n, dtype=torch.float64, device=prob.device)
    work = torch.empty(16 * ((n + 15) // 16) + 16, dtype=torch.uint8, device=prob.device)
    sw = C.c_longlong()
    _ck(_lib().pfnn_seed_connect(_p(prob), _p(phi_seed), _p(G), int(shape[0]), int(shape[1]), int(shape[2]),
                                 float(zeta), int(erode), int(halo), _p(work), _p(out),
                                 C.c_void_p(torch.cuda.current_stream().cuda_stream), C.byref(sw)), "seed_connect")
    return out, sw.value


def features(dT, sigma_scale):
    """Per-sample network features: log-supercooling and log-surface-tension scale, O(1)."""
    return [math.log10(dT) / 1.3, math.log10(sigma_scale) / 2.5]
