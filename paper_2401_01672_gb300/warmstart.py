"""Learned warm start of the micro-scale equilibrium (BF16 encoder-decoder + RKM relaxation).

generate(): equilibria of many small instances from batched binary32-field runs (the batched
            persistent solver), as training pairs (glass field, features) -> phase field.
train():    Adam on the library's own BF16 tensor-core forward/backward kernels.
predict():  network phase field for a (large) instance, kept in the ice region connected to the seed
            (clipped to [0, 1]) and equal to the seed's phase field elsewhere.
relax():    the plain binary64 Runge-Kutta-Merson integration from a given phase field to the
            equilibrium test (ice count unchanged for the time a free front needs to cross 20 cells and
            no pore interface faster than 1 % of the free-front speed), which stays the judge of the result.
"""
from __future__ import annotations

import math
import time

import numpy as np

from . import inputs as I
from . import nn as NN
from . import pf

from . import sweep

EQ_REL_TOL = sweep.EQ_REL_TOL


def generate(instances, max_steps=4000, batch=128, t_end_factor=50.0):
    """Run the instances to the equilibrium test in batches (the end time, t_end_factor times the nominal
    one, is only a backstop); return device tensors G, feat, phi_eq and the per-instance results."""
    import torch
    Gs, Ps, F, stats = [], [], [], []
    for k in range(0, len(instances), batch):
        chunk = instances[k:k + batch]
        stream = torch.cuda.Stream()
        grids = [sweep._grid(inst, I.PREC_FP32, stream) for inst in chunk]
        b = pf.Batch(grids)
        res = b.run_to([i.t_end * t_end_factor for i in chunk], 1e-6, max_steps,
                       eq_window=[i.eq_window for i in chunk], eq_rel_tol=EQ_REL_TOL,
                       eq_rate=[sweep.eq_rate(i) for i in chunk])
        for inst, g, r in zip(chunk, grids, res):
            Gs.append(torch.from_numpy(g.get_glass().astype(np.float32)))
            Ps.append(torch.from_numpy(g.get_state()[1].astype(np.float32)))
            F.append(NN.features(inst.dT, inst.sigma_scale))
            stats.append(r)
        b.close()
    G = torch.stack(Gs).cuda()
    P = torch.stack(Ps).cuda()
    feat = torch.tensor(F, dtype=torch.float32, device="cuda")
    return G, feat, P, stats


def train(G, feat, P, steps=600, batch=4, lr=2e-3, seed=0, log_every=0):
    """Adam on mean binary cross-entropy; returns the network and the loss history."""
    import torch
    net = NN.UNet(seed=seed)
    g = np.random.default_rng(seed)
    n = G.shape[0]
    hist = []
    for it in range(steps):
        idx = torch.from_numpy(g.choice(n, size=min(batch, n), replace=False)).cuda()
        net.forward(G[idx].reshape(-1).contiguous(), feat[idx].contiguous(), P[idx].reshape(-1).contiguous())
        net.backward()
        cur = lr * 0.5 * (1 + math.cos(math.pi * it / steps))   # cosine decay
        net.adam_step(lr=cur)
        if log_every and it % log_every == 0:
            hist.append((it, net.loss_value()))
    hist.append((steps, net.loss_value()))
    NN.check_device()
    return net, hist


def predict(net, inst, G, halo=3, erode=0):
    """Network phase field for one instance (G: host glass field), as a host float64 array: the network's
    output kept in the ice region connected to the seed (the micro model has no nucleation), the seed's
    phase field elsewhere and in the cells whose water indicator is zero (they never change)."""
    import torch
    Gd = torch.from_numpy(G.astype(np.float32)).cuda()
    feat = torch.tensor([NN.features(inst.dT, inst.sigma_scale)], dtype=torch.float32, device="cuda")
    prob = net.forward(Gd, feat)
    NN.check_device()
    phi, _ = NN.seed_connect(prob, torch.from_numpy(np.ascontiguousarray(inst.phi0)).cuda(),
                             torch.from_numpy(np.ascontiguousarray(G)).cuda(), inst.shape, inst.params["zeta"], halo,
                             erode)
    return phi.cpu().numpy()


def relax(inst, phi_init, max_steps=20000, precision=I.PREC_FP64, t_end_factor=50.0, eq_frac=None):
    """Binary64 RKM from phi_init until the equilibrium test holds (the end time is only a backstop,
    t_end_factor times the instance's nominal t_end; eq_frac overrides the residual test's fraction of the
    free-front speed); returns (result, phi, wall seconds, G)."""
    import torch
    stream = torch.cuda.Stream()
    g = pf.Grid(inst.shape, inst.h, I.MODEL_MICRO, I.REACT_SIGMAP1P, precision, inst.params, stream=stream)
    g.set_geometry(inst.spheres)
    g.set_state(None, phi_init, 0.0, inst.dt0)
    b = pf.Batch([g])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    r = b.run_to([inst.t_end * t_end_factor], 1e-6, max_steps, eq_window=[inst.eq_window],
                 eq_rel_tol=EQ_REL_TOL, eq_rate=[sweep.eq_rate(inst, eq_frac)])[0]
    wall = time.perf_counter() - t0
    phi = g.get_state()[1]
    r["uwc"] = g.unfrozen_fraction()["uwc"]
    G = g.get_glass()
    b.close()
    return r, phi, wall, G
