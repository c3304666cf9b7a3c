"""What the learned warm start gains: a network trained (with the library's own BF16 kernels) on
equilibria of small instances predicts the equilibrium of a larger unseen instance; the prediction is
kept in the ice region connected to the seed (the micro model has no nucleation); the binary64
relaxation from it meets the equilibrium test (pore ice count settled and no pore interface faster than
1 % of the free-front speed) in fewer Merson attempts and less time than the plain run from the seed,
and ends at an equilibrium whose unfrozen-water fraction is within 1 % of the plain run's.  (The two
runs stop at valid equilibria that still differ in a few per cent of the cells, mostly where the water
indicator is small and the relaxation slow: max|dphi| is reported, not bounded by 1e-3.)"""
import numpy as np
import pytest

from paper_2401_01672_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2401_01672_gb300 import build
    build.build()
    from paper_2401_01672_gb300 import warmstart as WS
    from paper_2401_01672_gb300 import nn as NN
    return torch, WS, NN


def test_seed_connect_keeps_only_the_seeded_region(env):
    """Two predicted ice blobs, one touching the seed plane and one isolated in the pore space: the
    isolated one goes back to the seed's phase field, the connected one (and its `halo` cells) keeps the
    prediction; cells with a zero water indicator keep the seed's value."""
    torch, WS, NN = env
    n = (20, 18, 24)
    N = n[0] * n[1] * n[2]
    z, y, x = np.meshgrid(np.arange(n[2]), np.arange(n[1]), np.arange(n[0]), indexing="ij")
    prob = np.full((n[2], n[1], n[0]), 0.1, np.float32)
    connected = (x < 8) & (z < 12)               # touches the seed plane z = 0
    isolated = (x > 12) & (z > 16) & (y > 4)     # separated from it by prob <= 1/2
    prob[connected] = 0.9
    prob[isolated] = 0.8
    seed = np.zeros((n[2], n[1], n[0]))
    seed[0] = 1.0
    G = np.zeros((n[2], n[1], n[0]))
    G[20:, :, :4] = 1.0                          # glass: water indicator 0 there
    out, sweeps = NN.seed_connect(torch.from_numpy(prob.ravel()).cuda(), torch.from_numpy(seed.ravel()).cuda(),
                                  torch.from_numpy(G.ravel()).cuda(), n, 2.0, halo=2)
    o = out.cpu().numpy().reshape(n[2], n[1], n[0])
    assert sweeps >= 16
    assert np.all(o[0] == 1.0)                               # the seed stays ice
    assert np.all(o[connected & (z >= 1)] == np.float32(0.9))
    assert np.all(o[isolated] == 0.0)
    # halo: cells within 2 of the reached region keep the prediction, farther ones the seed value
    near = (x >= 8) & (x < 10) & (z >= 1) & (z < 12)
    assert np.all(o[near] == np.float32(0.1))
    far = (x >= 10) & (z >= 3) & (z < 12)
    assert np.all(o[far] == 0.0)
    assert np.all(o[G >= 0.5] == seed[G >= 0.5])


def test_warm_start_cuts_time_to_equilibrium(env):
    torch, WS, NN = env
    train = I.warmstart_instances(160, 32, seed=77, dT_range=(1.0, 3.0), scale_range=(1.0, 3.0))
    G, feat, P, stats = WS.generate(train)
    assert sum(r["equilibrium"] for r in stats) >= 0.8 * len(stats)
    net, hist = WS.train(G, feat, P, steps=500, batch=8, lr=3e-3, log_every=100)
    assert hist[-1][1] < 0.6 * hist[0][1]
    test = I.warmstart_instances(2, 64, seed=78, dT_range=(1.0, 3.0), scale_range=(1.0, 3.0))
    rows = []
    for inst in test:
        cold, phi_c, wall_c, Gt = WS.relax(inst, inst.phi0)
        torch.cuda.synchronize()
        import time
        t0 = time.perf_counter()
        pred = WS.predict(net, inst, Gt)
        t_inf = time.perf_counter() - t0
        warm, phi_w, wall_w, _ = WS.relax(inst, pred)
        assert cold["equilibrium"] and warm["equilibrium"]
        ac = cold["n_accepted"] + cold["n_rejected"]
        aw = warm["n_accepted"] + warm["n_rejected"]
        dphi = float(np.max(np.abs(phi_w - phi_c)))
        bulk = (1.0 - inst.params["zeta"] * Gt) > 0.5
        dphi_bulk = float(np.max(np.abs(phi_w - phi_c)[bulk]))
        off = float(np.mean(np.abs(phi_w - phi_c) > 1e-3))
        duwc = abs(warm["uwc"] - cold["uwc"]) / cold["uwc"]
        rows.append((ac, aw, wall_c, wall_w + t_inf, dphi, dphi_bulk, off, duwc))
    print("\n(cold attempts, warm attempts, cold s, warm s incl. inference, max|dphi|, max|dphi| pore bulk, "
          f"fraction of cells off by > 1e-3, UWC rel): {rows}, loss {hist[0][1]:.3f} -> {hist[-1][1]:.3f}")
    for ac, aw, wc, ww, dphi, dphi_bulk, off, duwc in rows:
        assert duwc <= 1e-2 and off <= 0.05
        assert ac / aw > 1.5 and wc / ww > 1.5
    net.close()
