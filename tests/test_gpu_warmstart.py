"""What the learned warm start gains: a network trained (with the library's own BF16 kernels) on
equilibria of small instances predicts the equilibrium of a larger unseen instance; the binary64
relaxation from that prediction meets the equilibrium test in fewer Merson attempts than the plain
run from the nucleation seed, and ends close to the plain run's equilibrium."""
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
    return torch, WS


def test_warm_start_cuts_attempts_to_equilibrium(env):
    torch, WS = env
    train = I.warmstart_instances(160, 32, seed=77, dT_range=(1.0, 3.0), scale_range=(1.0, 3.0))
    G, feat, P, stats = WS.generate(train)
    assert sum(r["equilibrium"] for r in stats) >= 0.8 * len(stats)
    net, hist = WS.train(G, feat, P, steps=500, batch=8, lr=3e-3, log_every=100)
    assert hist[-1][1] < 0.6 * hist[0][1]
    test = I.warmstart_instances(2, 64, seed=78, dT_range=(1.0, 3.0), scale_range=(1.0, 3.0))
    gains = []
    for inst in test:
        cold, phi_c, _, Gt = WS.relax(inst, inst.phi0)
        warm, phi_w, _, _ = WS.relax(inst, WS.predict(net, inst, Gt))
        print(f"\ncold {cold}\nwarm {warm}")
        print(f"equilibria in training data: {sum(r['equilibrium'] for r in stats)}/{len(stats)}, "
              f"mean t_eq {np.nanmean([r['t_eq'] for r in stats]):.4f}")
        assert cold["equilibrium"] and warm["equilibrium"]
        ac = cold["n_accepted"] + cold["n_rejected"]
        aw = warm["n_accepted"] + warm["n_rejected"]
        gains.append(ac / aw)
        # same equilibrium up to pores the seed cannot reach (several equilibria are valid)
        assert abs(warm["uwc"] - cold["uwc"]) <= 0.05
    print(f"\nattempt ratio cold/warm: {gains}, loss {hist[0][1]:.3f} -> {hist[-1][1]:.3f}")
    assert min(gains) > 1.5
