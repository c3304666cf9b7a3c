"""Macro-scale vessel of Sec. 3.1 through the library on a coarse mesh (N3 = 40) for the first 40
minutes of cooling: every model runs, the ice fraction grows once the cap is cold (the nucleation disk
may first lose some ice to the +20 K water), SigmaP1-P keeps phi in [0, 1] to the step tolerance (its
reaction term vanishes at 0 and 1), the Temp model's phi(theta) stays in [0, 1] by construction, and
no temperature falls below the cap's."""
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
    from paper_2401_01672_gb300 import macro
    return macro


@pytest.mark.parametrize("model,rx,sigma", [(I.MODEL_FULL, I.REACT_SIGMAP1P, "large"),
                                            (I.MODEL_FULL, I.REACT_SIGMAP1P, "tiny"),
                                            (I.MODEL_TEMP, I.REACT_SIGMAP1P, "large")])
def test_macro_vessel_cooling(env, model, rx, sigma):
    macro = env
    w = I.macro_case(40, model, rx, sigma=sigma)
    w.extra["t_end"] = 2400.0
    r = macro.run_case(w, n_samples=12, max_attempts=200000)
    assert r["status"] == "ok" and len(r["curve"]) == 12
    ice = np.array([p["ice_fraction"] for p in r["curve"]])
    assert np.all(np.diff(ice[len(ice) // 2:]) >= 0.0)
    assert ice[-1] > ice[0] and ice[-1] > 0.0
    lo = min(p["phi_min"] for p in r["curve"])
    hi = max(p["phi_max"] for p in r["curve"])
    assert lo >= -1e-6 and hi <= 1.0 + 1e-6
    # the cap is the only cold boundary: the coldest temperature is the cap's
    assert min(p["theta_min"] for p in r["curve"]) >= -25.0 - 1e-6


def test_macro_vessel_binary32_form_follows_binary64(env):
    """The vessel (N3 = 40, SigmaP1-P, small sigma, first 40 minutes of cooling) in the binary32-field
    form: its stage inputs are increments over a binary32 copy of the state, so the error estimate keeps
    no rounding floor above the tolerance and it takes at most twice the binary64 attempts (binary32
    stage values took several times more); the sampled ice fractions agree to 1e-3."""
    macro = env
    out = {}
    for prec in (I.PREC_FP64, I.PREC_FP32):
        w = I.macro_case(40, I.MODEL_FULL, I.REACT_SIGMAP1P, sigma="small")
        w.extra["t_end"] = 2400.0
        out[prec] = macro.run_case(w, n_samples=12, max_attempts=400000, precision=prec)
    r64, r32 = out[I.PREC_FP64], out[I.PREC_FP32]
    assert r64["status"] == "ok" and r32["status"] == "ok"
    i64 = np.array([p["ice_fraction"] for p in r64["curve"]])
    i32 = np.array([p["ice_fraction"] for p in r32["curve"]])
    print(f"\nbinary64 {r64['attempts']} attempts, binary32 form {r32['attempts']}, "
          f"max |d ice fraction| {np.max(np.abs(i64 - i32)):.2e}")
    assert i64[-1] > 0.0
    assert np.max(np.abs(i64 - i32)) <= 1e-3
    assert r32["attempts"] <= 2 * r64["attempts"]


def test_uwc_falls_with_supercooling_coarse(env):
    """Micro-scale vessel (bead radius 5 um) on a coarse mesh: at the larger supercooling the ice
    reaches into smaller pores (Gibbs-Thomson), so less water stays unfrozen in the bed."""
    from paper_2401_01672_gb300 import sweep
    inst = I.uwc_instances(dTs=(0.1, 2.0), beds=("settled",), n3=60)
    b = sweep.run_batched(inst, max_steps=30000)   # dT = 2 needs ~16,500 attempts at this mesh
    res = b["instances"]
    assert all(r["status"] == 0 for r in res)
    assert all(r["equilibrium"] for r in res)
    u = [r["uwc"] for r in res]
    assert 0.0 <= u[1] < u[0] <= 1.0
