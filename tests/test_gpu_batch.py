"""Batched persistent runs (one CUDA-graph launch with a device-side WHILE loop over all instances)
and the tile autotuner.

Each batched instance must reproduce its own single-grid run (same step counts, same state to
rounding), one instance is checked against the oracle, and the equilibrium test and the step cap
must stop instances independently.
"""
import math

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
    from paper_2401_01672_gb300 import pf
    import oracle
    oracle.build()
    return torch, pf, oracle


SHAPES = [(33, 40, 37), (48, 32, 29), (21, 21, 64), (40, 40, 40)]


def micro_instance(q, shape, h=5e-8):
    """Micro-scale instance q: own bead packing, supercooling and surface-tension scale."""
    scale = [1.0, 3.0, 1.0, 10.0][q]
    dT = [0.5, 2.0, 1.0, 5.0][q]
    sv = I.packing_rsa(shape, 3, 4.0, 6.0, 500 + q)
    c = I.pore_ball_center(shape, sv, 4.0, 600 + q)
    phi0 = I.ball_indicator(shape, c, 4.0)
    p = I.default_params(xi=h, xi_G=0.4 * h, zeta=2.0, theta_micro=-dT, alpha=I.TABLE1["alpha"] / scale)
    return sv * h, p, phi0, 0.1 * p["alpha"] * h * h


def make_grids(pf, prec):
    grids, meta = [], []
    for q, shape in enumerate(SHAPES):
        sp, p, phi0, dt0 = micro_instance(q, shape)
        g = pf.Grid(shape, 5e-8, I.MODEL_MICRO, I.REACT_SIGMAP1P, prec, p)
        g.set_geometry(sp)
        g.set_state(None, phi0, 0.0, dt0)
        grids.append(g)
        meta.append((sp, p, phi0, dt0))
    return grids, meta


@pytest.mark.parametrize("prec", [I.PREC_FP64, I.PREC_FP32])
def test_batch_matches_single_grid_runs(env, prec):
    torch, pf, oracle = env
    t_end = [0.004, 0.002, 0.003, 0.0015]
    single = []
    grids, meta = make_grids(pf, prec)
    for g, te in zip(grids, t_end):
        s = g.run_to(te, 1e-6, 400)
        single.append((s, g.get_state()[1]))
        g.close()
    grids, meta = make_grids(pf, prec)
    b = pf.Batch(grids)
    res = b.run_to(t_end, 1e-6, 400)
    assert b.iterations() <= 402
    for q, (r, (s, ph)) in enumerate(zip(res, single)):
        assert r["status"] == 0 and not r["equilibrium"]
        assert (r["n_accepted"], r["n_rejected"]) == (s["n_accepted"], s["n_rejected"]), q
        assert r["t"] == s["t"]
        phb = grids[q].get_state()[1]
        assert np.max(np.abs(phb - ph)) <= 1e-13 * max(1.0, np.max(np.abs(ph)))
    b.close()


def test_batch_instance_against_oracle(env):
    torch, pf, oracle = env
    grids, meta = make_grids(pf, I.PREC_FP64)
    b = pf.Batch(grids)
    t_end = [0.003, 0.001, 0.002, 0.001]
    res = b.run_to(t_end, 1e-6, 2000)
    q = 0
    sp, p, phi0, dt0 = meta[q]
    o = oracle.Oracle(SHAPES[q], 5e-8, "micro", "sigmap1p", p)
    G = o.glass(sp, p["xi_G"])
    r = o.run(G, None, phi0, 0.0, dt0, t_end[q], 1e-6, 2000)
    assert (res[q]["n_accepted"], res[q]["n_rejected"]) == (r["n_accepted"], r["n_rejected"])
    ph = grids[q].get_state()[1]
    assert np.max(np.abs(ph - r["phi"])) <= 1e-8
    b.close()


def test_batch_equilibrium_and_cap(env):
    """A sub-critical seed melts away (Gibbs-Thomson: R < R* = 2/(mu alpha dT)): its instance stops on
    the equilibrium test (ice count unchanged for eq_window) with no ice left; the other, without the
    test, runs into the step cap."""
    torch, pf, oracle = env
    h = 5e-8
    shape = (24, 24, 24)
    grids = []
    p0 = I.default_params(xi=h, xi_G=0.4 * h, theta_micro=-0.01, alpha=I.TABLE1["alpha"])
    for _ in range(2):
        g = pf.Grid(shape, h, I.MODEL_MICRO, 0, I.PREC_FP64, p0)
        g.set_state(None, I.ball_indicator(shape, (12, 12, 12), 3.0), 0.0, 0.1 * p0["alpha"] * h * h)
        grids.append(g)
    b = pf.Batch(grids)
    window = 0.01
    res = b.run_to([10.0, 10.0], 1e-6, 3000, eq_window=[window, 0.0])
    assert res[0]["equilibrium"] and window <= res[0]["t_eq"] < 10.0
    assert grids[0].unfrozen_fraction()["n_ice"] == 0
    assert not res[1]["equilibrium"]
    assert res[1]["n_accepted"] + res[1]["n_rejected"] == 3000
    b.close()


def test_autotune_changes_speed_not_results(env, tmp_path):
    torch, pf, oracle = env
    shape = (70, 50, 90)
    h = 3e-4
    w = I.full_bead_case(40, 9)  # parameters of the bead workload
    p = dict(w.params)
    th, ph, G = I.random_fields(shape, 31, theta_scale=2.0)
    out = []
    for tune in (False, True):
        g = pf.Grid(shape, h, I.MODEL_FULL, I.REACT_SIGMAP1P, I.PREC_FP64, p)
        g.set_glass(G)
        g.set_state(th, ph, 0.0, 0.01)
        if tune:
            cache = str(tmp_path / "tiles.txt")
            by, zc, ms = g.autotune(cache)
            assert by in (4, 8, 16) and zc in (2, 3, 4, 5, 6, 8, 10, 12, 16, 24, 32, 64) and ms > 0
            assert g.get_tiles() == (by, zc)
            assert open(cache).read().split()[1:3] == [str(by), str(zc)]
            # a cached shape is reused without timing
            g2 = pf.Grid(shape, h, I.MODEL_FULL, I.REACT_SIGMAP1P, I.PREC_FP64, p)
            assert g2.autotune(cache)[:2] == (by, zc)
            g2.close()
        s = g.run_to(1.0, 1e-6, 30)
        out.append((s, g.get_state()))
        g.close()
    (s0, st0), (s1, st1) = out
    assert (s0["n_accepted"], s0["n_rejected"]) == (s1["n_accepted"], s1["n_rejected"])
    assert np.array_equal(st0[0], st1[0]) and np.array_equal(st0[1], st1[1])
