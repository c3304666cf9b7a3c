"""z-slab multi-domain mode (the paper's 1-D decomposition along x3, Sec. 2.5) against the single-domain
grid: the domain cut into 2 or 3 slabs (even and uneven cuts) that exchange their cut planes every stage
and share one step control reproduces the single-domain run bit for bit: the same accepted and rejected
attempts, the same state at every cell, the same unfrozen-water counts."""
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
    return torch, pf


def bead_case(n3=44):
    """A full-model bead crop, cold top face switching to warm at t_freeze (so the run crosses the
    Dirichlet switch), ice seed on the top planes."""
    shape = (38, 30, n3)
    h = 3e-4
    sv, _ = I.packing_boolean(shape, 0.55, I.uniform_radius(5.0, 8.0), 31)
    p = I.default_params(xi=h, xi_G=0.4 * h, alpha=I.ALPHA_MACRO["large"], zeta=2.0, dirichlet_faces=I.FACE_ZP,
                         theta_freeze=-5.0, theta_thaw=2.0, t_freeze=1.0)
    th0 = np.full(int(np.prod(shape)), 1.0)
    ph0 = I.top_slab_indicator(shape, 3)
    return shape, h, sv * h, p, th0, ph0


def single(pf, shape, h, model, prec, p, sp, th0, ph0, t_end, tiles):
    g = pf.Grid(shape, h, model, I.REACT_SIGMAP1P, prec, p)
    g.set_geometry(sp)
    g.set_tiles(*tiles)
    g.set_state(th0, ph0, 0.0, 0.01 if model != I.MODEL_MICRO else 1e-4)
    s = g.run_to(t_end, 1e-6, 100000)
    th, ph, t, dt = g.get_state()
    u = g.unfrozen_fraction()
    g.close()
    return s, th, ph, t, dt, u


def slabs(pf, shape, h, model, prec, p, sp, th0, ph0, t_end, tiles, nslabs, planes):
    S = pf.Slabs(shape, h, model, I.REACT_SIGMAP1P, prec, p, nslabs=nslabs, planes=planes)
    S.set_geometry(sp)
    S.set_tiles(*tiles)
    S.set_state(th0, ph0, 0.0, 0.01 if model != I.MODEL_MICRO else 1e-4)
    s = S.run_to(t_end, 1e-6, 100000)
    th, ph, t, dt = S.get_state()
    u = S.unfrozen_fraction()
    hb = S.halo_bytes()
    S.close()
    return s, th, ph, t, dt, u, hb


@pytest.mark.parametrize("prec", [I.PREC_FP64, I.PREC_FP32])
@pytest.mark.parametrize("nslabs,planes", [(2, None), (3, [0, 5, 29, 44]), (4, [0, 1, 2, 30, 44])])
def test_slabs_equal_single_domain_full_model(env, prec, nslabs, planes):
    torch, pf = env
    shape, h, sp, p, th0, ph0 = bead_case()
    tiles = (8, 7)   # z chunks that do not divide the slabs: ragged chunks at every cut
    ref = single(pf, shape, h, I.MODEL_FULL, prec, p, sp, th0, ph0, 2.0, tiles)
    got = slabs(pf, shape, h, I.MODEL_FULL, prec, p, sp, th0, ph0, 2.0, tiles, nslabs, planes)
    s0, s1 = ref[0], got[0]
    assert s0["n_accepted"] > 20 and s0["t"] == 2.0
    assert (s1["n_accepted"], s1["n_rejected"]) == (s0["n_accepted"], s0["n_rejected"])
    assert s1["last_err"] == s0["last_err"]
    assert np.array_equal(got[1], ref[1]) and np.array_equal(got[2], ref[2])
    assert got[3] == ref[3] and got[4] == ref[4]
    assert (got[5]["n_ice"], got[5]["n_water"]) == (ref[5]["n_ice"], ref[5]["n_water"])
    # halo traffic: every cut, both directions, two fields, per attempt four exchanges of stage inputs and
    # one of the state (replays included); the binary32 form adds the binary32 copy of the state
    esz = 4 if prec == I.PREC_FP32 else 8
    nx = 5 if prec == I.PREC_FP32 else 4
    per_attempt = (nslabs - 1) * 2 * 2 * shape[0] * shape[1] * (nx * esz + 8)
    assert got[6] > 0 and got[6] % per_attempt == 0


def test_slabs_equal_single_domain_micro(env):
    torch, pf = env
    shape = (33, 28, 40)
    h = 5e-8
    sv = I.packing_rsa(shape, 5, 5.0, 7.0, 12)
    c = I.pore_ball_center(shape, sv, 4.0, 13)
    ph0 = I.ball_indicator(shape, c, 4.0)
    p = I.default_params(xi=h, xi_G=0.4 * h, zeta=2.0, theta_micro=-0.5, alpha=I.TABLE1["alpha"])
    t_end = 0.01
    ref = single(pf, shape, h, I.MODEL_MICRO, I.PREC_FP64, p, sv * h, None, ph0, t_end, (4, 9))
    got = slabs(pf, shape, h, I.MODEL_MICRO, I.PREC_FP64, p, sv * h, None, ph0, t_end, (4, 9), 3, None)
    assert ref[0]["n_accepted"] > 10
    assert (got[0]["n_accepted"], got[0]["n_rejected"]) == (ref[0]["n_accepted"], ref[0]["n_rejected"])
    assert np.array_equal(got[2], ref[2])
    assert (got[5]["n_ice"], got[5]["n_water"]) == (ref[5]["n_ice"], ref[5]["n_water"])


def test_slabs_reject_bad_cuts(env):
    torch, pf = env
    p = I.default_params(xi=1e-6)
    for nslabs, planes in ((3, [0, 4, 4, 10]), (2, [1, 5, 10]), (2, [0, 5, 9]), (11, None), (0, None)):
        with pytest.raises(pf.PfError):
            pf.Slabs((8, 8, 10), 1e-6, I.MODEL_MICRO, 0, 0, p, nslabs=nslabs, planes=planes)
