"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle.

Bar (binary64 path): max|gpu - oracle| / max|oracle| <= 1e-11 for fields, bit-exact counts,
identical accepted/rejected step counts under adaptive stepping.  Shapes are ragged with
respect to the 32 x 8 x 32 tiles and span several tiles; one case runs at 256^3.
"""
import math

import numpy as np
import pytest

from paper_2401_01672_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = 1e-11


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2401_01672_gb300 import build
    build.build()
    return torch


@pytest.fixture(scope="module")
def orc():
    import oracle
    oracle.build()
    return oracle


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    den = np.max(np.abs(b))
    return float(np.max(np.abs(a - b)) / (den if den > 0 else 1.0))


def both(orc, shape, h, model, rx, params, prec=0):
    from paper_2401_01672_gb300 import pf
    g = pf.Grid(shape, h, model, rx, prec, params)
    o = orc.Oracle(shape, h, model, rx, params)
    return g, o


def dev(torch, a, dtype=None):
    t = torch.as_tensor(np.ascontiguousarray(a))
    return t.to(device="cuda", dtype=dtype or torch.float64).contiguous()


CASES = [
    ("full", I.MODEL_FULL, I.REACT_SIGMAP1P),
    ("full-gradp", I.MODEL_FULL, I.REACT_GRADP),
    ("temp", I.MODEL_TEMP, I.REACT_SIGMAP1P),
    ("micro", I.MODEL_MICRO, I.REACT_SIGMAP1P),
    ("micro-gradp", I.MODEL_MICRO, I.REACT_GRADP),
]


def case_params(h, model, **over):
    base = dict(xi=1.3 * h, xi_G=0.4 * h, alpha=4.17e6 if model != I.MODEL_MICRO else 3.0e9,
                dirichlet_faces=I.FACE_ZP | I.FACE_XM | I.FACE_YP, theta_freeze=-5.0, theta_thaw=2.0,
                t_freeze=10.0, theta_micro=-0.7, zeta=2.0, gamma=2.0)
    base.update(over)
    return I.default_params(**base)


def test_glass_field_parity(torch_cuda, orc):
    shape = (45, 38, 29)
    h = 1e-6
    p = case_params(h, I.MODEL_MICRO, xi_G=0.45 * h)
    g, o = both(orc, shape, h, I.MODEL_MICRO, 0, p)
    rng = I.rng(7)
    sp = np.column_stack([rng.uniform(-3, 48, 14), rng.uniform(-3, 41, 14), rng.uniform(-3, 32, 14),
                          rng.uniform(2, 9, 14)]) * h
    for cap in (math.nan, 22.3 * h):
        g.set_geometry(sp, cap)
        Gg = g.get_glass()
        Go = o.glass(sp, p["xi_G"], cap)
        assert np.max(np.abs(Gg - Go)) <= 1e-14
        assert np.array_equal(Gg < 0.5, Go < 0.5)
    g.close()


@pytest.mark.parametrize("name,model,rx", CASES)
@pytest.mark.parametrize("shape", [(45, 38, 29), (37, 19, 70), (1, 1, 1), (3, 2, 1)])
def test_rhs_parity_fp64(torch_cuda, orc, name, model, rx, shape):
    torch = torch_cuda
    h = 2e-4 if model != I.MODEL_MICRO else 1e-6
    p = case_params(h, model)
    g, o = both(orc, shape, h, model, rx, p)
    th, ph, G = I.random_fields(shape, 100 + model * 10 + rx, theta_scale=3.0)
    g.set_glass(G)
    for t in (0.0, 10.0):
        oth, oph = o.rhs(G, th, ph, t=t)
        dth = torch.empty(g.N, device="cuda", dtype=torch.float64)
        dph = torch.empty(g.N, device="cuda", dtype=torch.float64)
        g.rhs(t, dev(torch, th) if model != I.MODEL_MICRO else None,
              dev(torch, ph) if model != I.MODEL_TEMP else None, dth, dph)
        torch.cuda.synchronize()
        if model != I.MODEL_MICRO:
            assert rel(dth.cpu().numpy(), oth) <= TOL
        else:
            assert np.all(dth.cpu().numpy() == 0)
        assert rel(dph.cpu().numpy(), oph) <= TOL
    g.close()


@pytest.mark.parametrize("name,model,rx", CASES)
def test_rkm_step_parity_fp64(torch_cuda, orc, name, model, rx):
    shape = (41, 23, 37)
    h = 2e-4 if model != I.MODEL_MICRO else 1e-6
    p = case_params(h, model)
    g, o = both(orc, shape, h, model, rx, p)
    th, ph, G = I.random_fields(shape, 300 + model, theta_scale=2.0)
    g.set_glass(G)
    dt = 0.02 if model != I.MODEL_MICRO else 0.05 * p["alpha"] * h * h
    g.set_state(th, ph, 9.0, dt)
    acc, err, dtn = g.rkm_step(dt, 1e-30, force_accept=True)
    gth, gph, t, _ = g.get_state()
    oth, oph, oerr = o.rkm_step(G, th, ph, 9.0, dt)
    assert acc and t == 9.0 + dt
    if model != I.MODEL_MICRO:
        assert rel(gth, oth) <= TOL
    if model != I.MODEL_TEMP:
        assert rel(gph, oph) <= TOL
    assert abs(err - oerr) <= 1e-8 * oerr
    g.close()


def test_micro32_fixed_then_adaptive(torch_cuda, orc):
    """32^3 micro-scale case: 200 fixed steps (1e-11), then adaptive to t_end with the same
    accepted and rejected counts and the same unfrozen-water counts."""
    w = I.micro_32()
    g, o = both(orc, w.shape, w.h, w.model, w.reaction, w.params)
    g.set_geometry(w.spheres, w.x3_cap)
    G = o.glass(w.spheres, w.params["xi_G"], w.x3_cap)
    assert np.max(np.abs(g.get_glass() - G)) <= 1e-14
    dt = w.extra["fixed_dt"]
    g.set_state(None, w.phi0, 0.0, dt)
    s = g.run_fixed(200, dt)
    assert s["n_accepted"] == 200
    r = o.run(G, None, w.phi0, 0.0, dt, math.inf, 1.0, 200, fixed=True)
    _, gph, gt, _ = g.get_state()
    assert rel(gph, r["phi"]) <= TOL and abs(gt - r["t"]) <= 1e-15 * r["t"]
    # adaptive continuation
    tol, t_end = w.extra["tol"], w.extra["t_end"]
    ga = g.run_to(t_end, tol, 100000)
    ra = o.run(G, None, r["phi"], r["t"], dt, t_end, tol, 100000)
    assert ra["status"] == 0
    assert (ga["n_accepted"], ga["n_rejected"]) == (ra["n_accepted"], ra["n_rejected"])
    assert ga["t"] == t_end == ra["t"]
    _, gph, _, _ = g.get_state()
    assert rel(gph, ra["phi"]) <= 1e-8
    ug = g.unfrozen_fraction()
    uo = o.uwc(G, ra["phi"])
    assert (ug["n_water"], ug["n_ice"]) == (uo["n_water"], uo["n_ice"])
    assert abs(ug["smooth"] - uo["smooth"]) <= 1e-9
    g.close()


@pytest.mark.parametrize("name,model,rx", CASES[:3])
def test_adaptive_counts_macro(torch_cuda, orc, name, model, rx):
    """Bead case with a Dirichlet top face switching at t_freeze: same step counts, landing
    exactly on t_freeze and t_end."""
    n = 24
    shape = (n, n + 5, n - 3)
    h = 3e-4
    sv, _ = I.packing_boolean(shape, 0.45, I.uniform_radius(3, 5), 77)
    p = I.default_params(xi=h, xi_G=0.4 * h, alpha=4.17e6, dirichlet_faces=I.FACE_ZP, theta_freeze=-5.0,
                         theta_thaw=2.0, t_freeze=2.0, zeta=2.0 if model != I.MODEL_TEMP else 1.0)
    g, o = both(orc, shape, h, model, rx, p)
    g.set_geometry(sv * h)
    G = o.glass(sv * h, p["xi_G"])
    th0 = np.full(g.N, 1.0)
    ph0 = I.top_slab_indicator(shape, 2)
    g.set_state(th0, ph0, 0.0, 0.01)
    ga = g.run_to(4.0, 1e-5, 20000)
    ra = o.run(G, th0, ph0, 0.0, 0.01, 4.0, 1e-5, 20000)
    assert ra["status"] == 0 and ga["t"] == 4.0
    assert (ga["n_accepted"], ga["n_rejected"]) == (ra["n_accepted"], ra["n_rejected"])
    gth, gph, _, _ = g.get_state()
    assert rel(gth, ra["theta"]) <= 1e-7
    g.close()


def test_uwc_parity(torch_cuda, orc):
    shape = (33, 17, 45)
    g, o = both(orc, shape, 1e-6, I.MODEL_MICRO, 0, case_params(1e-6, I.MODEL_MICRO))
    _, ph, G = I.random_fields(shape, 55)
    ph[::9] = 0.5
    G[::11] = 0.5
    g.set_glass(G)
    g.set_state(None, ph, 0.0, 1e-6)
    for region in (None, (3, 30, 0, 17, 10, 44), (0, 1, 0, 1, 0, 1), (5, 5, 0, 17, 0, 45)):
        a = g.unfrozen_fraction(region)
        b = o.uwc(G, ph, region)
        assert (a["n_water"], a["n_ice"]) == (b["n_water"], b["n_ice"])
        if b["n_water"]:
            assert a["uwc"] == b["uwc"]
            assert abs(a["smooth"] - b["smooth"]) <= 1e-12
    g.close()


def test_temp_uwc_and_state(torch_cuda, orc):
    shape = (20, 21, 22)
    h = 3e-4
    p = case_params(h, I.MODEL_TEMP, zeta=1.0)
    g, o = both(orc, shape, h, I.MODEL_TEMP, 0, p)
    th, _, G = I.random_fields(shape, 8, theta_scale=1.0)
    g.set_glass(G)
    g.set_state(th, None, 0.0, 1e-3)
    _, gph, _, _ = g.get_state()
    oph = o.temp_phi(G, th)
    assert rel(gph, oph) <= 1e-14
    a = g.unfrozen_fraction()
    b = o.uwc(G, oph)
    assert (a["n_water"], a["n_ice"]) == (b["n_water"], b["n_ice"])
    g.close()


def test_max_phase_rate(torch_cuda, orc):
    shape = (30, 20, 40)
    h = 1e-6
    p = case_params(h, I.MODEL_MICRO)
    g, o = both(orc, shape, h, I.MODEL_MICRO, 0, p)
    _, ph, G = I.random_fields(shape, 12)
    g.set_glass(G)
    g.set_state(None, ph, 0.0, 1e-6)
    _, oph = o.rhs(G, None, ph)
    assert abs(g.max_phase_rate() - np.max(np.abs(oph))) <= 1e-12 * np.max(np.abs(oph))
    g.close()


def test_checkpoint_resume_bitwise(torch_cuda):
    from paper_2401_01672_gb300 import pf
    w = I.micro_32()
    g = pf.Grid(w.shape, w.h, w.model, w.reaction, 0, w.params)
    g.set_geometry(w.spheres)
    g.set_state(None, w.phi0, 0.0, w.extra["fixed_dt"])
    g.run_to(0.01, 1e-6)
    _, ph, t, dt = g.get_state()
    g.run_to(0.02, 1e-6)
    _, a, ta, _ = g.get_state()
    g2 = pf.Grid(w.shape, w.h, w.model, w.reaction, 0, w.params)
    g2.set_geometry(w.spheres)
    g2.set_state(None, ph, t, dt)
    g2.run_to(0.02, 1e-6)
    _, b, tb, _ = g2.get_state()
    assert ta == tb and np.array_equal(a, b)
    g.close()
    g2.close()


def test_error_statuses(torch_cuda):
    from paper_2401_01672_gb300 import pf
    p = case_params(1e-6, I.MODEL_MICRO)
    with pytest.raises(pf.PfError) as e:
        pf.Grid((0, 4, 4), 1e-6, I.MODEL_MICRO, 0, 0, p)
    assert e.value.status == pf.PF_E_INVALID
    with pytest.raises(pf.PfError):
        pf.Grid((4, 4, 4), -1.0, I.MODEL_MICRO, 0, 0, p)
    g = pf.Grid((8, 8, 8), 1e-6, I.MODEL_MICRO, 0, 0, p)
    with pytest.raises(pf.PfError) as e:
        g.unfrozen_fraction((0, 9, 0, 8, 0, 8))
    assert e.value.status == pf.PF_E_INVALID
    ph = np.zeros(512)
    ph[100] = np.nan
    g.set_state(None, ph, 0.0, 1e-4)
    with pytest.raises(pf.PfError) as e:
        g.run_to(1.0, 1e-6)
    assert e.value.status == pf.PF_E_NONFINITE
    _, back, t, _ = g.get_state()
    assert t == 0.0 and np.isnan(back[100])
    g.close()
    p2 = case_params(1e-6, I.MODEL_MICRO, dt_min=1e-3)
    g = pf.Grid((8, 8, 8), 1e-6, I.MODEL_MICRO, 0, 0, p2)
    _, ph, G = I.random_fields((8, 8, 8), 3)
    g.set_glass(G)
    g.set_state(None, ph, 0.0, 1e-2)
    with pytest.raises(pf.PfError) as e:
        g.run_to(1.0, 1e-14)
    assert e.value.status == pf.PF_E_DT_UNDERFLOW
    g.close()


@pytest.mark.slow
def test_full_size_rhs_and_step_256(torch_cuda, orc):
    """256^3 full model (the benchmark size; the step in the autotuned launch configuration the bench
    times): right-hand side and one forced Merson step element by element against the oracle, random
    G/theta/phi."""
    torch = torch_cuda
    shape = (256, 256, 256)
    h = 3e-4
    p = I.default_params(xi=h, xi_G=0.4 * h, alpha=4.17e6, dirichlet_faces=I.FACE_ZP, theta_freeze=-5.0)
    g, o = both(orc, shape, h, I.MODEL_FULL, I.REACT_SIGMAP1P, p)
    th, ph, G = I.random_fields(shape, 2024, theta_scale=2.0, smooth=1)
    g.set_glass(G)
    oth, oph = o.rhs(G, th, ph)
    dth = torch.empty(g.N, device="cuda", dtype=torch.float64)
    dph = torch.empty_like(dth)
    g.rhs(0.0, dev(torch, th), dev(torch, ph), dth, dph)
    torch.cuda.synchronize()
    assert rel(dth.cpu().numpy(), oth) <= TOL
    assert rel(dph.cpu().numpy(), oph) <= TOL
    del oth, oph, dth, dph
    dt = 0.01
    g.set_state(th, ph, 0.0, dt)
    g.autotune(None)   # the launch configuration the bench times
    g.rkm_step(dt, 1.0, force_accept=True)
    gth, gph, _, _ = g.get_state()
    sth, sph, _ = o.rkm_step(G, th, ph, 0.0, dt)
    assert rel(gth, sth) <= TOL and rel(gph, sph) <= TOL
    g.close()


def test_full_size_geometry_sampled(torch_cuda, orc):
    """256^3 bead packing at ~60% solid: G at sampled cells (oracle visits every sphere)."""
    w = I.full_bead_case(256, 20240106)
    from paper_2401_01672_gb300 import pf
    g = pf.Grid(w.shape, w.h, w.model, w.reaction, 0, w.params)
    g.set_geometry(w.spheres)
    Gg = g.get_glass()
    o = orc.Oracle(w.shape, w.h, w.model, w.reaction, w.params)
    cells = I.rng(5).integers(0, w.n_cells, 3000)
    Go = o.glass(w.spheres, w.params["xi_G"], cells=cells)
    # conditioning: a rounding of |x - x_i| (up to eps * L) is amplified by 1/(2 xi_G) in the tanh
    # argument and by at most 1/2 in G: bound eps * L / (4 xi_G), L = 256 h
    bound = 4 * np.finfo(float).eps * 256 * w.h / (4 * w.params["xi_G"])
    assert np.max(np.abs(Gg[cells] - Go)) <= bound
    frac = np.mean(Gg >= 0.5)
    assert 0.5 < frac < 0.7
    g.close()


@pytest.mark.parametrize("model", [I.MODEL_FULL, I.MODEL_TEMP])
@pytest.mark.parametrize("harmonic,faces", [(1, I.FACE_ZP), (0, 63), (1, 63)])
def test_rhs_parity_face_options(torch_cuda, orc, model, harmonic, faces):
    """Harmonic-mean face conductivity and Dirichlet temperature on every face."""
    torch = torch_cuda
    shape = (35, 19, 41)
    h = 2e-4
    p = case_params(h, model, harmonic_mean=harmonic, dirichlet_faces=faces)
    g, o = both(orc, shape, h, model, I.REACT_SIGMAP1P, p)
    th, ph, G = I.random_fields(shape, 700 + harmonic + faces, theta_scale=3.0)
    G[::13] = 1.0   # glass-only cells: lambda of both sides exercised
    g.set_glass(G)
    for t in (0.0, 20.0):
        oth, oph = o.rhs(G, th, ph, t=t)
        dth = torch.empty(g.N, device="cuda", dtype=torch.float64)
        dph = torch.empty(g.N, device="cuda", dtype=torch.float64)
        g.rhs(t, dev(torch, th), dev(torch, ph) if model != I.MODEL_TEMP else None, dth, dph)
        torch.cuda.synchronize()
        assert rel(dth.cpu().numpy(), oth) <= TOL
        assert rel(dph.cpu().numpy(), oph) <= TOL
    g.close()
