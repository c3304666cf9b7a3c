"""Seeded input generators that feed both sides: the macro vessel of Sec. 3.1 (settled bead bed
stand-in, nucleation disk of eq. nucleation-site) checked against their definitions."""
import math

import numpy as np

from paper_2401_01672_gb300 import inputs as I


def test_settled_bed_is_a_valid_packing():
    L1 = L2 = 0.03
    r = 0.003
    top = 0.036
    sp = I.settled_bed(L1, L2, r, top, seed=5)
    assert len(sp) > 50 and np.all(sp[:, 3] == r)
    c = sp[:, :3]
    # inside the walls and on or above the floor, below the bed top
    assert np.all(c[:, 0] >= r) and np.all(c[:, 0] <= L1 - r)
    assert np.all(c[:, 1] >= r) and np.all(c[:, 1] <= L2 - r)
    assert np.all(c[:, 2] >= r * (1 - 1e-12)) and np.all(c[:, 2] + r <= top * (1 + 1e-12))
    # no two spheres overlap (touching allowed to rounding)
    d = np.sqrt(((c[:, None, :] - c[None, :, :]) ** 2).sum(-1))
    np.fill_diagonal(d, np.inf)
    assert d.min() >= 2 * r * (1 - 1e-9)
    # every sphere rests on the floor or on an earlier sphere
    for q in range(len(c)):
        if c[q, 2] > r * (1 + 1e-9):
            assert np.any(np.abs(d[q, :q] - 2 * r) <= 1e-9 * r)
    # deterministic under its seed
    assert np.array_equal(sp, I.settled_bed(L1, L2, r, top, seed=5))


def test_nucleation_disk_matches_its_definition():
    n3 = 100
    shape = (n3 // 2, n3 // 2, n3)
    L3 = I.MACRO_L3
    h = L3 / n3
    f = I.nucleation_disk(shape, h, L3 / 2, L3 / 2, L3).reshape(n3, n3 // 2, n3 // 2)
    assert set(np.unique(f)) == {0.0, 1.0}
    k = np.nonzero(f.any(axis=(1, 2)))[0]
    z = (k + 0.5) * h
    assert np.all(z > 0.87 * L3) and np.all(z < 0.97 * L3)
    # cell count close to the disk volume (pi (L1/3)^2 x 0.1 L3) in cells
    vol = math.pi * (L3 / 6) ** 2 * 0.1 * L3 / h ** 3
    assert abs(f.sum() - vol) / vol < 0.08


def test_macro_case_parameters_follow_table2():
    w = I.macro_case(100, I.MODEL_FULL, I.REACT_SIGMAP1P, sigma="small")
    p = w.params
    assert w.shape == (50, 50, 100) and math.isclose(w.h, 6e-4)
    assert math.isclose(p["xi"], 0.06 / 100) and math.isclose(p["xi_G"], 0.06 / 500)
    assert p["alpha"] == 1.25e7 and p["zeta"] == 2.0 and p["dirichlet_faces"] == I.FACE_ZP
    assert (p["theta_freeze"], p["theta_thaw"], p["t_freeze"]) == (-25.0, 20.0, 5 * 3600.0)
    assert math.isclose(w.x3_cap, 11 / 12 * 0.06) and np.all(w.theta0 == 20.0)
    t = I.macro_case(100, I.MODEL_TEMP, gamma=10.0)
    assert t.phi0 is None and t.params["zeta"] == 1.0 and t.params["gamma"] == 10.0


def test_fcc_bed_is_a_jittered_lattice():
    L1 = L2 = 50e-6
    r = 5e-6
    top = 60e-6
    gap = 0.02
    sp = I.fcc_bed(L1, L2, top, r, seed=3, gap=gap)
    c = sp[:, :3]
    assert len(sp) > 60
    assert np.all(c[:, :2] >= r) and np.all(c[:, 0] <= L1 - r) and np.all(c[:, 1] <= L2 - r)
    assert np.all(c[:, 2] >= r) and np.all(c[:, 2] <= top - r)
    d = np.sqrt(((c[:, None, :] - c[None, :, :]) ** 2).sum(-1))
    np.fill_diagonal(d, np.inf)
    nn = d.min(axis=1)
    # no contacts; every sphere within the jitter of the lattice's nearest-neighbour distance
    assert nn.min() > 2 * r
    assert np.all(nn <= 2 * r * (1 + gap) + 0.98 * gap * r + 1e-12)
    # 12 lattice neighbours for spheres away from the walls
    inner = np.all((c > 3 * r) & (c < np.array([L1, L2, top]) - 3 * r), axis=1)
    assert np.any(inner)
    counts = (d[inner] < 2 * r * (1 + 2 * gap)).sum(axis=1)
    assert np.all(counts == 12)


def test_uwc_instances_region_and_time_scales():
    ins = I.uwc_instances(dTs=(0.1, 1.0), beds=("fcc", "settled"), n3=60)
    assert [i.label for i in ins] == ["fcc", "fcc", "settled", "settled"]
    i = ins[1]
    assert i.shape == (30, 30, 60) and i.region == (0, 30, 0, 30, 0, 30)
    assert math.isclose(i.params["theta_micro"], -1.0) and i.params["alpha"] == I.TABLE1["alpha"]
    v = i.params["mu"] * 1.0
    assert math.isclose(i.eq_window, 20 * i.h / v) and math.isclose(i.t_end, 20 * 100e-6 / v)
