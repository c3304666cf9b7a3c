"""Pins of the CPU oracle against facts the paper and the mathematics fix.

Each test names the passage or the mathematical fact it relies on.  None of
them re-uses the oracle's own formula to produce the expected value: they use
closed forms (eigenvalues, travelling waves, stability polynomials), exact
invariants, brute force, library ODE solvers, or the paper's printed tables.
"""
import json
import math
import os

import numpy as np
import pytest
from scipy import integrate

from paper_2401_01672_gb300 import inputs as I

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def mk(oracle_mod, shape, h, model, reaction="sigmap1p", **over):
    p = I.default_params(**over)
    return oracle_mod.Oracle(shape, h, model, reaction, p)


# ------------------------------------------------------------------ Table 1/2
def test_table1_constants_consistent():
    """Table 1 (Sec. 2.1): delta_s = rho_I L / T* and alpha = delta_s/(mu sigma) reproduce the printed values."""
    g = json.load(open(os.path.join(GOLD, "table1_materials.json")))
    ds = g["rho"]["I"] * g["latent_L"] / g["T_star"]
    assert abs(ds - g["delta_s_printed"]) / g["delta_s_printed"] < 5e-4
    alpha = ds / (g["mu"] * g["sigma"])
    assert abs(alpha - g["alpha_printed"]) / g["alpha_printed"] < 5e-5
    assert I.TABLE1["rho"] == (g["rho"]["L"], g["rho"]["I"], g["rho"]["G"])
    assert I.TABLE1["c"] == (g["c"]["L"], g["c"]["I"], g["c"]["G"])
    assert I.TABLE1["lambda"] == (g["lambda"]["L"], g["lambda"]["I"], g["lambda"]["G"])
    assert I.TABLE1["alpha"] == g["alpha_printed"]


def test_table2_alpha_regimes():
    """Sec. 3.1: 'large' alpha = rho_L c_L; 'small' is three times larger; 'tiny' sigma ~1000x realistic."""
    g2 = json.load(open(os.path.join(GOLD, "table2_macro_parameters.json")))
    g1 = json.load(open(os.path.join(GOLD, "table1_materials.json")))
    large = g1["rho"]["L"] * g1["c"]["L"]
    assert abs(large - g2["alpha"]["large"]) / large < 2e-3
    assert abs(g2["alpha"]["small"] / g2["alpha"]["large"] - 3) < 0.01
    # sigma_tiny / sigma_real = alpha_real / alpha_tiny ~ 1000 (approximately, as printed)
    assert 500 < g1["alpha_printed"] / g2["alpha"]["tiny"] < 2000
    assert I.ALPHA_MACRO == g2["alpha"]


# ------------------------------------------------------------ Runge-Kutta-Merson
# (closed-form pins first: with -x a broken tableau or estimate fails here in milliseconds, before
# the adaptive runs below, which it would only slow down)
def test_merson_linear_stability_polynomial(oracle_mod):
    """Merson's method applied to y' = lambda y multiplies y by R(z) = 1 + z + z^2/2 + z^3/6 + z^4/24 + z^5/144
    (z = lambda dt), and its error estimate tracks the true local error e^z - R(z) ~ z^5/720 as z -> 0.
    Two cells of uniform water with insulated walls: the difference mode has lambda = -2D/h^2."""
    h = 1e-3
    o = mk(oracle_mod, (2, 1, 1), h, "full", latent=0.0)
    D = 0.6 / (997.0 * 4180.0)
    lam = -2 * D / h ** 2
    for z in (-0.01, -0.1, -0.5, -1.0, -2.5, -3.5):
        dt = z / lam
        a = 0.7
        th, ph, E = o.rkm_step(np.zeros(2), np.array([1.0 + a, 1.0 - a]), np.zeros(2), 0.0, dt)
        R = 1 + z + z * z / 2 + z ** 3 / 6 + z ** 4 / 24 + z ** 5 / 144
        assert abs((th[0] - 1.0) / a - R) < 1e-13
        assert abs(th[0] + th[1] - 2.0) < 1e-14
        # for linear problems the estimate is exactly |z^5 y|/720, the leading term of e^z - R(z)
        # (the combination 2k1-9k3+8k4-k5 cancels to z^4/24 of |k|: allow that cancellation's rounding)
        assert abs(E / (a * abs(z) ** 5 / 720) - 1) < max(1e-9, 2e-14 * 24 / z ** 4)
        if abs(z) <= 0.01:
            assert abs(E / (a * abs(math.exp(z) - R)) - 1) < 0.02


def test_merson_fourth_order_nonlinear(oracle_mod):
    """Fixed-step Merson integration of the one-cell Allen-Cahn ODE phi' = f(phi)/(alpha xi^2) converges
    at order 4 against scipy's DOP853 at tight tolerance (a library routine, independent of the oracle)."""
    h = 1e-6
    xi = 2e-6
    dT = 0.2
    alpha, mu = 1e9, 1e-4
    o = mk(oracle_mod, (1, 1, 1), h, "micro", xi=xi, theta_micro=-dT, alpha=alpha)
    K = 0.5 * xi * mu * alpha * dT
    rate = 1.0 / (alpha * xi * xi)

    def f(t, y):
        p = y[0]
        return [rate * 2 * p * (1 - p) * (p - 0.5 + K)]   # both limiters are 1 on [0.2, 0.8]

    T = 0.4 / rate
    ref = integrate.solve_ivp(f, (0, T), [0.3], method="DOP853", rtol=1e-13, atol=1e-15).y[0, -1]
    assert 0.2 < ref < 0.8 and abs(ref - 0.3) > 0.02  # stays where both limiters are 1
    errs = []
    for n in (8, 16, 32):
        r = o.run(np.zeros(1), None, np.array([0.3]), 0.0, T / n, T, 1.0, n, fixed=True)
        errs.append(abs(r["phi"][0] - ref))
    assert 12 < errs[0] / errs[1] < 20 and 12 < errs[1] / errs[2] < 20


# ------------------------------------------------------------------ geometry
def test_glass_field_sphere_levels(oracle_mod):
    """Sec. 2.1 G_balls: G = 1/2 on the sphere surface, 1/4 and 3/4 at |x-x_i| - r = +-2 xi_G atanh(1/2)."""
    h = 1.0
    xi_G = 0.7
    o = mk(oracle_mod, (40, 3, 3), h, "micro")
    r = 7.0
    # centre on the x axis through cell centres (j = k = 1); cell i has x = i + 1/2
    c = np.array([[10.5, 1.5, 1.5, r]])
    G = o.glass(c, xi_G).reshape(3, 3, 40)[1, 1]
    assert G[10 + 7] == 0.5                      # distance exactly r
    assert abs(G[10] - 0.5 * (1 + math.tanh(r / (2 * xi_G)))) < 1e-15
    # a sphere with r chosen so that a cell centre sits at r + 2 xi_G atanh(1/2): G = 1/4
    for target, sgn in ((0.25, +1), (0.75, -1)):
        rr = 9.0 - sgn * 2 * xi_G * math.atanh(0.5)
        G2 = o.glass(np.array([[10.5, 1.5, 1.5, rr]]), xi_G).reshape(3, 3, 40)[1, 1]
        assert abs(G2[19] - target) < 1e-14
    # monotone decrease away from the centre, in [0, 1]
    assert np.all(np.diff(G[10:]) <= 0) and G.min() >= 0 and G.max() <= 1


def test_glass_field_max_and_cap(oracle_mod):
    """Sec. 2.1: G is the max over beads (overlaps allowed) and the cap term 1/2(1+tanh((x3-x3cap)/(2xi_G)))."""
    h = 1.0
    o = mk(oracle_mod, (6, 6, 12), h, "micro")
    a = o.glass(np.array([[3.0, 3.0, 3.0, 2.0]]), 0.5)
    b = o.glass(np.array([[3.0, 3.0, 6.0, 2.5]]), 0.5)
    ab = o.glass(np.array([[3.0, 3.0, 3.0, 2.0], [3.0, 3.0, 6.0, 2.5]]), 0.5)
    assert np.array_equal(ab, np.maximum(a, b))
    cap = o.glass(np.zeros((0, 4)), 0.5, x3_cap=8.5).reshape(12, 6, 6)
    assert np.all(cap[8] == 0.5)                 # cell centre z = 8.5 on the cap's bottom
    assert np.all(cap[11] > 0.99) and np.all(cap[3] < 1e-4)
    both = o.glass(np.array([[3.0, 3.0, 3.0, 2.0]]), 0.5, x3_cap=8.5)
    assert np.array_equal(both, np.maximum(a, cap.ravel()))


def test_glass_cells_subset_matches_full(oracle_mod):
    o = mk(oracle_mod, (9, 7, 5), 1.0, "micro")
    sp = np.array([[2.0, 3.0, 1.0, 2.2], [6.5, 2.0, 4.0, 1.7]])
    full = o.glass(sp, 0.4)
    cells = np.array([0, 5, 17, 100, 314])
    assert np.array_equal(o.glass(sp, 0.4, cells=cells), full[cells])


# ------------------------------------------------------------- heat equation
def _mode_fields(shape, axis, values):
    n = shape[axis]
    arr = np.zeros(shape[::-1])
    sl = [None, None, None]
    sl[2 - axis] = slice(None)
    arr[...] = values.reshape([n if a == 2 - axis else 1 for a in range(3)])
    return arr.ravel()


@pytest.mark.parametrize("material", ["water", "ice", "glass"])
@pytest.mark.parametrize("axis", [0, 1, 2])
def test_heat_neumann_eigenmode(oracle_mod, material, axis):
    """Textbook FV fact: on a uniform medium with insulated walls, cos(k pi (i+1/2)/N) is an
    eigenvector of the 3-point operator with eigenvalue -(4 D/h^2) sin^2(k pi/(2N)),
    D = lambda/(rho c) of the material in Table 1 (pins the blend corners, the h^2 scaling
    and the zero-flux walls, along each axis)."""
    N = 24
    shape = [2, 3, 4]
    shape[axis] = N
    shape = tuple(shape)
    h = 1e-3
    o = mk(oracle_mod, shape, h, "full", latent=0.0)
    col = {"water": (0, 0.0, 0), "ice": (0, 1.0, 1), "glass": (1.0, 0.37, 2)}[material]
    G = np.full(o.N, float(col[0]))
    phi = np.full(o.N, col[1])
    D = I.TABLE1["lambda"][col[2]] / (I.TABLE1["rho"][col[2]] * I.TABLE1["c"][col[2]])
    for k in (1, 3, 7):
        x = (np.arange(N) + 0.5) / N
        th = _mode_fields(shape, axis, np.cos(k * math.pi * x))
        dth, _ = o.rhs(G, th, phi)
        lam = -(4 * D / h ** 2) * math.sin(k * math.pi / (2 * N)) ** 2
        assert np.max(np.abs(dth - lam * th)) <= 1e-12 * abs(lam)


def test_heat_dirichlet_eigenmode(oracle_mod):
    """Insulated at x=0, Dirichlet T_b on the face x=L (eq. BC-temperature-cap) with the boundary value
    half a cell from the last centre: theta - theta_b = cos((m+1/2) pi (i+1/2)/N) is an eigenvector with
    eigenvalue -(4D/h^2) sin^2((m+1/2) pi/(2N)).  A wrong Dirichlet factor (1 instead of 2) fails it."""
    N = 20
    h = 2e-3
    for tb in (0.0, -3.5):
        o = mk(oracle_mod, (N, 2, 2), h, "full", latent=0.0, dirichlet_faces=I.FACE_XP, theta_freeze=tb)
        G = np.zeros(o.N)
        phi = np.zeros(o.N)
        D = 0.6 / (997.0 * 4180.0)
        for m in (0, 2, 5):
            x = (np.arange(N) + 0.5) / N
            v = np.cos((m + 0.5) * math.pi * x)
            th = _mode_fields((N, 2, 2), 0, v) + tb
            dth, _ = o.rhs(G, th, phi, t=0.0)
            lam = -(4 * D / h ** 2) * math.sin((m + 0.5) * math.pi / (2 * N)) ** 2
            assert np.max(np.abs(dth - lam * (th - tb))) <= 1e-11 * abs(lam)


def test_dirichlet_switch_time(oracle_mod):
    """eq. (BC-temperature-cap): T_freeze before t_freeze, T_thaw after."""
    o = mk(oracle_mod, (4, 1, 1), 1e-3, "full", latent=0.0, dirichlet_faces=I.FACE_XM,
           theta_freeze=-5.0, theta_thaw=3.0, t_freeze=10.0)
    th = np.zeros(4)
    a, _ = o.rhs(np.zeros(4), th, np.zeros(4), t=9.999)
    b, _ = o.rhs(np.zeros(4), th, np.zeros(4), t=10.0)
    assert a[0] < 0 and b[0] > 0 and abs(a[0] / b[0] + 5.0 / 3.0) < 1e-14
    assert np.all(a[1:] == 0) and np.all(b[1:] == 0)


def _blend(G, phi, w):
    return G * w[2] + (1 - G) * (phi * w[1] + (1 - phi) * w[0])


@pytest.mark.parametrize("faces", [0, I.FACE_ZP | I.FACE_XM])
def test_enthalpy_identity_full(oracle_mod, faces):
    """eq. (heat-equation) summed over finite volumes: sum_i [rho c dtheta - rho L dphi]_i h^3 equals the
    net boundary heat flow (interior face fluxes cancel pairwise).  Zero for insulated walls."""
    shape = (7, 6, 5)
    h = 1e-3
    o = mk(oracle_mod, shape, h, "full", dirichlet_faces=faces, theta_freeze=-4.0, alpha=4.17e6, xi=h)
    th, ph, G = I.random_fields(shape, 11)
    dth, dph = o.rhs(G, th, ph)
    p = o.params
    rho = _blend(G, ph, p["rho"])
    c = _blend(G, ph, p["c"])
    lam = _blend(G, ph, p["lambda"])
    total = np.sum(rho * c * dth - rho * p["latent"] * dph)
    bnd = 0.0
    t3 = th.reshape(5, 6, 7)
    l3 = lam.reshape(5, 6, 7)
    if faces & I.FACE_ZP:
        bnd += np.sum(2 * l3[-1] * (-4.0 - t3[-1])) / h ** 2
    if faces & I.FACE_XM:
        bnd += np.sum(2 * l3[:, :, 0] * (-4.0 - t3[:, :, 0])) / h ** 2
    scale = np.sum(np.abs(rho * c * dth)) + 1.0
    assert abs(total - bnd) <= 1e-12 * scale


def test_enthalpy_conserved_by_rkm(oracle_mod):
    """With rho and c equal for ice and water, H = sum(rho c theta - rho L phi) is a linear first integral
    of the insulated semi-discrete system, so every Runge-Kutta step keeps it to rounding."""
    shape = (6, 5, 7)
    h = 1e-3
    o = mk(oracle_mod, shape, h, "full", rho=(997.0, 997.0, 2500.0), c=(4180.0, 4180.0, 840.0),
           alpha=4.17e6, xi=h)
    th, ph, G = I.random_fields(shape, 5, theta_scale=2.0)
    p = o.params
    rho = _blend(G, ph, p["rho"])        # phi-independent here
    c = _blend(G, ph, p["c"])
    H0 = np.sum(rho * c * th - rho * p["latent"] * ph)
    res = o.run(G, th, ph, 0.0, 0.02, 0.5, 1e-6, 30, fixed=True)
    H1 = np.sum(rho * c * res["theta"] - rho * p["latent"] * res["phi"])
    assert res["n_accepted"] == 25
    assert abs(H1 - H0) <= 1e-13 * np.sum(np.abs(rho * p["latent"] * ph) + np.abs(rho * c * th))


def test_temp_model_identity(oracle_mod):
    """eq. (combined-heat-xfer-phase-transition) with rho, c equal for ice and water:
    sum rho (c theta' - L phi'(T) theta') = sum div(lambda grad T) = 0 for insulated walls; and
    the Temp phase field is eq. (explicit-p-dependence-on-T)."""
    shape = (5, 6, 7)
    h = 1e-3
    o = mk(oracle_mod, shape, h, "temp", rho=(997.0, 997.0, 2500.0), c=(4180.0, 4180.0, 840.0), gamma=2.0)
    th, _, G = I.random_fields(shape, 9, theta_scale=1.0)
    dth, dph = o.rhs(G, th, None)
    p = o.params
    rho = _blend(G, 0.0, p["rho"])
    c = _blend(G, 0.0, p["c"])
    total = np.sum(rho * c * dth - rho * p["latent"] * dph)
    assert abs(total) <= 1e-12 * np.sum(np.abs(rho * c * dth))
    phi = o.temp_phi(G, th)
    IW = np.maximum(0.0, 1 - 2.0 * G)
    assert np.allclose(phi[IW == 0], 0.0)
    # phi = 1/2 I_W at theta = 0, -> I_W for theta << 0, -> 0 for theta >> 0
    z = o.temp_phi(G, np.zeros(o.N))
    assert np.allclose(z, 0.5 * IW, rtol=0, atol=1e-15)
    assert np.allclose(o.temp_phi(G, np.full(o.N, -50.0)), IW, atol=1e-15)
    assert np.allclose(o.temp_phi(G, np.full(o.N, 50.0)), 0.0, atol=1e-15)


# ----------------------------------------------------------- Allen-Cahn part
def _interface_position(phi_line, h):
    """x where phi crosses 1/2 (linear interpolation between cell centres)."""
    s = np.where((phi_line[:-1] - 0.5) * (phi_line[1:] - 0.5) <= 0)[0]
    i = s[0]
    a, b = phi_line[i], phi_line[i + 1]
    return (i + 0.5 + (0.5 - a) / (b - a)) * h


def test_planar_profile_stationary_second_order(oracle_mod):
    """Sec. 2.2: phi = 1/2(1 + tanh((x-x0)/(2 xi))) solves xi^2 phi'' + 2 phi (1-phi)(phi-1/2) = 0, so at
    T = T* the discrete right-hand side vanishes as (h/xi)^2 (pins the Laplacian scaling and the
    double-well term's sign)."""
    res = []
    for m in (2, 4, 8):
        h = 1e-6
        xi = m * h
        N = 40 * m
        o = mk(oracle_mod, (N, 1, 1), h, "micro", xi=xi, theta_micro=0.0, alpha=1e9)
        x = (np.arange(N) + 0.5) * h
        phi = 0.5 * (1 + np.tanh((x - N * h / 2) / (2 * xi)))
        _, dph = o.rhs(np.zeros(N), None, phi)
        res.append(np.max(np.abs(dph)) * o.params["alpha"] * xi * xi)
    assert res[0] / res[1] > 3.5 and res[1] / res[2] > 3.8
    assert res[2] < 2e-4


def _front_speed(oracle_mod, reaction, xi_over_h, dT, alpha, N, t_end):
    h = 1e-6
    xi = xi_over_h * h
    o = mk(oracle_mod, (N, 1, 1), h, "micro", reaction, xi=xi, theta_micro=-dT, alpha=alpha)
    x = (np.arange(N) + 0.5) * h
    x0 = 0.75 * N * h
    phi = 0.5 * (1 + np.tanh((x - x0) / (2 * xi)))   # ice on the right
    G = np.zeros(N)
    # relax the profile shape first, then time the motion
    r0 = o.run(G, None, phi, 0.0, 1e-5, 0.2 * t_end, 1e-9, 10 ** 6)
    p0 = _interface_position(r0["phi"], h)
    r1 = o.run(G, None, r0["phi"], r0["t"], r0["dt"], t_end, 1e-9, 10 ** 6)
    p1 = _interface_position(r1["phi"], h)
    return (p0 - p1) / (r1["t"] - r0["t"])            # speed of ice growth to the left


def test_gradp_travelling_wave_speed(oracle_mod):
    """eq. (reaction-term-GradP): at constant supercooling dT the tanh profile travels exactly at
    v = mu dT (ice grows), since xi^2 mu alpha |grad phi| dT = xi mu alpha dT phi(1-phi).
    Gibbs-Thomson law, eq. (Gibbs-Thomson), for a planar front (kappa = 0)."""
    mu, dT, alpha = 1e-4, 10.0, 1e9
    v = _front_speed(oracle_mod, "gradp", 8, dT, alpha, 400, 0.1)
    assert abs(v / (mu * dT) - 1.0) < 0.02


def test_sigmap1p_front_speed_matches_solvability(oracle_mod):
    """eq. (reaction-term-SigmaP1-P) with small xi mu alpha dT: first-order solvability gives
    v = 6 b mu dT * int_0^1 phi(1-phi) Sigma(phi) Sigma(1-phi) dphi (the integral is 1/6 without the
    limiter).  The ratio to the GradP speed on the same mesh cancels most of the mesh error.
    A dropped or mis-shaped limiter (eq. Sigma-limiter) changes the ratio by ~10%."""
    e0, e1 = 0.05, 0.2

    def S(w):
        if w <= e0:
            return 0.0
        if w >= e1:
            return 1.0
        s = (w - e0) / (e1 - e0)
        return s * s * (3 - 2 * s)

    Iint = integrate.quad(lambda p: p * (1 - p) * S(p) * S(1 - p), 0, 1, points=[e0, e1, 1 - e1, 1 - e0],
                          epsabs=1e-14)[0]
    expect = 6 * Iint
    assert 0.89 < expect < 0.93
    mu, alpha = 1e-4, 1e9
    xi = 8e-6
    dT = 0.02 / (xi * mu * alpha)
    t_end = 40e-6 / (mu * dT)
    vs = _front_speed(oracle_mod, "sigmap1p", 8, dT, alpha, 300, t_end)
    vg = _front_speed(oracle_mod, "gradp", 8, dT, alpha, 300, t_end)
    assert abs(vs / vg - expect) < 0.015
    assert abs(vg / (mu * dT) - 1) < 0.03


@pytest.mark.parametrize("reaction", ["sigmap1p", "gradp"])
def test_gibbs_thomson_critical_radius(oracle_mod, reaction):
    """eq. (Gibbs-Thomson) with v = 0 and kappa = 2/R (sphere): a grain of ice at supercooling dT is in
    (unstable) equilibrium at R* = 2/(mu alpha dT).  Smaller grains melt, larger grains grow.
    Octant of a sphere in a corner with mirror walls = a full sphere."""
    h = 1e-6
    N = 30
    xi = 1.5 * h
    alpha, mu = 1e9, 1e-4
    Rstar = 11.0 * h
    dT = 2.0 / (mu * alpha * Rstar)
    o = mk(oracle_mod, (N, N, N), h, "micro", reaction, xi=xi, theta_micro=-dT, alpha=alpha)
    z, y, x = np.meshgrid(*(np.arange(N) + 0.5,) * 3, indexing="ij")
    r = np.sqrt(x * x + y * y + z * z).ravel() * h
    G = np.zeros(o.N)
    vols = {}
    for f in (0.7, 1.4):
        R0 = f * Rstar
        phi = 0.5 * (1 - np.tanh((r - R0) / (2 * xi)))
        # let the diffuse profile form, then measure the volume trend
        t1 = 0.25 * Rstar / (mu * dT)
        a = o.run(G, None, phi, 0.0, 1e-5, t1, 1e-7, 10 ** 5)
        b = o.run(G, None, a["phi"], a["t"], a["dt"], 2 * t1, 1e-7, 10 ** 5)
        vols[f] = (a["phi"].sum(), b["phi"].sum())
    assert vols[0.7][1] < vols[0.7][0]          # subcritical: melts
    assert vols[1.4][1] > vols[1.4][0]          # supercritical: grows


def test_sigma_limiter_special_values(oracle_mod):
    """eq. (Sigma-limiter) through a one-cell micro model (no Laplacian): below eps0 the latent driving
    term vanishes; between eps1 and 1-eps1 both limiters are 1; at (eps0+eps1)/2 the smoothstep is 1/2."""
    h = 1e-6
    xi = 2e-6
    dT = 0.3
    alpha, mu = 1e9, 1e-4
    o = mk(oracle_mod, (1, 1, 1), h, "micro", xi=xi, theta_micro=-dT, alpha=alpha)
    K = 0.5 * xi * mu * alpha * dT

    def f_of(phi):
        _, d = o.rhs(np.zeros(1), None, np.array([phi]))
        return d[0] * alpha * xi * xi

    for p in (0.0, 0.01, 0.05, 0.95, 1.0):
        assert abs(f_of(p) - 2 * p * (1 - p) * (p - 0.5)) < 1e-15
    for p in (0.2, 0.35, 0.5, 0.8):
        assert abs(f_of(p) - 2 * p * (1 - p) * (p - 0.5 + K)) < 1e-14
    pm = 0.125
    assert abs(f_of(pm) - 2 * pm * (1 - pm) * (pm - 0.5 + 0.5 * K)) < 1e-14
    # continuity of f at the limiter's corners
    for c in (0.05, 0.2, 0.8, 0.95):
        assert abs(f_of(c + 1e-9) - f_of(c - 1e-9)) < 1e-8


def test_water_indicator_freezes_glass(oracle_mod):
    """eq. (water-indicator) with zeta = 2 (Sec. 3.1): I_W = 0 where G >= 1/2, so phi never changes
    there; with zeta = 1, I_W > 0 for G < 1."""
    shape = (8, 7, 6)
    o = mk(oracle_mod, shape, 1e-6, "micro", xi=1e-6, alpha=1e9, zeta=2.0, theta_micro=-0.4)
    th, ph, G = I.random_fields(shape, 3)
    _, dph = o.rhs(G, None, ph)
    assert np.all(dph[G >= 0.5] == 0.0)
    o1 = mk(oracle_mod, shape, 1e-6, "micro", xi=1e-6, alpha=1e9, zeta=1.0, theta_micro=-0.4)
    _, dph1 = o1.rhs(G, None, ph)
    sel = (G >= 0.5) & (G < 1.0) & (np.abs(dph1) > 0)
    assert sel.sum() > 10


def test_micro_model_invariants(oracle_mod):
    """Sec. 2.4 (lambda = L = 0): temperature stays at T* - dT exactly, phi stays in [0, 1] for
    SigmaP1-P, and cells with I_W = 0 keep their phi bit for bit over many steps."""
    w = I.micro_32()
    n = 16
    shape = (n, n, n)
    o = mk(oracle_mod, shape, w.h, "micro", **{k: w.params[k] for k in ("xi", "xi_G", "zeta", "theta_micro")})
    sp = np.array([[4e-7, 4e-7, 4e-7, 2.5e-7], [6e-7, 2e-7, 5e-7, 2.0e-7]])
    G = o.glass(sp, w.params["xi_G"])
    phi = I.ball_indicator(shape, (12.0, 11.0, 4.0), 3.0)
    phi = np.maximum(phi, (G > 0.7).astype(float))   # ice planted inside glass too
    r = o.run(G, None, phi, 0.0, 2e-5, 0.01, 1e-6, 200)
    assert r["status"] == 0 and r["n_accepted"] > 20
    out = r["phi"]
    assert out.min() >= -1e-12 and out.max() <= 1 + 1e-12
    frozen = G >= 0.5
    assert np.array_equal(out[frozen], phi[frozen])


def test_gradp_may_leave_unit_interval_sigmap1p_does_not(oracle_mod):
    """Sec. 3.2: GradP can produce phi > 1 where the diffuse interface is distorted by glass, while
    SigmaP1-P keeps phi in [0, 1].  Ice fills the water half of the box; phi is pinned to 0 in the
    glass half (I_W = 0 with zeta = 2), so |grad phi| > 0 on ice cells where phi = 1."""
    n = 8
    shape = (n, n, n)
    h = 1e-6
    base = dict(xi=h, alpha=1e9, zeta=2.0, theta_micro=-40.0)
    G = np.zeros((n, n, n))
    G[:, :, 4:] = 1.0
    G = G.ravel()
    phi = (G == 0).astype(float)
    hi = {}
    for rx in ("gradp", "sigmap1p"):
        o = mk(oracle_mod, shape, h, "micro", rx, **base)
        r = o.run(G, None, phi, 0.0, 1e-6, 2e-3, 1e-7, 400)
        hi[rx] = r["phi"].max()
    assert hi["sigmap1p"] <= 1 + 1e-12
    assert hi["gradp"] > 1 + 1e-3


def test_run_lands_on_switch_times_and_counts(oracle_mod):
    """Adaptive stepping never crosses t_freeze or t_end (eq. BC-temperature-cap switches there) and
    every attempt is either accepted (E <= tol) or rejected."""
    shape = (6, 4, 5)
    h = 1e-3
    o = mk(oracle_mod, shape, h, "full", dirichlet_faces=I.FACE_ZP, theta_freeze=-5.0, theta_thaw=2.0,
           t_freeze=3.0, alpha=4.17e6, xi=h)
    th = np.full(o.N, 1.0)
    ph = I.top_slab_indicator(shape, 1)
    G = np.zeros(o.N)
    r = o.run(G, th, ph, 0.0, 0.05, 5.0, 1e-5, 5000, trace=True)
    tr = r["trace"]
    assert r["t"] == 5.0 and r["status"] == 0
    acc = tr[tr[:, 3] == 1]
    ends = acc[:, 0] + acc[:, 1]
    assert np.any(np.abs(ends - 3.0) < 1e-15)
    starts = acc[:, 0]
    assert np.all((starts >= 3.0) | (ends <= 3.0 + 1e-15))
    assert r["n_accepted"] == int((tr[:, 3] == 1).sum())
    assert np.all(tr[tr[:, 3] == 1, 2] <= 1e-5)
    assert np.all(tr[tr[:, 3] == 0, 2] > 1e-5)
    # proposal law (reading): next dt = dt * min(5, 0.8 (tol/E)^(1/5))
    for a, b in zip(tr[:-1], tr[1:]):
        if b[0] + b[1] >= 3.0 - 1e-12 and abs(b[0] + b[1] - 3.0) < 1e-12:
            continue
        if abs(b[0] + b[1] - 5.0) < 1e-12:
            continue
        exp = a[1] * (5.0 if a[2] == 0 else min(5.0, 0.8 * (1e-5 / a[2]) ** 0.2))
        assert abs(b[1] - exp) <= 1e-15 * exp


def test_dt_underflow_status(oracle_mod):
    shape = (4, 4, 4)
    o = mk(oracle_mod, shape, 1e-3, "full", alpha=4.17e6, xi=1e-3, dt_min=1.0)
    th, ph, G = I.random_fields(shape, 2)
    r = o.run(G, th, ph, 0.0, 5.0, 100.0, 1e-12, 50)
    assert r["status"] == -4


# ------------------------------------------------------------- symmetry / UWC
def test_rhs_symmetries(oracle_mod):
    """The operator commutes with axis permutations and reflections of the grid (isotropic
    stencil, symmetric face conductivity, mirror walls).  A transposed stride or a one-sided
    index fails this on a non-cubic grid."""
    shape = (7, 9, 11)
    h = 1e-3
    for model, rx in (("full", "sigmap1p"), ("full", "gradp"), ("temp", "sigmap1p")):
        o = mk(oracle_mod, shape, h, model, rx, alpha=4.17e6, xi=h)
        th, ph, G = I.random_fields(shape, 21)
        a_th, a_ph = o.rhs(G, th, ph)
        A = lambda v: v.reshape(11, 9, 7)
        # reflect x
        rf = lambda v: A(v)[:, :, ::-1].ravel()
        b_th, b_ph = o.rhs(rf(G), rf(th), rf(ph))
        assert np.allclose(b_th, rf(a_th), rtol=1e-12, atol=1e-12 * np.abs(a_th).max())
        assert np.allclose(b_ph, rf(a_ph), rtol=1e-12, atol=1e-12 * np.abs(a_ph).max())
        # swap x <-> z : shape becomes (11, 9, 7)
        o2 = mk(oracle_mod, (11, 9, 7), h, model, rx, alpha=4.17e6, xi=h)
        tp = lambda v: np.transpose(A(v), (2, 1, 0)).ravel()
        c_th, c_ph = o2.rhs(tp(G), tp(th), tp(ph))
        assert np.allclose(c_th, tp(a_th), rtol=1e-12, atol=1e-12 * np.abs(a_th).max())
        assert np.allclose(c_ph, tp(a_ph), rtol=1e-12, atol=1e-12 * np.abs(a_ph).max())


def test_uwc_brute_force(oracle_mod):
    """eqs. (water-occupied-subdomain), (frozen-subdomain), (UWC-formula) by a numpy count."""
    shape = (13, 10, 9)
    o = mk(oracle_mod, shape, 1.0, "micro")
    _, ph, G = I.random_fields(shape, 4)
    ph[::7] = 0.5
    G[::5] = 0.5
    for region in (None, (2, 11, 0, 10, 4, 9), (0, 13, 0, 10, 0, 5)):
        r = o.uwc(G, ph, region)
        g3, p3 = G.reshape(9, 10, 13), ph.reshape(9, 10, 13)
        if region is not None:
            i0, i1, j0, j1, k0, k1 = region
            g3, p3 = g3[k0:k1, j0:j1, i0:i1], p3[k0:k1, j0:j1, i0:i1]
        w = g3 < 0.5
        ice = w & (p3 > 0.5)
        assert r["n_water"] == int(w.sum()) and r["n_ice"] == int(ice.sum())
        assert abs(r["uwc"] - (1 - ice.sum() / w.sum())) < 1e-15
        assert abs(r["smooth"] - (1 - ((1 - g3) * p3).sum() / (1 - g3).sum())) < 1e-12


def test_temp_phase_rate_is_chain_rule(oracle_mod):
    """Sec. 2.3: dphi/dt = phi'(T) dT/dt with phi(T) of eq. (explicit-p-dependence-on-T); phi' is checked
    against central finite differences of phi(T) itself."""
    shape = (6, 5, 4)
    for gamma in (2.0, 10.0):
        o = mk(oracle_mod, shape, 1e-3, "temp", gamma=gamma, zeta=1.0)
        th, _, G = I.random_fields(shape, 14, theta_scale=0.5)
        dth, dph = o.rhs(G, th, None)
        d = 1e-6
        fd = (o.temp_phi(G, th + d) - o.temp_phi(G, th - d)) / (2 * d)
        sel = np.abs(dth) > 1e-12 * np.max(np.abs(dth))
        assert np.allclose(dph[sel] / dth[sel], fd[sel], rtol=1e-6, atol=1e-9 * np.max(np.abs(fd)))


def test_steps_land_exactly_on_switch_times(oracle_mod):
    """Steps are shortened to end exactly at t_freeze and t_end (eq. BC-temperature-cap switches there):
    the step after the landing one starts at t_freeze exactly, for switching times that are not
    representable sums of the step sizes."""
    shape = (5, 4, 4)
    h = 1e-3
    for tf, te in ((1.0 / 3.0 * 10, 5.1), (2.718281828459045, 4.9), (1.4142135623730951, 3.3)):
        o = mk(oracle_mod, shape, h, "full", dirichlet_faces=I.FACE_ZP, theta_freeze=-5.0, theta_thaw=2.0,
               t_freeze=tf, alpha=4.17e6, xi=h)
        r = o.run(np.zeros(o.N), np.full(o.N, 1.0), I.top_slab_indicator(shape, 1), 0.0, 0.07, te, 1e-5, 5000,
                  trace=True)
        acc = r["trace"][r["trace"][:, 3] == 1]
        assert r["t"] == te
        assert np.any(acc[:, 0] == tf)
        assert np.all(acc[:, 1] > 1e-9)


def test_long_step_lands_exactly(oracle_mod):
    """A step shortened to reach t_freeze from t = 0.7 ends exactly at t_freeze even where
    0.7 + (t_freeze - 0.7) rounds past it (t_freeze = 10/3 and e): the following step starts at t_freeze."""
    for tf in (10.0 / 3.0, 2.718281828459045):
        o = mk(oracle_mod, (1, 1, 1), 1e-6, "micro", xi=1e-6, alpha=1e9, t_freeze=tf)
        r = o.run(np.zeros(1), None, np.array([0.3]), 0.7, 100.0, 50.0, 1.0, 2, fixed=True, trace=True)
        assert r["trace"][1, 0] == tf


# ------------------------------------------------------------------ threads and non-finite estimates
def test_results_do_not_depend_on_thread_count(oracle_mod):
    """The loops over cells may run on several threads: a Merson step, the glass field and an adaptive
    run are bit-identical with one thread and with all of them."""
    shape = (23, 17, 19)
    h = 3e-4
    o = mk(oracle_mod, shape, h, "full", alpha=4.17e6, xi=h, xi_G=0.4 * h, dirichlet_faces=I.FACE_ZP,
           theta_freeze=-5.0)
    sv, _ = I.packing_boolean(shape, 0.5, I.uniform_radius(3.0, 5.0), 5)
    th0, ph0, _ = I.random_fields(shape, 9, theta_scale=2.0)
    full = oracle_mod.threads()
    out = []
    try:
        for n in (1, max(full, 2)):
            oracle_mod.threads(n)
            G = o.glass(sv * h, 0.4 * h)
            th, ph, E = o.rkm_step(G, th0, ph0, 0.0, 0.01)
            r = o.run(G, th0, ph0, 0.0, 0.01, 0.3, 1e-6, 100)
            out.append((G, th, ph, E, r["theta"], r["phi"], r["n_accepted"], r["n_rejected"]))
    finally:
        oracle_mod.threads(full)
    a, b = out
    for x, y in zip(a, b):
        assert np.array_equal(np.asarray(x), np.asarray(y))


def test_error_estimate_keeps_a_nan(oracle_mod):
    """A NaN anywhere in the state makes the error estimate NaN (the run then stops as non-finite),
    wherever the NaN sits in the visiting order and however many threads visit the cells."""
    shape = (16, 4, 4)
    o = mk(oracle_mod, shape, 1e-6, "micro", xi=1e-6, alpha=3e9, theta_micro=-0.5)
    full = oracle_mod.threads()
    try:
        for n in (1, max(full, 2)):
            oracle_mod.threads(n)
            for pos in (0, 5, o.N - 1):
                ph = np.full(o.N, 0.25)
                ph[pos] = math.nan
                _, _, E = o.rkm_step(np.zeros(o.N), None, ph, 0.0, 1e-9)
                assert math.isnan(E), (n, pos)
    finally:
        oracle_mod.threads(full)
