"""Seeded synthetic inputs shared by the CUDA path, the oracle tests and the bench.

This module holds NO arithmetic of the method (no glass field, no blends, no
right-hand side, no integrator).  It only produces the inputs the method is
run on: the paper's printed material constants (Table 1), parameter sets
(Table 2 and the voxel readings of the workloads), sphere packings, initial
fields and random test fields.  Every random draw comes from numpy's PCG64
generator with an explicit seed, so the same call gives the same input on any
machine.

Geometry is produced in voxel units and returned in metres (x, y, z, r) rows:
cell (i, j, k) has its centre at ((i+1/2)h, (j+1/2)h, (k+1/2)h).  The solid
fraction used to stop the Boolean packer is a sharp voxel count of points
inside some sphere; it is a property of the synthetic packing, not of the
paper's smooth glass field G.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

LIQUID, ICE, GLASS = 0, 1, 2

# Table 1 of the paper (Sec. 2.1): physical properties, SI units.
TABLE1 = {
    "rho": (997.0, 917.0, 2500.0),      # kg m^-3      liquid, ice, glass
    "c": (4180.0, 2050.0, 840.0),       # J kg^-1 K^-1
    "lambda": (0.6, 2.22, 1.1),         # W m^-1 K^-1
    "latent": 3.34e5,                   # J kg^-1
    "T_star": 273.15,                   # K
    "sigma": 0.033,                     # J m^-2
    "delta_s": 1.121e6,                 # J m^-3 K^-1 (printed)
    "mu": 1.0e-4,                       # m s^-1 K^-1
    "alpha": 3.39782e11,                # s m^-2 (printed)
}

# Table 2 of the paper (Sec. 3.1): alpha for the "large", "small", "tiny" sigma cases.
ALPHA_MACRO = {"large": 4.17e6, "small": 1.25e7, "tiny": 3.7e8}

MODEL_FULL, MODEL_TEMP, MODEL_MICRO = 0, 1, 2
REACT_SIGMAP1P, REACT_GRADP = 0, 1
PREC_FP64, PREC_FP32 = 0, 1

# Face bits for Dirichlet temperature faces: x-, x+, y-, y+, z-, z+.
FACE_XM, FACE_XP, FACE_YM, FACE_YP, FACE_ZM, FACE_ZP = 1, 2, 4, 8, 16, 32


def default_params(**over) -> dict:
    """Parameter dictionary with Table 1 materials and the Table 2 limiter values.

    Keys mirror the C-ABI struct ``pf_params``; temperatures are offsets
    theta = T - T* in kelvin.  ``over`` replaces entries.
    """
    p = {
        "rho": TABLE1["rho"],
        "c": TABLE1["c"],
        "lambda": TABLE1["lambda"],
        "latent": TABLE1["latent"],
        "mu": TABLE1["mu"],
        "alpha": TABLE1["alpha"],
        "xi": 1.0e-3,
        "xi_G": 1.0e-3,
        "eps0": 0.05,
        "eps1": 0.2,
        "b": 1.0,
        "gamma": 2.0,
        "zeta": 2.0,
        "theta_micro": -0.5,
        "theta_freeze": -25.0,
        "theta_thaw": 20.0,
        "t_freeze": math.inf,
        "dt_min": 1e-300,
        "dt_max": math.inf,
        "dirichlet_faces": 0,
        "harmonic_mean": 0,
    }
    for k, v in over.items():
        if k not in p:
            raise KeyError(f"unknown parameter {k!r}")
        p[k] = v
    return p


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


# ----------------------------------------------------------------- packings
def _stamp(mask: np.ndarray, c, r):
    """Mark voxels whose centres are inside the sphere (c, r) (voxel units, centre at i+1/2)."""
    n1, n2, n3 = mask.shape[2], mask.shape[1], mask.shape[0]
    lo = [max(0, int(math.floor(c[d] - r - 0.5))) for d in range(3)]
    hi = [min((n1, n2, n3)[d], int(math.ceil(c[d] + r + 0.5)) + 1) for d in range(3)]
    if any(lo[d] >= hi[d] for d in range(3)):
        return
    xs = np.arange(lo[0], hi[0]) + 0.5 - c[0]
    ys = np.arange(lo[1], hi[1]) + 0.5 - c[1]
    zs = np.arange(lo[2], hi[2]) + 0.5 - c[2]
    d2 = zs[:, None, None] ** 2 + ys[None, :, None] ** 2 + xs[None, None, :] ** 2
    mask[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]] |= d2 < r * r


def packing_rsa(shape, n_spheres, r_lo, r_hi, seed, max_tries=200000):
    """Random sequential addition of non-overlapping spheres lying inside the box.

    shape = (n1, n2, n3) cells; radii uniform in [r_lo, r_hi] voxels.
    Returns an (n, 4) array of (x, y, z, r) in voxel units.
    """
    g = rng(seed)
    n1, n2, n3 = shape
    out = []
    tries = 0
    while len(out) < n_spheres:
        tries += 1
        if tries > max_tries:
            raise RuntimeError("RSA packing did not converge")
        r = g.uniform(r_lo, r_hi)
        c = (g.uniform(r, n1 - r), g.uniform(r, n2 - r), g.uniform(r, n3 - r))
        ok = True
        for (x, y, z, rr) in out:
            if (x - c[0]) ** 2 + (y - c[1]) ** 2 + (z - c[2]) ** 2 < (r + rr) ** 2:
                ok = False
                break
        if ok:
            out.append((c[0], c[1], c[2], r))
    return np.array(out, dtype=np.float64)


def packing_boolean(shape, solid_fraction, radius_sampler, seed, max_spheres=10_000_000):
    """Overlap-allowed (Boolean) placement until the sharp voxel solid fraction reaches the target.

    Centres are uniform over the box; spheres may cross the walls.  Spheres are added in groups sized
    to a quarter of the remaining deficit (at least one), so small boxes do not overshoot.
    radius_sampler(g) draws one radius in voxels.
    Returns (spheres (n, 4) voxel units, achieved sharp solid fraction).
    """
    g = rng(seed)
    n1, n2, n3 = shape
    mask = np.zeros((n3, n2, n1), dtype=bool)
    total = mask.size
    out = []
    solid = 0
    vol_sum, vol_n = 0.0, 0
    while solid < solid_fraction * total:
        deficit = solid_fraction * total - solid
        mean_vol = vol_sum / vol_n if vol_n else None
        batch = 1 if mean_vol is None else int(max(1, min(64, 0.25 * deficit / mean_vol)))
        for _ in range(batch):
            r = float(radius_sampler(g))
            c = (g.uniform(0, n1), g.uniform(0, n2), g.uniform(0, n3))
            out.append((c[0], c[1], c[2], r))
            _stamp(mask, c, r)
            vol_sum += 4.0 / 3.0 * math.pi * r ** 3
            vol_n += 1
        solid = int(mask.sum())
        if len(out) > max_spheres:
            raise RuntimeError("Boolean packing did not reach the target")
    return np.array(out, dtype=np.float64), solid / total


def uniform_radius(lo, hi):
    return lambda g: g.uniform(lo, hi)


def lognormal_radius(mean, sigma_ln):
    """Lognormal radii with the given arithmetic mean (voxels) and log-standard deviation."""
    mu_ln = math.log(mean) - 0.5 * sigma_ln * sigma_ln
    return lambda g: g.lognormal(mu_ln, sigma_ln)


def sharp_solid_mask(shape, spheres_vox):
    """Voxel mask (z, y, x) of centres inside any sphere (voxel units)."""
    n1, n2, n3 = shape
    mask = np.zeros((n3, n2, n1), dtype=bool)
    for s in spheres_vox:
        _stamp(mask, s[:3], s[3])
    return mask


def pore_ball_center(shape, spheres_vox, radius, seed, margin=1.0, max_tries=100000):
    """First drawn centre whose ball of `radius` keeps `margin` voxels from every sphere and wall."""
    g = rng(seed)
    n1, n2, n3 = shape
    for _ in range(max_tries):
        c = np.array([g.uniform(radius + margin, n - radius - margin) for n in (n1, n2, n3)])
        d = np.sqrt(((spheres_vox[:, :3] - c) ** 2).sum(axis=1)) - spheres_vox[:, 3]
        if len(d) == 0 or d.min() >= radius + margin:
            return c
    raise RuntimeError("no pore-space seed position found")


# ------------------------------------------------------------ initial fields
def ball_indicator(shape, center_vox, radius_vox) -> np.ndarray:
    """Sharp 0/1 field (flattened x fastest) of cell centres strictly inside the ball."""
    n1, n2, n3 = shape
    z, y, x = np.meshgrid(np.arange(n3) + 0.5, np.arange(n2) + 0.5, np.arange(n1) + 0.5, indexing="ij")
    d2 = (x - center_vox[0]) ** 2 + (y - center_vox[1]) ** 2 + (z - center_vox[2]) ** 2
    return (d2 < radius_vox * radius_vox).astype(np.float64).ravel()


def top_slab_indicator(shape, planes) -> np.ndarray:
    """Sharp 0/1 field equal to 1 on the top `planes` x3-planes (k >= n3 - planes)."""
    n1, n2, n3 = shape
    f = np.zeros((n3, n2, n1))
    f[n3 - planes:] = 1.0
    return f.ravel()


def random_fields(shape, seed, theta_scale=5.0, smooth=2):
    """Random theta (K), phi in [0,1] and G in [0,1] with a few passes of box smoothing.

    Used for right-hand-side parity on arbitrary states; contains cells in the
    Sigma-limiter bands, in bulk water/ice and in glass.
    """
    g = rng(seed)
    n1, n2, n3 = shape

    def sm(a):
        for _ in range(smooth):
            a = (a + np.roll(a, 1, 0) + np.roll(a, -1, 0) + np.roll(a, 1, 1) + np.roll(a, -1, 1)
                 + np.roll(a, 1, 2) + np.roll(a, -1, 2)) / 7.0
        return a

    th = sm(g.standard_normal((n3, n2, n1))) * theta_scale
    ph = sm(g.uniform(-1.5, 2.5, (n3, n2, n1)))
    ph = np.clip(ph, 0.0, 1.0)
    G = np.clip(sm(g.uniform(-1.0, 2.0, (n3, n2, n1))), 0.0, 1.0)
    return th.ravel().copy(), ph.ravel().copy(), G.ravel().copy()


# ----------------------------------------------------------------- workloads
@dataclass
class Workload:
    """A complete seeded input: grid, parameters, geometry and initial state."""
    name: str
    shape: tuple
    h: float
    model: int
    reaction: int
    params: dict
    spheres: np.ndarray            # (n, 4) metres
    x3_cap: float                  # nan = no cap
    theta0: np.ndarray             # flattened, x fastest
    phi0: np.ndarray
    extra: dict = field(default_factory=dict)

    @property
    def n_cells(self):
        return self.shape[0] * self.shape[1] * self.shape[2]


def micro_32(seed=20240104):
    """32^3 micro-scale constant-supercooling case: 6 RSA spheres r~U[6,9] voxels, ice ball r=4.

    h = 5e-8 m, xi = h, xi_G = 0.4 h, realistic alpha, dT = 0.5 K, zeta = 2, insulated.
    """
    shape = (32, 32, 32)
    h = 5e-8
    sv = packing_rsa(shape, 6, 6.0, 9.0, seed)
    c = pore_ball_center(shape, sv, 4.0, seed + 1)
    phi0 = ball_indicator(shape, c, 4.0)
    p = default_params(xi=h, xi_G=0.4 * h, zeta=2.0, theta_micro=-0.5, alpha=TABLE1["alpha"])
    sp = sv.copy()
    sp *= h
    return Workload("micro_32", shape, h, MODEL_MICRO, REACT_SIGMAP1P, p, sp, math.nan,
                    np.full(phi0.shape, -0.5), phi0,
                    extra={"fixed_dt": 0.1 * p["alpha"] * h * h, "fixed_steps": 200,
                           "t_end": 4 * 32 * h / (p["mu"] * 0.5), "tol": 1e-6,
                           "seed_center_vox": c})


def full_bead_case(n, seed, solid=0.60, r_lo=10.0, r_hi=16.0, radius_sampler=None,
                   h=3e-4, theta_ini=1.0, theta_cold=-5.0, name=None):
    """Full-model glass-bead case on an n^3 grid (the 256^3 freezing workload and its crops).

    Boolean packing to the sharp solid fraction `solid`, top face x3 = L3 held at
    theta_cold (Dirichlet), other faces insulated, theta = theta_ini initially,
    ice seed = the two top x3-planes.  alpha = "large sigma" value of Table 2,
    xi = h, xi_G = 0.4 h, zeta = 2.
    """
    shape = (n, n, n)
    sampler = radius_sampler or uniform_radius(r_lo, r_hi)
    sv, frac = packing_boolean(shape, solid, sampler, seed)
    p = default_params(xi=h, xi_G=0.4 * h, zeta=2.0, alpha=ALPHA_MACRO["large"],
                       dirichlet_faces=FACE_ZP, theta_freeze=theta_cold, theta_thaw=2.0)
    sp = sv.copy()
    sp *= h
    theta0 = np.full(n ** 3, float(theta_ini))
    phi0 = top_slab_indicator(shape, 2)
    return Workload(name or f"full_{n}", shape, h, MODEL_FULL, REACT_SIGMAP1P, p, sp, math.nan,
                    theta0, phi0, extra={"solid_fraction_sharp": frac, "tol": 1e-6,
                                         "n_spheres": len(sp)})


def lognormal_case(n=512, seed=20240112, t_freeze=math.inf):
    """Full-model freeze-then-thaw workload on an n^3 grid (512^3: about 14,600 beads): radii lognormal
    with mean 12 voxels and log-standard deviation 0.25, Boolean placement to 60 % solid, h = 0.3 mm,
    theta = +1 K, top face at -5 K until t_freeze and at +2 K after it (eq. BC-temperature-cap), ice seed
    in the two top planes.  (A bead count of 40,000 at this mean radius would fill 2.2 times the box, so
    the placement stops at the solid fraction instead.)"""
    w = full_bead_case(n, seed, radius_sampler=lognormal_radius(12.0, 0.25), name=f"full_lognormal_{n}")
    w.params["t_freeze"] = float(t_freeze)
    return w


def midfront_state(w, G, front=0.5, theta_cold=-5.0, theta_warm=1.0):
    """A state of a bead workload (top face cold) with its freezing front at the fraction `front` of the
    height: phi = 1/2 (1 + tanh((z - z_f) / (2 xi))) in the pore cells (G < 1/2; the planar interface
    profile of the Allen-Cahn equation, Sec. 2.2) and 0 in the glass; theta rising linearly from 0 at
    the front to theta_cold at the top face, and from 0 at the front to theta_warm 20 cells below it.
    Used to time the stage kernels on the mix of cells a run meets half way, without running there."""
    n1, n2, n3 = w.shape
    xi = w.params["xi"]
    z = (np.arange(n3) + 0.5) * w.h
    L = n3 * w.h
    zf = front * L
    prof = 0.5 * (1.0 + np.tanh((z - zf) / (2.0 * xi)))
    th_z = np.where(z >= zf, theta_cold * (z - zf) / (L - zf), theta_warm * np.minimum(1.0, (zf - z) / (20 * w.h)))
    G3 = np.asarray(G).reshape(n3, n2, n1)
    phi = np.where(G3 < 0.5, prof[:, None, None], 0.0)
    theta = np.broadcast_to(th_z[:, None, None], (n3, n2, n1))
    return np.ascontiguousarray(theta, dtype=np.float64).ravel(), np.ascontiguousarray(phi, dtype=np.float64).ravel()


def top_crop(w, crop, t_freeze, name=None):
    """The crop x [off, off + crop) of a bead workload at the top centre of its box, as a problem of its
    own: the beads whose glass terms reach the crop (beyond r + 40 xi_G they are below 1e-17), shifted;
    the same top face (Dirichlet, freeze then thaw at t_freeze) and seed planes; the cut faces insulated."""
    n1, n2, n3 = w.shape
    c1, c2, c3 = crop
    off = np.array([(n1 - c1) // 2, (n2 - c2) // 2, n3 - c3], dtype=np.float64)
    lo = off * w.h
    hi = (off + np.array(crop, dtype=np.float64)) * w.h
    sp = w.spheres
    reach = sp[:, 3] + 40 * w.params["xi_G"]
    near = np.all((sp[:, :3] > lo - reach[:, None]) & (sp[:, :3] < hi + reach[:, None]), axis=1)
    sps = sp[near].copy()
    sps[:, :3] -= lo
    p = dict(w.params)
    p["t_freeze"] = float(t_freeze)
    ncell = c1 * c2 * c3
    return Workload(name or f"{w.name}_crop{c1}", tuple(crop), w.h, w.model, w.reaction, p, sps, w.x3_cap,
                    np.full(ncell, float(w.theta0[0])), top_slab_indicator(tuple(crop), 2),
                    extra={"offset_vox": off.astype(int).tolist(), "n_spheres": len(sps)})


# Surface-tension scales and supercoolings of the micro-scale parametric sweep.
SIGMA_SCALES = (1.0, 3.0, 10.0, 30.0, 100.0, 300.0)
SUPERCOOLINGS = (0.1, 0.2, 0.5, 1.0, 2.0, 5.0, 10.0, 20.0)


@dataclass
class SweepInstance:
    shape: tuple
    h: float
    params: dict
    spheres: np.ndarray       # metres
    phi0: np.ndarray
    dt0: float
    t_end: float
    eq_window: float          # equilibrium: ice count unchanged for the time a free front (mu dT) crosses 20 cells
    sigma_scale: float
    dT: float
    x3_cap: float = math.nan  # glass cap (nan = none)
    region: tuple = None      # unfrozen-water region {i0, i1, j0, j1, k0, k1} (None = whole grid)
    label: str = ""


def sweep_instances(n=48, seed=20240108, h=1e-7, solid=0.60, sizes=None, seed_radius=4.0):
    """Micro-scale parametric sweep: instance i has an n_i^3 grid (n_i = 8 round(12 2^(i/(n-1))), 96..192,
    in a seeded permutation), its own Boolean packing (radii uniform in [10, 16] voxels, `solid` sharp
    solid fraction), surface-tension scale s and supercooling dT from the 6 x 8 table (alpha = alpha_Table1 / s),
    an ice ball of `seed_radius` voxels in the pore space, t_end = 4 L / (mu dT)."""
    g = rng(seed)
    if sizes is None:
        sizes = [8 * int(round(12 * 2 ** (i / max(n - 1, 1)))) for i in range(n)]
    perm = g.permutation(len(sizes))
    combos = [(sc, dT) for sc in SIGMA_SCALES for dT in SUPERCOOLINGS]
    out = []
    for i in range(n):
        N = int(sizes[perm[i] % len(sizes)])
        sc, dT = combos[(i * len(combos)) // n]
        shape = (N, N, N)
        sv, _ = packing_boolean(shape, solid, uniform_radius(10.0, 16.0), seed + 1 + i)
        c = pore_ball_center(shape, sv, seed_radius, seed + 1001 + i, margin=0.5)
        phi0 = ball_indicator(shape, c, seed_radius)
        p = default_params(xi=h, xi_G=0.4 * h, zeta=2.0, theta_micro=-dT, alpha=TABLE1["alpha"] / sc)
        sp = sv.copy()
        sp *= h
        out.append(SweepInstance(shape, h, p, sp, phi0, 0.1 * p["alpha"] * h * h, 4 * N * h / (p["mu"] * dT),
                                 20 * h / (p["mu"] * dT), sc, dT))
    return out


def warmstart_instances(n, side=64, seed=20240109, h=1e-7, solid=0.5, dT_range=(0.5, 5.0), scale_range=(1.0, 10.0)):
    """Micro-scale equilibria for the learned warm start: n cubes of `side`^3 cells, each with its own
    Boolean bead packing (radii uniform in [10, 16] voxels, sharp solid fraction `solid`), supercooling
    and surface-tension scale drawn log-uniformly, ice seeded on the bottom plane (nucleation at a
    cooled face, as under the paper's cap), t_end = 4 L / (mu dT)."""
    g = rng(seed)
    out = []
    for i in range(n):
        shape = (side, side, side)
        dT = float(math.exp(g.uniform(math.log(dT_range[0]), math.log(dT_range[1]))))
        sc = float(math.exp(g.uniform(math.log(scale_range[0]), math.log(scale_range[1]))))
        sv, _ = packing_boolean(shape, solid, uniform_radius(10.0, 16.0), seed + 7 + 13 * i)
        phi0 = np.zeros((side, side, side))
        phi0[0] = 1.0
        p = default_params(xi=h, xi_G=0.4 * h, zeta=2.0, theta_micro=-dT, alpha=TABLE1["alpha"] / sc)
        sp = sv.copy()
        sp *= h
        out.append(SweepInstance(shape, h, p, sp, phi0.ravel(), 0.1 * p["alpha"] * h * h,
                                 4 * side * h / (p["mu"] * dT), 20 * h / (p["mu"] * dT), sc, dT))
    return out


# ------------------------------------------------------------------ macro-scale vessel (Sec. 3.1)
# Table 2: vessel interior L3 x L3/2 x L3/2 with L3 = 6 cm, glass cap above 11/12 L3, bead radius
# L3/20, xi_G = L3/500, xi = L3/N3, cooled through the cap at -25 K for 5 h, then heated at +20 K
# for 5 h, initial temperature +20 K, nucleation disk of eq. (nucleation-site).
MACRO_L3 = 0.06
MACRO_T_FREEZE = 5 * 3600.0
MACRO_T_END = 10 * 3600.0


def settled_bed(L1, L2, r, bed_top, seed, candidates=64, max_fails=200):
    """Stand-in for the paper's DEM-settled bead bed (the DEM positions are not available).  Spheres of
    radius r are added one at a time: each of `candidates` uniformly random (x1, x2) positions inside
    the walls is given the height where a vertically falling sphere first touches the floor or an
    earlier sphere, and the lowest of them is taken (a sphere settles into the deepest pocket within
    reach).  A sphere is kept if its top stays below bed_top; the bed is complete after max_fails
    consecutive sets of candidates that are not.  Returns (n, 4) rows (x, y, z, r) in metres."""
    g = rng(seed)
    cs = np.zeros((0, 3))
    fails = 0
    while fails < max_fails:
        x = g.uniform(r, L1 - r, candidates)
        y = g.uniform(r, L2 - r, candidates)
        z = np.full(candidates, r)
        if len(cs):
            d2 = (cs[None, :, 0] - x[:, None]) ** 2 + (cs[None, :, 1] - y[:, None]) ** 2
            rest = np.where(d2 < 4.0 * r * r, cs[None, :, 2] + np.sqrt(np.maximum(4.0 * r * r - d2, 0.0)), r)
            z = np.maximum(z, rest.max(axis=1))
        q = int(np.argmin(z))
        if z[q] + r <= bed_top:
            cs = np.vstack([cs, [x[q], y[q], z[q]]])
            fails = 0
        else:
            fails += 1
    return np.hstack([cs, np.full((len(cs), 1), r)])


def nucleation_disk(shape, h, L1, L2, L3) -> np.ndarray:
    """Sharp 0/1 indicator of eq. (nucleation-site) at the cell centres: 0.87 L3 < x3 < 0.97 L3 and
    (x1 - L1/2)^2 + (x2 - L2/2)^2 < (L1/3)^2."""
    n1, n2, n3 = shape
    x = (np.arange(n1) + 0.5) * h
    y = (np.arange(n2) + 0.5) * h
    z = (np.arange(n3) + 0.5) * h
    rad = (x[None, None, :] - L1 / 2) ** 2 + (y[None, :, None] - L2 / 2) ** 2 < (L1 / 3) ** 2
    slab = (z > 0.87 * L3) & (z < 0.97 * L3)
    return (slab[:, None, None] & rad).astype(np.float64).ravel()


def macro_case(n3, model, reaction=REACT_SIGMAP1P, sigma="large", gamma=2.0, seed=20240110, bed_fraction=0.6):
    """The paper's macro-scale vessel (Table 2) on N3 = n3 cells along x3 (n1 = n2 = n3/2, h = L3/n3).
    Phase-field models: alpha of the sigma class, zeta = 2, nucleation disk; Temp model: zeta = 1,
    gamma as given, no phase-field state.  The bead bed fills the vessel up to bed_fraction L3."""
    if n3 % 2:
        raise ValueError("n3 must be even")
    L3 = MACRO_L3
    L1 = L2 = L3 / 2
    h = L3 / n3
    shape = (n3 // 2, n3 // 2, n3)
    r = L3 / 20
    spheres = settled_bed(L1, L2, r, bed_fraction * L3, seed)
    temp = model == MODEL_TEMP
    p = default_params(xi=L3 / n3, xi_G=L3 / 500, zeta=1.0 if temp else 2.0, gamma=gamma,
                       alpha=ALPHA_MACRO[sigma], dirichlet_faces=FACE_ZP, theta_freeze=-25.0, theta_thaw=20.0,
                       t_freeze=MACRO_T_FREEZE)
    theta0 = np.full(int(np.prod(shape)), 20.0)
    phi0 = None if temp else nucleation_disk(shape, h, L1, L2, L3)
    tag = "temp" if temp else ("gradp" if reaction == REACT_GRADP else "sigmap1p")
    name = f"macro{n3}_{tag}_" + (f"gamma{gamma:g}" if temp else sigma)
    return Workload(name, shape, h, model, reaction, p, spheres, 11.0 / 12.0 * L3, theta0, phi0,
                    extra={"n_spheres": len(spheres), "t_end": MACRO_T_END, "sigma": None if temp else sigma,
                           "gamma": gamma if temp else None, "bed_top": bed_fraction * L3})


def fcc_bed(L1, L2, bed_top, r, seed, gap=0.02):
    """Ordered bed: a face-centred cubic lattice of spheres of radius r with nearest-neighbour distance
    2r(1 + gap), centred in the walls, every sphere whose top stays below bed_top kept, each moved by a
    seeded random offset shorter than half the gap (so no two touch).  Returns (n, 4) rows in metres."""
    g = rng(seed)
    a = 2.0 * r * (1.0 + gap) * math.sqrt(2.0)          # cubic cell of the fcc lattice
    basis = np.array([[0, 0, 0], [0.5, 0.5, 0], [0.5, 0, 0.5], [0, 0.5, 0.5]]) * a
    nx, ny, nz = int(L1 / a) + 2, int(L2 / a) + 2, int(bed_top / a) + 2
    ijk = np.stack(np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij"), -1).reshape(-1, 3)
    pts = (ijk[:, None, :] * a + basis[None, :, :]).reshape(-1, 3)
    lo = np.array([r, r, r])
    hi = np.array([L1 - r, L2 - r, bed_top - r])
    best, best_pts = -1, None
    for ox in np.linspace(0, a, 9, endpoint=False):      # lattice shift keeping the most spheres
        for oy in np.linspace(0, a, 9, endpoint=False):
            q = pts + np.array([ox, oy, 0.0]) + lo
            keep = np.all((q >= lo) & (q <= hi), axis=1)
            if keep.sum() > best:
                best, best_pts = int(keep.sum()), q[keep]
    jit = g.normal(size=best_pts.shape)
    jit *= (0.49 * gap * r) / np.maximum(np.linalg.norm(jit, axis=1, keepdims=True), 1e-300) * g.uniform(0, 1, (len(jit), 1))
    c = np.clip(best_pts + jit, lo, hi)
    return np.hstack([c, np.full((len(c), 1), r)])


def uwc_instances(dTs=(0.05, 0.1, 0.2, 0.5, 1.0, 2.0), beds=("fcc", "settled"), n3=200, r=5e-6, seed=20240111):
    """Micro-scale unfrozen-water study (Sec. 3.3): the vessel of Table 2 scaled so that the bead radius
    is r (L3 = 20 r: polystyrene, r = 5 um), constant supercooling dT (micro model), realistic alpha of
    Table 1, ice from the nucleation disk, unfrozen water counted in the bottom half of the vessel (which
    the bed fills).  One instance per (bed, dT); beds: "fcc" (ordered, dense) and "settled" (random,
    looser).  t_end = 20 L3/(mu dT) is a backstop: the runs stop on the equilibrium test (ice count
    unchanged for the time a free front needs to cross 20 cells)."""
    L3 = 20.0 * r
    L1 = L2 = L3 / 2
    h = L3 / n3
    shape = (n3 // 2, n3 // 2, n3)
    out = []
    for b, bed in enumerate(beds):
        if bed == "fcc":
            sp = fcc_bed(L1, L2, 0.6 * L3, r, seed + b)
        else:
            sp = settled_bed(L1, L2, r, 0.6 * L3, seed + b)
        phi0 = nucleation_disk(shape, h, L1, L2, L3)
        for dT in dTs:
            p = default_params(xi=L3 / n3, xi_G=L3 / 500, zeta=2.0, theta_micro=-float(dT), alpha=TABLE1["alpha"])
            v = p["mu"] * dT
            out.append(SweepInstance(shape, h, p, sp, phi0, 0.1 * p["alpha"] * h * h, 20 * L3 / v, 20 * h / v, 1.0,
                                     float(dT), x3_cap=11.0 / 12.0 * L3,
                                     region=(0, shape[0], 0, shape[1], 0, n3 // 2), label=bed))
    return out
