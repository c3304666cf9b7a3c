"""Mutation check of the oracle's pins: each plausible mistake (a dropped term, a wrong sign, factor,
index or stage coefficient) is planted in a copy of the oracle source, compiled, and the pin suite
(tests/test_oracle_pins.py) must fail against it.  Mistakes are planted on the CPU only."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "pf_oracle.c")

MUTANTS = {
    "dirichlet_factor": ("div += 2.0 * lam_i * (th_b - th_i) / h2;", "div += 1.0 * lam_i * (th_b - th_i) / h2;"),
    "blend_swapped": ("(phi * w[IC] + (1.0 - phi) * w[LQ])", "(phi * w[LQ] + (1.0 - phi) * w[IC])"),
    "driving_sign": ("S * under);", "S * (-under));"),
    "latent_dropped": ("(div + rho * m->L * dph) / (rho * c)", "(div + 0.0 * dph) / (rho * c)"),
    "laplacian_two_axes": ("        for (int d = 0; d < 3; ++d) {\n                double lo", "        for (int d = 0; d < 2; ++d) {\n                double lo"),
    "merson_estimate": ("9.0 * k[3][f][q]", "8.0 * k[3][f][q]"),
    "merson_stage4_index": ("3.0 * dt / 8.0 * k[3][0][q]", "3.0 * dt / 8.0 * k[2][0][q]"),
    "controller_exponent": ("pow(tol / E, 0.2)", "pow(tol / E, 0.25)"),
    "gradp_scale": ("double g = (hi - lo) / (2.0 * h);", "double g = (hi - lo) / h;"),
    "limiter_power": ("3.0 * (a * a) / (d * d)", "3.0 * (a * a) / d"),
    "uwc_strictness": ("if (G[id] < 0.5) {", "if (G[id] <= 0.5) {"),
    "glass_width": ("spheres[4 * s + 3]) / (2.0 * xi_G)", "spheres[4 * s + 3]) / xi_G"),
    "water_indicator": ("double v = 1.0 - zeta * G;", "double v = 1.0 - G;"),
    "face_mean": ("lam_f = 0.5 * (lam_i + lam_j);", "lam_f = lam_j;"),
    "temp_gamma": ("return -0.5 * water_indicator(G, m->zeta) * m->gamma * (1.0 - th * th);",
                   "return -0.5 * water_indicator(G, m->zeta) * (1.0 - th * th);"),
    "landing": ("*t = land ? target : *t + h;", "*t = *t + h;"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site not unique for {name}"
    mut = tmp_path / "mutant.c"
    mut.write_text(src.replace(old, new))
    so = tmp_path / "libmutant.so"
    subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-o", str(so), str(mut), "-lm"])
    env = dict(os.environ, PF_ORACLE_SO=str(so))
    # a timeout is not a catch: only a pin that fails counts
    r = subprocess.run([sys.executable, "-m", "pytest", os.path.join(ROOT, "tests", "test_oracle_pins.py"), "-x", "-q",
                        "-p", "no:cacheprovider"], cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 1, f"no pin caught the mutant {name} (exit {r.returncode}):\n{r.stdout[-800:]}"
    assert " failed" in r.stdout, r.stdout[-800:]
