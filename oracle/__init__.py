"""CPU oracle of the phase-field freezing model (plain FP64 C, built with gcc).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA library and never imports it.

Every function follows the paper (Strachota, arXiv 2401.01672) step by step;
the C source ``pf_oracle.c`` cites the section or equation of each step and
lists the readings taken where the paper is silent.

Parity status: every function here is pinned by ``tests/test_oracle_pins.py``
(closed forms, invariants, brute force, library routines).  The Temp model's
behaviour at large gamma (sharp Stefan limit) is "parity unpinned".
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pf_oracle.c")
_LIB = os.path.join(_HERE, "liboracle_pf.so")
# tests/test_oracle_mutants.py points this at a library built from a deliberately broken copy
_OVERRIDE = os.environ.get("PF_ORACLE_SO")
_lib = None

MODEL = {"full": 0, "temp": 1, "micro": 2}
REACTION = {"sigmap1p": 0, "gradp": 1}


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2 -ffp-contract=off, IEEE rounding as written), with OpenMP
    over the loops on cells where the compiler has it (results do not depend on the thread count)."""
    if _OVERRIDE:
        return _OVERRIDE
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        base = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        if subprocess.run(base[:1] + ["-fopenmp"] + base[1:], capture_output=True).returncode != 0:
            subprocess.check_call(base)
        os.replace(tmp, _LIB)
    return _LIB


def threads(n: int = 0) -> int:
    """Threads of the oracle's loops over cells: n > 0 sets the count; returns the count in use."""
    return int(_load().or_threads(int(n)))


class ORModel(C.Structure):
    _fields_ = [
        ("n1", C.c_int), ("n2", C.c_int), ("n3", C.c_int),
        ("h", C.c_double),
        ("model", C.c_int), ("reaction", C.c_int),
        ("rho", C.c_double * 3), ("c", C.c_double * 3), ("lam", C.c_double * 3),
        ("L", C.c_double), ("mu", C.c_double), ("alpha", C.c_double), ("xi", C.c_double),
        ("eps0", C.c_double), ("eps1", C.c_double), ("b", C.c_double), ("gamma", C.c_double),
        ("zeta", C.c_double),
        ("theta_micro", C.c_double),
        ("theta_freeze", C.c_double), ("theta_thaw", C.c_double), ("t_freeze", C.c_double),
        ("dt_min", C.c_double), ("dt_max", C.c_double),
        ("dirichlet", C.c_int), ("harmonic", C.c_int),
    ]


def _load():
    global _lib
    if _lib is None:
        lib = C.CDLL(build())
        P = C.POINTER
        d, i, ll = C.c_double, C.c_int, C.c_longlong
        pd, pll = P(d), P(ll)
        lib.or_glass.argtypes = [P(ORModel), pd, ll, d, d, i, pll, ll, pd]
        lib.or_temp_phi.argtypes = [P(ORModel), pd, pd, pd]
        lib.or_rhs.argtypes = [P(ORModel), pd, d, pd, pd, pll, ll, pd, pd]
        lib.or_rkm_step.argtypes = [P(ORModel), pd, d, d, pd, pd, pd, pd, pd]
        lib.or_controller.argtypes = [d, d, d, d]
        lib.or_controller.restype = d
        lib.or_run.argtypes = [P(ORModel), pd, pd, pd, pd, pd, d, d, ll, i, pll, pll, pd, pd]
        lib.or_run.restype = i
        lib.or_uwc.argtypes = [P(ORModel), pd, pd, P(C.c_int), pll, pll, pd, pd]
        lib.or_threads.argtypes = [i]
        lib.or_threads.restype = i
        _lib = lib
    return _lib


def _p(a):
    if a is None:
        return None
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _arr(a, n=None):
    if a is None:
        return None
    a = np.ascontiguousarray(a, dtype=np.float64).ravel()
    if n is not None and a.size != n:
        raise ValueError(f"expected {n} values, got {a.size}")
    return a


class Oracle:
    """One grid configuration: shape (n1, n2, n3), cell size h, model, reaction and parameters."""

    def __init__(self, shape, h, model, reaction, params):
        self.shape = tuple(int(s) for s in shape)
        self.N = self.shape[0] * self.shape[1] * self.shape[2]
        m = ORModel()
        m.n1, m.n2, m.n3 = self.shape
        m.h = h
        m.model = MODEL[model] if isinstance(model, str) else int(model)
        m.reaction = REACTION[reaction] if isinstance(reaction, str) else int(reaction)
        m.rho = (C.c_double * 3)(*params["rho"])
        m.c = (C.c_double * 3)(*params["c"])
        m.lam = (C.c_double * 3)(*params["lambda"])
        m.L = params["latent"]
        m.mu = params["mu"]
        m.alpha = params["alpha"]
        m.xi = params["xi"]
        m.eps0 = params["eps0"]
        m.eps1 = params["eps1"]
        m.b = params["b"]
        m.gamma = params["gamma"]
        m.zeta = params["zeta"]
        m.theta_micro = params["theta_micro"]
        m.theta_freeze = params["theta_freeze"]
        m.theta_thaw = params["theta_thaw"]
        m.t_freeze = params["t_freeze"]
        m.dt_min = params["dt_min"]
        m.dt_max = params["dt_max"]
        m.dirichlet = int(params["dirichlet_faces"])
        m.harmonic = int(params.get("harmonic_mean", 0))
        self.m = m
        self.params = dict(params)
        self.lib = _load()

    # -- Sec. 2.1
    def glass(self, spheres, xi_G, x3_cap=math.nan, cells=None):
        sp = _arr(spheres)
        ns = 0 if sp is None else sp.size // 4
        if sp is None or sp.size == 0:
            sp = np.zeros(4)
        has_cap = not math.isnan(x3_cap)
        if cells is None:
            out = np.empty(self.N)
            cp, nc = None, 0
        else:
            cells = np.ascontiguousarray(cells, dtype=np.int64)
            out = np.empty(cells.size)
            cp, nc = cells.ctypes.data_as(C.POINTER(C.c_longlong)), cells.size
        self.lib.or_glass(C.byref(self.m), _p(sp), ns, xi_G, 0.0 if not has_cap else x3_cap,
                          int(has_cap), cp, nc, _p(out))
        return out

    # -- Sec. 2.3
    def temp_phi(self, G, theta):
        G, theta = _arr(G, self.N), _arr(theta, self.N)
        out = np.empty(self.N)
        self.lib.or_temp_phi(C.byref(self.m), _p(G), _p(theta), _p(out))
        return out

    # -- Secs. 2.2-2.5
    def rhs(self, G, theta, phi, t=0.0, cells=None):
        G = _arr(G, self.N)
        theta = _arr(theta, self.N)
        phi = _arr(phi, self.N)
        if cells is None:
            n = self.N
            cp, nc = None, 0
        else:
            cells = np.ascontiguousarray(cells, dtype=np.int64)
            n = cells.size
            cp, nc = cells.ctypes.data_as(C.POINTER(C.c_longlong)), cells.size
        dth, dph = np.empty(n), np.empty(n)
        self.lib.or_rhs(C.byref(self.m), _p(G), t, _p(theta), _p(phi), cp, nc, _p(dth), _p(dph))
        return dth, dph

    def rkm_step(self, G, theta, phi, t, dt):
        G = _arr(G, self.N)
        theta = _arr(theta, self.N) if theta is not None else np.zeros(self.N)
        phi = _arr(phi, self.N) if phi is not None else np.zeros(self.N)
        ot, op = np.empty(self.N), np.empty(self.N)
        err = C.c_double()
        self.lib.or_rkm_step(C.byref(self.m), _p(G), t, dt, _p(theta), _p(phi), _p(ot), _p(op), C.byref(err))
        return ot, op, err.value

    def controller(self, E, tol, dt):
        return self.lib.or_controller(E, tol, dt, self.m.dt_max)

    def run(self, G, theta, phi, t, dt, t_end, tol, max_steps, fixed=False, trace=False):
        """Integrate in place copies; returns dict with state, time, dt, counters and status."""
        G = _arr(G, self.N)
        th = _arr(theta, self.N).copy() if theta is not None else np.zeros(self.N)
        ph = _arr(phi, self.N).copy() if phi is not None else np.zeros(self.N)
        tt, dd = C.c_double(t), C.c_double(dt)
        na, nr = C.c_longlong(), C.c_longlong()
        le = C.c_double(0.0)
        tr = np.zeros(4 * max_steps) if trace else None
        st = self.lib.or_run(C.byref(self.m), _p(G), _p(th), _p(ph), C.byref(tt), C.byref(dd), t_end, tol,
                             int(max_steps), int(bool(fixed)), C.byref(na), C.byref(nr), C.byref(le), _p(tr))
        out = {"theta": th, "phi": ph, "t": tt.value, "dt": dd.value, "n_accepted": na.value,
               "n_rejected": nr.value, "last_err": le.value, "status": st}
        if trace:
            n = na.value + nr.value
            out["trace"] = tr[: 4 * n].reshape(n, 4)
        return out

    # -- Sec. 3.1 / 3.3
    def uwc(self, G, phi, region=None):
        G, phi = _arr(G, self.N), _arr(phi, self.N)
        nw, ni = C.c_longlong(), C.c_longlong()
        sn, sd = C.c_double(), C.c_double()
        rp = None
        if region is not None:
            rp = (C.c_int * 6)(*[int(v) for v in region])
        self.lib.or_uwc(C.byref(self.m), _p(G), _p(phi), rp, C.byref(nw), C.byref(ni), C.byref(sn), C.byref(sd))
        n_water, n_ice = nw.value, ni.value
        return {"n_water": n_water, "n_ice": n_ice,
                "uwc": (1.0 - n_ice / n_water) if n_water else math.nan,
                "smooth": (1.0 - sn.value / sd.value) if sd.value else math.nan}
