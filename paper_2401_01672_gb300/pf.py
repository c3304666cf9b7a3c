"""Python binding of the C ABI in include/pf.h (ctypes; argument marshalling only).

Every function keeps the C name.  Host arrays are numpy float64 (or pinned
torch CPU tensors); device arrays are torch CUDA tensors.  A non-zero status
raises ``PfError`` with the library's message.  There is no fallback: if the
CUDA library is missing the import of this module's functions fails loudly.
"""
from __future__ import annotations

import ctypes as C
import math
import os

import numpy as np

from . import inputs as _inputs

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpfgb300.so")

PF_OK, PF_E_INVALID, PF_E_CUDA, PF_E_OOM, PF_E_DT_UNDERFLOW, PF_E_NONFINITE, PF_E_RANGE, PF_E_TIMEOUT, PF_E_STATE = (
    0, -1, -2, -3, -4, -5, -6, -7, -8)
STATUS_NAMES = {0: "PF_OK", -1: "PF_E_INVALID", -2: "PF_E_CUDA", -3: "PF_E_OOM", -4: "PF_E_DT_UNDERFLOW",
                -5: "PF_E_NONFINITE", -6: "PF_E_RANGE", -7: "PF_E_TIMEOUT", -8: "PF_E_STATE"}

# Every symbol declared in include/pf.h (checked by the CPU tests).
EXPORTS = ["pf_create_grid", "pf_destroy_grid", "pf_set_geometry", "pf_set_glass", "pf_get_glass", "pf_set_state",
           "pf_get_state", "pf_rhs", "pf_rkm_step", "pf_run_to", "pf_run_fixed", "pf_unfrozen_fraction",
           "pf_max_phase_rate", "pf_profile_stages", "pf_measure_peaks", "pf_unfrozen_fraction_noalloc", "pf_last_error",
           "pf_kernel_launches", "pf_set_tiles", "pf_get_tiles", "pf_autotune", "pf_batch_create",
           "pf_batch_destroy", "pf_batch_grid", "pf_batch_autotune", "pf_batch_run_to", "pf_batch_iterations",
           "pf_batch_last_error", "pf_slabs_create", "pf_slabs_destroy", "pf_slabs_grid", "pf_slabs_set_geometry",
           "pf_slabs_set_tiles", "pf_slabs_set_state", "pf_slabs_get_state", "pf_slabs_run_to",
           "pf_slabs_unfrozen_fraction", "pf_slabs_halo_bytes", "pf_slabs_last_error"]


class PfError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class pf_params(C.Structure):
    _fields_ = [("rho", C.c_double * 3), ("c", C.c_double * 3), ("lambda_", C.c_double * 3),
                ("latent", C.c_double), ("mu", C.c_double), ("alpha", C.c_double), ("xi", C.c_double),
                ("xi_G", C.c_double), ("eps0", C.c_double), ("eps1", C.c_double), ("b", C.c_double),
                ("gamma", C.c_double), ("zeta", C.c_double), ("theta_micro", C.c_double),
                ("theta_freeze", C.c_double), ("theta_thaw", C.c_double), ("t_freeze", C.c_double),
                ("dt_min", C.c_double), ("dt_max", C.c_double), ("dirichlet_faces", C.c_int),
                ("harmonic_mean", C.c_int)]


class pf_run_stats(C.Structure):
    _fields_ = [("n_accepted", C.c_longlong), ("n_rejected", C.c_longlong), ("t", C.c_double),
                ("dt", C.c_double), ("last_err", C.c_double), ("launches", C.c_longlong)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class pf_batch_result(C.Structure):
    _fields_ = [("stats", pf_run_stats), ("t_eq", C.c_double), ("rate", C.c_double), ("equilibrium", C.c_int),
                ("status", C.c_int)]

    def as_dict(self):
        d = self.stats.as_dict()
        d.update(t_eq=self.t_eq, rate=self.rate, equilibrium=bool(self.equilibrium), status=self.status)
        return d


_lib = None


def load_library(path: str = LIB_PATH):
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"CUDA library not built: {path} (run __graft_entry__.build())")
    lib = C.CDLL(path)
    vp, d, i, ll = C.c_void_p, C.c_double, C.c_int, C.c_longlong
    pd, pi, pll = C.POINTER(d), C.POINTER(i), C.POINTER(ll)
    sig = {
        "pf_create_grid": [i, i, i, d, i, i, i, C.POINTER(pf_params), vp, C.POINTER(vp)],
        "pf_destroy_grid": [vp],
        "pf_set_geometry": [vp, vp, ll, d],
        "pf_set_glass": [vp, vp],
        "pf_get_glass": [vp, vp],
        "pf_set_state": [vp, vp, vp, d, d],
        "pf_get_state": [vp, vp, vp, pd, pd],
        "pf_rhs": [vp, d, vp, vp, vp, vp],
        "pf_rkm_step": [vp, pd, d, i, pi, pd],
        "pf_run_to": [vp, d, d, ll, C.POINTER(pf_run_stats)],
        "pf_run_fixed": [vp, ll, d, C.POINTER(pf_run_stats)],
        "pf_unfrozen_fraction": [vp, vp, pd, pll, pll, pd],
        "pf_max_phase_rate": [vp, pd],
        "pf_profile_stages": [vp, i, pd],
        "pf_measure_peaks": [pd, pd, pd],
        "pf_set_tiles": [vp, i, i],
        "pf_get_tiles": [vp, pi, pi],
        "pf_autotune": [vp, C.c_char_p, pi, pi, pd],
        "pf_batch_create": [i, C.POINTER(vp), C.POINTER(vp)],
        "pf_batch_destroy": [vp],
        "pf_batch_autotune": [vp, C.c_char_p],
        "pf_batch_run_to": [vp, pd, pd, d, pd, d, ll, C.POINTER(pf_batch_result)],
        "pf_unfrozen_fraction_noalloc": [vp, vp, i, i, i, vp, vp, pd, pll, pll, pd],
        "pf_slabs_create": [i, i, i, d, i, i, i, C.POINTER(pf_params), i, vp, vp, C.POINTER(vp)],
        "pf_slabs_destroy": [vp],
        "pf_slabs_set_geometry": [vp, vp, ll, d],
        "pf_slabs_set_tiles": [vp, i, i],
        "pf_slabs_set_state": [vp, vp, vp, d, d],
        "pf_slabs_get_state": [vp, vp, vp, pd, pd],
        "pf_slabs_run_to": [vp, d, d, ll, C.POINTER(pf_run_stats)],
        "pf_slabs_unfrozen_fraction": [vp, pd, pll, pll],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = C.c_int
    lib.pf_last_error.argtypes = [vp]
    lib.pf_last_error.restype = C.c_char_p
    lib.pf_kernel_launches.argtypes = []
    lib.pf_kernel_launches.restype = C.c_longlong
    lib.pf_batch_grid.argtypes = [vp, i]
    lib.pf_batch_grid.restype = vp
    lib.pf_batch_iterations.argtypes = [vp]
    lib.pf_batch_iterations.restype = C.c_longlong
    lib.pf_batch_last_error.argtypes = [vp]
    lib.pf_batch_last_error.restype = C.c_char_p
    lib.pf_slabs_grid.argtypes = [vp, i]
    lib.pf_slabs_grid.restype = vp
    lib.pf_slabs_halo_bytes.argtypes = [vp]
    lib.pf_slabs_halo_bytes.restype = C.c_longlong
    lib.pf_slabs_last_error.argtypes = [vp]
    lib.pf_slabs_last_error.restype = C.c_char_p
    _lib = lib
    return lib


def _check(st, handle):
    if st != PF_OK:
        msg = _lib.pf_last_error(handle)
        raise PfError(st, msg.decode() if msg else "")


def make_params(d: dict) -> pf_params:
    p = pf_params()
    p.rho = (C.c_double * 3)(*d["rho"])
    p.c = (C.c_double * 3)(*d["c"])
    p.lambda_ = (C.c_double * 3)(*d["lambda"])
    for k in ("latent", "mu", "alpha", "xi", "xi_G", "eps0", "eps1", "b", "gamma", "zeta", "theta_micro",
              "theta_freeze", "theta_thaw", "t_freeze", "dt_min", "dt_max"):
        setattr(p, k, float(d[k]))
    p.dirichlet_faces = int(d["dirichlet_faces"])
    p.harmonic_mean = int(d.get("harmonic_mean", 0))
    return p


def _host(a, n=None):
    """(pointer, keepalive) for a host float64 array (numpy or torch CPU tensor)."""
    if a is None:
        return None, None
    try:
        import torch
        if isinstance(a, torch.Tensor):
            if a.is_cuda or a.dtype != torch.float64 or not a.is_contiguous():
                raise ValueError("host tensor must be contiguous float64 on the CPU")
            if n is not None and a.numel() != n:
                raise ValueError(f"expected {n} values")
            return a.data_ptr(), a
    except ImportError:
        pass
    arr = np.ascontiguousarray(a, dtype=np.float64).ravel()
    if n is not None and arr.size != n:
        raise ValueError(f"expected {n} values, got {arr.size}")
    return arr.ctypes.data, arr


def _dev(t):
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("device arrays must be contiguous CUDA tensors")
    return t.data_ptr()


class Grid:
    """Owning handle of a pf_grid (the C object).  Methods map one-to-one to C calls."""

    def __init__(self, shape, h, model, reaction=0, precision=0, params=None, stream=None):
        lib = load_library()
        self.shape = tuple(int(s) for s in shape)
        self.N = self.shape[0] * self.shape[1] * self.shape[2]
        self.model, self.reaction, self.precision = int(model), int(reaction), int(precision)
        self.params = dict(params or _inputs.default_params())
        self._cparams = make_params(self.params)
        import torch
        self.stream = stream if stream is not None else torch.cuda.Stream()
        h_ptr = C.c_void_p()
        st = lib.pf_create_grid(self.shape[0], self.shape[1], self.shape[2], float(h), self.model,
                                self.reaction, self.precision, C.byref(self._cparams),
                                C.c_void_p(self.stream.cuda_stream), C.byref(h_ptr))
        _check(st, None)
        self.handle = h_ptr
        self.h = float(h)

    @property
    def field_dtype(self):
        import torch
        return torch.float32 if self.precision == _inputs.PREC_FP32 else torch.float64

    def close(self):
        if getattr(self, "handle", None) and not getattr(self, "_owned_by_batch", False):
            _lib.pf_destroy_grid(self.handle)
        self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # ---- thin wrappers
    def set_geometry(self, spheres, x3_cap=math.nan):
        sp = np.ascontiguousarray(spheres, dtype=np.float64).reshape(-1, 4)
        _check(_lib.pf_set_geometry(self.handle, sp.ctypes.data if sp.size else None, sp.shape[0], x3_cap),
               self.handle)

    def set_glass(self, G):
        p, keep = _host(G, self.N)
        _check(_lib.pf_set_glass(self.handle, p), self.handle)

    def get_glass(self):
        out = np.empty(self.N)
        _check(_lib.pf_get_glass(self.handle, out.ctypes.data), self.handle)
        return out

    def set_state(self, theta, phi, t=0.0, dt=1e-3):
        pt, k1 = _host(theta, self.N)
        pp, k2 = _host(phi, self.N)
        _check(_lib.pf_set_state(self.handle, pt, pp, float(t), float(dt)), self.handle)

    def get_state(self, theta_out=None, phi_out=None):
        th = np.empty(self.N) if theta_out is None else theta_out
        ph = np.empty(self.N) if phi_out is None else phi_out
        pt, _ = _host(th, self.N)
        pp, _ = _host(ph, self.N)
        t, dt = C.c_double(), C.c_double()
        _check(_lib.pf_get_state(self.handle, pt, pp, C.byref(t), C.byref(dt)), self.handle)
        return th, ph, t.value, dt.value

    def rhs(self, t, theta_in, phi_in, dtheta_out, dphi_out):
        """Right-hand side on device tensors of the grid's field type; enqueued on the grid's stream."""
        import torch
        cur = torch.cuda.current_stream()
        self.stream.wait_stream(cur)
        _check(_lib.pf_rhs(self.handle, float(t), _dev(theta_in), _dev(phi_in), _dev(dtheta_out), _dev(dphi_out)),
               self.handle)
        cur.wait_stream(self.stream)

    def rkm_step(self, dt, tol, force_accept=False):
        d = C.c_double(dt)
        acc, err = C.c_int(), C.c_double()
        _check(_lib.pf_rkm_step(self.handle, C.byref(d), float(tol), int(bool(force_accept)), C.byref(acc),
                                C.byref(err)), self.handle)
        return bool(acc.value), err.value, d.value

    def run_to(self, t_end, tol, max_steps=10 ** 9):
        s = pf_run_stats()
        _check(_lib.pf_run_to(self.handle, float(t_end), float(tol), int(max_steps), C.byref(s)), self.handle)
        return s.as_dict()

    def run_fixed(self, n_steps, dt):
        s = pf_run_stats()
        _check(_lib.pf_run_fixed(self.handle, int(n_steps), float(dt), C.byref(s)), self.handle)
        return s.as_dict()

    def unfrozen_fraction(self, region=None):
        r = None if region is None else (C.c_int * 6)(*[int(v) for v in region])
        u, sm = C.c_double(), C.c_double()
        ni, nw = C.c_longlong(), C.c_longlong()
        _check(_lib.pf_unfrozen_fraction(self.handle, r, C.byref(u), C.byref(ni), C.byref(nw), C.byref(sm)),
               self.handle)
        return {"uwc": u.value, "n_ice": ni.value, "n_water": nw.value, "smooth": sm.value}

    def set_tiles(self, by, zc):
        _check(_lib.pf_set_tiles(self.handle, int(by), int(zc)), self.handle)

    def get_tiles(self):
        by, zc = C.c_int(), C.c_int()
        _check(_lib.pf_get_tiles(self.handle, C.byref(by), C.byref(zc)), self.handle)
        return by.value, zc.value

    def autotune(self, cache_path=None):
        by, zc, ms = C.c_int(), C.c_int(), C.c_double()
        _check(_lib.pf_autotune(self.handle, cache_path.encode() if cache_path else None, C.byref(by), C.byref(zc),
                                C.byref(ms)), self.handle)
        return by.value, zc.value, ms.value

    def profile_stages(self, n_attempts):
        out = (C.c_double * 6)()
        _check(_lib.pf_profile_stages(self.handle, int(n_attempts), out), self.handle)
        return list(out)

    def max_phase_rate(self):
        v = C.c_double()
        _check(_lib.pf_max_phase_rate(self.handle, C.byref(v)), self.handle)
        return v.value


# C-named entry points (same names as include/pf.h)
def pf_create_grid(n1, n2, n3, h, model, reaction, precision, params, stream=None):
    return Grid((n1, n2, n3), h, model, reaction, precision, params, stream)


def pf_destroy_grid(g):
    g.close()


def pf_set_geometry(g, spheres, x3_cap=math.nan):
    g.set_geometry(spheres, x3_cap)


def pf_set_glass(g, G):
    g.set_glass(G)


def pf_get_glass(g):
    return g.get_glass()


def pf_set_state(g, theta, phi, t=0.0, dt=1e-3):
    g.set_state(theta, phi, t, dt)


def pf_get_state(g):
    return g.get_state()


def pf_rhs(g, t, theta_in, phi_in, dtheta_out, dphi_out):
    g.rhs(t, theta_in, phi_in, dtheta_out, dphi_out)


def pf_rkm_step(g, dt, tol, force_accept=False):
    return g.rkm_step(dt, tol, force_accept)


def pf_run_to(g, t_end, tol, max_steps=10 ** 9):
    return g.run_to(t_end, tol, max_steps)


def pf_run_fixed(g, n_steps, dt):
    return g.run_fixed(n_steps, dt)


def pf_unfrozen_fraction(g, region=None):
    return g.unfrozen_fraction(region)


def pf_max_phase_rate(g):
    return g.max_phase_rate()


def pf_profile_stages(g, n_attempts):
    return g.profile_stages(n_attempts)


class Batch:
    """Owning handle of a pf_batch: the grids passed in become batch-owned (their Python handles are
    detached and must not be used except through Batch.grid_state)."""

    def __init__(self, grids):
        lib = load_library()
        self.grids = list(grids)
        arr = (C.c_void_p * len(self.grids))(*[g.handle for g in self.grids])
        out = C.c_void_p()
        st = lib.pf_batch_create(len(self.grids), arr, C.byref(out))
        if st != PF_OK:
            msg = lib.pf_batch_last_error(None)
            raise PfError(st, msg.decode() if msg else "")
        for g in self.grids:
            g._owned_by_batch = True
        self.handle = out
        self.n = len(self.grids)

    def _check(self, st):
        if st != PF_OK:
            msg = _lib.pf_batch_last_error(self.handle)
            raise PfError(st, msg.decode() if msg else "")

    def autotune(self, cache_path=None):
        self._check(_lib.pf_batch_autotune(self.handle, cache_path.encode() if cache_path else None))
        return [g.get_tiles() for g in self.grids]

    def run_to(self, t_end, tol, max_steps, eq_window=None, eq_rel_tol=0.0, eq_rate=None):
        te = (C.c_double * self.n)(*[float(v) for v in t_end])
        er = None if eq_window is None else (C.c_double * self.n)(*[float(v) for v in eq_window])
        rr = None if eq_rate is None else (C.c_double * self.n)(*[float(v) for v in eq_rate])
        res = (pf_batch_result * self.n)()
        self._check(_lib.pf_batch_run_to(self.handle, te, er, float(eq_rel_tol), rr, float(tol), int(max_steps), res))
        return [r.as_dict() for r in res]

    def iterations(self):
        return _lib.pf_batch_iterations(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            _lib.pf_batch_destroy(self.handle)
            self.handle = None
            for g in self.grids:
                g.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Slabs:
    """Owning handle of a pf_slabs group: the n1 x n2 x n3 grid cut along x3 into slabs that exchange
    their cut planes every stage and share one step control (the paper's 1-D decomposition, Sec. 2.5,
    in one process on one GPU).  Host arrays hold the whole grid."""

    def __init__(self, shape, h, model, reaction=0, precision=0, params=None, nslabs=2, planes=None, stream=None):
        lib = load_library()
        self.shape = tuple(int(v) for v in shape)
        self.N = self.shape[0] * self.shape[1] * self.shape[2]
        self.params = dict(params or _inputs.default_params())
        self._cparams = make_params(self.params)
        import torch
        self.stream = stream if stream is not None else torch.cuda.Stream()
        pl = None if planes is None else (C.c_int * (nslabs + 1))(*[int(v) for v in planes])
        out = C.c_void_p()
        st = lib.pf_slabs_create(self.shape[0], self.shape[1], self.shape[2], float(h), int(model), int(reaction),
                                 int(precision), C.byref(self._cparams), int(nslabs), pl,
                                 C.c_void_p(self.stream.cuda_stream), C.byref(out))
        if st != PF_OK:
            msg = lib.pf_slabs_last_error(None)
            raise PfError(st, msg.decode() if msg else "")
        self.handle = out
        self.nslabs = int(nslabs)

    def _check(self, st):
        if st != PF_OK:
            msg = _lib.pf_slabs_last_error(self.handle)
            raise PfError(st, msg.decode() if msg else "")

    def set_geometry(self, spheres, x3_cap=math.nan):
        sp = np.ascontiguousarray(spheres, dtype=np.float64).reshape(-1, 4)
        self._check(_lib.pf_slabs_set_geometry(self.handle, sp.ctypes.data if sp.size else None, sp.shape[0], x3_cap))

    def set_tiles(self, by, zc):
        self._check(_lib.pf_slabs_set_tiles(self.handle, int(by), int(zc)))

    def set_state(self, theta, phi, t=0.0, dt=1e-3):
        pt, k1 = _host(theta, self.N)
        pp, k2 = _host(phi, self.N)
        self._check(_lib.pf_slabs_set_state(self.handle, pt, pp, float(t), float(dt)))

    def get_state(self):
        th, ph = np.empty(self.N), np.empty(self.N)
        t, dt = C.c_double(), C.c_double()
        self._check(_lib.pf_slabs_get_state(self.handle, th.ctypes.data, ph.ctypes.data, C.byref(t), C.byref(dt)))
        return th, ph, t.value, dt.value

    def run_to(self, t_end, tol, max_steps):
        s = pf_run_stats()
        self._check(_lib.pf_slabs_run_to(self.handle, float(t_end), float(tol), int(max_steps), C.byref(s)))
        return s.as_dict()

    def unfrozen_fraction(self):
        u = C.c_double()
        ni, nw = C.c_longlong(), C.c_longlong()
        self._check(_lib.pf_slabs_unfrozen_fraction(self.handle, C.byref(u), C.byref(ni), C.byref(nw)))
        return {"uwc": u.value, "n_ice": ni.value, "n_water": nw.value}

    def halo_bytes(self):
        return _lib.pf_slabs_halo_bytes(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            _lib.pf_slabs_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pf_batch_create(grids):
    return Batch(grids)


def pf_batch_run_to(b, t_end, tol, max_steps, eq_window=None, eq_rel_tol=0.0, eq_rate=None):
    return b.run_to(t_end, tol, max_steps, eq_window, eq_rel_tol, eq_rate)


def pf_autotune(g, cache_path=None):
    return g.autotune(cache_path)


def pf_measure_peaks():
    """(fp64 TFLOP/s, fp32 TFLOP/s, copy GB/s) measured on the current device."""
    lib = load_library()
    a, b, c = C.c_double(), C.c_double(), C.c_double()
    st = lib.pf_measure_peaks(C.byref(a), C.byref(b), C.byref(c))
    if st != PF_OK:
        raise PfError(st, "pf_measure_peaks failed")
    return a.value, b.value, c.value


def _check_noalloc_arrays(G_dev, phi_dev, shape):
    """Arguments of pf_unfrozen_fraction_noalloc: binary64 tensors of at least n1*n2*n3 elements on the
    current CUDA device.  The kernel reads every cell of the grid's box, so a shorter or narrower array,
    or one on another GPU, would be read out of bounds; raise ValueError before the call instead."""
    n = int(shape[0]) * int(shape[1]) * int(shape[2])
    for name, t in (("G", G_dev), ("phi", phi_dev)):
        if t is None:
            raise ValueError(f"{name} is required")
        if str(t.dtype) != "torch.float64":
            raise ValueError(f"{name} must be float64, got {t.dtype}")
        if t.numel() < n:
            raise ValueError(f"{name} has {t.numel()} elements, the grid needs {n}")
        if not t.is_cuda or not t.is_contiguous():
            raise ValueError(f"{name} must be a contiguous CUDA tensor")
        import torch
        if t.device.index != torch.cuda.current_device():
            raise ValueError(f"{name} is on cuda:{t.device.index}, the current device is cuda:{torch.cuda.current_device()}")


def pf_unfrozen_fraction_noalloc(G_dev, phi_dev, shape, region=None, stream=None):
    """Unfrozen-water counts on caller-owned device arrays, without any device allocation.

    For callers that cannot allocate GPU memory (the library's reduction scratch is a fixed
    module global).  Returns (status, dict); status is returned, not raised, so callers can
    tell PF_E_RANGE (region above the fixed scratch's limit) from other errors.
    """
    _check_noalloc_arrays(G_dev, phi_dev, shape)
    lib = load_library()
    r = None if region is None else (C.c_int * 6)(*[int(v) for v in region])
    u, sm = C.c_double(), C.c_double()
    ni, nw = C.c_longlong(), C.c_longlong()
    st = lib.pf_unfrozen_fraction_noalloc(_dev(G_dev), _dev(phi_dev), int(shape[0]), int(shape[1]), int(shape[2]),
                                          r, None if stream is None else C.c_void_p(stream), C.byref(u),
                                          C.byref(ni), C.byref(nw), C.byref(sm))
    return st, {"uwc": u.value, "n_ice": ni.value, "n_water": nw.value, "smooth": sm.value}


def pf_kernel_launches():
    return load_library().pf_kernel_launches()
