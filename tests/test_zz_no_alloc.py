"""The allocation-free unfrozen-water entry point against the grid-based one.

pf_unfrozen_fraction_noalloc serves callers that cannot call cudaMalloc (a plug-in whose host
application owns all device memory, a loop that cannot take an allocation's implicit
synchronisation, a fixed GPU memory budget).  Its reduction scratch is a module-global device
array shared by every call, so two calls in a row on different data must not see each other's
partials.  This file sorts last so that a run stopping at the first failure has already run
every other test; it builds what it needs itself and also passes alone in a fresh process.
"""
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
    pf.load_library()
    return torch, pf


def _grid_counts(pf, shape, G, ph, region):
    g = pf.Grid(shape, 1e-6, I.MODEL_MICRO, I.REACT_SIGMAP1P, I.PREC_FP64, I.default_params(xi=1e-6))
    try:
        g.set_glass(G)
        g.set_state(None, ph, 0.0, 1e-6)
        return g.unfrozen_fraction(region)
    finally:
        g.close()


def test_noalloc_matches_grid_entry_point_twice(env):
    torch, pf = env
    calls = [((45, 38, 29), 31, None), ((70, 33, 41), 32, (3, 61, 0, 33, 5, 40))]
    stream = torch.cuda.current_stream()
    for shape, seed, region in calls:
        _, ph, G = I.random_fields(shape, seed)
        ph[::13] = 0.5
        G[::17] = 0.5
        ref = _grid_counts(pf, shape, G, ph, region)
        Gd = torch.from_numpy(G).cuda()
        pd = torch.from_numpy(ph).cuda()
        torch.cuda.synchronize()
        st, got = pf.pf_unfrozen_fraction_noalloc(Gd, pd, shape, region, stream.cuda_stream)
        assert st == pf.PF_OK
        assert (got["n_water"], got["n_ice"]) == (ref["n_water"], ref["n_ice"])
        assert got["uwc"] == ref["uwc"]
        assert abs(got["smooth"] - ref["smooth"]) <= 1e-12


def test_noalloc_rejects_bad_arguments_and_oversize_regions(env):
    torch, pf = env
    shape = (8, 8, 8)
    Gd = torch.zeros(512, dtype=torch.float64, device="cuda")
    st, _ = pf.pf_unfrozen_fraction_noalloc(Gd, Gd, shape, (0, 9, 0, 8, 0, 8))
    assert st == pf.PF_E_INVALID
    # arrays the kernel would read out of bounds are refused before the call
    for bad in (torch.zeros(512, dtype=torch.float32, device="cuda"),
                torch.zeros(511, dtype=torch.float64, device="cuda"),
                torch.zeros(512, dtype=torch.float64)):
        with pytest.raises(ValueError):
            pf.pf_unfrozen_fraction_noalloc(bad, Gd, shape)
        with pytest.raises(ValueError):
            pf.pf_unfrozen_fraction_noalloc(Gd, bad, shape)
    # host memory handed to the C entry point directly is refused there (not device memory)
    import ctypes as C
    host = (C.c_double * 512)()
    lib = pf.load_library()
    nw = C.c_longlong(-1)
    st = lib.pf_unfrozen_fraction_noalloc(C.cast(host, C.c_void_p), C.c_void_p(Gd.data_ptr()), 8, 8, 8, None, None,
                                          None, None, C.byref(nw), None)
    assert st == pf.PF_E_INVALID and nw.value == -1
    # 1024 x 1024 x 257 cells is above the 2^28-cell limit of the fixed scratch; the arrays are
    # really that large, so nothing could be read out of bounds even without the check.
    big = (1024, 1024, 257)
    n = big[0] * big[1] * big[2]
    Gb = torch.ones(n, dtype=torch.float64, device="cuda")
    pb = torch.zeros(n, dtype=torch.float64, device="cuda")
    st, _ = pf.pf_unfrozen_fraction_noalloc(Gb, pb, big)
    assert st == pf.PF_E_RANGE
    st, got = pf.pf_unfrozen_fraction_noalloc(Gb, pb, big, (0, 1024, 0, 1024, 0, 256))
    assert st == pf.PF_OK and got["n_water"] == 0
    del Gb, pb
    torch.cuda.empty_cache()
