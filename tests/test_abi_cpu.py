"""CPU checks of the C-ABI boundary: the library builds, loads and exports every symbol
include/*.h declares, and the ctypes mirrors of the structs match the C layout.
No compute call is made (no GPU here)."""
import ctypes as C
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
INCLUDE = os.path.join(ROOT, "include")


def _declared(header):
    src = open(os.path.join(INCLUDE, header)).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b((?:pf|pfnn|pfb)_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2401_01672_gb300 import build
    build.build()
    from paper_2401_01672_gb300 import pf
    return pf.load_library()


def test_every_declared_symbol_is_exported(lib):
    from paper_2401_01672_gb300 import pf
    headers = [h for h in os.listdir(INCLUDE) if h.endswith(".h")]
    names = []
    for h in headers:
        names += _declared(h)
    assert "pf_create_grid" in names and "pf_run_to" in names
    out = subprocess.run(["nm", "-D", "--defined-only", pf.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (\w+)$", out, flags=re.M))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    for n in names:
        getattr(lib, n)


def test_binding_lists_match_header():
    from paper_2401_01672_gb300 import pf
    assert sorted(pf.EXPORTS) == _declared("pf.h")


def _c_layout(struct, fields):
    code = ['#include <stdio.h>', '#include <stddef.h>', '#include "pf.h"', 'int main(void){',
            f'printf("%zu\\n", sizeof({struct}));']
    for f in fields:
        code.append(f'printf("%zu\\n", offsetof({struct}, {f}));')
    code.append("return 0;}")
    d = os.path.join(ROOT, "paper_2401_01672_gb300", "_build")
    os.makedirs(d, exist_ok=True)
    src = os.path.join(d, f"layout_{struct}.c")
    exe = src[:-2]
    open(src, "w").write("\n".join(code))
    subprocess.check_call(["gcc", "-I", INCLUDE, "-o", exe, src])
    vals = [int(v) for v in subprocess.check_output([exe]).split()]
    return vals[0], vals[1:]


def test_params_struct_layout():
    from paper_2401_01672_gb300 import pf
    cf = [n for n, _ in pf.pf_params._fields_]
    cnames = [("lambda" if n == "lambda_" else n) for n in cf]
    size, offs = _c_layout("pf_params", cnames)
    assert size == C.sizeof(pf.pf_params)
    assert offs == [getattr(pf.pf_params, n).offset for n in cf]


def test_run_stats_struct_layout():
    from paper_2401_01672_gb300 import pf
    cf = [n for n, _ in pf.pf_run_stats._fields_]
    size, offs = _c_layout("pf_run_stats", cf)
    assert size == C.sizeof(pf.pf_run_stats)
    assert offs == [getattr(pf.pf_run_stats, n).offset for n in cf]


def test_product_path_does_not_import_oracle():
    """The library package never imports the oracle (test infrastructure only)."""
    pkg = os.path.join(ROOT, "paper_2401_01672_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".c")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt and "pf_oracle" not in txt, f


def test_missing_library_fails_loudly(tmp_path):
    from paper_2401_01672_gb300 import pf
    saved = pf._lib
    pf._lib = None
    try:
        with pytest.raises(ImportError):
            pf.load_library(str(tmp_path / "nope.so"))
    finally:
        pf._lib = saved


def test_noalloc_wrapper_refuses_arrays_it_would_overrun():
    """pf_unfrozen_fraction_noalloc reads n1*n2*n3 binary64 values from each array: the binding refuses
    narrower, shorter or host arrays before the C call (checked without a GPU)."""
    torch = pytest.importorskip("torch")
    from paper_2401_01672_gb300 import pf
    good = torch.zeros(512, dtype=torch.float64)
    for bad in (torch.zeros(512, dtype=torch.float32), torch.zeros(511, dtype=torch.float64), good, None):
        with pytest.raises(ValueError):
            pf.pf_unfrozen_fraction_noalloc(bad, good, (8, 8, 8))
        with pytest.raises(ValueError):
            pf.pf_unfrozen_fraction_noalloc(good, bad, (8, 8, 8))
