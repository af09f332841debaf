"""The C ABI builds for sm_103a, loads without a GPU and exports every entry point that
include/bgk.h declares; the CUDA path and the oracle share no code. CPU only (no compute calls)."""
import os
import re
import subprocess

import pytest

from paper_2308_06196_gb300 import _build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    txt = open(os.path.join(ROOT, "include", "bgk.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(bgk_[a-z_0-9]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def libpath():
    return _build.build()


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (bgk_\w+)", out))
    decl = declared_symbols()
    assert len(decl) >= 15
    missing = [s for s in decl if s not in exported]
    assert not missing, f"declared but not exported: {missing}"


def test_binding_loads_and_names_match(libpath):
    from paper_2308_06196_gb300 import bgk

    L = bgk.lib()
    for s in declared_symbols():
        assert hasattr(L, s)
    assert sorted(bgk.SYMBOLS) == declared_symbols()


def test_oracle_and_library_share_no_code():
    pkg = os.path.join(ROOT, "paper_2308_06196_gb300")
    for dirpath, _, files in os.walk(pkg):
        for fn in files:
            if fn.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                txt = open(os.path.join(dirpath, fn)).read()
                assert "oracle" not in txt.lower() or fn == "workloads.py", f"{fn} mentions the oracle"
    for fn in os.listdir(os.path.join(ROOT, "oracle")):
        if fn.endswith((".py", ".c", ".h")):
            txt = open(os.path.join(ROOT, "oracle", fn)).read()
            assert "paper_2308_06196_gb300" not in txt and "bgk.h" not in txt



def test_noalloc_wrapper_checks_buffers_before_any_launch():
    # the C entry point cannot see buffer sizes, so the binding checks dtype, shape and device of every
    # tensor and raises before calling into the library (CPU tensors here: nothing reaches a GPU)
    torch = pytest.importorskip("torch")
    from paper_2308_06196_gb300 import bgk

    nv, lo, hi = (4, 4, 4), (-3.0,) * 3, (3.0,) * 3
    good_f = torch.zeros((5, 64), dtype=torch.float32)
    good_q = torch.zeros((5, 5), dtype=torch.float64)
    cases = [
        (torch.zeros((5, 64), dtype=torch.float64), good_q, good_q),   # f in FP64
        (torch.zeros((5, 63), dtype=torch.float32), good_q, good_q),   # f of another velocity grid
        (torch.zeros((320,), dtype=torch.float32), good_q, good_q),    # f not [npts, N_v]
        (good_f, torch.zeros((5, 5), dtype=torch.float32), good_q),    # Q in FP32
        (good_f, good_q, torch.zeros((4, 5), dtype=torch.float64)),    # prim too short
        (good_f, torch.zeros((5, 4), dtype=torch.float64), good_q),    # Q of 4 components
        (good_f, good_q, good_q),                                      # host tensors
    ]
    for f, q, p in cases:
        with pytest.raises(ValueError):
            bgk.equilibrium_noalloc(f, nv, lo, hi, q, p)
