"""The C-ABI library builds, loads without a GPU and exports every symbol
declared in include/*.h.  No compute call is made here."""
import ctypes
import glob
import os
import re

import pytest

from conftest import ROOT

import paper_2503_18198_gb300 as spm
from paper_2503_18198_gb300 import _build, binding


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        for m in re.finditer(r"\b([A-Za-z_][A-Za-z0-9_]*)\s*\(", text):
            name = m.group(1)
            if name.startswith(("spm", "cpd_")) and not name.isupper() \
                    and not name.startswith(("SPM_",)):
                names.add(name)
    return names


def test_library_builds_and_exports_every_declared_symbol():
    path = _build.build()
    lib = ctypes.CDLL(path)
    names = declared_functions()
    assert {"spmttkrp_plan", "spmttkrp_run", "cpd_als_step"} <= names
    for n in sorted(names):
        assert hasattr(lib, n), f"{n} declared in include/ but not exported"
    assert set(binding.SYMBOLS) <= names
    # the Python binding has a function of the same name for every entry point
    for n in sorted(names):
        assert callable(getattr(binding, n, None)), f"{n} has no binding function"


def test_status_strings_and_no_device_behaviour():
    spm.load(build_if_missing=True)
    assert spm.spm_status_string(0) == "ok"
    assert "range" in spm.spm_status_string(2)
    assert spm.spm_status_string(99) == "unknown status"


def test_invalid_arguments_rejected_on_host():
    lib = spm.load(build_if_missing=True)
    h = ctypes.c_void_p()
    dims = (ctypes.c_int64 * 3)(4, 4, 4)
    # bad mode count, bad rank, bad dims: rejected before any device work
    assert lib.spmttkrp_plan(ctypes.byref(h), 1, dims, 0, None, None, 4, 0, None) == 1
    assert lib.spmttkrp_plan(ctypes.byref(h), 3, dims, 0, None, None, 0, 0, None) == 1
    assert lib.spmttkrp_plan(ctypes.byref(h), 3, dims, 0, None, None, 999, 0, None) == 1
    bad = (ctypes.c_int64 * 3)(4, 0, 4)
    assert lib.spmttkrp_plan(ctypes.byref(h), 3, bad, 0, None, None, 4, 0, None) == 1
    # unknown flag bits
    assert lib.spmttkrp_plan(ctypes.byref(h), 3, dims, 0, None, None, 4, 1 << 10, None) == 1
    # the fibre layout outside its shapes: rank 4, four modes (SPM_ERR_UNSUPPORTED)
    assert lib.spmttkrp_plan(ctypes.byref(h), 3, dims, 0, None, None, 4, spm.SPM_PLAN_FIBRE,
                             None) == 7
    dims4 = (ctypes.c_int64 * 4)(4, 4, 4, 4)
    assert lib.spmttkrp_plan(ctypes.byref(h), 4, dims4, 0, None, None, 32, spm.SPM_PLAN_FIBRE,
                             None) == 7
    # null plan handles
    assert lib.spmttkrp_run(None, 0, None, None, None) == 1
    assert lib.cpd_als_step(None, None, None, None, None) == 1
    lib.spmttkrp_plan_destroy(None)


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    monkeypatch.setattr(binding, "_lib", None)
    monkeypatch.setattr(binding, "library_path", lambda: str(tmp_path / "nope.so"))
    with pytest.raises(RuntimeError, match="missing"):
        binding.load()
