"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/hsma.h declares (no compute call: this runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "hsma.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(hsma_\w+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_1806_04801_gb300 import build
    build.build()
    from paper_1806_04801_gb300 import hsma
    return hsma.lib()


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("hsma_plan", "hsma_energy_forces", "hsma_energy_forces_batched", "hsma_plan_destroy",
                 "hsma_strerror", "hsma_plan_footprint"):
        assert must in names


def test_every_declared_symbol_is_exported_and_bound(lib):
    from paper_1806_04801_gb300 import hsma
    for name in declared_functions():
        assert hasattr(lib, name), name
        assert name in hsma.SIGNATURES, f"{name} has no ctypes signature in the binding"


def test_host_only_calls(lib):
    from paper_1806_04801_gb300 import hsma
    assert "sm_103a" in hsma.version()
    assert hsma.strerror(0) == "ok"
    assert "neutral" in hsma.strerror(-2)
    o = hsma.hsma_opts()
    assert lib.hsma_opts_default(ctypes.byref(o)) == 0
    assert o.precision == hsma.FP32_ACC64 and o.use_graphs == 1
    assert lib.hsma_opts_default(None) == -1
    assert hsma.kernel_launches() >= 0


def test_library_is_built_for_sm_103a_only():
    import subprocess
    from paper_1806_04801_gb300 import build
    src = open(os.path.join(ROOT, "paper_1806_04801_gb300", "build.py")).read()
    assert "arch=compute_103a,code=sm_103a" in src
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_binding_refuses_to_run_without_library(tmp_path, monkeypatch):
    from paper_1806_04801_gb300 import hsma
    monkeypatch.setattr(hsma, "_LIB", None)
    monkeypatch.setattr(hsma, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError, match="not built"):
        hsma.lib()
