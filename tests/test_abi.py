"""The C-ABI library builds for sm_103a, loads, and exports every function that
include/tim.h declares. No GPU calls here."""
import os
import subprocess

import pytest

from paper_1404_0900_gb300 import build as B
from paper_1404_0900_gb300 import tim


def test_header_declares_the_boundary():
    names = tim.declared_functions()
    for want in ("tim_create", "tim_destroy", "tim_load_graph", "tim_sample_rr",
                 "tim_kpt_estimate", "tim_refine_kpt", "tim_node_select", "tim_run",
                 "tim_strerror"):
        assert want in names


def test_library_loads_and_exports_every_declared_symbol():
    L = tim.lib()
    out = subprocess.run(["nm", "-D", "--defined-only", tim.library_path()],
                         capture_output=True, text=True, check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    for name in tim.declared_functions():
        assert name in exported, name
        assert hasattr(L, name)


def test_library_is_built_for_sm_103a_only():
    out = subprocess.run(["cuobjdump", "--list-elf", tim.library_path()],
                         capture_output=True, text=True)
    if out.returncode != 0:
        pytest.skip("cuobjdump unavailable")
    arches = set()
    for line in out.stdout.splitlines():
        for tok in line.replace(".", " ").split():
            if tok.startswith("sm_"):
                arches.add(tok)
    assert arches == {"sm_103a"}, arches


def test_strerror_without_gpu():
    L = tim.lib()
    assert L.tim_strerror(0) == b"ok"
    assert L.tim_strerror(-1) == b"invalid argument"
    assert L.tim_strerror(-6) == b"call out of order"


def test_create_fails_cleanly_without_device(monkeypatch):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(tim.TimError):
        tim.tim_create(0)


def test_missing_library_fails_loudly(monkeypatch):
    # no fallback: without libtim.so the binding raises instead of computing anything
    monkeypatch.setattr(B, "LIB", "/nonexistent/libtim.so")
    monkeypatch.setattr(tim, "_lib", None)
    with pytest.raises(OSError):
        tim.lib(build_if_missing=False)


def test_product_package_never_imports_the_oracle():
    pkg = os.path.dirname(os.path.abspath(tim.__file__))
    for name in os.listdir(pkg):
        if name.endswith(".py"):
            text = open(os.path.join(pkg, name)).read()
            assert "import oracle" not in text and "from oracle" not in text, name
