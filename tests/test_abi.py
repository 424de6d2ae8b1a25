"""The C-ABI library builds, loads without a GPU, and exports every function
that include/feasm.h declares; the binding exposes the same names."""

import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "feasm.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(fe_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("fe_create", "fe_destroy", "fe_pattern_build", "fe_pattern_csr", "fe_pattern_crac",
                     "fe_assemble_csr", "fe_assemble_crac", "fe_pattern_free", "fe_strerror"):
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_2012_00585_gb300 import _build
    lib = _build.build()
    out = subprocess.run(["nm", "-D", "--defined-only", lib], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (fe_\w+)$", out, flags=re.M))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing


def test_library_loads_and_binding_names_match():
    from paper_2012_00585_gb300 import feasm
    lib = feasm.load()
    for name in declared_functions():
        assert hasattr(lib, name)
        assert hasattr(feasm, name), f"binding lacks {name}"
    assert feasm.fe_strerror(feasm.FE_ERR_DUP_DOF) == "DOF listed twice in one element"
    assert feasm.fe_strerror(12345) == "unknown error"


def test_header_constants_match_binding():
    from paper_2012_00585_gb300 import feasm
    text = open(HEADER).read()
    for name, val in re.findall(r"#define (FE_\w+) \(?(-?(?:0x)?[0-9A-Fa-f]+)u?\)?", text):
        if hasattr(feasm, name):
            assert getattr(feasm, name) == int(val, 0), name


def test_no_cpu_fallback_in_product_package():
    pkg = os.path.join(ROOT, "paper_2012_00585_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".cpp", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f


@pytest.mark.parametrize("bad", ["fe_create"])
def test_create_without_gpu_fails_cleanly(bad):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2012_00585_gb300 import feasm
    with pytest.raises(feasm.FeError):
        feasm.fe_create(0)
