"""The C-ABI library loads and exports every entry point include/qmc.h
declares; without a GPU it refuses to create a context (no CPU fallback)."""
import os
import re
import subprocess

import pytest

from paper_2305_19768_gb300 import qmc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(qmc_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


def test_header_declares_the_binding_names():
    assert set(declared_functions()) == set(qmc.exported_symbols())


def test_library_exports_every_declared_symbol():
    path = qmc.lib() and qmc.library_path()
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (qmc_[a-z0-9_]+)", out))
    missing = set(declared_functions()) - exported
    assert not missing, missing


def test_no_context_without_gpu():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(qmc.QmcError) as ei:
        qmc.qmc_create(0)
    assert ei.value.code == -3
