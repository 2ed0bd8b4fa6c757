"""The C-ABI library builds, loads without a GPU, and exports every symbol include/abg.h
declares (no compute calls here)."""
import ctypes
import os
import re

import pytest

from conftest import ROOT


@pytest.fixture(scope="module")
def built():
    from paper_2405_11922_gb300 import build as b
    return b.build()


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "abg.h")).read()
    return sorted(set(re.findall(r"ABG_API\s+[\w\s\*]+?\b(abg_\w+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_symbols()
    for required in ("abg_create", "abg_destroy", "abg_cluster", "abg_propagate",
                     "abg_random_features", "abg_seed_factors", "abg_onmf", "abg_nci",
                     "abg_objective", "abg_strerror"):
        assert required in names


def test_library_exports_every_declared_symbol(built):
    lib = ctypes.CDLL(built)
    missing = [n for n in declared_symbols() if not hasattr(lib, n)]
    assert not missing, f"not exported: {missing}"


def test_binding_covers_header(built):
    import paper_2405_11922_gb300 as abg
    assert set(declared_symbols()) <= set(abg.SIGNATURES)
    L = abg.lib()
    assert L.abg_strerror(0) == b"ok"
    assert L.abg_strerror(-1) == b"invalid argument"


def test_no_oracle_in_product_path():
    # the package never imports the oracle, and the oracle never imports the package
    pkg = os.path.join(ROOT, "paper_2405_11922_gb300")
    for base, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                src = open(os.path.join(base, f)).read()
                assert "oracle" not in re.findall(r"^\s*(?:from|import)\s+(\w+)", src, re.M)
    for f in os.listdir(os.path.join(ROOT, "oracle")):
        if f.endswith(".py"):
            src = open(os.path.join(ROOT, "oracle", f)).read()
            assert "paper_2405_11922_gb300" not in src
