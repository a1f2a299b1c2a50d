"""The C-ABI library loads and exports every function include/ccm.h declares
(no CUDA call is made: this runs without a GPU)."""

from __future__ import annotations

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "ccm.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(ccm_\w+)\s*\(", text, flags=re.M)))


@pytest.fixture(scope="module")
def libpath():
    from paper_1905_00565_gb300 import build
    return build.build()


def test_header_declares_the_abi():
    names = declared_functions()
    for n in ["ccm_plan", "ccm_run", "ccm_submit", "ccm_poll", "ccm_context_create"]:
        assert n in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_names_match_the_header(libpath):
    from paper_1905_00565_gb300 import ccm
    assert sorted(ccm.EXPORTED) == declared_functions()
    for n in ccm.EXPORTED:
        assert callable(getattr(ccm, n))
    assert "sm_103a" in ccm.ccm_version()


def test_oracle_and_cuda_library_share_no_code():
    """The oracle imports nothing from the package and vice versa."""
    import ast
    bad = []
    for d, forbidden in (("oracle", "paper_1905_00565_gb300"),
                         ("paper_1905_00565_gb300", "oracle")):
        for f in os.listdir(os.path.join(ROOT, d)):
            if f.endswith(".py"):
                tree = ast.parse(open(os.path.join(ROOT, d, f)).read())
                for node in ast.walk(tree):
                    if isinstance(node, (ast.Import, ast.ImportFrom)):
                        mods = [a.name for a in node.names] if isinstance(node, ast.Import) \
                            else [node.module or ""]
                        bad += [(d, f, m) for m in mods if m.split(".")[0] == forbidden]
    assert not bad, bad
    for f in os.listdir(os.path.join(ROOT, "paper_1905_00565_gb300", "csrc")):
        src = open(os.path.join(ROOT, "paper_1905_00565_gb300", "csrc", f)).read()
        assert "oracle" not in src.lower().replace("oracles", ""), f
