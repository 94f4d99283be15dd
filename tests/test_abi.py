"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/hydro.h declares (no GPU needed)."""
import os
import re
import subprocess

import pytest

from paper_1510_06340_b300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    src = open(os.path.join(ROOT, "include", "hydro.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hydro_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    return B.build(verbose=False)


def test_header_declares_the_entry_points():
    names = declared()
    for n in ("hydro_create", "hydro_step", "hydro_batch_step", "hydro_get_primitives"):
        assert n in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (hydro_[a-z0-9_]+)$", out, flags=re.M))
    missing = [n for n in declared() if n not in exported]
    assert not missing, missing


def test_library_loads_and_reports_constants(libpath):
    from paper_1510_06340_b300 import hydro
    assert hydro.lib().hydro_mlp_nparam() == 1189
    from oracle import oracle as O
    assert O.mlp_nparam() == 1189


def test_kernels_are_built_for_sm_103a_only():
    """Every unit is compiled, and the library linked, for sm_103a alone
    (checked on the build commands, not by reading the compiled code)."""
    assert B.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
    for flag in B.ARCH:
        assert flag in B.BASE
    assert not any("compute_" in f or "sm_" in f for f in B.EXTRA)
