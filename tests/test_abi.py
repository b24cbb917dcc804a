"""CPU checks of the boundary: the C ABI library builds, loads, and exports
every function that include/iluk.h declares (no GPU work is launched)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "iluk.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^[A-Za-z_][\w \*]*?\b(\w+)\s*\(", src, flags=re.M)
    return sorted(set(n for n in names if n not in ("if", "defined")))


@pytest.fixture(scope="module")
def lib_path():
    from paper_0803_0048_gb300 import build
    return build.build()


def test_header_parses():
    names = declared_functions()
    for must in ("iluk_symbolic", "iluk_numeric", "iluk_apply", "iiluk_build", "gmres_solve"):
        assert must in names


def test_library_exports_every_declared_function(lib_path):
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True,
                         text=True, check=True).stdout
    exported = set(line.split()[-1] for line in out.splitlines() if " T " in line)
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing


def test_binding_covers_every_declared_function(lib_path):
    from paper_0803_0048_gb300 import _lib
    assert sorted(_lib.exported_symbols()) == declared_functions()
    lib = _lib.load()
    for name in declared_functions():
        assert getattr(lib, name) is not None
    assert lib.iluk_strerror(4) == b"zero pivot"


def test_status_codes_match_header():
    from paper_0803_0048_gb300 import _lib
    src = open(os.path.join(ROOT, "include", "iluk.h")).read()
    for name, val in re.findall(r"ILUK_(E\w+|OK) = (\d+)", src):
        assert getattr(_lib, name) == int(val), name


def test_product_path_does_not_import_oracle():
    pkg = os.path.join(ROOT, "paper_0803_0048_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "iluk_oracle" not in text, f
