"""Host-only checks of the C-ABI boundary: the library builds for sm_103a,
loads, and exports every function include/ndiag.h declares; the product path
and the oracle share no code."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ndiag.h")
PKG = os.path.join(ROOT, "paper_1008_3699_gb300")


def header_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    text = re.sub(r"typedef[^;]*;", "", text, flags=re.S)
    names = re.findall(r"^\s*[A-Za-z_][\w\s\*]*?\b([A-Za-z_]\w*)\s*\([^;{]*?\)\s*;", text, flags=re.M | re.S)
    return sorted(set(n for n in names if not n.endswith("_fn")))


@pytest.fixture(scope="module")
def lib_path():
    from paper_1008_3699_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = header_functions()
    for need in ["ndiag_create", "ndiag_destroy", "sor_sweep", "ssor_apply", "ilu0_factor", "ilu0_apply",
                 "krylov_solve"]:
        assert need in names


def test_library_exports_every_declared_symbol(lib_path):
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True, check=True)
    exported = set(re.findall(r"\sT\s+(\w+)$", out.stdout, flags=re.M))
    missing = [n for n in header_functions() if n not in exported]
    assert not missing, missing


def test_binding_loads_and_lists_the_same_symbols(lib_path):
    from paper_1008_3699_gb300 import ndiag
    L = ndiag.load()
    assert sorted(ndiag.EXPORTED) == header_functions()
    for name in header_functions():
        assert hasattr(L, name)


def test_product_path_never_touches_the_oracle():
    for dirpath, _, files in os.walk(PKG):
        for f in files:
            if f.endswith((".py", ".cu", ".h", ".cpp")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "liboracle" not in text and "oracle.cpp" not in text, f


def test_oracle_shares_no_code_with_the_cuda_library():
    src = open(os.path.join(ROOT, "oracle", "oracle.cpp")).read()
    includes = re.findall(r'#include\s+[<"]([^>"]+)[>"]', src)
    assert all("/" not in i and not i.endswith((".h", ".cuh")) for i in includes), includes
    code = re.sub(r"//[^\n]*", "", src)
    assert "ndiag" not in code and "csrc" not in code


def test_missing_library_fails_loudly(tmp_path):
    from paper_1008_3699_gb300 import ndiag
    with pytest.raises(ImportError):
        ndiag.load(str(tmp_path / "absent.so"))
