"""The C-ABI library builds for sm_103a, loads, and exports every entry point
include/imdp.h declares. No compute call runs here (no GPU needed)."""
import os
import re
import subprocess

import pytest

import paper_2401_04068_gb300 as pkg
from paper_2401_04068_gb300 import build as pbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"\b(imdp_[a-z0-9_]+)\s*\(", text)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib_path():
    return pbuild.build()


def _declared_statuses():
    text = open(os.path.join(ROOT, "include", "imdp.h")).read()
    return {name: int(v) for name, v in re.findall(r"\b(IMDP_E[A-Z]+|IMDP_OK)\s*=\s*(\d+)", text)}


def test_binding_status_codes_match_the_header():
    declared = _declared_statuses()
    assert sorted(declared.values()) == sorted(pkg.STATUS_NAMES)
    for name, v in declared.items():
        assert getattr(pkg, name) == v, name


def test_header_declares_the_boundary():
    names = _declared_functions()
    for must in ("imdp_create_csc", "imdp_value_iteration", "imdp_value_iteration_batch", "imdp_model_destroy"):
        assert must in names
    assert sorted(pkg.EXPORTED) == sorted(names)


def test_library_exports_every_declared_symbol(lib_path):
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\s[TW]\s+(\S+)", out))
    missing = [n for n in _declared_functions() if n not in exported]
    assert not missing, missing


def test_library_is_built_for_sm_103a(lib_path):
    assert "arch=compute_103a,code=sm_103a" in " ".join(pbuild.ARCH)
    assert os.path.getsize(lib_path) > 0


def test_loads_and_reports_status_strings(lib_path):
    lib = pkg.load()
    assert pkg.imdp_status_string(0) == "ok"
    assert pkg.imdp_status_string(2) == "infeasible interval model"
    # every status the header defines has its own name in the library and the binding
    names = {pkg.imdp_status_string(c) for c in pkg.STATUS_NAMES}
    assert len(names) == len(pkg.STATUS_NAMES) and "unknown status" not in names
    assert pkg.imdp_status_string(pkg.IMDP_EIO) == "file input/output error"
    assert pkg.imdp_version().count(".") == 2
    assert lib is pkg.load()


def test_product_path_has_no_oracle_dependency():
    # the package and its sources never import or link the oracle
    for dirpath, _, files in os.walk(os.path.join(ROOT, "paper_2401_04068_gb300")):
        if "_build" in dirpath:
            continue
        for f in files:
            if f.endswith((".py", ".cu", ".h", ".cuh")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text and "imdp_oracle" not in text, f


def test_plain_c_client(lib_path, tmp_path):
    # include/imdp.h compiles as strict C99, and a C program links the library and
    # uses the host-only calls (no GPU): bmdp-tool read, write, read back
    import shutil
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    exe = str(tmp_path / "abi_client")
    libdir = os.path.dirname(lib_path)
    libname = os.path.basename(lib_path)[3:-3]  # libNAME.so -> NAME
    subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I", os.path.join(ROOT, "include"),
                    os.path.join(ROOT, "tests", "abi_client.c"), "-L", libdir, f"-l{libname}",
                    f"-Wl,-rpath,{libdir}", "-o", exe], check=True, capture_output=True, text=True)
    out = subprocess.run([exe, os.path.join(ROOT, "tests", "golden", "worked_example.bmdp"),
                          str(tmp_path / "copy.bmdp")], capture_output=True, text=True, timeout=60)
    assert out.returncode == 0, out.stdout + out.stderr
    text = out.stdout
    assert f"version {pkg.imdp_version()}" in text
    assert "status infeasible interval model" in text
    assert "model 3 states 5 columns 13 transitions, terminal 2" in text
    assert "round trip same" in text
    assert "missing file: file input/output error\n" in text
