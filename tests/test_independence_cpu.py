"""The CUDA path and the oracle share no code, and the product path has no
CPU fallback.  Source-level checks (no GPU):

* no module of the package, kernel source or header imports, includes or
  loads anything under oracle/;
* no oracle module imports the package (the tests hand it the seeded
  inputs);
* the binding raises VmcError when libvmc.so is missing, before any CUDA
  call.
"""
import os
import re
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_1711_11418_gb300")


def sources(folder, exts):
    for base, _, files in os.walk(folder):
        if "__pycache__" in base or "_build" in base:
            continue
        for f in files:
            if f.endswith(exts):
                yield os.path.join(base, f)


def code_lines(path):
    """Lines of code with comments and docstrings removed (rough, enough
    for import / include statements)."""
    src = open(path, encoding="utf-8").read()
    if path.endswith(".py"):
        src = re.sub(r'""".*?"""', "", src, flags=re.S)
        return [l.split("#")[0] for l in src.splitlines()]
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return [l.split("//")[0] for l in src.splitlines()]


def test_product_does_not_reference_the_oracle():
    files = list(sources(PKG, (".py", ".cu", ".cuh", ".h"))) + \
        list(sources(os.path.join(ROOT, "include"), (".h",)))
    assert files
    for path in files:
        for line in code_lines(path):
            assert "oracle" not in line, (path, line)


def test_oracle_does_not_import_the_product():
    for path in sources(os.path.join(ROOT, "oracle"), (".py",)):
        for line in code_lines(path):
            assert "paper_1711_11418_gb300" not in line, (path, line)
            assert "libvmc" not in line, (path, line)


def test_binding_fails_loudly_without_the_library():
    code = ("import sys\n"
            "from paper_1711_11418_gb300 import vmc\n"
            "try:\n"
            "    vmc.load('/nonexistent/libvmc.so')\n"
            "except vmc.VmcError as e:\n"
            "    print('raised', e.code)\n"
            "    sys.exit(0)\n"
            "sys.exit(1)\n")
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True)
    assert r.returncode == 0 and "raised" in r.stdout, r.stdout + r.stderr
