"""Host-side checks of the C ABI: the library builds, loads and exports every
entry point that include/vmc.h declares (no CUDA call is made here)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "vmc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(vmc_[a-z_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_symbols()
    for n in ["vmc_create", "vmc_sample", "vmc_measure", "vmc_sr_step", "vmc_destroy"]:
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_1711_11418_gb300 import build, vmc
    lib = build.build()
    L = vmc.load(lib)
    for n in declared_symbols():
        assert hasattr(L, n), n
    assert set(vmc.EXPORTS) == set(declared_symbols())


def test_strerror_is_host_only():
    from paper_1711_11418_gb300 import build, vmc
    L = vmc.load(build.build())
    assert L.vmc_strerror(0) == b"ok"
    assert b"invalid" in L.vmc_strerror(-1)


def test_context_rejects_per_site_local_spin():
    """The CUDA path has no per-site local-spin constraint: a Kondo-lattice
    problem is refused before any CUDA call."""
    from paper_1711_11418_gb300 import build, inputs, vmc
    vmc.load(build.build())
    with pytest.raises(vmc.VmcError):
        vmc.Context(inputs.kondo_chain(2), 2)
