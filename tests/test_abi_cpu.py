"""Host-side checks of the C ABI: the library builds, loads and exports every
entry point that include/vmc.h declares (no CUDA call is made here)."""
import os
import re

import numpy as np
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


def test_context_rejects_an_unfillable_local_site_mask():
    """Kondo local spins: every marked site must take exactly one electron.
    Four marked sites and two electrons cannot satisfy that; the library
    refuses the problem before any CUDA call."""
    from paper_1711_11418_gb300 import build, inputs, vmc
    vmc.load(build.build())
    p = inputs.kondo_chain(2)
    bad = p.copy_with(Ne=2, local_sites=np.ones(p.Ns, bool))
    with pytest.raises(vmc.VmcError) as e:
        vmc.Context(bad, 2)
    assert e.value.code == -1


def test_kondo_placements_fill_each_local_site_once():
    from paper_1711_11418_gb300 import inputs
    p = inputs.kondo_chain(8)
    cfg = inputs.initial_configs(p.Ns, p.Ne, 20, False, 3, local_sites=p.local_sites)
    for e in cfg:
        up, dn = e[:p.N], e[p.N:]
        assert len(set(up)) == p.N and len(set(dn)) == p.N
        occ = np.bincount(e, minlength=p.Ns)
        assert np.all(occ[p.local_sites] == 1)
