"""Host-side pins of the seeded workload generators (no method arithmetic):
the shapes the benchmark workloads are defined by."""
import numpy as np

from paper_1711_11418_gb300 import inputs as I


def test_batched_systems_filling_and_couplings():
    """64 systems, L in {4..16}; Ne = 0.875 Ns rounded to the nearest even
    number; U/t uniform in [2, 8] (seeded)."""
    probs = I.batched_hubbard(64, seed=0)
    assert len(probs) == 64
    ne = sorted({(p.lat.Lx, p.Ne) for p in probs})
    assert ne == [(4, 14), (6, 32), (8, 56), (10, 88), (12, 126), (14, 172), (16, 224)]
    for p in probs:
        assert p.Ne % 2 == 0 and p.lat.Lx == p.lat.Ly
        U = np.asarray(p.U)
        assert np.all((U >= 2.0) & (U <= 8.0)) and np.ptp(U) == 0.0
    assert len({float(np.asarray(p.U)[0]) for p in probs}) == 64
    again = I.batched_hubbard(64, seed=0)
    assert all(np.array_equal(a.params, b.params) for a, b in zip(probs, again))


def test_workload_parameter_counts():
    """16x16 Hubbard: Gutzwiller 1 + distance Jastrow 44 + 2x2-sublattice
    pair orbitals 1024 = 1069; with the MLP factor (512 -> 1024 -> 1)
    another 1024*512 + 1024 + 1024 + 1 = 526,337; J1-J2 16x16 with one
    parameter per site pair: 65,536; 8x8: 1 + 14 + 256 = 271; 8-ring:
    1 + 2 + 16 = 19."""
    p = I.square16_hubbard()
    assert (p.n_g, p.n_v, p.n_f, p.Np) == (1, 44, 1024, 1069)
    assert (p.lat.Ns, p.Ne) == (256, 224)
    assert I.square16_hubbard_mlp().Np == 1069 + 1024 * 512 + 1024 + 1024 + 1
    j = I.j1j2_heisenberg(16, 0.5)
    assert j.Np == 65536 and j.local_spin and j.Ne == 256
    q = I.square8_hubbard()
    assert (q.n_g, q.n_v, q.n_f) == (1, 14, 256)
    r = I.ring8_hubbard()
    assert (r.n_g, r.n_v, r.n_f) == (1, 2, 16)


def test_translation_ops_match_the_oracle_translations():
    """inputs.translation_ops (the bench's operation set) against the oracle's
    translations on periodic and anti-periodic lattices: same site maps and
    boundary signs, in the same order (g = dx + Lx dy)."""
    import numpy as np
    from oracle.projection import translations
    from paper_1711_11418_gb300 import inputs as I
    for lat in (I.square(4, 4, -1, -1), I.square(3, 2, 1, -1), I.chain(6, -1)):
        perm, sign = I.translation_ops(lat)
        ref = translations(lat)
        assert perm.shape == (len(ref), lat.Ns)
        for g, (op, _) in enumerate(ref):
            assert np.array_equal(perm[g], np.array(op.perm))
            assert np.array_equal(sign[g], np.array(op.sign, np.int8))
        assert np.all(np.sort(perm, axis=1) == np.arange(lat.Ns))
