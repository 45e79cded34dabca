"""CPU oracle for the many-variable VMC hot path (test infrastructure).

A plain, slow, FP64 restatement of what the method computes, written from
the mVMC paper (Misawa et al., arXiv:1711.11418).  It exists only to check
the CUDA path: tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg
of ``bench.py`` may import it; the product library never does.  It shares
no code with the CUDA path; both receive their inputs from the seeded
generators in ``paper_1711_11418_gb300.inputs``.

Modules
-------
philox        Philox4x32-10 counter-based generator (Salmon et al., SC'11).
pfaffian      Pfaffian by Parlett-Reid elimination; brute-force expansion.
fock          Canonical Fock basis with Jordan-Wigner signs; operator algebra.
wavefunction  psi(x) = P_G P_J <x|phi_AP-Pf> (Sec. 3.2) and O_k (Sec. 3.3.1).
hamiltonian   Local energy E_loc(x) (Eq. MC, Sec. 3.1.1) and ED matrices.
sampler       Metropolis chains with hop / exchange updates (Sec. 3.1.2).
sr            SR matrices S, g and the solve: Cholesky or CG (Sec. 3.3.1-2,
              Algorithm 1).
exact         Exact enumeration over all configurations (tiny systems).
physics       Pair correlations by Eq. MC (measurement mode, Sec. 2.2.3) and the
              structure factors of Sec. 2.4.2.
projection    Momentum and point-group projection of the pair-product part
              (Sec. 3.2.2, Eqs. momP and pointP).
lanczos       First-step power-Lanczos moments and alpha_1 (Sec. 3.4).

Every function cites the passage it follows.  Pins against values the paper
or mathematics fix live in ``tests/test_oracle_*.py``.
"""
