"""CPU oracle for the periodic coupled-cluster Green's function (CCGF).

TEST INFRASTRUCTURE ONLY. Nothing in the product path imports, links or runs
this package: only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` use it. It shares no code with the CUDA path; the two meet
only through arrays produced by the seeded input generator.

Modules (all FP64 / complex128, plain and slow on purpose):

* ``fockspace``  Second-quantised brute force. Builds the Hamiltonian, the
                 cluster operators T and Lambda, and the CCGF of Eqs. 4-8 (and
                 its k-point form, Eq. 9) from their definitions as explicit
                 operators on the Fock space of a tiny system; also the exact
                 (FCI) Green's function of Eq. 1 by a Lehmann / direct solve.
* ``supercell``  Maps a k-point system onto its supercell (a "molecule" of
                 nk*nmo orbitals) with explicit momentum-conservation zeros.
* ``spinorb``    Spin-orbital EOM-IP/EA-CCSD (1h+2h1p / 1p+2p1h, Eq. 8) for a
                 molecule or supercell: similarity-transformed Hamiltonian
                 blocks, sigma vectors, right-hand sides and left vectors.
* ``kccsd``      Spin-adapted closed-shell k-point EOM-IP/EA-CCSD, the
                 formulation the CUDA path also computes, written as plain
                 einsum loops over k-blocks (the timed CPU baseline).
* ``solvers``    Dense LU, eigendecomposition (Lehmann) and restarted GMRES
                 solutions of the shifted systems of Eq. 6, and the
                 contraction of Eq. 7.
"""
