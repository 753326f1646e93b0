"""Plain FP64 CPU oracle for the CheFSI hot path -- TEST INFRASTRUCTURE ONLY.

Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline / reference arm may
import this package.  The CUDA library never calls it and shares no code with it.

What it computes (paper: real-space high-order finite-difference Kohn-Sham with
Chebyshev-filtered subspace iteration, CheFSI):
  fd.py          order-2M central second-derivative weights (high-order FD, Intro)
  grid.py        spherical Dirichlet grid (or box), lexicographic order (Intro, Method)
  potential.py   synthetic local potential + Kleinman-Bylander projectors
                 (Computational details: norm-conserving pseudopotentials in KB form)
  hamiltonian.py H = -1/2 Laplacian_h + V_loc + V_NL as a sparse operator
  chefsi.py      Chebyshev filter p_m(H)X, Cholesky-QR, Rayleigh-Ritz, density,
                 spectral bounds and the CheFSI outer loop (CheFSI paragraph)

Everything is float64 numpy/scipy.  Pins against closed forms live in tests/.
Parity pinned: FD weights, kinetic operator (box spectrum, polynomial exactness),
KB operator (dense assembly), filter (Chebyshev closed form), Cholesky-QR
(orthonormality), Rayleigh-Ritz (brute-force spectra, harmonic oscillator),
density (electron count, analytic ground state of the harmonic oscillator), SCF
total energy (the Kohn-Sham functional evaluated directly from the orbitals), LDA,
Poisson, mixing and occupations (scf.py), learned-start descriptors, network forward
pass (single-path closed form), gradients and Adam (learned.py).  Parity unpinned:
the absolute eigenvalues of the synthetic silicon Hamiltonian (the paper prints none
for any reproducible system).
"""
