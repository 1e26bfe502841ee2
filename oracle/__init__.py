"""FP64 CPU oracle for the plane-wave TDA-BSE excitation energy and its nuclear forces.

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, complex128 restatement
of the method of arXiv 2607.20728 (main text Eqs. 1-7, Supplemental Sec. SI)
on the synthetic Gaussian-well model.  Only ``tests/``, ``__graft_entry__.smoke()``
and ``bench.py``'s CPU-baseline leg may import it.  It shares no code with the
CUDA library (``paper_2607_20728_gb300``); the only shared module is the seeded
input generator ``bse_inputs``, which holds none of the method's arithmetic.

Modules:
  basis      plane-wave spheres, FFT grid, real-basis conversion
  model      local Gaussian potential (+ Gaussian ionic charges), dense Hamiltonian, ground
             state: non-SCF, or self-consistent in the Hartree potential (f_Hxc = v_c)
  screening  bare Coulomb and the low-rank PDEP screened interaction W (Eq. 3)
  liouville  the DMPT Liouville operator D + 2K1e - K1d (Eqs. 1-2), P_c, and the coupling
             block B = 2K2e - K2d beyond the TDA (Sec. SI)
  dense_bse  the TDA-BSE matrix and the coupling block B of the full BSE in the explicit
             transition basis (check a); full-BSE excitation energies
  davidson   block Davidson eigensolver on the P_c space
  wannier    Gamma-point Wannier localisation (joint Jacobi diagonalisation) and the K1d
             pair-pruned Liouville operator in the Wannier basis
  forces     U vector (Sec. SI), Z-vector (Eq. 7; coupled by the KS kernels in the Hartree
             model), densities (Eqs. 5-6),
             force contraction (Eq. 4), finite differences

Parity pins: see tests/test_oracle_*.py.  Every function here is pinned by at
least one check that does not re-run its own formula (closed forms, brute force,
finite differences, dense diagonalisation); none is "parity unpinned".
"""
