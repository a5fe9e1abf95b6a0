"""CPU FP64 oracle for the DMRG effective-Hamiltonian path (TEST INFRASTRUCTURE ONLY).

This package is the correctness reference for the CUDA library.  It is plain,
slow NumPy written from the paper (Nakatani, Wouters, Van Neck, Chan, "Linear
response theory for the density matrix renormalization group", 2013) and from
the textbook definitions it builds on.  Only the test suite, the smoke check
and the benchmark's CPU-baseline leg may import it; the product path never
does, and the two share no code (inputs come from the separate `synth`
module).

Modules:
  fock    determinant-space and Fock-space operators, FCI (the plain definition
          of H; Sec. "Time-Independent DMRG Equation").
  mps     block-sparse MPS: expansion to determinants, canonical forms,
          decimation (Eqs. mps_wave_gen, mps_wave, gauge-shift).
  blocks  renormalized normal/complementary operator sets, blocking,
          renormalization and the superblock sigma vector (Eqs. dmrg,
          hzero_sb, lopr1st; the "x" summation over complementary operators).
  dmrg    ground-state Davidson sweeps (Eq. dmrg and the sweep around it).
  tda     DMRG-TDA: the sweep algorithm of Fig. alg:dmrgtda and the
          tangent-space Rayleigh-Ritz definition it approximates (Eqs.
          dmrgrpa with W = 0, hsub ... param).
  transition  one-particle transition densities of the TDA states and their
          square norm (Table site_excitation).
  rpa     DMRG-RPA: the second-order matrix W of Eq. dmrgrpa as the energy
          functional's Hessian in a chart, by the paper's pairwise construction and
          through the sweep (Eq. bmatrix), the RPA frequencies, and the
          reduced-problem Davidson of Eq. reducedrpa.
  response  frequency-dependent linear response to a one-body perturbation at the
          TDA and RPA levels, and the exact response function (Eqs. pt_ext,
          realresp, imagresp).

Parity status: every function is pinned by a `-m "not gpu"` test against a
closed form, a brute-force determinant-space computation, an invariant or a
special case; none is "parity unpinned".
"""
