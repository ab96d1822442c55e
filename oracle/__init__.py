"""FP64 CPU oracle for the PSTD quantum-scattering hot path (arXiv 2403.04053).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline leg (and its ``--impl reference`` arm) may import,
call or execute anything in this package.  The product path (the CUDA library and
its Python binding) never does, and this package imports nothing from it: the two
share no code.  Inputs come from ``paper_2403_04053_gb300.inputs`` (seeded
generators only) and are passed in as arrays.

Modules
  pstd_oracle : tables, the leapfrog PSTD update (both TF/SF forms), the running
                single-frequency DFT on the six virtual planes
  ntdf_oracle : the near-to-distant-field transform as the literal per-cell mode
                sum of Eqs. bottomPsi_lm ... Psi, and its far-field limit
  analytic    : textbook closed forms that pin the oracle (partial waves, Born,
                spherical wave, leapfrog mode evolution)
  spinor_oracle : the two-component leapfrog with a gamma sigma . B coupling (EXACT form),
                pinned by its exact splitting into two scalar problems for B = b(r) nhat
  aux_oracle  : the 1-D auxiliary incident wave of Section 2.2.3 (free 1-D leapfrog along
                the incidence axis, read at each node's d by Eqs. pstd_psiinc, pstd_dpsiinc)
  adjoint_oracle : the discrete adjoint (transpose) of the leapfrog run, of the running
                DFT and of the surface transform, and the gradient of a Fresnel-field
                magnitude misfit with respect to V (no counterpart in the paper; pinned by
                central finite differences of the oracle's own forward loss)
"""
