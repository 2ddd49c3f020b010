"""Plain, slow, obviously-correct FP64 CPU oracle of the space-charge tracking step.

TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check of the package entry
module and the CPU-baseline leg of the benchmark may import, call or link
anything here.  The product path (the CUDA library and its Python binding)
never does, and shares no code with it.

What it computes follows arXiv:2208.02382 (ImpactX v22.08):
  * §Model Assumptions: s-based tracking with linear symplectic maps; space
    charge is electrostatic in the bunch rest frame, applied by a map-based
    split-operator step;
  * §ImpactX / Listing 1: particle shape (B-spline order), space-charge switch,
    lattice of sliced elements, reference particle set from kinetic energy;
  * the reused PIC routines (charge deposition, Poisson solve, beam statistics).
The paper prints no formulas.  Every formula here is the textbook reading of
those statements, and each function says which reading it takes.

Modules:
  physics      constants, reference particle, element maps, slice schedule
  spacecharge  rest-frame box rule, CIC deposit, IGF Green's function,
               Hockney doubled-grid solve, field, gather + kick
  igf_quad.c   the integrated Green's function antiderivative in __float128
  track        the split-operator tracking loop and beam moments
  distribution Waterbag and Gaussian bunches in the Listing-1 parametrisation
  adjoint      reverse-mode gradients of final rms sizes / emittances with
               respect to quadrupole strengths and initial Twiss parameters

Parity pins (closed forms, invariants, the paper's worked example, brute force)
are in tests/test_oracle_*.py.  Functions without such a pin say "parity
unpinned" in their docstring.
"""
