"""FP64 CPU oracle for batched multi-Debye fitting -- TEST INFRASTRUCTURE ONLY.

A plain, slow, obviously correct numpy implementation of what the CUDA library
computes, written from the paper (Majchrowska et al., "Modelling Arbitrary
Complex Dielectric Properties -- an automated implementation for gprMax",
arXiv:2109.01928). Only the test suite, the smoke check and the benchmark's
CPU-baseline leg may import it; the library itself never does, and this
package imports nothing from the library.

Modules
  models  target permittivity models, Eqs. 1 and 3-7
  dls     Debye basis (Eq. 7) and the damped least-squares cost with the
          negative-weight sign flip (Sec. III-B)
  varpro  analytic gradient of that cost w.r.t. log10(tau)
  rng     SplitMix64 counter-based random numbers
  pso     particle-swarm search over log10(tau) (Sec. III-A, Kennedy-Eberhart)
  de      differential evolution over log10(tau) (Sec. III-B, Storn-Price)
  da      dual annealing over log10(tau) (Sec. III-B, Tsallis-Stariolo)
  dmath   log, exp and normal deviates as fixed sequences of IEEE operations
  lbfgs   projected L-BFGS polish
  fit     the whole fit of one spectrum and the reported result (Listing 2)

Every function states the passage it follows. Where the paper is silent the
reading taken is stated in the function's docstring.
"""
