"""FP64 CPU oracle for vectorised multi-chain Hamiltonian Monte Carlo.

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, obviously correct
restatement of the method of "tfp.mcmc: Modern Markov Chain Monte Carlo Tools
Built for Modern Hardware" (Lao et al., 2020) in float64 numpy.  It exists to
check the CUDA path; it is not a fallback for it.  Only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import it, and it imports nothing from the CUDA package: the two sides share
only the seeded input generators, which hold none of the method's arithmetic.

Modules
  philox      Philox4x32-10 counter RNG and Box-Muller (the paper is silent on
              the generator; both sides implement the published definition).
  targets     log-densities and analytic gradients of the four targets.
  hmc         bootstrap, momentum draw, leapfrog, Metropolis-Hastings,
              dual-averaging step-size adaptation and the sample_chain driver.
  diagnostics multi-chain effective sample size and Monte Carlo standard error.
"""
