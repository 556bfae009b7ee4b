"""FP64 CPU oracle for the photoacoustic RTO hot path -- TEST INFRASTRUCTURE ONLY.

A plain, slow, readable restatement of what the method computes, written from
the paper (arXiv 2607.21373) in double precision with NumPy/SciPy.  It exists to
check the CUDA library, never to run in its place: only the tests,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline / reference arm may
import it.  It shares no code with the CUDA path (it has its own assembly,
detector location, time stepping, transpose, CGLS and statistics).

Modules
  fem        P1 matrices M, M_L, K, B of Section 3 (eq. semi-discrete, mass lumping)
             and sensor interpolation Pi (eq. lagrange and the general-Pi remark of 5.1)
  wave       Stoermer-Verlet forward map (eq. fully-discrete), the one-step
             propagator (eq. matrix-stromer), the backward recursion for G^T
             (eq. backward-recursion) with the transposed step (eq. adjoint-verlet)
  rto        noise model (eq. noise-model), extended least-squares system
             (eq. extended-matrices), CGLS, one RTO sample (Algorithm 1),
             ergodic mean/std (eq. ergodic), dense posterior (Appendix A)
  gradient   derivative of a data misfit with respect to per-element c^2,
             by finite differences of the forward map (no adjoint trick)
  matern     Whittle-Matern field by a spectral filter on a periodic box grid,
             trilinear interpolation to the nodes and its transpose, RTO in the
             latent space (Section 4.1.2 eq. matern-cov-op, Section 6.4)
  rng        counter-based N(0,1) draws (SplitMix64 and Box-Muller, from their
             published definitions) keyed by seed, stream, sample and element

Parity status: every function is pinned by a test in tests/test_oracle_*.py
against a closed form, an invariant or a brute-force evaluation, except the
Monte Carlo quality of small-sample std fields (statistical only; parity
unpinned beyond the Monte Carlo bound).
"""
