"""FP64 CPU oracle for the monolithic n-field block-preconditioned GMRES.

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, step-by-step CPU
restatement of the method (numpy / scipy.sparse, float64) used to check the
CUDA path.  Only the test-suite, the smoke check and the CPU-baseline leg of
the benchmark may import it; the solver library never calls it and shares no
code with it.

Modules and the passages they follow:

* ``rng``      - SplitMix64 counter generator (Steele, Lea & Flood 2014) used
                 for aggregation priorities and power-iteration start vectors.
* ``amg``      - smoothed-aggregation AMG setup (Sec. 3.3, the Galerkin coarse
                 operator A^{l+1} = R^l A^l P^l; aggregation after Vanek et al.).
* ``cycles``   - Chebyshev smoother and the multigrid V-cycle (Algorithm 1).
* ``precond``  - BGS(AMG) (Sec. 4.1), n-field SIMPLE(AMG) with merging
                 (Sec. 4.2) and monolithic AMG(BGS) (Sec. 4.3).
* ``krylov``   - right-preconditioned flexible GMRES(m) (Sec. 3.1-3.2).
"""
