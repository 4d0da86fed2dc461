"""Plain FP64 CPU oracle for SoftAbs-RMHMC on hierarchical (additive multiple-kernel)
Gaussian-process models.

THIS PACKAGE IS TEST INFRASTRUCTURE. It exists to check the CUDA path, never to serve it:
only the test suite, the package smoke check and the benchmark's CPU-baseline leg may import
it. It shares no code with the CUDA path (no kernels, headers, helpers, constants or
pre/post-processing); both receive the same seeded synthetic inputs and nothing else.

Every function computes the plain definition with NumPy/LAPACK in float64:
  * kernels.py    kernel matrices and their hyperparameter derivatives (Eq. BMKL, Eq. hpar_prior)
  * model.py      U(q), its gradient, Hessian and third-derivative slices (Eq. data_likelihood,
                  Sec. 2.3)
  * softabs.py    the soft-absolute map g, g', and the divided-difference matrix T (Sec. 2.2,
                  Eq. d3_transform)
  * geometry.py   eigendecomposition (LAPACK eigh), G, W1, W2, dH/dq via the full
                  third-derivative tensor (Eqs. Hamiltonian, d_Hamiltonian, Betancourt_formula)
  * integrator.py the generalized (implicit) leapfrog with fixed-point iterations (Eq. leapfrog)
  * sampler.py    Algorithm 1 with Metropolis-Hastings and momentum p ~ N(0, G)
  * philox.py     Philox4x64-10 counter-based generator (Salmon et al. 2011) + Box-Muller
  * jacobi.py     a separate cyclic Jacobi eigensolver used only for sweep-count checks (Sec. 2.4)
  * primal.py     the reduced-rank (primal) model of Sec. 2.5: features, spectral weights, U and
                  its derivatives, and the mean/variance model of Example 1 (J = 2)
  * bme.py        thermodynamic integration for the model evidence (the BME appendix) and the
                  closed-form tempered means of a Gaussian-likelihood GP

Pins (see tests/test_oracle_*.py): finite differences of U and its derivatives, closed-form
soft-abs limits, the Gaussian-likelihood GP posterior, brute-force quadrature at tiny N,
leapfrog reversibility, eps^2 energy-error scaling, numpy's library Philox, scipy's MVN. The pins'
sharpness is tested too: tests/test_oracle_mutations.py plants single-text mistakes in copies of
these modules and requires a pin to fail for each.
"""
