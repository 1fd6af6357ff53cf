"""Plain FP64 CPU oracle of the online Bayesian inversion (test infrastructure).

This package is test infrastructure, not part of the product.  Only the tests,
`__graft_entry__.smoke()` and the CPU-baseline leg of `bench.py` may import it.
It shares no code with the GPU path; the only common module is `synth`, which
produces seeded inputs and holds none of the method's arithmetic.

Every function is a plain, slow, readable restatement of a definition in the
paper (arXiv 2504.16344):

* `toeplitz` -- the p2o / p2q map as the block lower-triangular Toeplitz
  matrix of Eq. (ShiftInvariance), applied by its direct time-domain sum, and
  its Euclidean adjoint;
* `prior`    -- the Matern prior covariance Gamma_pr (block diagonal in time,
  Sec. "State of the art"), as a spectral filter on the periodic parameter
  grid written with explicit DFT matrices;
* `posterior` -- the data-space Hessian K = Gamma_n + F Gamma_pr F*, its
  Cholesky factor, the posterior mean m = Gamma_pr F* K^{-1} d and forecast
  q = F_q m (Phase 4 of Sec. "Real-time Bayesian inference and prediction
  framework"), the parameter-space MAP system of Eq. (mmap-problem) for
  cross-checks, observation windows and posterior samples;
* `qoi`      -- Phase 3: the data-to-QoI map Q = F_q Gamma_post F* Gamma_n^{-1}
  and the QoI posterior covariance F_q Gamma_post F_q*, formed from QoI unit
  vectors, and their dense parameter-space definitions for tiny cases.

Library primitives used as single steps: numpy matmul, numpy.linalg.cholesky
and scipy.linalg.solve_triangular.  No FFT library is used by the oracle.
"""
from . import toeplitz, prior, posterior, qoi  # noqa: F401
