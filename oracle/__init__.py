"""Plain FP64 CPU oracle for the sketched flexible Golub-Kahan solvers.

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's CPU
baseline leg are the only code allowed to import it.  It shares no code with
the GPU library (paper_2605_22281_gb300) and the GPU library never imports it.

Modules:
  sketch  - SplitMix64 and the sparse-sign / Gaussian / identity sketches (Section 2.7)
  sfl     - Algorithm 1 (sFLSQR) and Algorithm 2 (sFLSMR) with window-ell
            orthogonalization (eq. (FGK)), Householder small least squares,
            identity / fixed-diagonal / reweighting flexible operators, and the
            discrepancy stop of eq. (discrP).
  lowrank - the rank-r truncation operator of Section 1.2 (truncated SVD of
            the basis vector reshaped to an image) and its randomized-SVD form
            (the -RND variants of Section 4.1).
  adjoint - fixed-k sFLSQR with tau = diag(d) in plain PyTorch CPU FP64 ops,
            differentiated by autograd (imported on demand: `oracle.adjoint`).
"""
from .sketch import (SRHT, DenseSketch, GaussianHash, IdentitySketch, SparseSign, draw_hash, gaussian,
                     gaussian_hash_dense, sparse_sign_column, srht_dense, srht_rows, srht_signs,
                     sparse_sign_rows, splitmix64_stream)
from .sfl import (STOP_BREAKDOWN, STOP_DISCREPANCY, STOP_MAXIT, FixedDiag, Identity, Reweighting,
                  discrepancy_tol, householder_lstsq, sflsmr, sflsqr, sketches_for)
from .lowrank import LowRank, LowRankRandomized, randomized_svd_truncation, truncated_svd
