"""Low-rank truncation flexible operators for the FP64 CPU oracle.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py): only the tests, the smoke
check and the benchmark's CPU legs may use it; it shares no code with the GPU
library.

Section 1.2 (definition of the rank-r truncation operator) reshapes a basis
vector c into a 2D array C and replaces it by its rank-r truncated SVD:
    tau_r(c) = vec(C_r),  C_r = U_r Sigma_r V_r^T.
The paper stacks columns; the vectors here are row-major images (index
row * cols + col), i.e. they hold C^T.  Since (C^T)_r = (C_r)^T, both
orderings give the same map on vectors.

Section 4.1's -RND variants replace the truncated SVD by the randomized SVD
of Halko, Martinsson and Tropp (SIAM Review 53, 2011): a Gaussian test matrix
Omega (cols x (r + p)), the randomized range finder with q steps of subspace
iteration (their Algorithm 4.4), then the direct SVD of the small projected
matrix (their Algorithm 5.1), truncated to rank r.  The paper gives neither
the oversampling p nor q; the library and the oracle take them as parameters
(p = 10, q = 1 by default).  Omega is an input: the same matrix is used at
every step of a solve.
"""
from __future__ import annotations

import numpy as np

from .sfl import Precond


def truncated_svd(C: np.ndarray, r: int) -> np.ndarray:
    """C_r, the rank-r truncated SVD of C (LAPACK SVD as the library step)."""
    U, s, Vt = np.linalg.svd(C, full_matrices=False)
    r = min(r, len(s))
    return (U[:, :r] * s[:r]) @ Vt[:r]


def randomized_svd_truncation(C: np.ndarray, r: int, Omega: np.ndarray, q: int = 1) -> np.ndarray:
    """Rank-r approximation of C by the randomized SVD (HMT 2011, Algorithms
    4.4 and 5.1) with the given test matrix Omega (cols x l, l >= r):
        Y = C Omega,  Q = orth(Y);
        q times:  Q~ = orth(C^T Q),  Q = orth(C Q~);
        B = Q^T C = U~ S V^T;  C_r = Q U~_r S_r V_r^T.
    orth() is a Householder QR (numpy), keeping the first l columns."""
    Q, _ = np.linalg.qr(C @ Omega)
    for _ in range(q):
        Qt, _ = np.linalg.qr(C.T @ Q)
        Q, _ = np.linalg.qr(C @ Qt)
    B = Q.T @ C
    Ub, s, Vt = np.linalg.svd(B, full_matrices=False)
    r = min(r, len(s))
    return (Q @ (Ub[:, :r] * s[:r])) @ Vt[:r]


class LowRank(Precond):
    """tau_r(p): the rank-r truncated SVD of p reshaped to `shape` (row-major)."""

    def __init__(self, r: int, shape: tuple):
        self.r = int(r)
        self.shape = (int(shape[0]), int(shape[1]))

    def __call__(self, p, x_prev):
        return truncated_svd(np.asarray(p).reshape(self.shape), self.r).ravel()


class LowRankRandomized(Precond):
    """tau_r(p) by the randomized SVD with the fixed test matrix Omega
    (shape[1] x (r + p)) and q subspace-iteration steps."""

    def __init__(self, r: int, shape: tuple, Omega: np.ndarray, q: int = 1):
        self.r = int(r)
        self.shape = (int(shape[0]), int(shape[1]))
        self.Omega = np.asarray(Omega, dtype=np.float64)
        self.q = int(q)
        if self.Omega.shape[0] != self.shape[1] or self.Omega.shape[1] < self.r:
            raise ValueError("Omega must be cols x l with l >= r")

    def __call__(self, p, x_prev):
        C = np.asarray(p).reshape(self.shape)
        return randomized_svd_truncation(C, self.r, self.Omega, self.q).ravel()
