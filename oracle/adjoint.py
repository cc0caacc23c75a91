"""Differentiable fixed-k sFLSQR (test infrastructure only, like all of oracle/).

Algorithm 1 (sFLSQR) run for exactly k steps (no stop test) with the flexible
operator tau = diag(d), written with plain PyTorch CPU operations in FP64 so
that torch.autograd yields the exact derivative of x_k with respect to b and
d (up to rounding).  It follows the same readings as oracle.sfl: the window of
eq. (FGK) orthogonalizes the new vector against the previous p_j (pre-tau,
unit norm) and the w_j, each coefficient taken from the current vector
(modified Gram-Schmidt, ascending j); the sketched least-squares problem
min ||S A Z_k y - S b|| is solved through a QR factorization of S A Z_k; and
x_k = Z_k y_k.

Only the tests import this module (the GPU library never does).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import torch


def torch_operator(A) -> torch.Tensor:
    """A (scipy sparse or the workloads CSR) as a torch sparse COO tensor (FP64, CPU)."""
    S = A.scipy() if hasattr(A, "scipy") else A
    S = sp.coo_matrix(S)
    idx = torch.as_tensor(np.vstack([S.row, S.col]).astype(np.int64))
    return torch.sparse_coo_tensor(idx, torch.as_tensor(S.data, dtype=torch.float64), S.shape,
                                   check_invariants=True).coalesce()


def sflsqr_fixed_k(A: torch.Tensor, b: torch.Tensor, d: torch.Tensor, S: torch.Tensor, k: int, ell: int):
    """x_k of Algorithm 1 with tau = diag(d), k steps, window ell.

    A: sparse or dense (m x n), b: (m,), d: (n,), S: dense (s x m); returns x (n,)."""
    AT = A.t()

    def mv(M, v):
        return torch.sparse.mm(M, v[:, None])[:, 0] if M.is_sparse else M @ v

    beta = torch.linalg.vector_norm(b)
    W = [b / beta]                       # w_1
    t = mv(AT, W[0])                     # A^T w_1
    P, Z, AZ = [], [], []
    for j in range(1, k + 1):
        q = t
        for i in range(max(1, j - ell), j):              # MGS against p_{j-ell} .. p_{j-1}
            q = q - torch.dot(P[i - 1], q) * P[i - 1]
        p = q / torch.linalg.vector_norm(q)              # p_j
        P.append(p)
        z = d * p                                        # z_j = tau(p_j)
        Z.append(z)
        q = mv(A, z)                                     # A z_j
        AZ.append(q)
        for i in range(max(1, j - ell), j + 1):          # MGS against w_{j-ell} .. w_j
            q = q - torch.dot(W[i - 1], q) * W[i - 1]
        W.append(q / torch.linalg.vector_norm(q))        # w_{j+1}
        t = mv(AT, W[-1])
    M = S @ torch.stack(AZ, 1)                           # S A Z_k
    Q, R = torch.linalg.qr(M)
    y = torch.linalg.solve_triangular(R, (Q.t() @ (S @ b))[:, None], upper=True)[:, 0]
    return torch.stack(Z, 1) @ y


def gradients(A, b: np.ndarray, d: np.ndarray, S_dense: np.ndarray, k: int, ell: int, xbar: np.ndarray):
    """(x, dL/db, dL/dd) for L = <xbar, x_k(b, d)>, by autograd."""
    At = torch_operator(A)
    bt = torch.tensor(b, dtype=torch.float64, requires_grad=True)
    dt = torch.tensor(d, dtype=torch.float64, requires_grad=True)
    St = torch.as_tensor(S_dense, dtype=torch.float64)
    x = sflsqr_fixed_k(At, bt, dt, St, k, ell)
    (x * torch.as_tensor(xbar, dtype=torch.float64)).sum().backward()
    return x.detach().numpy(), bt.grad.numpy(), dt.grad.numpy()
