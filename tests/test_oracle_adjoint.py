"""Pins of the differentiable fixed-k oracle (oracle.adjoint), CPU only.

* its forward is the numpy oracle's sFLSQR run to the same k (an independent
  transcription of Algorithm 1);
* its gradients agree with central finite differences along random
  directions;
* a special case with a closed form: S = I, a full window and k = n on a
  small full-column-rank A make x_k the least-squares solution A^+ b for
  every positive d, so dL/db = (A^+)^T xbar and dL/dd = 0.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle as O
import workloads as wl

torch = pytest.importorskip("torch")
OA = pytest.importorskip("oracle.adjoint")


def small_problem(N=16, n_angles=12, seed=3):
    A = wl.siddon_projector(N, n_angles, wl.detector_bins(N))
    rng = np.random.default_rng(seed)
    x = wl.ellipse_phantom(N, rng)
    b, _ = wl.add_noise(A.matvec(x), 0.01, rng)
    return A, b


U = np.finfo(np.float64).eps / 2


@pytest.mark.parametrize("k", [1, 4, 8])
def test_forward_matches_numpy_oracle(k):
    """Two transcriptions of Algorithm 1 agree to rounding, widened by the
    small problem's conditioning (kappa(S A Z_8) ~ 1e3 here)."""
    A, b = small_problem()
    n = A.shape[1]
    d = np.random.default_rng(4).uniform(0.5, 1.5, n)
    S = O.SparseSign(9, 41, 8, A.shape[0])
    r = O.sflsqr(A.scipy(), b, S, maxit=k, tol=0.0, ell=2, tau=O.FixedDiag(d), keep_basis=True)
    kappa = np.linalg.cond(S.mat @ (A.scipy() @ r.Z))
    x, _, _ = OA.gradients(A, b, d, S.dense(), k, 2, np.zeros(n))
    assert np.linalg.norm(x - r.x) <= max(1e-13, 64 * U * kappa) * np.linalg.norm(r.x)


@pytest.mark.parametrize("ell", [1, 2, 3])
def test_gradients_match_finite_differences(ell):
    A, b = small_problem()
    m, n = A.shape
    rng = np.random.default_rng(10 + ell)
    d = rng.uniform(0.5, 1.5, n)
    S = O.SparseSign(9, 31, 8, m).dense()
    xbar = rng.standard_normal(n)
    k = 6
    _, gb, gd = OA.gradients(A, b, d, S, k, ell, xbar)
    At = OA.torch_operator(A)
    St = torch.as_tensor(S)

    def L(bb, dd):
        with torch.no_grad():
            x = OA.sflsqr_fixed_k(At, torch.as_tensor(bb), torch.as_tensor(dd), St, k, ell)
        return float(x.numpy() @ xbar)

    for trial in range(3):
        vb = rng.standard_normal(m)
        vd = rng.standard_normal(n)
        h = 1e-6
        fd_b = (L(b + h * vb, d) - L(b - h * vb, d)) / (2 * h)
        fd_d = (L(b, d + h * vd) - L(b, d - h * vd)) / (2 * h)
        assert abs(fd_b - gb @ vb) <= 1e-6 * max(abs(fd_b), np.linalg.norm(gb) * np.linalg.norm(vb))
        assert abs(fd_d - gd @ vd) <= 1e-6 * max(abs(fd_d), np.linalg.norm(gd) * np.linalg.norm(vd))


def test_full_space_is_least_squares_with_closed_form_gradients():
    rng = np.random.default_rng(5)
    m, n = 14, 6
    A = sp.csr_matrix(rng.standard_normal((m, n)))
    b = rng.standard_normal(m)
    d = rng.uniform(0.5, 2.0, n)
    xbar = rng.standard_normal(n)
    x, gb, gd = OA.gradients(A, b, d, np.eye(m), n, n, xbar)
    Ap = np.linalg.pinv(A.toarray())
    assert np.linalg.norm(x - Ap @ b) <= 1e-10 * np.linalg.norm(Ap @ b)
    assert np.linalg.norm(gb - Ap.T @ xbar) <= 1e-9 * np.linalg.norm(Ap.T @ xbar)
    assert np.linalg.norm(gd) <= 1e-9 * np.linalg.norm(gb) * np.linalg.norm(b) / np.linalg.norm(d)
