"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: published
generator outputs, textbook LSQR / LSMR (SciPy, run as libraries), dense
Krylov projections and dense SVD least squares (LAPACK), Theorem 1 and its
remarks, Corollary 1 by Monte Carlo, and structural invariants of eq. (FGK).
"""
import math
import os

import numpy as np
import pytest
import scipy.sparse.linalg as spla

import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def well_conditioned(m, n, seed, smin=0.5, smax=2.0):
    rng = np.random.default_rng(seed)
    U, _ = np.linalg.qr(rng.standard_normal((m, n)))
    V, _ = np.linalg.qr(rng.standard_normal((n, n)))
    sv = np.linspace(smax, smin, n)
    return (U * sv) @ V.T, rng


def decaying(m, n, rho, seed):
    """The artificial problem of Section 2.4: singular values rho^(1-i),
    x_true = ones, ||b_true|| = 1 (singular vectors seeded random orthogonal)."""
    rng = np.random.default_rng(seed)
    U, _ = np.linalg.qr(rng.standard_normal((m, n)))
    V, _ = np.linalg.qr(rng.standard_normal((n, n)))
    sv = rho ** (1.0 - np.arange(1, n + 1))
    A = (U * sv) @ V.T
    bt = A @ np.ones(n)
    A /= np.linalg.norm(bt)
    bt = A @ np.ones(n)
    return A, bt, rng


def dense_krylov(M, v, k):
    """Orthonormal basis of K_k(M, v) by QR of the explicit Krylov matrix."""
    cols = [v / np.linalg.norm(v)]
    for _ in range(k - 1):
        u = M @ cols[-1]
        cols.append(u / np.linalg.norm(u))
    Q, _ = np.linalg.qr(np.column_stack(cols))
    return Q


# ---------------------------------------------------------------- sketch

def test_splitmix64_published_outputs():
    want = [int(l, 16) for l in open(os.path.join(GOLDEN, "splitmix64_seed0.txt")) if l.strip() and not l.startswith("#")]
    assert O.splitmix64_stream(0, len(want)) == want


def test_sparse_sign_structure():
    s, zeta, ncols = 200, 8, 3000
    rows, signs = O.sparse_sign_rows(42, s, zeta, ncols)
    for c in range(ncols):
        assert len(set(rows[c].tolist())) == zeta
    assert rows.min() >= 0 and rows.max() < s
    assert set(np.unique(signs).tolist()) == {-1, 1}
    S = O.SparseSign(42, s, zeta, ncols).dense()
    assert np.allclose(np.linalg.norm(S, axis=0), 1.0, rtol=0, atol=1e-15)
    assert np.allclose(np.abs(S[S != 0]), 1 / math.sqrt(zeta), rtol=0, atol=0)
    # rows are uniform: chi-square of the row counts (df = s - 1)
    counts = np.bincount(rows.ravel(), minlength=s)
    e = zeta * ncols / s
    chi2 = ((counts - e) ** 2 / e).sum()
    assert chi2 < s + 6 * math.sqrt(2 * s)
    # signs are balanced
    assert abs(signs.mean()) < 5 / math.sqrt(signs.size)


def test_sparse_sign_vectorised_equals_definition():
    for seed, s, zeta in [(42, 200, 8), (7, 5, 5), (123456789012345, 600, 1), (2**63 + 11, 401, 8)]:
        rows, signs = O.sparse_sign_rows(seed, s, zeta, 64)
        for c in range(64):
            col = O.sparse_sign_column(seed, s, zeta, c)
            assert [r for r, _ in col] == rows[c].tolist()
            assert [g for _, g in col] == signs[c].tolist()


def test_sparse_sign_embedding_in_expectation():
    # E[S^T S] = I: ||S v||^2 averaged over independent seeds approaches ||v||^2
    rng = np.random.default_rng(3)
    v = rng.standard_normal(500)
    v /= np.linalg.norm(v)
    vals = [np.linalg.norm(O.SparseSign(seed, 50, 4, 500).apply(v)) ** 2 for seed in range(400)]
    assert abs(np.mean(vals) - 1.0) < 0.03


# ---------------------------------------------------------------- small LS

def test_householder_lstsq_matches_lapack():
    rng = np.random.default_rng(0)
    for s, k in [(10, 1), (30, 7), (200, 40), (41, 41)]:
        M = rng.standard_normal((s, k)) @ np.diag(np.logspace(0, -4, k))
        r = rng.standard_normal(s)
        y, res, ok = O.householder_lstsq(M, r)
        y_ref = np.linalg.lstsq(M, r, rcond=None)[0]
        assert ok
        assert np.linalg.norm(y - y_ref) <= 1e-9 * np.linalg.norm(y_ref)
        assert abs(res - np.linalg.norm(r - M @ y_ref)) <= 1e-12 * np.linalg.norm(r)


def test_householder_detects_rank_deficiency():
    rng = np.random.default_rng(1)
    M = rng.standard_normal((20, 3))
    M = np.column_stack([M, M[:, 0] + M[:, 1]])
    _, _, ok = O.householder_lstsq(M, rng.standard_normal(20))
    assert not ok


# ---------------------------------------------------------------- textbook special cases

@pytest.mark.parametrize("k", [1, 2, 5, 12, 20])
def test_sflsqr_identity_full_orth_is_lsqr(k):
    """tau = id, S = I, full orthogonalization: sFLSQR is LSQR (footnote of Section 2.4)."""
    A, rng = well_conditioned(60, 40, 10)
    b = rng.standard_normal(60)
    r = O.sflsqr(A, b, O.IdentitySketch(60), maxit=k, ell=-1)
    x_ref = spla.lsqr(A, b, damp=0.0, atol=0.0, btol=0.0, conlim=0.0, iter_lim=k)[0]
    assert r.iters == k
    assert np.linalg.norm(r.x - x_ref) <= 1e-8 * np.linalg.norm(x_ref)
    # the exact Krylov projection x_k = V_k (A V_k)^+ b, V_k spanning K_k(A^T A, A^T b)  (eq. (xlsqr))
    if k <= 12:
        V = dense_krylov(A.T @ A, A.T @ b, k)
        x_kr = V @ np.linalg.lstsq(A @ V, b, rcond=None)[0]
        assert np.linalg.norm(r.x - x_kr) <= 1e-10 * np.linalg.norm(x_kr)


@pytest.mark.parametrize("k", [1, 3, 8, 15])
def test_sflsmr_identity_full_orth_is_lsmr(k):
    """tau = id, S = I, full orthogonalization: sFLSMR is LSMR (eq. (xlsmr))."""
    A, rng = well_conditioned(50, 30, 11)
    b = rng.standard_normal(50)
    r = O.sflsmr(A, b, O.IdentitySketch(30), S_stop=O.IdentitySketch(50), maxit=k, ell=-1)
    x_ref = spla.lsmr(A, b, damp=0.0, atol=0.0, btol=0.0, conlim=0.0, maxiter=k)[0]
    assert np.linalg.norm(r.x - x_ref) <= 1e-8 * np.linalg.norm(x_ref)
    if k <= 8:
        V = dense_krylov(A.T @ A, A.T @ b, k)
        x_kr = V @ np.linalg.lstsq(A.T @ A @ V, A.T @ b, rcond=None)[0]
        assert np.linalg.norm(r.x - x_kr) <= 1e-10 * np.linalg.norm(x_kr)


def test_fixed_diagonal_flexible_space_is_preconditioned_krylov():
    """tau = diag(d) fixed, full orth, S = I: range(Z_k) = K_k(D A^T A, D A^T b),
    and x_k minimises ||b - A x|| over it (eq. (FLSQR))."""
    A, rng = well_conditioned(40, 25, 12)
    b = rng.standard_normal(40)
    d = rng.uniform(0.5, 1.5, 25)
    for k in (2, 4, 7):
        r = O.sflsqr(A, b, O.IdentitySketch(40), maxit=k, ell=-1, tau=O.FixedDiag(d))
        V = dense_krylov((d[:, None] * A.T) @ A, d * (A.T @ b), k)
        x_kr = V @ np.linalg.lstsq(A @ V, b, rcond=None)[0]
        assert np.linalg.norm(r.x - x_kr) <= 1e-10 * np.linalg.norm(x_kr)


def test_unmatched_backprojector_is_ab_gmres_space():
    """With B != A^T in place of A^T and tau = id (Section 3.2): FLSQR builds
    K_k(B A, B b); sFLSQR with S = I and full orth minimises ||b - A x|| over it
    and sFLSMR minimises ||B (b - A x)||."""
    A, rng = well_conditioned(35, 20, 13)
    B = A.T + 0.05 * rng.standard_normal((20, 35))
    b = rng.standard_normal(35)
    for k in (1, 3, 6):
        V = dense_krylov(B @ A, B @ b, k)
        r1 = O.sflsqr(A, b, O.IdentitySketch(35), maxit=k, ell=-1, AT=B)
        x1 = V @ np.linalg.lstsq(A @ V, b, rcond=None)[0]
        assert np.linalg.norm(r1.x - x1) <= 1e-10 * np.linalg.norm(x1)
        r2 = O.sflsmr(A, b, O.IdentitySketch(20), S_stop=O.IdentitySketch(35), maxit=k, ell=-1, AT=B)
        x2 = V @ np.linalg.lstsq(B @ A @ V, B @ b, rcond=None)[0]
        assert np.linalg.norm(r2.x - x2) <= 1e-10 * np.linalg.norm(x2)


@pytest.mark.parametrize("tau", ["id", "diag", "irw"])
def test_full_space_reaches_dense_sketched_lstsq(tau):
    """After k = n steps (no breakdown) range(Z_n) = R^n for any invertible tau,
    so x_n = argmin ||S (A x - b)|| (sFLSQR) and argmin ||S (A^T A x - A^T b)||
    (sFLSMR), computed here by dense SVD least squares."""
    m, n = 12, 8
    rng = np.random.default_rng(20)
    A = rng.standard_normal((m, n))
    b = rng.standard_normal(m)
    pre = {"id": O.Identity(), "diag": O.FixedDiag(rng.uniform(0.5, 2, n)), "irw": O.Reweighting(1e-2)}[tau]
    Sm = O.gaussian(rng, 10, m)
    r = O.sflsqr(A, b, Sm, maxit=n, ell=2, tau=pre)
    assert r.iters == n
    x_ref = np.linalg.lstsq(Sm.S @ A, Sm.S @ b, rcond=None)[0]
    assert np.linalg.norm(r.x - x_ref) <= 1e-9 * np.linalg.norm(x_ref)
    Sn = O.gaussian(rng, 9, n)
    r2 = O.sflsmr(A, b, Sn, S_stop=O.IdentitySketch(m), maxit=n, ell=2, tau=pre)
    assert r2.iters == n
    x_ref2 = np.linalg.lstsq(Sn.S @ A.T @ A, Sn.S @ A.T @ b, rcond=None)[0]
    assert np.linalg.norm(r2.x - x_ref2) <= 1e-9 * np.linalg.norm(x_ref2)
    # s >= n and S full rank: the sketched normal equations give A^+ b
    assert np.linalg.norm(r2.x - np.linalg.lstsq(A, b, rcond=None)[0]) <= 1e-9 * np.linalg.norm(x_ref2)


def test_small_ls_step_in_isolation():
    """y_k equals the dense least-squares solution of (S A Z_k, S b) rebuilt from
    the oracle's own basis (eq. (sFLSQR)), and the sFLSMR y_k that of
    (S A^T A Z_k, S A^T b) (eq. (sFLSMR))."""
    A, rng = well_conditioned(80, 50, 21, smin=0.05)
    b = rng.standard_normal(80)
    S = O.SparseSign(5, 41, 4, 80)
    r = O.sflsqr(A, b, S, maxit=20, ell=2, tau=O.Reweighting(1e-3))
    for k in (1, 7, 20):
        Zk = r.Z[:, :k]
        y_ref = np.linalg.lstsq(S.dense() @ A @ Zk, S.apply(b), rcond=None)[0]
        assert np.linalg.norm(r.ys[k - 1] - y_ref) <= 1e-9 * np.linalg.norm(y_ref)
    Sn = O.SparseSign(6, 41, 4, 50)
    r2 = O.sflsmr(A, b, Sn, S_stop=O.SparseSign(7, 41, 4, 80), maxit=20, ell=2)
    for k in (1, 9, 20):
        Zk = r2.Z[:, :k]
        y_ref = np.linalg.lstsq(Sn.dense() @ A.T @ A @ Zk, Sn.apply(A.T @ b), rcond=None)[0]
        assert np.linalg.norm(r2.ys[k - 1] - y_ref) <= 1e-9 * np.linalg.norm(y_ref)


# ---------------------------------------------------------------- structure of eq. (FGK)

@pytest.mark.parametrize("ell", [0, 1, 2, 4])
def test_fgk_relations_and_band(ell):
    A, rng = well_conditioned(90, 60, 30, smin=0.01)
    b = rng.standard_normal(90)
    d = rng.uniform(0.5, 1.5, 60)
    r = O.sflsqr(A, b, O.SparseSign(1, 61, 8, 90), maxit=30, ell=ell, tau=O.FixedDiag(d))
    k = r.Z.shape[1]
    AZ = A @ r.Z
    assert np.linalg.norm(AZ - r.W @ r.H) <= 1e-13 * np.linalg.norm(AZ)
    # A^T W_k = P_k T_k with T upper triangular and banded (bandwidth ell)
    ATW = A.T @ r.W[:, :k]
    assert np.linalg.norm(ATW - r.P @ r.T) <= 1e-13 * np.linalg.norm(ATW)
    for j in range(k):
        for i in range(k + 1):
            if not (j - ell <= i <= j + 1):
                assert r.H[i, j] == 0.0
        for i in range(k):
            if not (j - ell <= i <= j):
                assert r.T[i, j] == 0.0
    # window orthogonality (the partial orthogonalization of Section 2.3):
    # w_{k+1} is orthogonal to w_j, j = k-ell..k, and p_k to p_j, j = k-ell..k-1
    for i in range(r.W.shape[1]):
        for j in range(max(0, i - ell - 1), i):
            assert abs(r.W[:, i] @ r.W[:, j]) <= 1e-13
    for i in range(k):
        for j in range(max(0, i - ell), i):
            assert abs(r.P[:, i] @ r.P[:, j]) <= 1e-13
    # unit norms of the partially orthogonal bases
    assert np.allclose(np.linalg.norm(r.W, axis=0), 1, atol=1e-14)
    assert np.allclose(np.linalg.norm(r.P, axis=0), 1, atol=1e-14)
    # Z = tau(P)
    assert np.array_equal(r.Z, d[:, None] * r.P)


def test_window_zero_still_orthogonalises_w_against_last():
    A, rng = well_conditioned(40, 30, 31)
    r = O.sflsqr(A, rng.standard_normal(40), O.IdentitySketch(40), maxit=10, ell=0)
    for j in range(1, r.W.shape[1]):
        assert abs(r.W[:, j] @ r.W[:, j - 1]) <= 1e-14


def test_orthogonalise_against_z_literal_matches_p_for_identity():
    A, rng = well_conditioned(40, 30, 32)
    b = rng.standard_normal(40)
    S = O.SparseSign(3, 25, 4, 40)
    r1 = O.sflsqr(A, b, S, maxit=10, ell=2, orth_against="p")
    r2 = O.sflsqr(A, b, S, maxit=10, ell=2, orth_against="z")
    assert np.array_equal(r1.x, r2.x)


def test_reweighting_operator_at_second_step():
    """tau_2(p) = diag((x_1^2 + eps)^(1/4)) p, where x_1 = z_1 y_1 is the one-term
    sketched least-squares solution (closed form for k = 1)."""
    A, rng = well_conditioned(30, 20, 33)
    b = rng.standard_normal(30)
    S = O.SparseSign(9, 15, 4, 30)
    eps = 3e-3
    r = O.sflsqr(A, b, S, maxit=3, ell=2, tau=O.Reweighting(eps))
    p1 = A.T @ b / np.linalg.norm(A.T @ b)
    z1 = eps ** 0.25 * p1
    c = S.apply(A @ z1)
    y1 = (c @ S.apply(b)) / (c @ c)
    x1 = y1 * z1
    assert np.allclose(r.Z[:, 0], z1, rtol=1e-13, atol=0)
    assert np.allclose(r.Z[:, 1] / r.P[:, 1], (x1 ** 2 + eps) ** 0.25, rtol=1e-12, atol=0)


# ---------------------------------------------------------------- Section 2.5 / 2.6 theory

def test_remark_sflsmr_is_sflsqr_with_sketch_SAt():
    """Remark after Algorithm 2: sFLSMR with S equals sFLSQR with S A^T."""
    A, rng = well_conditioned(50, 30, 40, smin=0.05)
    b = rng.standard_normal(50)
    Sn = O.SparseSign(11, 31, 8, 30)
    r_mr = O.sflsmr(A, b, Sn, S_stop=O.IdentitySketch(50), maxit=15, ell=2)
    r_qr = O.sflsqr(A, b, O.DenseSketch(Sn.dense() @ A.T), maxit=15, ell=2)
    for k in range(15):
        assert np.linalg.norm(r_mr.ys[k] - r_qr.ys[k]) <= 1e-11 * np.linalg.norm(r_qr.ys[k])


def test_scale_and_row_permutation_invariance():
    A, rng = well_conditioned(60, 40, 41, smin=0.05)
    b = rng.standard_normal(60)
    S = O.SparseSign(12, 41, 8, 60).dense()
    perm = rng.permutation(41)
    r0 = O.sflsqr(A, b, O.DenseSketch(S), maxit=20, ell=2)
    r1 = O.sflsqr(A, b, O.DenseSketch(3.7 * S), maxit=20, ell=2)
    r2 = O.sflsqr(A, b, O.DenseSketch(S[perm]), maxit=20, ell=2)
    for k in range(20):
        nrm = np.linalg.norm(r0.ys[k])
        assert np.linalg.norm(r0.ys[k] - r1.ys[k]) <= 1e-12 * nrm
        assert np.linalg.norm(r0.ys[k] - r2.ys[k]) <= 1e-12 * nrm


def _residual_terms(A, Zk, b, S):
    Q, _ = np.linalg.qr(A @ Zk)
    Qc = np.linalg.svd(np.eye(A.shape[0]) - Q @ Q.T)[0][:, :A.shape[0] - Q.shape[1]]
    r_opt = np.linalg.norm(b - Q @ (Q.T @ b))
    return Q, Qc, r_opt


def test_theorem1_deterministic_bounds():
    """r_opt <= r_sFLSQR <= r_opt sqrt(1 + ||(SQ)^+ S Q_perp||^2) and the sFLSMR
    bound with S A^T, eqs. (bound1) and (bound2), at every k, for several sketches."""
    A, bt, rng = decaying(60, 30, 1.15, 50)
    b = bt + 0.1 * rng.standard_normal(60) / math.sqrt(60)
    for sk in range(3):
        Sm = O.gaussian(rng, 25, 60) if sk == 0 else O.DenseSketch(O.SparseSign(sk, 25, 4, 60).dense())
        Sn = O.gaussian(rng, 25, 30) if sk == 0 else O.DenseSketch(O.SparseSign(sk + 10, 25, 4, 30).dense())
        rq = O.sflsqr(A, b, Sm, maxit=10, ell=2)
        rm = O.sflsmr(A, b, Sn, S_stop=O.IdentitySketch(60), maxit=10, ell=2)
        for k in range(1, 11):
            Zk = rq.Z[:, :k]
            Q, Qc, r_opt = _residual_terms(A, Zk, b, Sm)
            r_q = np.linalg.norm(A @ rq.xs[k - 1] - b) if rq.xs else np.linalg.norm(A @ (Zk @ rq.ys[k - 1]) - b)
            b1 = r_opt * math.sqrt(1 + np.linalg.norm(np.linalg.pinv(Sm.S @ Q) @ Sm.S @ Qc, 2) ** 2)
            assert r_opt * (1 - 1e-12) <= r_q <= b1 * (1 + 1e-10)
            r_m = np.linalg.norm(A @ (rm.Z[:, :k] @ rm.ys[k - 1]) - b)
            SAt = Sn.S @ A.T
            Q2, Qc2, r_opt2 = _residual_terms(A, rm.Z[:, :k], b, Sn)
            b2 = r_opt2 * math.sqrt(1 + np.linalg.norm(np.linalg.pinv(SAt @ Q2) @ SAt @ Qc2, 2) ** 2)
            assert r_opt2 * (1 - 1e-12) <= r_m <= b2 * (1 + 1e-10)


def test_rank_k_remark_sflsmr_is_optimal():
    """Remark after Theorem 1: for A of exact rank k, after k steps r_sFLSMR = r_opt."""
    rng = np.random.default_rng(60)
    m, n, k = 40, 25, 6
    U, _ = np.linalg.qr(rng.standard_normal((m, k)))
    V, _ = np.linalg.qr(rng.standard_normal((n, k)))
    A = (U * np.linspace(3, 1, k)) @ V.T
    b = rng.standard_normal(m)
    Sn = O.gaussian(rng, 13, n)
    r = O.sflsmr(A, b, Sn, S_stop=O.IdentitySketch(m), maxit=k, ell=2)
    assert r.iters == k
    r_m = np.linalg.norm(A @ r.x - b)
    Q, _ = np.linalg.qr(A @ r.Z)
    r_opt = np.linalg.norm(b - Q @ (Q.T @ b))
    assert abs(r_m - r_opt) <= 1e-10 * r_opt
    # sFLSQR with a Gaussian sketch is not optimal in general
    rq = O.sflsqr(A, b, O.gaussian(rng, 13, m), maxit=k, ell=2)
    assert np.linalg.norm(A @ rq.x - b) > r_opt * (1 + 1e-6)


@pytest.mark.slow
def test_corollary1_gaussian_expectation():
    """Corollary 1 (Gaussian S): E[r^2] = r_opt^2 (1 + c).  Proposition 10.2 of
    Halko-Martinsson-Tropp gives E||(SQ)^+||_F^2 = k/(s-k-1) for an s x k
    standard Gaussian, which is the constant checked here (the printed
    s/(s-k-1) is the reading noted in the design notes)."""
    A, bt, rng = decaying(200, 100, 1.02, 61)
    b = bt + 0.1 * rng.standard_normal(200) / math.sqrt(200)
    k, s = 10, 21
    base = O.sflsqr(A, b, O.IdentitySketch(200), maxit=k, ell=2)
    Zk = base.Z
    Q, _ = np.linalg.qr(A @ Zk)
    r_opt = np.linalg.norm(b - Q @ (Q.T @ b))
    ratios = []
    for t in range(2000):
        S = O.gaussian(np.random.default_rng(1000 + t), s, 200)
        r = O.sflsqr(A, b, S, maxit=k, ell=2, keep_basis=False)
        ratios.append((np.linalg.norm(A @ r.x - b) / r_opt) ** 2)
    want = 1 + k / (s - k - 1)
    assert abs(np.mean(ratios) / want - 1) < 0.05
    assert abs(np.mean(ratios) - (1 + s / (s - k - 1))) > 0.3


def test_section24_sketched_residual_above_lsqr_large_noise():
    """Section 2.4 (artificial problem, rho = 1.01, 10% noise, Gaussian s = 2k+1):
    the sLSQR residual ends above LSQR's (about 30% in the paper), and sLSMR
    tracks the optimal residual more closely than sLSQR (Section 2.5)."""
    m, n, k = 1024, 512, 50
    A, bt, rng = decaying(m, n, 1.01, 70)
    e = rng.standard_normal(m)
    b = bt + 0.10 * e / np.linalg.norm(e)
    lsqr = O.sflsqr(A, b, O.IdentitySketch(m), maxit=k, ell=-1, keep_basis=False)
    r_lsqr = np.linalg.norm(A @ lsqr.x - b)
    ratios_q, ratios_m = [], []
    for t in range(3):
        g = np.random.default_rng(500 + t)
        sq = O.sflsqr(A, b, O.gaussian(g, 2 * k + 1, m), maxit=k, ell=-1, keep_basis=False)
        sm = O.sflsmr(A, b, O.gaussian(g, 2 * k + 1, n), S_stop=O.IdentitySketch(m), maxit=k, ell=-1,
                      keep_basis=False)
        ratios_q.append(np.linalg.norm(A @ sq.x - b) / r_lsqr)
        ratios_m.append(np.linalg.norm(A @ sm.x - b) / r_lsqr)
    assert 1.05 < np.mean(ratios_q) < 1.8
    assert np.mean(ratios_m) < np.mean(ratios_q)


# ---------------------------------------------------------------- stop rule and breakdown

def test_discrepancy_stop_is_first_crossing():
    A, rng = well_conditioned(60, 40, 80, smin=0.01)
    b = rng.standard_normal(60)
    S = O.SparseSign(2, 41, 8, 60)
    full = O.sflsqr(A, b, S, maxit=25, tol=0.0, ell=2)
    rel = np.array(full.relres)
    j = 11
    tol = 0.5 * (rel[j - 1] + rel[:j - 1].min()) if rel[j - 1] < rel[:j - 1].min() else None
    if tol is None:
        pytest.skip("sequence not decreasing at the probe index")
    r = O.sflsqr(A, b, S, maxit=25, tol=tol, ell=2)
    first = int(np.argmax(rel < tol)) + 1
    assert r.status == O.STOP_DISCREPANCY and r.iters == first
    assert np.array_equal(r.x, full.Z[:, :first] @ full.ys[first - 1])


def test_breakdown_in_invariant_subspace():
    """b in a 1-D invariant subspace: w_2 vanishes, the solve stops with the
    exact solution of the first step."""
    A = np.diag([2.0, 1.0, 0.5, 0.25])
    b = np.array([3.0, 0.0, 0.0, 0.0])
    for solve in (lambda: O.sflsqr(A, b, O.IdentitySketch(4), maxit=4, ell=2),
                  lambda: O.sflsmr(A, b, O.IdentitySketch(4), S_stop=O.IdentitySketch(4), maxit=4, ell=2)):
        r = solve()
        assert r.status == O.STOP_BREAKDOWN and r.iters == 1
        assert np.allclose(r.x, [1.5, 0, 0, 0], rtol=0, atol=1e-15)
