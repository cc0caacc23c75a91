"""Plain FP64 CPU oracle for sFLSQR (Algorithm 1) and sFLSMR (Algorithm 2).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute this module: only the tests, the smoke check and the benchmark's CPU
baseline leg use it.  It shares no code with the GPU library.

The oracle follows the two algorithms of Section 2 step by step, in the
paper's order and notation, in FP64, with library primitives (sparse matvec,
numpy vector ops) as steps and no blocking, fusion or reordering:

  FGK with window-ell orthogonalization, eq. (FGK) in Section 2.3:
      A^T W = P T,   A Z = W H,   Z = tau(P)
  sFLSQR, eq. (sFLSQR):  y_k = argmin || S_m (A Z_k y - b) ||
  sFLSMR, eq. (sFLSMR):  y_k = argmin || s_{A^T b} - [S A^T W, S z] H y ||

The small least-squares problem is solved from scratch at every iteration by
Householder QR (Golub & Van Loan, Algorithm 5.3.2) and back substitution.

Readings of points the paper leaves open (each one is also listed in the
design notes):
  * orthogonalize against p_j (pre-tau, unit norm; the relation A^T W = P T of
    eq. (FGK)) by default; `orth_against="z"` gives the literal z_j of the
    algorithm listings.  The two coincide for tau = identity.
  * "ell" is the orthogonalization window; ell < 0 means full orthogonalization.
  * Modified Gram-Schmidt: each coefficient is taken from the current vector.
  * The reweighting preconditioner P_k = diag((x_{k-1}^2 + eps)^(1/4)) uses the
    latest available iterate x_{k-1} = Z_{k-1} y_{k-1}, with x_0 = 0.
  * Discrepancy stop (eq. (discrP)): tol = eta * ||e|| / ||b||; sFLSQR stops
    when ||s_b - S_AZ y_k|| < tol ||s_b||.  sFLSMR by default keeps an m-side
    sketch S_m of A z_k and applies the same test to ||S_m (b - A Z y_k)||;
    stop_rule="normal" uses the residual sFLSMR actually minimises,
    ||s_{A^T b} - M_k y_k|| < tol ||s_{A^T b}||.
  * Breakdown: ||z|| <= 1e-300 or <= 1e-14 times its norm before
    orthogonalization, or |R_kk| <= 1e-14 |R_11| in the small QR, ends the
    solve with status BREAKDOWN and the last completed iterate.  The same test
    on ||w|| is a lucky breakdown (A z_k in span(W_k)): step k's small LS is
    still solved (it needs no w_{k+1}) and its iterate returned.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .sketch import Sketch, SparseSign

STOP_DISCREPANCY = 1
STOP_MAXIT = 2
STOP_BREAKDOWN = 3

BREAKDOWN_ABS = 1e-300
BREAKDOWN_REL = 1e-14


def householder_lstsq(M: np.ndarray, rhs: np.ndarray) -> tuple[np.ndarray, float, bool]:
    """min_y ||rhs - M y||_2 for a tall s x k matrix by Householder QR.

    Returns (y, residual norm ||rhs - M y||, rank_ok).  Each reflector is
    H_j = I - beta v v^T with v[0] = x[0] - alpha, alpha = -sign(x[0]) ||x||.
    """
    R = np.array(M, dtype=np.float64, copy=True)
    g = np.array(rhs, dtype=np.float64, copy=True)
    s, k = R.shape
    for j in range(k):
        x = R[j:, j]
        nx = np.linalg.norm(x)
        if nx == 0.0:
            continue
        alpha = -nx if x[0] >= 0 else nx
        v = x.copy()
        v[0] -= alpha
        beta = 2.0 / (v @ v)
        R[j:, j:] -= beta * np.outer(v, v @ R[j:, j:])
        g[j:] -= beta * v * (v @ g[j:])
    d = np.abs(np.diag(R[:k, :k]))
    rank_ok = k == 0 or (d.min() > BREAKDOWN_REL * d[0] and d[0] > 0)
    y = np.zeros(k)
    if rank_ok:
        for i in range(k - 1, -1, -1):
            y[i] = (g[i] - R[i, i + 1:k] @ y[i + 1:]) / R[i, i]
    res = float(np.linalg.norm(rhs - M @ y))
    return y, res, rank_ok


class Precond:
    """The flexible operator tau of eq. (modbasis): z_k = tau_k(p_k)."""

    def __call__(self, p: np.ndarray, x_prev: np.ndarray) -> np.ndarray:
        raise NotImplementedError


class Identity(Precond):
    def __call__(self, p, x_prev):
        return p.copy()


class FixedDiag(Precond):
    """tau(p) = diag(w) p with a fixed weight vector w."""

    def __init__(self, w):
        self.w = np.asarray(w, dtype=np.float64)

    def __call__(self, p, x_prev):
        return self.w * p


class Reweighting(Precond):
    """Iteratively reweighted right preconditioner (Section 1.2):
    tau_k(p) = diag((x_{k-1}^2 + eps)^(1/4)) p, x_0 = 0."""

    def __init__(self, eps: float = 1e-4):
        self.eps = eps

    def __call__(self, p, x_prev):
        return np.power(x_prev * x_prev + self.eps, 0.25) * p


@dataclass
class Result:
    x: np.ndarray
    y: np.ndarray
    iters: int
    status: int
    relres: list = field(default_factory=list)       # stop-test ratio numerator/denominator per k
    xs: list = field(default_factory=list)           # x_k per iteration (if record_x)
    ys: list = field(default_factory=list)
    Z: np.ndarray | None = None
    P: np.ndarray | None = None
    W: np.ndarray | None = None
    H: np.ndarray | None = None
    T: np.ndarray | None = None
    alpha: list = field(default_factory=list)        # ||z|| after orthogonalization
    beta: list = field(default_factory=list)         # H_{k+1,k}


def _window(k: int, ell: int, upto: int) -> range:
    """1-based indices j = max(1, k - ell) .. upto (full when ell < 0)."""
    lo = 1 if ell < 0 else max(1, k - ell)
    return range(lo, upto + 1)


def _fgk_solve(A, b, *, method: str, S_ls: Sketch, S_stop: Sketch | None, maxit: int, tol: float,
               ell: int, tau: Precond, AT=None, orth_against: str = "p", stop_rule: str = "residual",
               record_x: bool = False, keep_basis: bool = True) -> Result:
    """Shared driver of Algorithms 1 and 2 (they differ only in the sketched LS)."""
    matvec = (lambda v: A @ v)
    rmatvec = (lambda v: A.T @ v) if AT is None else (lambda v: AT @ v)
    m, n = A.shape
    b = np.asarray(b, dtype=np.float64)

    # initialisation (first statements of Algorithms 1 and 2)
    beta0 = float(np.linalg.norm(b))
    w1 = b / beta0
    z = rmatvec(w1)
    W = [w1]                      # W[j-1] = w_j
    P: list[np.ndarray] = []
    Z: list[np.ndarray] = []
    Hmat = np.zeros((maxit + 1, maxit))
    Tmat = np.zeros((maxit, maxit))
    if method == "sflsqr":
        s_b = S_ls.apply(b)
        SAZ: list[np.ndarray] = []
        stop_den = float(np.linalg.norm(s_b))
    else:
        s_Atb = beta0 * S_ls.apply(z)
        SAtW = [s_Atb / beta0]    # columns S A^T w_j
        if stop_rule == "residual":
            s_b = S_stop.apply(b)
            SAZ = []
            stop_den = float(np.linalg.norm(s_b))
        else:
            stop_den = float(np.linalg.norm(s_Atb))

    res = Result(x=np.zeros(n), y=np.zeros(0), iters=0, status=STOP_MAXIT)
    x_prev = np.zeros(n)
    y = np.zeros(0)
    for k in range(1, maxit + 1):
        # window orthogonalization of z (MGS, ascending j)
        zraw_norm = float(np.linalg.norm(z))
        V = P if orth_against == "p" else Z
        for j in _window(k, ell, k - 1):
            c = float(V[j - 1] @ z)
            z = z - c * V[j - 1]
            Tmat[j - 1, k - 1] = c
        alpha = float(np.linalg.norm(z))
        if alpha <= BREAKDOWN_ABS or alpha <= BREAKDOWN_REL * zraw_norm:
            res.status = STOP_BREAKDOWN
            break
        Tmat[k - 1, k - 1] = alpha
        p = z / alpha
        P.append(p)
        zk = tau(p, x_prev)
        Z.append(zk)
        res.alpha.append(alpha)

        w = matvec(zk)
        if method == "sflsqr" or stop_rule == "residual":
            SAZ.append((S_ls if method == "sflsqr" else S_stop).apply(w))

        # window orthogonalization of w, recording H
        wraw_norm = float(np.linalg.norm(w))
        for j in _window(k, ell, k):
            h = float(W[j - 1] @ w)
            Hmat[j - 1, k - 1] = h
            w = w - h * W[j - 1]
        hk = float(np.linalg.norm(w))
        # lucky breakdown: A z_k lies in span(W_k); the small LS of step k needs
        # no w_{k+1} (its H_{k+1,k} is 0), so step k is completed and the solve ends
        lucky = hk <= BREAKDOWN_ABS or hk <= BREAKDOWN_REL * wraw_norm
        if not lucky:
            Hmat[k, k - 1] = hk
            W.append(w / hk)
            res.beta.append(hk)
            z = rmatvec(W[-1])

        # small sketched least-squares problem
        if method == "sflsqr":
            Mk = np.column_stack(SAZ)
            yk, r_ls, ok = householder_lstsq(Mk, s_b)
            r_stop = r_ls
        else:
            Sz = np.zeros(S_ls.s) if lucky else S_ls.apply(z)
            Mk = np.column_stack(SAtW + [Sz]) @ Hmat[:k + 1, :k]
            yk, r_ls, ok = householder_lstsq(Mk, s_Atb)
            if stop_rule == "residual":
                r_stop = float(np.linalg.norm(s_b - np.column_stack(SAZ) @ yk))
            else:
                r_stop = r_ls
        if not ok:
            res.status = STOP_BREAKDOWN      # keep the last completed iterate
            break
        y = yk
        x_prev = np.column_stack(Z) @ y
        res.iters = k
        res.relres.append(r_stop / stop_den)
        res.ys.append(y.copy())
        if record_x:
            res.xs.append(x_prev.copy())
        if r_stop < tol * stop_den:
            res.status = STOP_DISCREPANCY
            break
        if lucky:
            res.status = STOP_BREAKDOWN
            break
        if method != "sflsqr":
            SAtW.append(Sz)

    k = res.iters
    res.y = y
    res.x = np.column_stack(Z[:k]) @ y if k > 0 else np.zeros(n)
    if keep_basis:
        res.Z = np.column_stack(Z) if Z else np.zeros((n, 0))
        res.P = np.column_stack(P) if P else np.zeros((n, 0))
        res.W = np.column_stack(W)
        res.H = Hmat[:len(W), :len(W) - 1]
        res.T = Tmat[:len(P), :len(P)]
    return res


def sflsqr(A, b, S: Sketch, *, maxit: int, tol: float = 0.0, ell: int = 2, tau: Precond | None = None,
           AT=None, orth_against: str = "p", record_x: bool = False, keep_basis: bool = True) -> Result:
    """Algorithm 1 (sFLSQR).  S is the s x m sketch; AT, if given, replaces A^T
    (an unmatched back-projector)."""
    return _fgk_solve(A, b, method="sflsqr", S_ls=S, S_stop=None, maxit=maxit, tol=tol, ell=ell,
                      tau=tau or Identity(), AT=AT, orth_against=orth_against, record_x=record_x,
                      keep_basis=keep_basis)


def sflsmr(A, b, S: Sketch, *, maxit: int, tol: float = 0.0, ell: int = 2, tau: Precond | None = None,
           AT=None, S_stop: Sketch | None = None, stop_rule: str = "residual", orth_against: str = "p",
           record_x: bool = False, keep_basis: bool = True) -> Result:
    """Algorithm 2 (sFLSMR).  S is the s x n sketch; S_stop (s x m) carries the
    m-side discrepancy estimate when stop_rule == "residual"."""
    if stop_rule == "residual" and S_stop is None:
        raise ValueError("stop_rule='residual' needs S_stop (an s x m sketch)")
    return _fgk_solve(A, b, method="sflsmr", S_ls=S, S_stop=S_stop, maxit=maxit, tol=tol, ell=ell,
                      tau=tau or Identity(), AT=AT, orth_against=orth_against, stop_rule=stop_rule,
                      record_x=record_x, keep_basis=keep_basis)


def discrepancy_tol(eta: float, noise_norm: float, b_norm: float) -> float:
    """tol of the relative stop test from eq. (discrP): eta * ||e|| / ||b||."""
    return eta * noise_norm / b_norm


def sketches_for(method: str, seed: int, s: int, zeta: int, m: int, n: int) -> tuple:
    """The sparse-sign sketches a solve uses: sFLSQR draws S_m from `seed`;
    sFLSMR draws S_n from `seed` and its m-side stop sketch from `seed + 1`."""
    if method == "sflsqr":
        return SparseSign(seed, s, zeta, m), None
    return SparseSign(seed, s, zeta, n), SparseSign(seed + 1, s, zeta, m)
