"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle.

Bars: bit-exact for the sketch's integer draws; FP64 iterates within relative
1e-10 per iteration; FP64 sparse products within 1e-14 (only the summation
order differs); reduced-precision products against the oracle run on the same
rounded operator.
"""
import ctypes
import math

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import oracle as O
import workloads as wl

pytestmark = pytest.mark.gpu

import torch  # noqa: E402

from paper_2605_22281_gb300 import api as G  # noqa: E402


@pytest.fixture(autouse=True)
def _needs_cuda():
    if not torch.cuda.is_available():
        raise RuntimeError("GPU test selected but no CUDA device is available")

RTOL_ITER = 1e-10


def to_csr(S) -> wl.CSR:
    S = sp.csr_matrix(S)
    return wl.CSR(S.shape, S.indptr.astype(np.int64), S.indices.astype(np.int32), S.data.astype(np.float64))


def rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def dev(x):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


@pytest.fixture(scope="module")
def ct64():
    p = wl.make("ct64_sflsqr")
    return p, G.Plan(p.A)


@pytest.fixture(scope="module")
def ct64_unmatched():
    N, na = 64, 60
    nb = wl.detector_bins(N)
    A = wl.siddon_projector(N, na, nb)
    B = wl.pixel_backprojector(N, na, nb)
    rng = np.random.default_rng(11)
    x = wl.sparse_phantom(N, rng, 0.05)
    b, en = wl.add_noise(A.matvec(x), 0.02, rng)
    return A, B, x, b, en, G.Plan(A, B)


def edge_matrix(seed=0, m=37, n=53):
    """Ragged CSR: empty rows, one 600-entry row, empty columns, sizes not multiples of 4."""
    rng = np.random.default_rng(seed)
    rows, cols, vals = [], [], []
    for r in range(m):
        if r % 7 == 3:
            continue                       # empty row
        k = 600 if r == 5 else int(rng.integers(1, 9))
        c = rng.choice(n - 3, size=min(k, n - 3), replace=k > n - 3)
        rows += [r] * len(c); cols += list(c); vals += list(rng.standard_normal(len(c)))
    S = sp.coo_matrix((vals, (rows, cols)), shape=(m, n)).tocsr()
    S.sum_duplicates()
    return S


# ---------------------------------------------------------------- sketch

@pytest.mark.parametrize("seed,s,zeta,ncols", [(42, 200, 8, 5460), (7, 5, 5, 100), (2**63 + 11, 401, 8, 1000),
                                               (3, 600, 16, 777), (9, 2048, 1, 3000), (43, 400, 8, 65536)])
def test_sketch_draws_bit_exact(seed, s, zeta, ncols):
    rows, signs = G.sketch_export(seed, s, zeta, ncols)
    r_or, s_or = O.sparse_sign_rows(seed, s, zeta, ncols)
    assert np.array_equal(rows.cpu().numpy(), r_or)
    assert np.array_equal(signs.cpu().numpy(), s_or)


@pytest.mark.parametrize("seed,s,zeta,n", [(1, 200, 8, 5460), (5, 33, 3, 1001), (8, 600, 16, 70000)])
def test_sketch_apply_matches_oracle(seed, s, zeta, n):
    v = np.random.default_rng(seed).standard_normal(n)
    got = G.sketch_apply(seed, s, zeta, dev(v)).cpu().numpy()
    want = O.SparseSign(seed, s, zeta, n).apply(v)
    assert rel(got, want) <= 1e-14


# ---------------------------------------------------------------- sparse products

@pytest.mark.parametrize("which", ["ct64", "edge", "edge2"])
def test_spmv_fp64(which, ct64):
    if which == "ct64":
        S = ct64[0].A.scipy()
        plan = ct64[1]
    else:
        S = edge_matrix(0 if which == "edge" else 1, *((37, 53) if which == "edge" else (130, 9)))
        plan = G.Plan(to_csr(S))
    rng = np.random.default_rng(4)
    x = rng.standard_normal(S.shape[1])
    u = rng.standard_normal(S.shape[0])
    assert rel(plan.apply(dev(x)).cpu().numpy(), S @ x) <= 1e-14
    assert rel(plan.apply(dev(u), transpose=True).cpu().numpy(), S.T @ u) <= 1e-14


def test_spmv_unmatched_backprojector(ct64_unmatched):
    A, B, *_, plan = ct64_unmatched
    u = np.random.default_rng(5).standard_normal(A.shape[0])
    assert rel(plan.apply(dev(u), transpose=True).cpu().numpy(), B.scipy() @ u) <= 1e-14


@pytest.mark.parametrize("vdt,tol", [("f32", 2e-6), ("bf16", 2e-6)])
def test_spmv_reduced_precision_on_rounded_operator(vdt, tol, ct64):
    S = ct64[0].A.scipy().astype(np.float64)
    if vdt == "f32":
        Sr = S.astype(np.float32).astype(np.float64)
    else:
        Sr = S.copy()
        Sr.data = torch.as_tensor(S.data).to(torch.bfloat16).to(torch.float64).numpy()
    plan = G.Plan(ct64[0].A, value_dtype=vdt)
    x = np.random.default_rng(6).standard_normal(S.shape[1]).astype(np.float32).astype(np.float64)
    u = np.random.default_rng(7).standard_normal(S.shape[0]).astype(np.float32).astype(np.float64)
    assert rel(plan.apply(dev(x)).cpu().numpy(), Sr @ x) <= tol
    assert rel(plan.apply(dev(u), transpose=True).cpu().numpy(), Sr.T @ u) <= tol


# ---------------------------------------------------------------- solvers: per-iteration parity

U = 2.0 ** -53   # FP64 unit roundoff


def run_oracle_sflsqr(A, b, s, zeta, seed, maxit, tol, ell, tau=None, AT=None, orth_against="p"):
    S = O.SparseSign(seed, s, zeta, A.shape[0])
    r = O.sflsqr(A, b, S, maxit=maxit, tol=tol, ell=ell, tau=tau, AT=AT, record_x=True, keep_basis=True,
                 orth_against=orth_against)
    r.M = S.mat @ (A @ r.Z)                                  # sketched LS matrix S A Z (eq. (sFLSQR))
    return r


def run_oracle_sflsmr(A, b, s, zeta, seed, maxit, tol, ell, tau=None, AT=None, stop_rule="residual",
                      orth_against="p"):
    Sn = O.SparseSign(seed, s, zeta, A.shape[1])
    Sm = O.SparseSign(seed + 1, s, zeta, A.shape[0])
    r = O.sflsmr(A, b, Sn, S_stop=Sm, maxit=maxit, tol=tol, ell=ell, tau=tau, AT=AT, stop_rule=stop_rule,
                 record_x=True, keep_basis=True, orth_against=orth_against)
    BT = A.T if AT is None else AT
    r.M = Sn.mat @ (BT @ (A @ r.Z))                          # S A^T A Z (eq. (sFLSMR))
    return r


def iterate_tolerance(kappa: float) -> float:
    """Bar of the stress runs only (fixed step counts far past the discrepancy
    point): relative 1e-10, or the first-order perturbation size 32 u kappa of
    the small least-squares problem when that is larger (two backward-stable
    FP64 solvers that differ only in rounding order cannot agree better once
    kappa(S A Z_k) exceeds ~3e4)."""
    return max(RTOL_ITER, 32 * U * kappa)


def assert_stop_step(r, info, tol_stop):
    """Same stop step as the oracle unless its last stop ratio lies within
    1e-8 (relative) of the threshold."""
    if tol_stop <= 0 or abs(r.relres[-1] / tol_stop - 1) > 1e-8:
        assert info.iters == r.iters, (info.iters, r.iters)


def assert_iterates_flat(r, x_gpu_hist, relres_gpu, info, tol_stop):
    """Configured workloads (solves that end at the discrepancy stop): x_k and
    the stop ratio of EVERY step up to the stop within relative 1e-10 of the
    oracle's, with no allowance for the small problem's conditioning.
    Returns the number of steps checked."""
    assert info.status == r.status, (info.status, r.status)
    assert_stop_step(r, info, tol_stop)
    kk = min(r.iters, info.iters)
    assert kk >= 1
    xh = x_gpu_hist.cpu().numpy()
    rh = relres_gpu.cpu().numpy()
    worst = 0.0
    for j in range(kk):
        e = rel(xh[j], r.xs[j])
        worst = max(worst, e)
        assert e <= RTOL_ITER, f"iterate {j + 1}: rel err {e:.3e} (bar {RTOL_ITER:.0e})"
        assert abs(rh[j] - r.relres[j]) <= RTOL_ITER * abs(r.relres[j]), f"stop ratio {j + 1}"
    print(f"flat bar: {kk} steps checked, worst relative error {worst:.2e}")
    return kk


def assert_iterates_conditioned(r, x_gpu_hist, relres_gpu, info, tol_stop, min_checked=10):
    """Stress runs past the discrepancy point: x_k and the stop ratio of every
    step whose small problem is still determined (kappa(S A Z_k) <= 1e12)
    against the oracle at the bar iterate_tolerance(kappa); the stop ratio
    also gets an accumulated-rounding floor of 64 k u.  Steps with kappa >
    1e12 are counted, not checked, and at least min(min_checked, steps run)
    steps must be checked.  Returns the number of steps checked."""
    conds = [np.linalg.cond(r.M[:, :j + 1]) for j in range(r.M.shape[1])]
    k = r.iters
    if info.iters < k and info.status == O.STOP_BREAKDOWN:
        # the GPU's rank test |R_kk| <= 1e-14 |R_11| fired first: only where the
        # oracle's matrix is numerically rank deficient
        assert conds[info.iters] > 1e12, (info.iters, conds[info.iters])
    else:
        assert_stop_step(r, info, tol_stop)
    kk = min(k, info.iters)
    xh = x_gpu_hist.cpu().numpy()
    rh = relres_gpu.cpu().numpy()
    checked = skipped = 0
    for j in range(kk):
        if conds[j] > 1e12:
            skipped += 1     # numerically rank-deficient small problem: x_k is not determined
            continue
        tj = iterate_tolerance(conds[j])
        e = rel(xh[j], r.xs[j])
        assert e <= tj, f"iterate {j + 1}: rel err {e:.3e} (bar {tj:.1e}, cond {conds[j]:.1e})"
        assert abs(rh[j] - r.relres[j]) <= tj * abs(r.relres[j]) + 64 * (j + 1) * U, f"stop ratio {j + 1}"
        checked += 1
    assert checked >= min(min_checked, kk), f"only {checked} of {kk} steps checked ({skipped} rank deficient)"
    return checked


SKETCH_APPLY = ["kernel", "fused"]


@pytest.mark.parametrize("sketch_apply", SKETCH_APPLY)
def test_sflsqr_ct64_per_iteration(ct64, sketch_apply):
    p, plan = ct64
    st = p.settings
    tol = O.discrepancy_tol(st["eta"], p.noise_norm[0], np.linalg.norm(p.b))
    r = run_oracle_sflsqr(p.A.scipy(), p.b, st["s"], st["zeta"], st["seed"], st["maxit"], tol, st["window"])
    x, info, h = plan.solve("sflsqr", dev(p.b), s=st["s"], zeta=st["zeta"], seed=st["seed"], window=st["window"],
                            maxit=st["maxit"], noise_norm=p.noise_norm[0], eta=st["eta"], x_history=True,
                            relres_history=True, sketch_apply=sketch_apply)
    assert info.status == O.STOP_DISCREPANCY == r.status
    assert_iterates_flat(r, h["x"], h["relres"], info, tol)
    assert rel(x.cpu().numpy(), r.x) <= RTOL_ITER
    assert abs(info.tol - tol) <= 1e-15 * tol


@pytest.mark.parametrize("ell", [0, 1, 2, 5, 8])
@pytest.mark.parametrize("sketch_apply", SKETCH_APPLY)
def test_sflsqr_fixed_iterations_windows(ct64, ell, sketch_apply):
    """No stop rule, past the discrepancy point, while the small problem stays
    determined (its condition number grows to ~1e10 by the last step)."""
    p, plan = ct64
    maxit = 12 if ell == 0 else 25
    r = run_oracle_sflsqr(p.A.scipy(), p.b, 101, 8, 42, maxit, 0.0, ell)
    x, info, h = plan.solve("sflsqr", dev(p.b), s=101, zeta=8, seed=42, window=ell, maxit=maxit, x_history=True,
                            relres_history=True, sketch_apply=sketch_apply)
    assert r.iters == maxit and info.status in (O.STOP_MAXIT, O.STOP_BREAKDOWN)
    assert_iterates_conditioned(r, h["x"], h["relres"], info, 0.0)


@pytest.mark.parametrize("precond", ["diag", "reweight"])
@pytest.mark.parametrize("sketch_apply", SKETCH_APPLY)
def test_sflsqr_flexible_operators(ct64, precond, sketch_apply):
    p, plan = ct64
    n = p.A.shape[1]
    w = np.random.default_rng(47).uniform(0.5, 1.5, n)
    tau = O.FixedDiag(w) if precond == "diag" else O.Reweighting(1e-4)
    r = run_oracle_sflsqr(p.A.scipy(), p.b, 61, 8, 46, 20, 0.0, 2, tau=tau)
    x, info, h = plan.solve("sflsqr", dev(p.b), s=61, zeta=8, seed=46, window=2, maxit=20, precond=precond,
                            diag_w=dev(w) if precond == "diag" else None, irw_eps=1e-4, x_history=True,
                            relres_history=True, sketch_apply=sketch_apply)
    assert_iterates_conditioned(r, h["x"], h["relres"], info, 0.0)


@pytest.mark.parametrize("sketch_apply", SKETCH_APPLY)
def test_sflsmr_unmatched_reweighted_per_iteration(ct64_unmatched, sketch_apply):
    A, B, x_true, b, en, plan = ct64_unmatched
    tol = O.discrepancy_tol(1.01, en, np.linalg.norm(b))
    r = run_oracle_sflsmr(A.scipy(), b, 201, 8, 43, 150, tol, 2, tau=O.Reweighting(1e-4), AT=B.scipy())
    x, info, h = plan.solve("sflsmr", dev(b), s=201, zeta=8, seed=43, window=2, maxit=150, noise_norm=en, eta=1.01,
                            precond="reweight", irw_eps=1e-4, x_history=True, relres_history=True,
                            sketch_apply=sketch_apply)
    assert info.status == r.status
    assert_iterates_conditioned(r, h["x"], h["relres"], info, tol)


@pytest.mark.parametrize("sketch_apply", SKETCH_APPLY)
def test_sflsmr_normal_equation_stop_rule(ct64, sketch_apply):
    p, plan = ct64
    r = run_oracle_sflsmr(p.A.scipy(), p.b, 81, 4, 5, 25, 0.0, 2, stop_rule="normal")
    x, info, h = plan.solve("sflsmr", dev(p.b), s=81, zeta=4, seed=5, window=2, maxit=25, stop_rule="normal",
                            x_history=True, relres_history=True, sketch_apply=sketch_apply)
    assert_iterates_conditioned(r, h["x"], h["relres"], info, 0.0)


def ls_smem_doubles(s, maxit, cl, stage_q, stage_saz):
    """The small least-squares kernel's shared-memory plan (doubles), restated:
    six vectors of maxit + 2, three row blocks, slice partials, and the staged
    Q / S_m A Z blocks with an odd row stride."""
    rb = -(-s // cl)
    n = 6 * (maxit + 2) + 3 * rb + max(rb, 256)
    return n + (stage_q + stage_saz) * rb * (maxit | 1)


@pytest.mark.parametrize("method", ["sflsqr", "sflsmr"])
def test_largest_sketch_runs_the_unstaged_small_problem(ct64, method):
    """s = 2048 (the largest sketch) with maxit = 300: a CTA's block of Q (and,
    under sFLSMR's residual rule, of S_m A Z) no longer fits the kernel's
    160 KB staging budget, so the small least-squares step reads them from
    global memory.  Staging depends on s and maxit only; the discrepancy stop
    ends the solve after a few well-conditioned steps."""
    assert ls_smem_doubles(2048, 300, 16, 1, 0) * 8 > 160 * 1024
    p, plan = ct64
    st = p.settings
    tol = O.discrepancy_tol(st["eta"], p.noise_norm[0], np.linalg.norm(p.b))
    kw = dict(s=2048, zeta=8, seed=st["seed"], window=2, maxit=300, noise_norm=p.noise_norm[0], eta=st["eta"],
              x_history=True, relres_history=True)
    if method == "sflsqr":
        r = run_oracle_sflsqr(p.A.scipy(), p.b, 2048, 8, st["seed"], 300, tol, 2)
    else:
        r = run_oracle_sflsmr(p.A.scipy(), p.b, 2048, 8, st["seed"], 300, tol, 2)
    x, info, h = plan.solve(method, dev(p.b), **kw)
    assert info.status == O.STOP_DISCREPANCY == r.status
    assert 2 <= info.iters <= 40
    assert_iterates_flat(r, h["x"], h["relres"], info, tol)


@pytest.mark.parametrize("precond,window", [("diag", 2), ("reweight", 2), ("diag", 5)])
def test_sflsqr_literal_z_window(ct64, precond, window):
    """The z window taken as the stored z_j = tau(p_j) (the window loop of
    Algorithm 1 as printed) against the oracle's literal reading."""
    p, plan = ct64
    n = p.A.shape[1]
    w = np.random.default_rng(47).uniform(0.5, 1.5, n)
    tau = O.FixedDiag(w) if precond == "diag" else O.Reweighting(1e-4)
    r = run_oracle_sflsqr(p.A.scipy(), p.b, 61, 8, 46, 20, 0.0, window, tau=tau, orth_against="z")
    r_p = run_oracle_sflsqr(p.A.scipy(), p.b, 61, 8, 46, 20, 0.0, window, tau=tau)
    assert rel(r.x, r_p.x) > 1e-6, "the two readings should differ when tau is not the identity"
    x, info, h = plan.solve("sflsqr", dev(p.b), s=61, zeta=8, seed=46, window=window, maxit=20, precond=precond,
                            diag_w=dev(w) if precond == "diag" else None, irw_eps=1e-4, x_history=True,
                            relres_history=True, orth_against="z")
    assert_iterates_conditioned(r, h["x"], h["relres"], info, 0.0)


def test_sflsmr_unmatched_literal_z_window(ct64_unmatched):
    A, B, x_true, b, en, plan = ct64_unmatched
    tol = O.discrepancy_tol(1.01, en, np.linalg.norm(b))
    r = run_oracle_sflsmr(A.scipy(), b, 201, 8, 43, 150, tol, 2, tau=O.Reweighting(1e-4), AT=B.scipy(),
                          orth_against="z")
    x, info, h = plan.solve("sflsmr", dev(b), s=201, zeta=8, seed=43, window=2, maxit=150, noise_norm=en, eta=1.01,
                            precond="reweight", irw_eps=1e-4, x_history=True, relres_history=True,
                            orth_against="z")
    assert info.status == r.status
    assert_iterates_conditioned(r, h["x"], h["relres"], info, tol)


def test_literal_z_window_is_the_default_for_identity(ct64):
    """For tau = id the stored z~_j are the p~_j bit for bit, so both readings
    run the same arithmetic."""
    p, plan = ct64
    kw = dict(s=101, zeta=8, seed=42, window=3, maxit=30)
    x1, i1, _ = plan.solve("sflsqr", dev(p.b), **kw)
    x2, i2, _ = plan.solve("sflsqr", dev(p.b), orth_against="z", **kw)
    assert i1.iters == i2.iters and torch.equal(x1, x2)
    o = plan._opts(101, 8, 42, 2, 30, 0.0, 1.01, "identity", "residual", None, 1e-4, "f64", None, None)
    o.orth_against_z = 2
    info = G.N.Info()
    st = plan.lib.sflsqr_solve(plan.handle, G._ptr(dev(p.b)), ctypes.byref(o), G._ptr(x1), ctypes.byref(info),
                               G._stream())
    assert st == G.N.SFL_EINVAL


@pytest.fixture(scope="module")
def ct24():
    """24x24 image, 30 angles x 34 bins (m = 1020, n = 576): small enough for
    an identity sketch on either side (s = m or s = n <= 2048)."""
    A = wl.siddon_projector(24, 30, wl.detector_bins(24))
    rng = np.random.default_rng(11)
    x = wl.ellipse_phantom(24, rng)
    b, en = wl.add_noise(A.matvec(x), 0.01, rng)
    return A, b, G.Plan(A)


def test_identity_sketch_with_full_window_is_textbook_lsqr(ct24):
    """S = I, tau = id and a window covering every earlier vector (ell = 8,
    k <= 9): x_k is the LSQR iterate, checked against SciPy's lsqr run for k
    iterations with no stopping tolerance (the pin on textbook LSQR, on the GPU
    path itself)."""
    A, b, plan = ct24
    m = A.shape[0]
    eye = torch.eye(m, dtype=torch.float64, device="cuda")
    x, info, h = plan.solve("sflsqr", dev(b), s=m, window=8, maxit=9, x_history=True, sketch_matrix=eye)
    assert info.iters == 9
    S = A.scipy()
    for k in range(1, 10):
        xk = spla.lsqr(S, b, atol=0.0, btol=0.0, conlim=0.0, iter_lim=k)[0]
        assert rel(h["x"][k - 1].cpu().numpy(), xk) <= 1e-8, k


def test_identity_sketches_with_full_window_are_textbook_lsmr(ct24):
    A, b, plan = ct24
    m, n = A.shape
    eye_n = torch.eye(n, dtype=torch.float64, device="cuda")
    # the m-side sketch only feeds the discrepancy estimate (no stop here); it has s = n rows
    stop = dev(np.random.default_rng(3).standard_normal((n, m)))
    x, info, h = plan.solve("sflsmr", dev(b), s=n, window=8, maxit=9, x_history=True, sketch_matrix=eye_n,
                            sketch_matrix_stop=stop)
    assert info.iters == 9
    S = A.scipy()
    for k in range(1, 10):
        xk = spla.lsmr(S, b, atol=0.0, btol=0.0, conlim=0.0, maxiter=k)[0]
        assert rel(h["x"][k - 1].cpu().numpy(), xk) <= 1e-8, k


@pytest.mark.parametrize("method", ["sflsqr", "sflsmr"])
def test_gaussian_sketch_matches_oracle(ct64, method):
    """An explicit Gaussian sketch (N(0,1) entries, unscaled as in Corollary
    1), the same matrices given to the oracle's dense sketch."""
    p, plan = ct64
    A = p.A.scipy()
    m, n = A.shape
    s, maxit = 61, 25
    rng = np.random.default_rng(2024)
    if method == "sflsqr":
        Sm = rng.standard_normal((s, m))
        r = O.sflsqr(A, p.b, O.DenseSketch(Sm), maxit=maxit, tol=0.0, ell=2, record_x=True, keep_basis=True)
        r.M = Sm @ (A @ r.Z)
        x, info, h = plan.solve("sflsqr", dev(p.b), s=s, window=2, maxit=maxit, x_history=True,
                                relres_history=True, sketch_matrix=dev(Sm))
    else:
        Sn, Sm = rng.standard_normal((s, n)), rng.standard_normal((s, m))
        r = O.sflsmr(A, p.b, O.DenseSketch(Sn), S_stop=O.DenseSketch(Sm), maxit=maxit, tol=0.0, ell=2,
                     record_x=True, keep_basis=True)
        r.M = Sn @ (A.T @ (A @ r.Z))
        x, info, h = plan.solve("sflsmr", dev(p.b), s=s, window=2, maxit=maxit, x_history=True,
                                relres_history=True, sketch_matrix=dev(Sn), sketch_matrix_stop=dev(Sm))
    assert_iterates_conditioned(r, h["x"], h["relres"], info, 0.0)


# ---------------------------------------------------------------- generated sketches (SRHT, hash-drawn Gaussian)

GEN_SKETCH = {"srht": O.SRHT, "gaussian": O.GaussianHash}


@pytest.mark.parametrize("kind", ["srht", "gaussian"])
def test_generated_sketch_sflsqr_matches_oracle(ct64, kind):
    """sFLSQR with a sketch the kernel regenerates from the seed in every
    application (no stored S): the stop step and every iterate within the
    flat 1e-10 of the oracle given the same matrix (built by its own
    restatement of the generator); two runs bitwise equal."""
    p, plan = ct64
    st = p.settings
    A = p.A.scipy()
    S = GEN_SKETCH[kind](st["seed"], st["s"], A.shape[0])
    tol = O.discrepancy_tol(st["eta"], p.noise_norm[0], np.linalg.norm(p.b))
    r = O.sflsqr(A, p.b, S, maxit=st["maxit"], tol=tol, ell=st["window"], record_x=True, keep_basis=True)
    r.M = S.S @ (A @ r.Z)
    kw = dict(s=st["s"], seed=st["seed"], window=st["window"], maxit=st["maxit"], noise_norm=p.noise_norm[0],
              eta=st["eta"], sketch_kind=kind)
    x, info, h = plan.solve("sflsqr", dev(p.b), x_history=True, relres_history=True, **kw)
    assert info.status == r.status == O.STOP_DISCREPANCY
    assert_iterates_flat(r, h["x"], h["relres"], info, tol)
    x2, info2, _ = plan.solve("sflsqr", dev(p.b), **kw)
    assert torch.equal(x, x2) and info2.iters == info.iters


@pytest.mark.parametrize("kind", ["srht", "gaussian"])
def test_generated_sketch_sflsmr_unmatched_matches_oracle(ct64_unmatched, kind):
    """sFLSMR with B and reweighting, both sketches generated (S_n from the
    seed, the stop sketch S_m from seed + 1), against the oracle."""
    A, B, x_true, b, en, plan = ct64_unmatched
    As, Bs = A.scipy(), B.scipy()
    m, n = As.shape
    Sn, Sm = GEN_SKETCH[kind](43, 201, n), GEN_SKETCH[kind](44, 201, m)
    tol = O.discrepancy_tol(1.01, en, np.linalg.norm(b))
    r = O.sflsmr(As, b, Sn, S_stop=Sm, maxit=150, tol=tol, ell=2, tau=O.Reweighting(1e-4), AT=Bs, record_x=True,
                 keep_basis=True)
    r.M = Sn.S @ (Bs @ (As @ r.Z))
    x, info, h = plan.solve("sflsmr", dev(b), s=201, seed=43, window=2, maxit=150, noise_norm=en, eta=1.01,
                            precond="reweight", irw_eps=1e-4, x_history=True, relres_history=True, sketch_kind=kind)
    assert info.status == r.status
    assert_iterates_conditioned(r, h["x"], h["relres"], info, tol)


def test_generated_sketch_argument_checks(ct64):
    p, plan = ct64
    m = p.A.shape[0]
    M = 1 << (m - 1).bit_length()
    with pytest.raises(G.N.SflError):   # more rows than the Hadamard matrix has
        plan.solve("sflsqr", dev(p.b), s=M + 1, maxit=20, sketch_kind="srht")
    S = torch.zeros((61, m), dtype=torch.float64, device="cuda")
    with pytest.raises(G.N.SflError):   # not with an explicit sketch
        plan.solve("sflsqr", dev(p.b), s=61, maxit=20, sketch_matrix=S, sketch_kind="gaussian")
    with pytest.raises(ValueError):
        plan.solve("sflsqr", dev(p.b), s=61, maxit=20, sketch_kind="fourier")


@pytest.fixture(scope="module")
def decay105():
    """The residual-size study's problem at rho = 1.05: dense 1024 x 512, 10% noise."""
    A, b, _, _ = wl.decaying(1024, 512, 1.05, 70, 0.10)
    return A, b, G.Plan(wl.dense_csr(A))


@pytest.mark.parametrize("method", ["sflsqr", "sflsmr"])
def test_decaying_dense_operator_with_gaussian_sketch_matches_oracle(decay105, method):
    """20 steps, window 8, Gaussian s = 2k + 1 = 41: per-iteration parity on a
    dense operator stored as CSR."""
    A, b, plan = decay105
    m, n = A.shape
    k, s = 20, 41
    g = np.random.default_rng(500)
    Sm, Sn = g.standard_normal((s, m)), g.standard_normal((s, n))
    if method == "sflsqr":
        r = O.sflsqr(A, b, O.DenseSketch(Sm), maxit=k, tol=0.0, ell=8, record_x=True, keep_basis=True)
        r.M = Sm @ (A @ r.Z)
        x, info, h = plan.solve("sflsqr", dev(b), s=s, window=8, maxit=k, x_history=True, relres_history=True,
                                sketch_matrix=dev(Sm))
    else:
        r = O.sflsmr(A, b, O.DenseSketch(Sn), S_stop=O.DenseSketch(Sm), maxit=k, tol=0.0, ell=8, record_x=True,
                     keep_basis=True)
        r.M = Sn @ (A.T @ (A @ r.Z))
        x, info, h = plan.solve("sflsmr", dev(b), s=s, window=8, maxit=k, x_history=True, relres_history=True,
                                sketch_matrix=dev(Sn), sketch_matrix_stop=dev(Sm))
    assert_iterates_conditioned(r, h["x"], h["relres"], info, 0.0)


def test_residual_size_study_ordering():
    """The paper's residual-size study (rho = 1.01, 10% noise, 20 steps,
    Gaussian s = 41), on the GPU path: sLSQR's residual ends well above LSQR's
    (about 30% in the paper), and sLSMR's stays the closer of the two to it
    (means over three sketches)."""
    A, b, _, _ = wl.decaying(1024, 512, 1.01, 70, 0.10)
    m, n = A.shape
    k, s = 20, 41
    r_opt = np.linalg.norm(A @ spla.lsqr(A, b, atol=0.0, btol=0.0, conlim=0.0, iter_lim=k)[0] - b)
    plan = G.Plan(wl.dense_csr(A))
    rq, rm = [], []
    for t in range(3):
        g = np.random.default_rng(500 + t)
        Sm, Sn = dev(g.standard_normal((s, m))), dev(g.standard_normal((s, n)))
        xq, _, _ = plan.solve("sflsqr", dev(b), s=s, window=8, maxit=k, sketch_matrix=Sm)
        xm, _, _ = plan.solve("sflsmr", dev(b), s=s, window=8, maxit=k, sketch_matrix=Sn, sketch_matrix_stop=Sm)
        rq.append(np.linalg.norm(A @ xq.cpu().numpy() - b) / r_opt)
        rm.append(np.linalg.norm(A @ xm.cpu().numpy() - b) / r_opt)
    plan.close()
    assert 1.05 < np.mean(rq) < 1.8
    assert abs(np.mean(rm) - 1.0) < abs(np.mean(rq) - 1.0)


def test_dense_sketch_argument_checks(ct64):
    p, plan = ct64
    m, n = p.A.shape
    Sn = torch.zeros((61, n), dtype=torch.float64, device="cuda")
    with pytest.raises(G.N.SflError):           # sFLSMR needs its m-side stop sketch too
        plan.solve("sflsmr", dev(p.b), s=61, window=2, maxit=10, sketch_matrix=Sn)
    with pytest.raises(ValueError):
        plan.solve("sflsqr", dev(p.b), s=61, window=2, maxit=10, sketch_matrix=Sn)   # wrong width


# ---------------------------------------------------------------- pixel-tiled A^T / B

@pytest.mark.parametrize("vdt", ["f64", "f32", "bf16"])
def test_tiled_transpose_products_are_bit_identical(ct64, ct64_unmatched, vdt):
    """Rows of A^T (or B) stored in 16x16 pixel tiles: every row is summed in
    the same order as in natural order, so the products agree bit for bit."""
    p, _ = ct64
    N = int(round(math.sqrt(p.A.shape[1])))
    rng = np.random.default_rng(5)
    for A, B in ((p.A, None), (ct64_unmatched[0], ct64_unmatched[1])):
        plain = G.Plan(A, B, value_dtype=vdt)
        tiled = G.Plan(A, B, value_dtype=vdt, image_shape=(N, N))
        assert tiled.stats()["tiled_At"] == 1 and plain.stats()["tiled_At"] == 0
        w = dev(rng.standard_normal(A.shape[0]))
        z = dev(rng.standard_normal(A.shape[1]))
        assert torch.equal(plain.apply(w, transpose=True), tiled.apply(w, transpose=True))
        assert torch.equal(plain.apply(z), tiled.apply(z))
        plain.close(); tiled.close()


@pytest.mark.slow
def test_tiled_transpose_with_interleaved_warps_is_bit_identical():
    """1024x1024 operator (481M entries, BF16 values): A^T has 2^20 rows, so a
    tiled plan's CTAs own many tiles and their warps take the blocks in turn;
    every row is still summed exactly as in natural order."""
    A = wl.siddon_projector(1024, 360, wl.detector_bins(1024))
    plain = G.Plan(A, value_dtype="bf16")
    tiled = G.Plan(A, value_dtype="bf16", image_shape=(1024, 1024))
    w = dev(np.random.default_rng(9).standard_normal(A.shape[0]))
    assert torch.equal(plain.apply(w, transpose=True), tiled.apply(w, transpose=True))
    plain.close(); tiled.close()


@pytest.mark.parametrize("vdt", ["f64", "f32", "bf16"])
@pytest.mark.parametrize("tiles", [False, True])
def test_16bit_column_deltas_are_bit_identical(ct64, ct64_unmatched, vdt, tiles):
    """The default plan reads 16-bit column deltas (every delta of a CT
    operator fits); index_bits=32 keeps the 32-bit indices.  The entries, their
    order and the gathers are the same, so products and whole solves agree
    bit for bit."""
    p, _ = ct64
    N = int(round(math.sqrt(p.A.shape[1])))
    shape = (N, N) if tiles else None
    rng = np.random.default_rng(6)
    st = p.settings
    for A, B in ((p.A, None), (ct64_unmatched[0], ct64_unmatched[1])):
        d16 = G.Plan(A, B, value_dtype=vdt, image_shape=shape)
        i32 = G.Plan(A, B, value_dtype=vdt, image_shape=shape, index_bits=32)
        sd, si = d16.stats(), i32.stats()
        assert (sd["index_bytes_A"], sd["index_bytes_At"]) == (2, 2)
        assert (si["index_bytes_A"], si["index_bytes_At"]) == (4, 4)
        assert sd["lanes_A"] == 8 and sd["lanes_At"] == 8
        w = dev(rng.standard_normal(A.shape[0]))
        z = dev(rng.standard_normal(A.shape[1]))
        assert torch.equal(d16.apply(z), i32.apply(z))
        assert torch.equal(d16.apply(w, transpose=True), i32.apply(w, transpose=True))
        b = dev(A.matvec(rng.standard_normal(A.shape[1])))
        method = "sflsqr" if B is None else "sflsmr"
        kw = dict(s=st["s"], zeta=st["zeta"], seed=st["seed"], window=2, maxit=12)
        xa, ia, _ = d16.solve(method, b, **kw)
        xb, ib, _ = i32.solve(method, b, **kw)
        assert ia.iters == ib.iters and torch.equal(xa, xb)
        d16.close(); i32.close()


def test_delta_columns_yield_to_the_device_byte_cap(ct64):
    """A plan capped at the bytes of its 32-bit form builds without the 16-bit
    deltas (no error) and gives the same products."""
    p, _ = ct64
    full = G.Plan(p.A)
    st = full.stats()
    assert (st["index_bytes_A"], st["index_bytes_At"]) == (2, 2)
    delta_bytes = sum(2 * (st[k] + 16) + 4 * r for k, r in (("padded_nnz_A", st["rows"]), ("padded_nnz_At", st["cols"])))
    capped = G.Plan(p.A, max_device_bytes=int(st["device_bytes"]) - delta_bytes)
    sc = capped.stats()
    assert (sc["index_bytes_A"], sc["index_bytes_At"]) == (4, 4)
    assert sc["device_bytes"] == st["device_bytes"] - delta_bytes
    z = dev(np.random.default_rng(2).standard_normal(p.A.shape[1]))
    assert torch.equal(full.apply(z), capped.apply(z))
    full.close(); capped.close()


def test_wide_columns_keep_32bit_indices():
    """An operator whose deltas do not fit in 16 bits (random columns over 2^20)
    keeps the 32-bit indices, and its products still match SciPy."""
    rng = np.random.default_rng(8)
    m, n, per = 300, 1 << 20, 64
    cols = np.sort(np.stack([rng.choice(n, per, replace=False) for _ in range(m)]), axis=1)
    A = wl.CSR((m, n), np.arange(0, m * per + 1, per, dtype=np.int64), cols.ravel().astype(np.int32),
               rng.standard_normal(m * per))
    plan = G.Plan(A)
    assert plan.stats()["index_bytes_A"] == 4
    z = rng.standard_normal(n)
    w = rng.standard_normal(m)
    assert rel(plan.apply(dev(z)).cpu().numpy(), A.scipy() @ z) <= 1e-14
    assert rel(plan.apply(dev(w), transpose=True).cpu().numpy(), A.scipy().T @ w) <= 1e-14
    plan.close()
    with pytest.raises(Exception):
        G.Plan(A, index_bits=16)


def test_tiled_plan_solves_match_oracle(ct64, ct64_unmatched):
    p, _ = ct64
    N = int(round(math.sqrt(p.A.shape[1])))
    st = p.settings
    tol = O.discrepancy_tol(st["eta"], p.noise_norm[0], np.linalg.norm(p.b))
    plan = G.Plan(p.A, image_shape=(N, N))
    r = run_oracle_sflsqr(p.A.scipy(), p.b, st["s"], st["zeta"], st["seed"], st["maxit"], tol, st["window"])
    x, info, h = plan.solve("sflsqr", dev(p.b), s=st["s"], zeta=st["zeta"], seed=st["seed"], window=st["window"],
                            maxit=st["maxit"], noise_norm=p.noise_norm[0], eta=st["eta"], x_history=True,
                            relres_history=True)
    assert info.status == r.status
    assert_iterates_flat(r, h["x"], h["relres"], info, tol)
    plan.close()
    A, B, x_true, b, en, _ = ct64_unmatched
    plan = G.Plan(A, B, image_shape=(N, N))
    tol = O.discrepancy_tol(1.01, en, np.linalg.norm(b))
    r = run_oracle_sflsmr(A.scipy(), b, 201, 8, 43, 150, tol, 2, tau=O.Reweighting(1e-4), AT=B.scipy())
    x, info, h = plan.solve("sflsmr", dev(b), s=201, zeta=8, seed=43, window=2, maxit=150, noise_norm=en, eta=1.01,
                            precond="reweight", irw_eps=1e-4, x_history=True, relres_history=True)
    assert info.status == r.status
    assert_iterates_conditioned(r, h["x"], h["relres"], info, tol)
    plan.close()


def test_operator_order_plan_matches_oracle(ct64):
    """Rows kept in the caller's entry order (no lane-interleaved slots): the
    single-solve products still cover every entry once."""
    p, _ = ct64
    st = p.settings
    tol = O.discrepancy_tol(st["eta"], p.noise_norm[0], np.linalg.norm(p.b))
    plan = G.Plan(p.A, slot_layout="operator")
    r = run_oracle_sflsqr(p.A.scipy(), p.b, st["s"], st["zeta"], st["seed"], st["maxit"], tol, st["window"])
    x, info, h = plan.solve("sflsqr", dev(p.b), s=st["s"], zeta=st["zeta"], seed=st["seed"], window=st["window"],
                            maxit=st["maxit"], noise_norm=p.noise_norm[0], eta=st["eta"], x_history=True,
                            relres_history=True)
    assert_iterates_flat(r, h["x"], h["relres"], info, tol)
    w = dev(np.random.default_rng(4).standard_normal(p.A.shape[0]))
    ref = p.A.scipy().T @ w.cpu().numpy()
    assert rel(plan.apply(w, transpose=True).cpu().numpy(), ref) <= 1e-14
    plan.close()


def test_image_shape_must_match_the_columns(ct64):
    p, _ = ct64
    N = int(round(math.sqrt(p.A.shape[1])))
    with pytest.raises(G.N.SflError):
        G.Plan(p.A, image_shape=(N - 1, N))
    with pytest.raises(G.N.SflError):
        G.Plan(p.A, image_shape=(0, N))


# ---------------------------------------------------------------- determinism and drivers

@pytest.mark.parametrize("sketch_apply", SKETCH_APPLY)
def test_bitwise_reproducible_and_drivers_agree(ct64_unmatched, sketch_apply):
    A, B, x_true, b, en, plan = ct64_unmatched
    kw = dict(s=201, zeta=8, seed=43, window=2, maxit=60, noise_norm=en, eta=1.01, precond="reweight",
              sketch_apply=sketch_apply)
    x1, i1, _ = plan.solve("sflsmr", dev(b), **kw)
    x2, i2, _ = plan.solve("sflsmr", dev(b), **kw)
    x3, i3, _ = plan.solve("sflsmr", dev(b), driver="host_loop", **kw)
    assert torch.equal(x1, x2) and torch.equal(x1, x3)
    assert i1.iters == i2.iters == i3.iters


def test_sketch_apply_modes_launch_what_they_say(ct64, ct64_unmatched):
    """'fused' runs no sketch kernel in the loop, 'kernel' one per step; on
    these short rows (under 512 entries per output) 'auto' is 'kernel'.  The
    two modes agree to rounding (fixed-point against FP64 sums)."""
    p, plan = ct64
    st = p.settings
    kw = dict(s=st["s"], zeta=st["zeta"], seed=st["seed"], window=st["window"], maxit=st["maxit"],
              noise_norm=p.noise_norm[0], eta=st["eta"], driver="profiled")
    runs = {m: plan.solve("sflsqr", dev(p.b), sketch_apply=m, **kw) for m in ("auto", "fused", "kernel")}
    step = {m: h["kernel_launches"]["sketch"] for m, (_, _, h) in runs.items()}
    assert step["fused"] == 0 and step["kernel"] == runs["kernel"][1].iters and step["auto"] == step["kernel"]
    assert runs["fused"][1].iters == runs["kernel"][1].iters
    xf, xk = runs["fused"][0].cpu().numpy(), runs["kernel"][0].cpu().numpy()
    assert rel(xf, xk) <= RTOL_ITER
    A, B, x_true, b, en, planu = ct64_unmatched
    kw = dict(s=201, zeta=8, seed=43, window=2, maxit=60, noise_norm=en, eta=1.01, precond="reweight",
              driver="profiled")
    _, i_f, h_f = planu.solve("sflsmr", dev(b), sketch_apply="fused", **kw)
    _, i_k, h_k = planu.solve("sflsmr", dev(b), sketch_apply="kernel", **kw)
    assert h_f["kernel_launches"]["sketch"] == 0 and h_k["kernel_launches"]["sketch"] == i_k.iters
    with pytest.raises(ValueError):
        plan.solve("sflsqr", dev(p.b), s=st["s"], sketch_apply="sometimes")


def test_host_buffers_entry_point(ct64):
    p, plan = ct64
    st = p.settings
    kw = dict(s=st["s"], zeta=st["zeta"], seed=st["seed"], window=st["window"], maxit=st["maxit"],
              noise_norm=p.noise_norm[0], eta=st["eta"])
    xd, info_d, _ = plan.solve("sflsqr", dev(p.b), **kw)
    xh, info_h = plan.solve_host("sflsqr", p.b, **kw)
    assert np.array_equal(xd.cpu().numpy(), xh) and info_d.iters == info_h.iters


# ---------------------------------------------------------------- edge cases

def test_minimum_sketch_and_single_step(ct64):
    p, plan = ct64
    for zeta, s, maxit in [(1, 2, 1), (1, 11, 10), (16, 17, 16)]:
        r = run_oracle_sflsqr(p.A.scipy(), p.b, s, zeta, 3, maxit, 0.0, 2)
        x, info, h = plan.solve("sflsqr", dev(p.b), s=s, zeta=zeta, seed=3, window=2, maxit=maxit, x_history=True,
                                relres_history=True)
        assert_iterates_conditioned(r, h["x"], h["relres"], info, 0.0)


def test_zero_rhs_returns_zero(ct64):
    p, plan = ct64
    x, info, _ = plan.solve("sflsqr", torch.zeros(p.A.shape[0], dtype=torch.float64, device="cuda"), s=21, maxit=20)
    assert info.status == O.STOP_BREAKDOWN and info.iters == 0
    assert torch.count_nonzero(x) == 0


def test_lucky_breakdown_matches_oracle():
    A = sp.diags([2.0, 1.0, 0.5, 0.25, 3.0, 1.5]).tocsr()
    b = np.array([3.0, 0, 0, 0, 0, 0])
    plan = G.Plan(to_csr(A))
    for method in ("sflsqr", "sflsmr"):
        x, info, _ = plan.solve(method, dev(b), s=7, zeta=2, seed=1, window=2, maxit=6)
        assert info.status == O.STOP_BREAKDOWN and info.iters == 1
        assert np.allclose(x.cpu().numpy(), [1.5, 0, 0, 0, 0, 0], rtol=0, atol=1e-14)


def test_invalid_inputs_are_rejected(ct64):
    p, plan = ct64
    b = dev(p.b)
    with pytest.raises(G.N.SflError) as e:
        plan.solve("sflsqr", b, s=10, maxit=10)            # needs s >= maxit + 1
    assert e.value.status == G.N.SFL_EINVAL
    with pytest.raises(G.N.SflError) as e:
        plan.solve("sflsqr", b, s=50, maxit=10, window=9)   # windows above 8 (negative: full orthogonalization)
    assert e.value.status == G.N.SFL_EINVAL
    bad = to_csr(sp.eye(5, format="csr"))
    bad.colidx = bad.colidx.copy(); bad.colidx[2] = 7
    with pytest.raises(G.N.SflError) as e:
        G.Plan(bad)
    assert e.value.status == G.N.SFL_EINVAL
    nanm = to_csr(sp.eye(5, format="csr"))
    nanm.values = nanm.values.copy(); nanm.values[1] = np.nan
    with pytest.raises(G.N.SflError) as e:
        G.Plan(nanm)
    assert e.value.status == G.N.SFL_ENONFINITE
    bn = p.b.copy(); bn[3] = np.inf
    with pytest.raises(G.N.SflError) as e:
        plan.solve("sflsqr", dev(bn), s=21, maxit=20)
    assert e.value.status == G.N.SFL_ENONFINITE


# ---------------------------------------------------------------- full-size workload

@pytest.mark.slow
def test_ct256_unmatched_full_size_matches_oracle():
    """The 256x256 unmatched sFLSMR workload at full size, in the launch
    configuration the benchmark times (pixel-tiled, lane-interleaved plan):
    the stop step, and x_k and the stop ratio of all steps up to the stop
    within relative 1e-10 of the oracle's."""
    p = wl.make("ct256_sflsmr_unmatched")
    st = p.settings
    plan = G.Plan(p.A, p.B, image_shape=(p.N, p.N))
    tol = O.discrepancy_tol(st["eta"], p.noise_norm[0], np.linalg.norm(p.b))
    r = run_oracle_sflsmr(p.A.scipy(), p.b, st["s"], st["zeta"], st["seed"], st["maxit"], tol, st["window"],
                          tau=O.Reweighting(st["irw_eps"]), AT=p.B.scipy())
    x, info, h = plan.solve("sflsmr", dev(p.b), s=st["s"], zeta=st["zeta"], seed=st["seed"], window=st["window"],
                            maxit=st["maxit"], noise_norm=p.noise_norm[0], eta=st["eta"], precond="reweight",
                            irw_eps=st["irw_eps"], x_history=True, relres_history=True)
    assert info.status == r.status == O.STOP_DISCREPANCY
    assert_iterates_flat(r, h["x"], h["relres"], info, tol)
    x2, info2, _ = plan.solve("sflsmr", dev(p.b), s=st["s"], zeta=st["zeta"], seed=st["seed"], window=st["window"],
                              maxit=st["maxit"], noise_norm=p.noise_norm[0], eta=st["eta"], precond="reweight",
                              irw_eps=st["irw_eps"])
    assert info2.iters == info.iters
    assert rel(x2.cpu().numpy(), r.x) <= RTOL_ITER


@pytest.mark.slow
def test_ct1024_fp64_full_size_matches_oracle():
    """The 1024x1024 FP64 workload the benchmark times (480.6M entries, s =
    600, zeta = 8, window 4), in its launch configuration (pixel-tiled A^T,
    lane-interleaved slots, 8 lanes per row, the sketch fused into the
    forward product): the stop step, and x_k and the stop ratio of every
    step up to the stop within relative 1e-10 of the oracle's."""
    p = wl.make("ct1024_sflsqr")
    st = p.settings
    plan = G.Plan(p.A, image_shape=(p.N, p.N))
    assert plan.stats()["lanes_A"] == 8
    tol = O.discrepancy_tol(st["eta"], p.noise_norm[0], np.linalg.norm(p.b))
    x, info, h = plan.solve("sflsqr", dev(p.b), s=st["s"], zeta=st["zeta"], seed=st["seed"], window=st["window"],
                            maxit=st["maxit"], noise_norm=p.noise_norm[0], eta=st["eta"], x_history=True,
                            relres_history=True, driver="profiled")
    assert h["kernel_launches"]["sketch"] == 0   # fused: no sketch kernel in the loop
    xh, rh = h["x"][: info.iters].clone(), h["relres"].clone()
    del h
    plan.close()
    r = run_oracle_sflsqr(p.A.scipy(), p.b, st["s"], st["zeta"], st["seed"], st["maxit"], tol, st["window"])
    assert info.status == r.status == O.STOP_DISCREPANCY
    assert_iterates_flat(r, xh, rh, info, tol)
    assert rel(x.cpu().numpy(), r.x) <= RTOL_ITER


# ---------------------------------------------------------------- reduced precision: solves

def rounded(S, vdt):
    if vdt == "f32":
        return S.astype(np.float32).astype(np.float64)
    R = S.copy()
    R.data = torch.as_tensor(S.data).to(torch.bfloat16).to(torch.float64).numpy()
    return R


def assert_reduced_iterates(r, xh, info, bar):
    """Reduced precision: every iterate up to the earlier of the two stops
    within `bar` of the oracle's (the stop steps may differ by one: a stop
    ratio near the threshold can fall on either side of it).  Returns the
    worst relative error."""
    assert abs(info.iters - r.iters) <= 1, (info.iters, r.iters)
    kk = min(info.iters, r.iters)
    assert kk >= 1
    worst = 0.0
    for j in range(kk):
        e = rel(xh[j], r.xs[j])
        worst = max(worst, e)
        assert e <= bar, f"step {j + 1}: rel err {e:.3e} (bar {bar:.0e})"
    return worst


@pytest.mark.parametrize("vdt,bar_same_op,bar_fp64,bar_recon", [("f32", 2e-5, 2e-5, 0.01), ("bf16", 2e-5, 2e-2, 0.05)])
def test_reduced_precision_solves_against_oracle(vdt, bar_same_op, bar_fp64, bar_recon, ct64):
    """FP32/BF16 operator values with FP32 vectors and accumulation (FP64 small
    problem).  Stated errors, at every step up to the earlier stop: against
    the FP64 oracle run on the same rounded operator (what FP32 vectors cost),
    against the FP64 oracle on the exact operator (what the value rounding
    costs); and the reconstruction error within 1% (FP32) or 5% (BF16 values,
    about three significant digits) of the FP64 solve's."""
    p, _ = ct64
    st = p.settings
    S = p.A.scipy()
    tol = O.discrepancy_tol(st["eta"], p.noise_norm[0], np.linalg.norm(p.b))
    plan = G.Plan(p.A, value_dtype=vdt)
    x, info, h = plan.solve("sflsqr", dev(p.b), s=st["s"], zeta=st["zeta"], seed=st["seed"], window=st["window"],
                            maxit=st["maxit"], noise_norm=p.noise_norm[0], eta=st["eta"], x_history=True)
    xg = x.cpu().numpy()
    xh = h["x"].cpu().numpy()
    assert np.array_equal(xh[info.iters - 1], xg)
    r_same = run_oracle_sflsqr(rounded(S, vdt), p.b, st["s"], st["zeta"], st["seed"], st["maxit"], tol, st["window"])
    r_exact = run_oracle_sflsqr(S, p.b, st["s"], st["zeta"], st["seed"], st["maxit"], tol, st["window"])
    assert_reduced_iterates(r_same, xh, info, bar_same_op)
    assert_reduced_iterates(r_exact, xh, info, bar_fp64)
    e_gpu = rel(xg, p.x_true)
    e_fp64 = rel(r_exact.x, p.x_true)
    assert abs(e_gpu - e_fp64) <= bar_recon * e_fp64
    plan.close()


@pytest.fixture(scope="module")
def recipe1024_at_256():
    """The 1024x1024 mixed-precision recipe (360 angles, 1% noise, ellipse
    phantom, s = 600, window 4, maxit 300) on a 256x256 image: 360 x 363 rays,
    m = 130,680, n = 65,536, 30M nonzeros."""
    return wl.make("ct1024_sflsqr", N=256, n_angles=360)


@pytest.mark.slow
def test_recipe_1024_fp64_fused_sketch_every_step(recipe1024_at_256):
    """The 1024x1024 recipe (s = 600, zeta = 8, window 4) at 256x256 in FP64
    with the sketch fused into the forward product's epilogue, in the
    benchmark's plan layout: the stop step, and every iterate and stop ratio
    within relative 1e-10 of the oracle's."""
    p = recipe1024_at_256
    st = p.settings
    tol = O.discrepancy_tol(st["eta"], p.noise_norm[0], np.linalg.norm(p.b))
    plan = G.Plan(p.A, image_shape=(p.N, p.N))
    x, info, h = plan.solve("sflsqr", dev(p.b), s=st["s"], zeta=st["zeta"], seed=st["seed"], window=st["window"],
                            maxit=st["maxit"], noise_norm=p.noise_norm[0], eta=st["eta"], x_history=True,
                            relres_history=True, sketch_apply="fused")
    r = run_oracle_sflsqr(p.A.scipy(), p.b, st["s"], st["zeta"], st["seed"], st["maxit"], tol, st["window"])
    assert info.status == r.status == O.STOP_DISCREPANCY
    assert_iterates_flat(r, h["x"], h["relres"], info, tol)
    plan.close()


@pytest.mark.parametrize("vdt,bar_same_op,bar_fp64", [("f32", 1e-4, 1e-4), ("bf16", 1e-4, 2e-2)])
def test_recipe_1024_reduced_precision_every_step(recipe1024_at_256, vdt, bar_same_op, bar_fp64):
    """The mixed-precision recipe with pixel-tiled, lane-interleaved plans as
    the benchmark builds them: every iterate within bar_same_op of the FP64
    oracle run on the same rounded operator, and within bar_fp64 of the
    oracle on the exact operator (BF16 values keep about three digits)."""
    p = recipe1024_at_256
    st = p.settings
    S = p.A.scipy()
    tol = O.discrepancy_tol(st["eta"], p.noise_norm[0], np.linalg.norm(p.b))
    plan = G.Plan(p.A, value_dtype=vdt, image_shape=(p.N, p.N))
    x, info, h = plan.solve("sflsqr", dev(p.b), s=st["s"], zeta=st["zeta"], seed=st["seed"], window=st["window"],
                            maxit=st["maxit"], noise_norm=p.noise_norm[0], eta=st["eta"], x_history=True)
    xh = h["x"].cpu().numpy()
    r_same = run_oracle_sflsqr(rounded(S, vdt), p.b, st["s"], st["zeta"], st["seed"], st["maxit"], tol, st["window"])
    r_exact = run_oracle_sflsqr(S, p.b, st["s"], st["zeta"], st["seed"], st["maxit"], tol, st["window"])
    w_same = assert_reduced_iterates(r_same, xh, info, bar_same_op)
    w_exact = assert_reduced_iterates(r_exact, xh, info, bar_fp64)
    print(f"{vdt}: {info.iters} steps, worst rel err vs oracle on the rounded operator {w_same:.2e}, "
          f"vs the exact operator {w_exact:.2e}")
    plan.close()
