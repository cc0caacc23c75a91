"""GPU parity of full orthogonalization (window < 0; eq. (FGK) with the band
filled) and of the unsketched FLSQR (eq. (FLSQR)), through the C ABI.

Bars: solves that end at the discrepancy stop, every iterate within relative
1e-10 of the FP64 oracle's (flat); stress runs without a stop rule, 1e-10
widened by the small problem's conditioning (32 u kappa); the textbook pins,
1e-9 against SciPy's lsqr / lsmr on a matrix (kappa = 20) on which SciPy's
recurrences, which never reorthogonalize, stay within 1e-11 of the
fully orthogonalized oracle for 50 steps.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import oracle as O
import workloads as wl

pytestmark = pytest.mark.gpu

import torch  # noqa: E402

from paper_2605_22281_gb300 import api as G  # noqa: E402
from tests.test_gpu_parity import (RTOL_ITER, assert_iterates_conditioned, assert_iterates_flat, dev,  # noqa: E402
                                   rel, run_oracle_sflsmr, run_oracle_sflsqr)


@pytest.fixture(autouse=True)
def _needs_cuda():
    if not torch.cuda.is_available():
        raise RuntimeError("GPU test selected but no CUDA device is available")


@pytest.fixture(scope="module")
def ct64():
    p = wl.make("ct64_sflsqr")
    return p, G.Plan(p.A)


@pytest.fixture(scope="module")
def kappa20():
    """Dense 1500 x 400 operator with singular values log-spaced in [1, 20]
    (seeded), stored as CSR, and a Gaussian right-hand side."""
    m, n = 1500, 400
    rng = np.random.default_rng(7)
    U, _ = np.linalg.qr(rng.standard_normal((m, n)))
    V, _ = np.linalg.qr(rng.standard_normal((n, n)))
    A = (U * np.geomspace(1.0, 20.0, n)) @ V.T
    b = rng.standard_normal(m)
    return A, b, G.Plan(wl.dense_csr(A))


@pytest.mark.parametrize("method", ["sflsqr", "sflsmr"])
def test_full_window_to_the_discrepancy_stop(ct64, method):
    p, plan = ct64
    st = p.settings
    tol = O.discrepancy_tol(st["eta"], p.noise_norm[0], np.linalg.norm(p.b))
    run = run_oracle_sflsqr if method == "sflsqr" else run_oracle_sflsmr
    r = run(p.A.scipy(), p.b, st["s"], st["zeta"], st["seed"], st["maxit"], tol, -1)
    x, info, h = plan.solve(method, dev(p.b), s=st["s"], zeta=st["zeta"], seed=st["seed"], window=-1,
                            maxit=st["maxit"], noise_norm=p.noise_norm[0], eta=st["eta"], x_history=True,
                            relres_history=True)
    assert info.status == O.STOP_DISCREPANCY
    assert_iterates_flat(r, h["x"], h["relres"], info, tol)
    assert rel(x.cpu().numpy(), r.x) <= RTOL_ITER


@pytest.mark.parametrize("method,precond", [("sflsqr", "diag"), ("sflsqr", "reweight"), ("sflsmr", "reweight")])
def test_full_window_flexible_operators_stress(ct64, method, precond):
    """30 steps with no stop rule past the discrepancy point, a flexible
    operator, every window vector kept."""
    p, plan = ct64
    n = p.A.shape[1]
    w = np.random.default_rng(47).uniform(0.5, 1.5, n)
    tau = O.FixedDiag(w) if precond == "diag" else O.Reweighting(1e-4)
    run = run_oracle_sflsqr if method == "sflsqr" else run_oracle_sflsmr
    r = run(p.A.scipy(), p.b, 91, 8, 46, 30, 0.0, -1, tau=tau)
    x, info, h = plan.solve(method, dev(p.b), s=91, zeta=8, seed=46, window=-1, maxit=30, precond=precond,
                            diag_w=dev(w) if precond == "diag" else None, irw_eps=1e-4, x_history=True,
                            relres_history=True)
    assert_iterates_conditioned(r, h["x"], h["relres"], info, 0.0)


def test_full_window_unmatched_backprojector():
    N, na = 64, 60
    nb = wl.detector_bins(N)
    A = wl.siddon_projector(N, na, nb)
    B = wl.pixel_backprojector(N, na, nb)
    rng = np.random.default_rng(11)
    x = wl.sparse_phantom(N, rng, 0.05)
    b, en = wl.add_noise(A.matvec(x), 0.02, rng)
    tol = O.discrepancy_tol(1.01, en, np.linalg.norm(b))
    plan = G.Plan(A, B, image_shape=(N, N))
    r = run_oracle_sflsmr(A.scipy(), b, 201, 8, 43, 60, tol, -1, tau=O.Reweighting(1e-4), AT=B.scipy())
    _, info, h = plan.solve("sflsmr", dev(b), s=201, zeta=8, seed=43, window=-1, maxit=60, noise_norm=en, eta=1.01,
                            precond="reweight", irw_eps=1e-4, x_history=True, relres_history=True)
    assert_iterates_conditioned(r, h["x"], h["relres"], info, tol)
    plan.close()


def test_full_window_identity_sketch_is_textbook_lsqr_to_50_steps(kappa20):
    """S = I (s = m), tau = id, full orthogonalization: x_k is the LSQR
    iterate, against SciPy's lsqr run for k iterations, k = 1..50."""
    A, b, plan = kappa20
    m = A.shape[0]
    eye = torch.eye(m, dtype=torch.float64, device="cuda")
    _, info, h = plan.solve("sflsqr", dev(b), s=m, window=-1, maxit=50, x_history=True, sketch_matrix=eye)
    assert info.iters == 50
    xh = h["x"].cpu().numpy()
    for k in range(1, 51):
        xk = spla.lsqr(A, b, atol=0.0, btol=0.0, conlim=0.0, iter_lim=k)[0]
        assert rel(xh[k - 1], xk) <= 1e-9, k


def test_full_window_identity_sketch_is_textbook_lsmr_to_50_steps(kappa20):
    A, b, plan = kappa20
    m, n = A.shape
    eye_n = torch.eye(n, dtype=torch.float64, device="cuda")
    stop = dev(np.random.default_rng(3).standard_normal((n, m)))   # only feeds the discrepancy estimate
    _, info, h = plan.solve("sflsmr", dev(b), s=n, window=-1, maxit=50, x_history=True, sketch_matrix=eye_n,
                            sketch_matrix_stop=stop)
    assert info.iters == 50
    xh = h["x"].cpu().numpy()
    for k in range(1, 51):
        xk = spla.lsmr(A, b, atol=0.0, btol=0.0, conlim=0.0, maxiter=k)[0]
        assert rel(xh[k - 1], xk) <= 1e-9, k


def test_flsqr_is_textbook_lsqr_to_50_steps(kappa20):
    """FLSQR (no sketch, exact projected problem through H) with tau = id."""
    A, b, plan = kappa20
    _, info, h = plan.solve("flsqr", dev(b), s=0, window=-1, maxit=50, x_history=True, relres_history=True)
    assert info.iters == 50
    xh = h["x"].cpu().numpy()
    rh = h["relres"].cpu().numpy()
    for k in range(1, 51):
        xk = spla.lsqr(A, b, atol=0.0, btol=0.0, conlim=0.0, iter_lim=k)[0]
        assert rel(xh[k - 1], xk) <= 1e-9, k
        # the stop ratio is the true relative residual ||b - A x_k|| / ||b||
        tr = np.linalg.norm(b - A @ xh[k - 1]) / np.linalg.norm(b)
        assert abs(rh[k - 1] - tr) <= 1e-10 * tr, k


@pytest.mark.parametrize("precond", ["identity", "reweight"])
def test_flsqr_matches_oracle_with_identity_sketch(ct64, precond):
    """FLSQR against the oracle's sFLSQR with S = I and a full window (the
    exact least-squares problem over A Z_k), to the discrepancy stop."""
    p, plan = ct64
    st = p.settings
    m = p.A.shape[0]
    tol = O.discrepancy_tol(st["eta"], p.noise_norm[0], np.linalg.norm(p.b))
    tau = O.Reweighting(1e-4) if precond == "reweight" else None
    r = O.sflsqr(p.A.scipy(), p.b, O.IdentitySketch(m), maxit=st["maxit"], tol=tol, ell=-1, tau=tau,
                 record_x=True, keep_basis=True)
    r.M = p.A.scipy() @ r.Z
    x, info, h = plan.solve("flsqr", dev(p.b), s=0, window=-1, maxit=st["maxit"], noise_norm=p.noise_norm[0],
                            eta=st["eta"], precond=precond, irw_eps=1e-4, x_history=True, relres_history=True)
    assert info.status == O.STOP_DISCREPANCY
    assert_iterates_flat(r, h["x"], h["relres"], info, tol)


def test_full_window_bitwise_reproducible_and_drivers_agree(ct64):
    p, plan = ct64
    kw = dict(s=121, zeta=8, seed=5, window=-1, maxit=40)
    x1, i1, _ = plan.solve("sflsqr", dev(p.b), **kw)
    x2, i2, _ = plan.solve("sflsqr", dev(p.b), driver="host_loop", **kw)
    x3, i3, _ = plan.solve("flsqr", dev(p.b), s=0, window=-1, maxit=40)
    x4, i4, _ = plan.solve("flsqr", dev(p.b), s=0, window=-1, maxit=40, driver="host_loop")
    assert torch.equal(x1, x2) and i1.iters == i2.iters
    assert torch.equal(x3, x4) and i3.iters == i4.iters


def test_full_window_argument_checks(ct64):
    p, plan = ct64
    with pytest.raises(G.N.SflError) as e:
        plan.solve("sflsqr", dev(p.b), s=61, window=-1, maxit=20, orth_against="z")
    assert e.value.status == G.N.SFL_EUNSUPPORTED
    with pytest.raises(G.N.SflError) as e:     # FLSQR needs the full window
        plan.solve("flsqr", dev(p.b), s=0, window=2, maxit=20)
    assert e.value.status == G.N.SFL_EINVAL


@pytest.mark.slow
def test_more_than_256_steps_reach_the_unstaged_inverse_rows():
    """300 steps of sFLSQR with every window vector kept (no stop rule), s = 700,
    on a dense 1500 x 1000 operator with singular values log-spaced in
    [1, 1000] (seeded): the small least-squares kernel keeps the first 256 rows
    of R^-1 in registers and takes the rest from global memory, which only
    steps past 257 reach.  The basis stays orthonormal (1e-14) and
    cond(S A Z_300) is 7e2 here, so every iterate is held to the flat 1e-10."""
    m, n = 1500, 1000
    rng = np.random.default_rng(7)
    U, _ = np.linalg.qr(rng.standard_normal((m, n)))
    V, _ = np.linalg.qr(rng.standard_normal((n, n)))
    A = (U * np.geomspace(1.0, 1000.0, n)) @ V.T
    b = rng.standard_normal(m)
    plan = G.Plan(wl.dense_csr(A))
    r = run_oracle_sflsqr(A, b, 700, 8, 71, 300, 0.0, -1)
    x, info, h = plan.solve("sflsqr", dev(b), s=700, zeta=8, seed=71, window=-1, maxit=300, x_history=True,
                            relres_history=True)
    assert info.iters == 300 and r.iters == 300
    assert np.linalg.cond(r.M) < 1e4
    checked = assert_iterates_conditioned(r, h["x"], h["relres"], info, 0.0, min_checked=300)
    assert checked == 300
    plan.close()
