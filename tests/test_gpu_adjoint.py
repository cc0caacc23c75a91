"""GPU hand-written adjoint of fixed-k batched sFLSQR against the oracle's
autograd gradients (oracle.adjoint), and through torch.autograd.

Bars: FP64 forward iterates as the batched solve; FP64 gradients within
relative 1e-8 (they go through the small QR twice, so the bar is the
iterate bar widened by the small problem's conditioning); FP32 gradients
within 2e-3 of the FP64 oracle's; the full-size case by a directional
finite difference of the GPU forward itself.
"""
import numpy as np
import pytest

import oracle as O
import workloads as wl

pytestmark = pytest.mark.gpu

import torch  # noqa: E402

from paper_2605_22281_gb300 import api as G  # noqa: E402

OA = pytest.importorskip("oracle.adjoint")
U = np.finfo(np.float64).eps / 2


@pytest.fixture(autouse=True)
def _needs_cuda():
    if not torch.cuda.is_available():
        raise RuntimeError("GPU test selected but no CUDA device is available")


def rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def dev(x):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


def problem(N=32, n_angles=24, R=3, seed=7):
    A = wl.siddon_projector(N, n_angles, wl.detector_bins(N))
    bs = []
    for j in range(R):
        rng = np.random.default_rng(seed + j)
        b, _ = wl.add_noise(A.matvec(wl.ellipse_phantom(N, rng)), 0.01, rng)
        bs.append(b)
    return A, np.stack(bs)


def oracle_grads(A, B, d, s, zeta, seed, k, ell, Xbar):
    S = O.SparseSign(seed, s, zeta, A.shape[0]).dense()
    xs, gbs, gd = [], [], 0.0
    for j in range(B.shape[0]):
        x, gb, gdj = OA.gradients(A, B[j], d, S, k, ell, Xbar[j])
        xs.append(x); gbs.append(gb); gd = gd + gdj
    return np.stack(xs), np.stack(gbs), gd


@pytest.fixture(scope="module")
def small():
    A, B = problem()
    return A, B, G.Plan(A)


@pytest.mark.parametrize("ell,k", [(2, 8), (1, 6), (3, 10)])
def test_fp64_adjoint_matches_oracle_gradients(small, ell, k):
    A, B, plan = small
    n = A.shape[1]
    rng = np.random.default_rng(20 + ell)
    d = rng.uniform(0.5, 1.5, n)
    Xbar = rng.standard_normal((B.shape[0], n))
    X, infos, _ = G.fixed_batched(plan, dev(B), dev(d), s=41, zeta=8, seed=3, window=ell, maxit=k)
    assert all(i.iters == k for i in infos)
    Bbar, dbar = G.adjoint(plan, dev(Xbar))
    xo, gb, gd = oracle_grads(A, B, d, 41, 8, 3, k, ell, Xbar)
    assert rel(X.cpu().numpy(), xo) <= 1e-10
    assert rel(Bbar.cpu().numpy(), gb) <= 1e-8
    assert rel(dbar.cpu().numpy(), gd) <= 1e-8


def test_tiled_plan_adjoint_matches_oracle_gradients(small):
    """The same gradients through a plan whose A^T rows are stored in pixel
    tiles (the SpMMs write through the original-row map)."""
    A, B, _ = small
    n = A.shape[1]
    N = int(round(np.sqrt(n)))
    tiled = G.Plan(A, image_shape=(N, N))
    assert tiled.stats()["tiled_At"] == 1
    rng = np.random.default_rng(33)
    d = rng.uniform(0.5, 1.5, n)
    Xbar = rng.standard_normal((B.shape[0], n))
    X, infos, _ = G.fixed_batched(tiled, dev(B), dev(d), s=41, zeta=8, seed=3, window=2, maxit=8)
    Bbar, dbar = G.adjoint(tiled, dev(Xbar))
    xo, gb, gd = oracle_grads(A, B, d, 41, 8, 3, 8, 2, Xbar)
    assert rel(X.cpu().numpy(), xo) <= 1e-10
    assert rel(Bbar.cpu().numpy(), gb) <= 1e-8
    assert rel(dbar.cpu().numpy(), gd) <= 1e-8
    tiled.close()


def test_identity_operator_weight_gradient_at_one(small):
    A, B, plan = small
    n = A.shape[1]
    Xbar = np.random.default_rng(31).standard_normal((B.shape[0], n))
    X, _, _ = G.fixed_batched(plan, dev(B), None, s=41, zeta=8, seed=3, window=2, maxit=8)
    Bbar, dbar = G.adjoint(plan, dev(Xbar))
    xo, gb, gd = oracle_grads(A, B, np.ones(n), 41, 8, 3, 8, 2, Xbar)
    assert rel(X.cpu().numpy(), xo) <= 1e-10
    assert rel(Bbar.cpu().numpy(), gb) <= 1e-8
    assert rel(dbar.cpu().numpy(), gd) <= 1e-8


def test_fp32_adjoint_against_fp64_oracle():
    A, B = problem(seed=40)
    n = A.shape[1]
    plan = G.Plan(A, value_dtype="f32")
    rng = np.random.default_rng(41)
    d = rng.uniform(0.5, 1.5, n)
    Xbar = rng.standard_normal((B.shape[0], n))
    X, _, _ = G.fixed_batched(plan, dev(B), dev(d), s=41, zeta=8, seed=3, window=2, maxit=8)
    Bbar, dbar = G.adjoint(plan, dev(Xbar))
    xo, gb, gd = oracle_grads(A, B, d, 41, 8, 3, 8, 2, Xbar)
    assert rel(X.cpu().numpy(), xo) <= 2e-4
    assert rel(Bbar.cpu().numpy(), gb) <= 2e-3
    assert rel(dbar.cpu().numpy(), gd) <= 2e-3
    plan.close()


def test_autograd_function_and_stale_state(small):
    A, B, plan = small
    n = A.shape[1]
    rng = np.random.default_rng(50)
    Bt = dev(B).requires_grad_(True)
    dt = dev(rng.uniform(0.5, 1.5, n)).requires_grad_(True)
    Xbar = dev(rng.standard_normal((B.shape[0], n)))
    kw = dict(s=41, zeta=8, seed=3, window=2, maxit=8)
    X = G.sflsqr_fixed_k(plan, Bt, dt, **kw)
    (X * Xbar).sum().backward()
    X2, _, _ = G.fixed_batched(plan, dev(B), dt.detach(), **kw)
    gb, gd = G.adjoint(plan, Xbar)
    assert torch.equal(X.detach(), X2)
    assert torch.equal(Bt.grad, gb) and torch.equal(dt.grad, gd)
    # a second forward replaces the kept state: the first one's backward refuses
    Y = G.sflsqr_fixed_k(plan, Bt, dt, **kw)
    G.fixed_batched(plan, dev(B), dt.detach(), **kw)
    with pytest.raises(RuntimeError):
        (Y * Xbar).sum().backward()


def test_adjoint_limits(small):
    A, B, plan = small
    with pytest.raises(G.N.SflError):
        G.fixed_batched(plan, dev(B), None, s=41, zeta=8, seed=3, window=4, maxit=8)
    fresh = G.Plan(A)
    with pytest.raises(G.N.SflError):
        G.adjoint(fresh, dev(np.zeros((B.shape[0], A.shape[1]))))
    fresh.close()


@pytest.mark.slow
def test_full_shape_gradients_match_oracle():
    """The differentiated workload's shape (256x256, 180 angles, s = 61,
    window 2, diagonal weight) for two of its sinograms at k = 10: the FP64
    forward and both gradients against the oracle's autograd at the
    small-case bars (kappa(S A Z_10) ~ 7e3)."""
    p = wl.make("ct256_diff16")
    st = p.settings
    plan = G.Plan(p.A, value_dtype="f64", image_shape=(p.N, p.N))
    B = p.b.T[[0, 9]].copy()
    d = st["weight"]
    Xbar = np.random.default_rng(61).standard_normal((B.shape[0], p.A.shape[1]))
    X, infos, _ = G.fixed_batched(plan, dev(B), dev(d), s=st["s"], zeta=st["zeta"], seed=st["seed"],
                                  window=st["window"], maxit=10)
    assert all(i.iters == 10 for i in infos)
    Bbar, dbar = G.adjoint(plan, dev(Xbar))
    xo, gb, gd = oracle_grads(p.A, B, d, st["s"], st["zeta"], st["seed"], 10, st["window"], Xbar)
    ex, eb, ed = rel(X.cpu().numpy(), xo), rel(Bbar.cpu().numpy(), gb), rel(dbar.cpu().numpy(), gd)
    print(f"full shape k=10: x {ex:.1e}, b-gradient {eb:.1e}, d-gradient {ed:.1e}")
    assert ex <= 1e-10 and eb <= 1e-8 and ed <= 1e-8
    plan.close()


@pytest.mark.slow
def test_full_size_directional_derivative():
    """16 sinograms of 256x256 phantoms with the diagonal weight, s = 61,
    window 2, FP64: <Xbar, dX[v]> from the adjoint against a central
    difference of the GPU forward along random directions in b and d.  k = 10
    (kappa(S A Z_10) ~ 7e3); at the configured k = 30 the sketched basis is
    numerically dependent (kappa ~ 1e15 from k ~ 20), where no derivative of
    the fixed-k map is determined."""
    p = wl.make("ct256_diff16")
    st = p.settings
    plan = G.Plan(p.A, value_dtype="f64")
    rng = np.random.default_rng(60)
    B = p.b.T.copy()
    d = st["weight"]
    Xbar = rng.standard_normal((B.shape[0], p.A.shape[1]))
    kw = dict(s=st["s"], zeta=st["zeta"], seed=st["seed"], window=st["window"], maxit=10)
    G.fixed_batched(plan, dev(B), dev(d), **kw)
    Bbar, dbar = G.adjoint(plan, dev(Xbar))
    vb = rng.standard_normal(B.shape)
    vd = rng.standard_normal(d.shape)
    hb = 1e-5 * np.linalg.norm(B) / np.linalg.norm(vb)
    hd = 1e-5 * np.linalg.norm(d) / np.linalg.norm(vd)

    def L(bb, dd):
        X, _, _ = G.fixed_batched(plan, dev(bb), dev(dd), **kw)
        return float((X.cpu().numpy() * Xbar).sum())

    fd_b = (L(B + hb * vb, d) - L(B - hb * vb, d)) / (2 * hb)
    fd_d = (L(B, d + hd * vd) - L(B, d - hd * vd)) / (2 * hd)
    assert abs(fd_b - float((Bbar.cpu().numpy() * vb).sum())) <= 1e-4 * abs(fd_b)
    assert abs(fd_d - float((dbar.cpu().numpy() * vd).sum())) <= 1e-4 * abs(fd_d)
    plan.close()
