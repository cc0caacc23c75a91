"""GPU parity of the matrix-free parallel-beam projectors (sfl_plan_create_ct)
against the stored operators of workloads/ (the same geometry, built by the C
generator) and against the FP64 oracle.

Bars: FP64 products within relative 16 N u of the CSR products (u = 2^-53;
a Siddon chord is the difference of two crossing parameters of size up to
N, each rounded, and the summation orders differ); FP32 products within
relative 4 N u32 (u32 = 2^-24: FP32 grid coordinates up to N, the same
chord argument);
solves on a matrix-free FP64 plan per iterate against the oracle on the CSR
operator: flat 1e-10 for a solve that ends at its discrepancy stop, the
conditioned bar for stress runs.
"""
import numpy as np
import pytest

import oracle as O
import workloads as wl

pytestmark = pytest.mark.gpu

import torch  # noqa: E402

from paper_2605_22281_gb300 import api as G  # noqa: E402
from tests.test_gpu_parity import (assert_iterates_conditioned, assert_iterates_flat, dev, rel,  # noqa: E402
                                   run_oracle_sflsmr, run_oracle_sflsqr)


@pytest.fixture(autouse=True)
def _needs_cuda():
    if not torch.cuda.is_available():
        raise RuntimeError("GPU test selected but no CUDA device is available")


GEOMS = [(64, 60), (24, 30), (33, 17), (128, 45)]   # (N, angles): bins = ceil(N sqrt 2)


@pytest.mark.parametrize("N,na", GEOMS)
def test_fp64_products_equal_the_stored_operators(N, na):
    nb = wl.detector_bins(N)
    A = wl.siddon_projector(N, na, nb).scipy()
    B = wl.pixel_backprojector(N, na, nb).scipy()
    rng = np.random.default_rng(N + na)
    z = rng.standard_normal(N * N)
    w = rng.standard_normal(na * nb)
    pm = G.Plan.ct(N, na, nb, back="matched")
    pu = G.Plan.ct(N, na, nb, back="unmatched")
    assert pm.stats()["matrix_free"] == 1
    e = [rel(pm.apply(dev(z)).cpu().numpy(), A @ z),
         rel(pm.apply(dev(w), transpose=True).cpu().numpy(), A.T @ w),
         rel(pu.apply(dev(w), transpose=True).cpu().numpy(), B @ w)]
    print(f"N={N} angles={na}: A z {e[0]:.1e}, A^T w {e[1]:.1e}, B w {e[2]:.1e}")
    assert max(e) <= 16 * N * 2.0 ** -53
    pm.close(); pu.close()


@pytest.mark.parametrize("N,na", [(64, 60), (256, 180)])
def test_fp32_products_against_the_stored_operators(N, na):
    nb = wl.detector_bins(N)
    A = wl.siddon_projector(N, na, nb).scipy()
    B = wl.pixel_backprojector(N, na, nb).scipy()
    rng = np.random.default_rng(3)
    z = rng.standard_normal(N * N).astype(np.float32).astype(np.float64)
    w = rng.standard_normal(na * nb).astype(np.float32).astype(np.float64)
    pm = G.Plan.ct(N, na, nb, back="matched", value_dtype="f32")
    pu = G.Plan.ct(N, na, nb, back="unmatched", value_dtype="f32")
    e = [rel(pm.apply(dev(z)).cpu().numpy(), A @ z),
         rel(pm.apply(dev(w), transpose=True).cpu().numpy(), A.T @ w),
         rel(pu.apply(dev(w), transpose=True).cpu().numpy(), B @ w)]
    print(f"fp32 N={N}: A z {e[0]:.1e}, A^T w {e[1]:.1e}, B w {e[2]:.1e}")
    assert max(e) <= 4 * N * 2.0 ** -24
    pm.close(); pu.close()


def test_matrix_free_sflsqr_to_the_discrepancy_stop():
    p = wl.make("ct64_sflsqr")
    st = p.settings
    tol = O.discrepancy_tol(st["eta"], p.noise_norm[0], np.linalg.norm(p.b))
    r = run_oracle_sflsqr(p.A.scipy(), p.b, st["s"], st["zeta"], st["seed"], st["maxit"], tol, st["window"])
    plan = G.Plan.ct(p.N, p.n_angles, p.n_bins)
    x, info, h = plan.solve("sflsqr", dev(p.b), s=st["s"], zeta=st["zeta"], seed=st["seed"], window=st["window"],
                            maxit=st["maxit"], noise_norm=p.noise_norm[0], eta=st["eta"], x_history=True,
                            relres_history=True)
    assert_iterates_flat(r, h["x"], h["relres"], info, tol)
    plan.close()


def test_matrix_free_unmatched_sflsmr_reweighted():
    N, na = 64, 60
    nb = wl.detector_bins(N)
    A = wl.siddon_projector(N, na, nb)
    B = wl.pixel_backprojector(N, na, nb)
    rng = np.random.default_rng(11)
    x = wl.sparse_phantom(N, rng, 0.05)
    b, en = wl.add_noise(A.matvec(x), 0.02, rng)
    tol = O.discrepancy_tol(1.01, en, np.linalg.norm(b))
    r = run_oracle_sflsmr(A.scipy(), b, 201, 8, 43, 60, tol, 2, tau=O.Reweighting(1e-4), AT=B.scipy())
    plan = G.Plan.ct(N, na, nb, back="unmatched")
    _, info, h = plan.solve("sflsmr", dev(b), s=201, zeta=8, seed=43, window=2, maxit=60, noise_norm=en, eta=1.01,
                            precond="reweight", irw_eps=1e-4, x_history=True, relres_history=True)
    assert_iterates_conditioned(r, h["x"], h["relres"], info, tol)
    plan.close()


def test_matrix_free_fp32_solve_against_the_oracle():
    """FP32 geometry, vectors and sums: every iterate within 1e-4 of the FP64
    oracle on the stored operator (the 1024^2 recipe at 128^2)."""
    p = wl.make("ct1024_sflsqr", N=128, n_angles=90)
    st = p.settings
    tol = O.discrepancy_tol(st["eta"], p.noise_norm[0], np.linalg.norm(p.b))
    r = run_oracle_sflsqr(p.A.scipy(), p.b, st["s"], st["zeta"], st["seed"], st["maxit"], tol, st["window"])
    plan = G.Plan.ct(p.N, p.n_angles, p.n_bins, value_dtype="f32")
    x, info, h = plan.solve("sflsqr", dev(p.b), s=st["s"], zeta=st["zeta"], seed=st["seed"], window=st["window"],
                            maxit=st["maxit"], noise_norm=p.noise_norm[0], eta=st["eta"], x_history=True)
    assert abs(info.iters - r.iters) <= 1
    xh = h["x"].cpu().numpy()
    errs = [rel(xh[j], r.xs[j]) for j in range(min(info.iters, r.iters))]
    print(f"fp32 matrix-free: {info.iters} steps, worst {max(errs):.2e}")
    assert max(errs) <= 1e-4
    plan.close()


def test_matrix_free_plans_refuse_batched_solves():
    plan = G.Plan.ct(32, 10, wl.detector_bins(32))
    B = torch.zeros((2, plan.m), dtype=torch.float64, device="cuda")
    with pytest.raises(G.N.SflError) as e:
        G.solve_batched(plan, B, [0.0, 0.0], s=21, maxit=10)
    assert e.value.status == G.N.SFL_EUNSUPPORTED
    plan.close()


def test_matrix_free_fused_sketch_at_512():
    """From 512^2 the sketch is fused into the forward product, whose CTAs then
    keep contiguous ray ranges (the sketch epilogue reads its own rows back):
    every iterate of the FP64 matrix-free solve within the flat bar of the
    oracle on the stored operator (the 1024^2 recipe at 512^2, 90 angles)."""
    p = wl.make("ct1024_sflsqr", N=512, n_angles=90)
    st = p.settings
    tol = O.discrepancy_tol(st["eta"], p.noise_norm[0], np.linalg.norm(p.b))
    r = run_oracle_sflsqr(p.A.scipy(), p.b, st["s"], st["zeta"], st["seed"], st["maxit"], tol, st["window"])
    plan = G.Plan.ct(p.N, p.n_angles, p.n_bins)
    x, info, h = plan.solve("sflsqr", dev(p.b), s=st["s"], zeta=st["zeta"], seed=st["seed"], window=st["window"],
                            maxit=st["maxit"], noise_norm=p.noise_norm[0], eta=st["eta"], sketch_apply="fused",
                            x_history=True, relres_history=True)
    assert_iterates_flat(r, h["x"], h["relres"], info, tol)
    plan.close()
