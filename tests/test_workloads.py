"""Sanity checks of the seeded synthetic CT inputs (geometry, sizes, noise)."""
import math

import numpy as np

import workloads as wl


def test_detector_bins_cover_diagonal():
    assert [wl.detector_bins(N) for N in (64, 256, 512, 1024)] == [91, 363, 725, 1449]


def test_siddon_geometry():
    N, na, nb = 32, 12, wl.detector_bins(32)
    A = wl.siddon_projector(N, na, nb)
    S = A.scipy()
    assert S.shape == (na * nb, N * N)
    # chord lengths are positive and no ray is longer than the image diagonal
    assert A.values.min() > 0 and np.asarray(S.sum(axis=1)).max() <= N * math.sqrt(2) + 1e-9
    # columns sorted within rows
    for r in range(S.shape[0]):
        c = A.colidx[A.rowptr[r]:A.rowptr[r + 1]]
        assert np.all(np.diff(c) > 0)
    # unit-spaced rays sample each pixel's width profile: mass 1 on average per angle
    for a in range(na):
        mass = np.asarray(S[a * nb:(a + 1) * nb].sum(axis=0)).ravel()
        assert abs(mass.mean() - 1.0) < 0.02 and mass.max() <= 2.0 + 1e-12


def test_pixel_backprojector_is_unmatched_adjoint():
    N, na = 32, 12
    nb = wl.detector_bins(N)
    A = wl.siddon_projector(N, na, nb).scipy()
    B = wl.pixel_backprojector(N, na, nb)
    assert B.shape == (N * N, na * nb)
    Bs = B.scipy()
    # interpolation weights sum to one per (pixel, angle)
    assert np.allclose(np.asarray(Bs.sum(axis=1)).ravel(), na)
    rng = np.random.default_rng(0)
    x = rng.standard_normal(N * N); x /= np.linalg.norm(x)
    y = rng.standard_normal(na * nb); y /= np.linalg.norm(y)
    mismatch = abs(y @ (A @ x) - x @ (Bs @ y))
    assert 1e-4 < mismatch < 0.2          # B != A^T, but close (Section 3.2 reports ~4e-2)


def test_noise_level_exact_and_seeded():
    p1 = wl.make("ct64_sflsqr")
    p2 = wl.make("ct64_sflsqr")
    assert np.array_equal(p1.b, p2.b)
    bt = p1.A.matvec(p1.x_true)
    assert abs(np.linalg.norm(p1.b - bt) - p1.noise_norm[0]) <= 1e-12 * p1.noise_norm[0]
    assert abs(p1.noise_norm[0] / np.linalg.norm(bt) - 0.01) < 1e-12
    assert p1.A.shape == (5460, 4096)


def test_sparse_phantom_fraction():
    x = wl.sparse_phantom(64, np.random.default_rng(2), 0.05)
    assert np.count_nonzero(x) == round(0.05 * 4096)
    assert x.min() >= 0 and x.max() <= 1
