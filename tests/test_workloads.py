"""Sanity checks of the seeded synthetic CT inputs (geometry, sizes, noise)."""
import math

import numpy as np
import pytest

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


def _clip_length(p0, u, lo, hi):
    """Length of the line p0 + s u inside the box [lo, hi] (Liang-Barsky clipping)."""
    s0, s1 = -math.inf, math.inf
    for k in range(2):
        if abs(u[k]) < 1e-15:
            if not (lo[k] <= p0[k] <= hi[k]):
                return 0.0
            continue
        a, b = (lo[k] - p0[k]) / u[k], (hi[k] - p0[k]) / u[k]
        s0, s1 = max(s0, min(a, b)), min(s1, max(a, b))
    return max(0.0, s1 - s0)


@pytest.mark.parametrize("N,na", [(8, 7), (11, 9)])
def test_siddon_entries_are_clipped_chords(N, na):
    """Every entry of the Siddon operator is the length of its ray clipped to
    its unit pixel, and every ray's sum is the chord through the whole image
    (checked for the angles off the axes; axis-aligned rays on grid lines
    follow the walk's floor rule instead)."""
    nb = wl.detector_bins(N)
    S = wl.siddon_projector(N, na, nb).scipy().toarray()
    h = N / 2
    checked = 0
    for a in range(na):
        th = a * math.pi / na
        c, s = math.cos(th), math.sin(th)
        if abs(c) < 1e-9 or abs(s) < 1e-9:
            continue
        u = (-s, c)
        for d in range(nb):
            t = d - 0.5 * (nb - 1)
            p0 = (t * c, t * s)
            row = a * nb + d
            whole = _clip_length(p0, u, (-h, -h), (h, h))
            assert abs(S[row].sum() - whole) <= 1e-12 * max(1.0, whole)
            for iy in range(N):
                for ix in range(N):
                    ref = _clip_length(p0, u, (ix - h, iy - h), (ix + 1 - h, iy + 1 - h))
                    got = S[row, iy * N + ix]
                    assert abs(got - ref) <= 1e-12, (a, d, ix, iy, got, ref)
            checked += 1
    assert checked >= (na - 1) * nb // 2


@pytest.mark.parametrize("N,na", [(8, 7), (11, 9)])
def test_backprojector_entries_are_hat_weights(N, na):
    """B[pixel, (a, d)] is the linear-interpolation (hat) weight max(0, 1 - |u - d|)
    of the pixel centre's bin coordinate u = x_c cos + y_c sin + (n_bins - 1)/2."""
    nb = wl.detector_bins(N)
    B = wl.pixel_backprojector(N, na, nb).scipy().toarray()
    h = N / 2
    off = 0.5 * (nb - 1)
    for a in range(na):
        th = a * math.pi / na
        c, s = math.cos(th), math.sin(th)
        for iy in range(N):
            for ix in range(N):
                u = (ix - h + 0.5) * c + (iy - h + 0.5) * s + off
                ref = np.maximum(0.0, 1.0 - np.abs(u - np.arange(nb)))
                ref[ref <= 1e-12] = 0.0
                got = B[iy * N + ix, a * nb:(a + 1) * nb]
                assert np.abs(got - ref).max() <= 1e-12, (a, ix, iy)
