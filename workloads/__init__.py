"""Seeded synthetic CT workloads (input data only).

This module builds the inputs that both the CPU oracle and the GPU solver are
run on: parallel-beam Siddon projectors A (CSR), pixel-driven unmatched
back-projectors B (CSR), random-ellipse and sparse phantoms, and noisy
sinograms b = A x_true + e with an exact noise level (the noise model of the
discrepancy principle, eq. (discrP) in Section 1.1).  It contains none of the
solver arithmetic and imports neither the oracle nor the GPU package.

The geometry conventions live in ``ctgen.c``.  The C helpers are compiled on
first use with the host gcc (OpenMP, ``-ffp-contract=off`` so that x86-64 and
aarch64 produce identical arrays).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ctgen.c")
_SO = os.path.join(_HERE, "_ctgen.so")
_lock = threading.Lock()
_lib = None


def build() -> str:
    """Compile ctgen.c into _ctgen.so next to it (idempotent)."""
    if os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(_SRC):
        return _SO
    tmp = _SO + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-ffp-contract=off",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i64p = ctypes.POINTER(ctypes.c_int64)
            i32p = ctypes.POINTER(ctypes.c_int32)
            f64p = ctypes.POINTER(ctypes.c_double)
            for name in ("siddon_count", "pixel_count"):
                getattr(lib, name).argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, i64p]
                getattr(lib, name).restype = None
            for name in ("siddon_fill", "pixel_fill"):
                getattr(lib, name).argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, i64p, i32p, f64p]
                getattr(lib, name).restype = None
            lib.csr_matvec.argtypes = [ctypes.c_int64, i64p, i32p, f64p, f64p, f64p]
            lib.csr_matvec.restype = None
            _lib = lib
    return _lib


def _ptr(a: np.ndarray, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


@dataclass
class CSR:
    """A CSR matrix as plain arrays: int64 row pointers, int32 columns, f64 values."""
    shape: tuple
    rowptr: np.ndarray
    colidx: np.ndarray
    values: np.ndarray

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    def rowptr32(self) -> np.ndarray:
        assert self.nnz < 2**31
        return self.rowptr.astype(np.int32)

    def scipy(self):
        import scipy.sparse as sp
        return sp.csr_matrix((self.values, self.colidx, self.rowptr), shape=self.shape)

    def matvec(self, x: np.ndarray) -> np.ndarray:
        """y = A x with the OpenMP C helper (used to synthesise b)."""
        x = np.ascontiguousarray(x, dtype=np.float64)
        y = np.empty(self.shape[0], dtype=np.float64)
        _load().csr_matvec(self.shape[0], _ptr(self.rowptr, ctypes.c_int64), _ptr(self.colidx, ctypes.c_int32),
                           _ptr(self.values, ctypes.c_double), _ptr(x, ctypes.c_double), _ptr(y, ctypes.c_double))
        return y


def _two_pass(count_fn, fill_fn, rows: int, N: int, n_angles: int, n_bins: int) -> tuple:
    cnt = np.zeros(rows, dtype=np.int64)
    count_fn(N, n_angles, n_bins, _ptr(cnt, ctypes.c_int64))
    rowptr = np.zeros(rows + 1, dtype=np.int64)
    np.cumsum(cnt, out=rowptr[1:])
    nnz = int(rowptr[-1])
    col = np.empty(nnz, dtype=np.int32)
    val = np.empty(nnz, dtype=np.float64)
    fill_fn(N, n_angles, n_bins, _ptr(rowptr, ctypes.c_int64), _ptr(col, ctypes.c_int32), _ptr(val, ctypes.c_double))
    return rowptr, col, val


def siddon_projector(N: int, n_angles: int, n_bins: int) -> CSR:
    """Ray-driven parallel-beam projector A (m = n_angles*n_bins rows, n = N*N columns)."""
    lib = _load()
    m = n_angles * n_bins
    rowptr, col, val = _two_pass(lib.siddon_count, lib.siddon_fill, m, N, n_angles, n_bins)
    return CSR((m, N * N), rowptr, col, val)


def pixel_backprojector(N: int, n_angles: int, n_bins: int) -> CSR:
    """Pixel-driven linear-interpolation back-projector B (n x m), B != A^T."""
    lib = _load()
    n = N * N
    rowptr, col, val = _two_pass(lib.pixel_count, lib.pixel_fill, n, N, n_angles, n_bins)
    return CSR((n, n_angles * n_bins), rowptr, col, val)


def detector_bins(N: int) -> int:
    """Number of unit bins that cover the image diagonal: ceil(N*sqrt(2))."""
    return int(math.ceil(N * math.sqrt(2.0) - 1e-9))


def ellipse_phantom(N: int, rng: np.random.Generator, count: int = 6) -> np.ndarray:
    """Sum of `count` random ellipses on [-1,1]^2 (centre uniform in the disc of
    radius 0.6, semi-axes U[0.1,0.5], orientation U[0,pi), intensity U[0.2,1]).
    Returned as a length N*N vector, index iy*N + ix."""
    c = (np.arange(N) + 0.5) / N * 2.0 - 1.0
    X, Y = np.meshgrid(c, c)  # Y[iy, ix], X[iy, ix]
    img = np.zeros((N, N))
    for _ in range(count):
        r = 0.6 * math.sqrt(rng.uniform())
        phi = rng.uniform(0.0, 2.0 * math.pi)
        cx, cy = r * math.cos(phi), r * math.sin(phi)
        a, b = rng.uniform(0.1, 0.5), rng.uniform(0.1, 0.5)
        psi = rng.uniform(0.0, math.pi)
        val = rng.uniform(0.2, 1.0)
        xr = (X - cx) * math.cos(psi) + (Y - cy) * math.sin(psi)
        yr = -(X - cx) * math.sin(psi) + (Y - cy) * math.cos(psi)
        img[(xr / a) ** 2 + (yr / b) ** 2 <= 1.0] += val
    return img.reshape(-1)


def sparse_phantom(N: int, rng: np.random.Generator, frac: float = 0.05) -> np.ndarray:
    """`frac` of the pixels (uniform, without replacement) set to U[0,1], the rest 0."""
    n = N * N
    x = np.zeros(n)
    k = int(round(frac * n))
    idx = rng.choice(n, size=k, replace=False)
    x[idx] = rng.uniform(0.0, 1.0, size=k)
    return x


def add_noise(b_true: np.ndarray, level: float, rng: np.random.Generator) -> tuple:
    """b = b_true + e with ||e||_2 = level * ||b_true||_2 exactly (white Gaussian
    direction).  Returns (b, ||e||_2)."""
    g = rng.standard_normal(b_true.shape[0])
    e = level * np.linalg.norm(b_true) * g / np.linalg.norm(g)
    return b_true + e, float(np.linalg.norm(e))


def dense_csr(M: np.ndarray) -> CSR:
    """A dense matrix stored as CSR (every entry kept)."""
    m, n = M.shape
    rowptr = np.arange(0, (m + 1) * n, n, dtype=np.int64)
    colidx = np.tile(np.arange(n, dtype=np.int32), m)
    return CSR((m, n), rowptr, colidx, np.ascontiguousarray(M, dtype=np.float64).ravel())


def decaying(m: int, n: int, rho: float, seed: int, level: float) -> tuple:
    """The artificial problem of the paper's residual-size study: A = U diag(rho^(1-i)) V^T
    with seeded random orthogonal U (m x n) and V (n x n), x_true = ones, A scaled so
    that ||b_true|| = 1, and b = b_true + e with ||e|| = level.  Returns
    (A dense, b, b_true, ||e||)."""
    rng = np.random.default_rng(seed)
    U, _ = np.linalg.qr(rng.standard_normal((m, n)))
    V, _ = np.linalg.qr(rng.standard_normal((n, n)))
    sv = rho ** (1.0 - np.arange(1, n + 1))
    A = (U * sv) @ V.T
    A /= np.linalg.norm(A @ np.ones(n))
    b_true = A @ np.ones(n)
    b, en = add_noise(b_true, level, rng)
    return A, b, b_true, en


def blur_inpaint_operator(N: int, psf_var: float, keep: float, rng: np.random.Generator, radius: int = 2) -> CSR:
    """The deblurring-and-inpainting operator of the paper's motivating example
    (Section 1.2, timings in Section 4.1): a Gaussian point-spread function of
    variance psf_var on an N x N image (stencil of (2 radius + 1)^2 taps,
    weights summing to 1, zero outside the image), followed by subsampling that
    keeps a seeded `keep` fraction of the pixels (rows in increasing pixel
    order).  Rows: kept pixels; columns: pixels (index row * N + col)."""
    n = N * N
    m = int(round(keep * n))
    kept = np.sort(rng.choice(n, size=m, replace=False))
    off = np.arange(-radius, radius + 1)
    dy, dx = np.meshgrid(off, off, indexing="ij")
    w = np.exp(-(dy ** 2 + dx ** 2) / (2.0 * psf_var))
    w = (w / w.sum()).ravel()
    dy, dx = dy.ravel(), dx.ravel()
    iy, ix = kept // N, kept % N
    yy = iy[:, None] + dy[None, :]
    xx = ix[:, None] + dx[None, :]
    ok = (yy >= 0) & (yy < N) & (xx >= 0) & (xx < N)
    counts = ok.sum(axis=1)
    rowptr = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    cols = (yy * N + xx)[ok].astype(np.int32)
    vals = np.broadcast_to(w, ok.shape)[ok].astype(np.float64)
    return CSR((m, n), rowptr, cols, vals)


def blocks_phantom(N: int, rng: np.random.Generator, nblocks: int = 12) -> np.ndarray:
    """A synthetic stand-in for the paper's 'house' photograph (not available
    here): a smooth background plus `nblocks` axis-aligned rectangles of
    intensity U[0.2, 1] (numerically low rank, as the low-rank truncation
    assumes).  Values in [0, ~2]."""
    y, x = np.meshgrid(np.linspace(0, 1, N), np.linspace(0, 1, N), indexing="ij")
    img = 0.3 + 0.2 * x + 0.1 * y
    for _ in range(nblocks):
        y0, x0 = rng.integers(0, N - N // 8, size=2)
        h, wd = rng.integers(N // 16, N // 3, size=2)
        img[y0:y0 + h, x0:x0 + wd] += rng.uniform(0.2, 1.0)
    return img.ravel()


@dataclass
class Problem:
    """One synthetic CT problem: operator(s), phantoms, data and solver settings."""
    name: str
    N: int
    n_angles: int
    n_bins: int
    A: CSR
    B: CSR | None
    x_true: np.ndarray          # (n,) or (n, nrhs)
    b: np.ndarray               # (m,) or (m, nrhs)
    noise_norm: np.ndarray      # (nrhs,)
    settings: dict = field(default_factory=dict)


# Workload definitions: named by what they are (image size, geometry, method).
WORKLOADS = {
    # sFLSQR on a 64x64 image, 60 angles x 91 bins, 6 ellipses, 1% noise.
    "ct64_sflsqr": dict(N=64, n_angles=60, phantom="ellipses", nrhs=1, levels=(0.01,), data_seed=1,
                        unmatched=False,
                        settings=dict(method="sflsqr", s=200, zeta=8, window=2, maxit=100, eta=1.01,
                                      precond="identity", seed=42)),
    # sFLSMR with an unmatched pixel-driven back-projector, 256x256 image,
    # 180 angles x 363 bins, 5%-sparse phantom, 2% noise, reweighting preconditioner.
    "ct256_sflsmr_unmatched": dict(N=256, n_angles=180, phantom="sparse", nrhs=1, levels=(0.02,), data_seed=2,
                                   unmatched=True,
                                   settings=dict(method="sflsmr", s=400, zeta=8, window=2, maxit=200, eta=1.01,
                                                 precond="irw", irw_eps=1e-4, seed=43)),
    # sFLSQR at scale: 1024x1024, 360 angles x 1449 bins, 1% noise.
    "ct1024_sflsqr": dict(N=1024, n_angles=360, phantom="ellipses", nrhs=1, levels=(0.01,), data_seed=3,
                          unmatched=False,
                          settings=dict(method="sflsqr", s=600, zeta=8, window=4, maxit=300, eta=1.01,
                                        precond="identity", seed=44)),
    # 64 sinograms of 512x512 phantoms through one 360 x 725 operator,
    # noise levels log-uniform in [0.5%, 5%].
    "ct512_batch64": dict(N=512, n_angles=360, phantom="ellipses", nrhs=64, levels="loguniform", data_seed=4,
                          unmatched=False,
                          settings=dict(method="sflsqr", s=401, zeta=8, window=2, maxit=200, eta=1.01,
                                        precond="identity", seed=45)),
    # deblurring and inpainting with a rank-30 truncation: 512x512 image, Gaussian
    # PSF of variance 0.25, half of the pixels kept, 5% noise, 50 steps, CountSketch
    # with s = 101 (the timing experiment of Section 4.1).
    "deblur512_lowrank": dict(N=512, operator="blur", psf_var=0.25, keep=0.5, phantom="blocks", nrhs=1,
                              levels=(0.05,), data_seed=6, unmatched=False,
                              settings=dict(method="sflsqr", s=101, zeta=1, window=2, maxit=50, eta=1.01,
                                            precond="lowrank", rank=30, oversample=10, power=1, seed=48,
                                            omega_seed=49)),
    # fixed-k = 30 differentiable solves, 256x256, batch 16, diagonal weight.
    "ct256_diff16": dict(N=256, n_angles=180, phantom="ellipses", nrhs=16, levels=(0.01,), data_seed=5,
                         unmatched=False,
                         settings=dict(method="sflsqr", s=61, zeta=8, window=2, maxit=30, eta=1.01,
                                       precond="diag", seed=46, weight_seed=47)),
}


def make(name: str, nrhs: int | None = None, **over) -> Problem:
    """Build a named workload.  `nrhs` may shrink a batched workload; `over`
    may override N / n_angles (for reduced-size test cases of the same recipe)."""
    spec = dict(WORKLOADS[name])
    N = over.get("N", spec["N"])
    n_angles = over.get("n_angles", spec.get("n_angles", 0))
    n_bins = detector_bins(N)
    if spec.get("operator") == "blur":
        A = blur_inpaint_operator(N, spec["psf_var"], over.get("keep", spec["keep"]),
                                  np.random.default_rng(spec["data_seed"] + 1000))
        n_angles = n_bins = 0
    else:
        A = siddon_projector(N, n_angles, n_bins)
    B = pixel_backprojector(N, n_angles, n_bins) if spec["unmatched"] else None
    k = spec["nrhs"] if nrhs is None else nrhs
    xs, bs, enorms = [], [], []
    for j in range(k):
        rng = np.random.default_rng(spec["data_seed"] + j)
        x = {"ellipses": ellipse_phantom, "sparse": sparse_phantom, "blocks": blocks_phantom}[spec["phantom"]](N, rng)
        if spec["levels"] == "loguniform":
            level = float(math.exp(rng.uniform(math.log(0.005), math.log(0.05))))
        else:
            level = spec["levels"][0]
        b, en = add_noise(A.matvec(x), level, rng)
        xs.append(x); bs.append(b); enorms.append(en)
    settings = dict(spec["settings"])
    if settings.get("precond") == "diag":
        settings["weight"] = np.random.default_rng(settings["weight_seed"]).uniform(0.5, 1.5, size=N * N)
    if settings.get("precond") == "lowrank":   # Gaussian test matrix of the randomized SVD (N x (r + p))
        settings["omega"] = np.random.default_rng(settings["omega_seed"]).standard_normal(
            (N, settings["rank"] + settings["oversample"]))
    if k == 1:
        x_true, b = xs[0], bs[0]
    else:
        x_true, b = np.stack(xs, axis=1), np.stack(bs, axis=1)
    return Problem(name, N, n_angles, n_bins, A, B, x_true, b, np.array(enorms), settings)
