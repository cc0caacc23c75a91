"""Python binding of the GB300 sFLSQR / sFLSMR library.

Argument marshalling only: device memory comes from PyTorch tensors, streams
from torch.cuda.current_stream(); every step of the solvers runs in the CUDA
kernels of libsfl.so (Algorithms 1 and 2 of the paper).
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np
import torch

from . import _native as N


def _require_cuda():
    if not torch.cuda.is_available():
        raise RuntimeError("paper_2605_22281_gb300 needs a CUDA device (GB300, sm_103a); none is available")


def _ptr(t: torch.Tensor | None):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _dev_csr(rowptr, colidx, values, shape, device):
    """Device copies of a host or device CSR (int32 indices, FP64/FP32 values)."""
    rp = torch.as_tensor(np.asarray(rowptr) if not torch.is_tensor(rowptr) else rowptr).to(device=device, dtype=torch.int32)
    ci = torch.as_tensor(np.asarray(colidx) if not torch.is_tensor(colidx) else colidx).to(device=device, dtype=torch.int32)
    va = torch.as_tensor(np.asarray(values) if not torch.is_tensor(values) else values).to(device=device)
    if va.dtype == torch.float64:
        dt = N.SFL_F64
    elif va.dtype == torch.float32:
        dt = N.SFL_F32
    elif va.dtype == torch.bfloat16:
        dt = N.SFL_BF16
    else:
        va = va.to(torch.float64)
        dt = N.SFL_F64
    c = N.Csr(shape[0], shape[1], int(ci.numel()), _ptr(rp), _ptr(ci), _ptr(va), dt)
    return c, (rp, ci, va)


METHODS = {"sflsqr": 0, "sflsmr": 1, "flsqr": 2}


@dataclass
class SolveInfo:
    iters: int
    status: int
    relres: float
    tol: float

    @property
    def status_name(self) -> str:
        return {0: "running", 1: "discrepancy", 2: "maxit", 3: "breakdown"}.get(self.status, "?")


class Plan:
    """A sparse operator A (m x n, CSR) and its transposed copy, or an unmatched
    back-projector B (n x m), stored on the GPU in `value_dtype`.  image_shape
    (rows, cols) with rows * cols = n declares the n-side an image (column
    index row * cols + col): the plan then stores the rows of A^T / B in pixel
    tiles (same products bit for bit, better cache reuse).  slot_layout:
    'interleaved' (single solves) or 'operator' (batched solves) entry order
    inside each row's chunk slots.  index_bits: 0 lets the single-solve
    products read 16-bit column deltas where the operator allows it (same
    products bit for bit, 2 bytes less per entry); 32 keeps 32-bit indices."""

    def __init__(self, A, B=None, value_dtype: str = "f64", device: str | int = 0, max_device_bytes: int = 0,
                 lanes_per_row: int = 0, image_shape: tuple | None = None, slot_layout: str = "interleaved",
                 index_bits: int = 0):
        _require_cuda()
        self.lib = N.load()
        self.device = torch.device("cuda", device) if isinstance(device, int) else torch.device(device)
        with torch.cuda.device(self.device):
            ca, keep_a = _dev_csr(A.rowptr, A.colidx, A.values, A.shape, self.device)
            cb, keep_b = (None, None)
            if B is not None:
                cb, keep_b = _dev_csr(B.rowptr, B.colidx, B.values, B.shape, self.device)
            ir, ic = (int(image_shape[0]), int(image_shape[1])) if image_shape is not None else (0, 0)
            if slot_layout not in ("interleaved", "operator"):
                raise ValueError(slot_layout)
            if index_bits not in (0, 32):
                raise ValueError(f"index_bits {index_bits!r}: 0 (16-bit deltas where they fit) or 32")
            po = N.PlanOpts(N.DTYPE[value_dtype], lanes_per_row, max_device_bytes, ir, ic,
                            0 if slot_layout == "interleaved" else 1, index_bits)
            h = ctypes.c_void_p()
            st = N.check(self.lib.sfl_plan_create(ctypes.byref(h), ctypes.byref(ca),
                                                  ctypes.byref(cb) if cb is not None else None,
                                                  ctypes.byref(po), _stream()), "sfl_plan_create")
            del keep_a, keep_b, st
        self.handle = h
        self.m, self.n = int(A.shape[0]), int(A.shape[1])
        self.value_dtype = value_dtype

    @classmethod
    def ct(cls, image_n: int, n_angles: int, n_bins: int, back: str = "matched", value_dtype: str = "f64",
           device: str | int = 0, max_device_bytes: int = 0):
        """A matrix-free plan for the parallel-beam CT geometry (image_n^2 pixels,
        n_angles x n_bins rays): A z by Siddon's ray walk and, for back =
        'matched', A^T w pixel-driven with exact chords, or for back =
        'unmatched' the pixel-driven linear-interpolation back-projector.  The
        products are computed on the fly in FP64 (value_dtype 'f64') or FP32."""
        _require_cuda()
        self = cls.__new__(cls)
        self.lib = N.load()
        self.device = torch.device("cuda", device) if isinstance(device, int) else torch.device(device)
        if back not in ("matched", "unmatched"):
            raise ValueError(back)
        g = N.CtGeometry(image_n, n_angles, n_bins, 0 if back == "matched" else 1, None)
        po = N.PlanOpts(N.DTYPE[value_dtype], 0, max_device_bytes, 0, 0, 0, 0)
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            N.check(self.lib.sfl_plan_create_ct(ctypes.byref(h), ctypes.byref(g), ctypes.byref(po), _stream()),
                    "sfl_plan_create_ct")
        self.handle = h
        self.m, self.n = n_angles * n_bins, image_n * image_n
        self.value_dtype = "f64" if value_dtype == "f64" else "f32"
        return self

    def close(self):
        if getattr(self, "handle", None):
            self.lib.sfl_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def stats(self) -> dict:
        s = N.PlanStats()
        N.check(self.lib.sfl_plan_get_stats(self.handle, ctypes.byref(s)), "sfl_plan_get_stats")
        return {f: getattr(s, f) for f, _ in N.PlanStats._fields_}

    def apply(self, x: torch.Tensor, transpose: bool = False) -> torch.Tensor:
        """y = A x, or y = A^T x (B x when the plan holds an unmatched B)."""
        x = x.to(device=self.device, dtype=torch.float64).contiguous()
        y = torch.empty(self.n if transpose else self.m, dtype=torch.float64, device=self.device)
        N.check(self.lib.sfl_plan_apply(self.handle, 1 if transpose else 0, _ptr(x), _ptr(y), _stream()),
                "sfl_plan_apply")
        return y

    def _opts(self, s, zeta, seed, window, maxit, noise_norm, eta, precond, stop_rule, diag_w, irw_eps,
              vec_dtype, x_hist, r_hist, orth_against="p", sk=None, sk_stop=None, lowrank=(0, 0, 0, None, 0),
              sketch_apply="auto", sketch_kind="sparse_sign"):
        if orth_against not in ("p", "z"):
            raise ValueError(orth_against)
        if sketch_apply not in N.SKETCH_APPLY:
            raise ValueError(f"sketch_apply {sketch_apply!r}: one of {sorted(N.SKETCH_APPLY)}")
        if sketch_kind not in N.SKETCH_KIND:
            raise ValueError(f"sketch_kind {sketch_kind!r}: one of {sorted(N.SKETCH_KIND)}")
        return N.Opts(s, zeta, seed, window, maxit, float(noise_norm), float(eta), N.PRECOND[precond],
                      N.STOP_RULE[stop_rule], _ptr(diag_w), float(irw_eps), N.DTYPE[vec_dtype], 0,
                      _ptr(x_hist), _ptr(r_hist), 1 if orth_against == "z" else 0, _ptr(sk), _ptr(sk_stop),
                      int(lowrank[0]), int(lowrank[1]), int(lowrank[2]), _ptr(lowrank[3]), int(lowrank[4]),
                      N.SKETCH_APPLY[sketch_apply], N.SKETCH_KIND[sketch_kind])

    def _lowrank(self, precond, rank, oversample, power, omega, fp64=False):
        """(rank, oversample, power, Omega) of the low-rank operator, Omega as a
        contiguous FP64 device tensor (image_cols x (rank + oversample))."""
        if precond != "lowrank":
            return (0, 0, 0, None, 0)
        if omega is None:
            raise ValueError("precond='lowrank' needs lowrank_omega (image_cols x (rank + oversample))")
        om = omega.to(device=self.device, dtype=torch.float64).contiguous()
        if om.dim() != 2 or om.shape[1] != rank + oversample:
            raise ValueError(f"lowrank_omega of shape {tuple(om.shape)}, expected (image_cols, {rank + oversample})")
        return (rank, oversample, power, om, 1 if fp64 else 0)

    def _dense_sketch(self, S, rows, cols):
        if S is None:
            return None
        S = S.to(device=self.device, dtype=torch.float64).contiguous()
        if tuple(S.shape) != (rows, cols):
            raise ValueError(f"sketch matrix of shape {tuple(S.shape)}, expected {(rows, cols)}")
        return S

    def solve(self, method: str, b: torch.Tensor, *, s: int, zeta: int = 8, seed: int = 0, window: int = 2,
              maxit: int = 100, noise_norm: float = 0.0, eta: float = 1.01, precond: str = "identity",
              stop_rule: str = "residual", diag_w: torch.Tensor | None = None, irw_eps: float = 1e-4,
              vec_dtype: str | None = None, x_history: bool = False, relres_history: bool = False,
              driver: str = "graph", out: torch.Tensor | None = None, sync: bool = True,
              orth_against: str = "p", sketch_matrix: torch.Tensor | None = None,
              sketch_matrix_stop: torch.Tensor | None = None, lowrank_rank: int = 30, lowrank_oversample: int = 10,
              lowrank_power: int = 1, lowrank_omega: torch.Tensor | None = None, lowrank_fp64: bool = False,
              sketch_apply: str = "auto", sketch_kind: str = "sparse_sign"):
        """Run sFLSQR (method='sflsqr', Algorithm 1), sFLSMR ('sflsmr', Algorithm
        2) or the unsketched FLSQR ('flsqr', eq. (FLSQR); needs window < 0).
        window < 0: full orthogonalization (block CGS2 against every earlier
        vector).

        orth_against: 'p' orthogonalizes the new z against the window's unit
        p_j (eq. (FGK)), 'z' against the stored z_j as the algorithms' loop is
        printed.  sketch_matrix: an explicit s x m (sFLSQR) or s x n (sFLSMR)
        sketch used instead of the sparse-sign one, with sketch_matrix_stop the
        s x m stop sketch of sFLSMR (kept alive by the caller until the solve
        has run when sync=False).  precond='lowrank': z = the rank-r randomized-SVD
        truncation of p reshaped to the plan's image (lowrank_rank r,
        lowrank_oversample p, lowrank_power q subspace-iteration steps, and the
        Gaussian test matrix lowrank_omega, image_cols x (r + p); FP32
        arithmetic, or FP64 with lowrank_fp64).  sketch_apply: 'fused' (the
        sketch is added in the products' epilogues, S drawn from the hash),
        'kernel' (a separate gather kernel over a table of S) or 'auto'
        (fused for long operator rows; see sfl_opts.sketch_apply).  sketch_kind:
        'sparse_sign' (default), 'srht' (subsampled randomized Hadamard
        transform) or 'gaussian' (N(0, 1/s) entries), all regenerated from
        the seed (see sfl_opts.sketch_kind).
        Returns (x, info, hist) where hist holds the
        optional per-step iterates (maxit x n) and stop ratios.  With sync=False
        the call does not wait and info is None."""
        if vec_dtype is None:
            vec_dtype = "f64" if self.value_dtype == "f64" else "f32"
        dev = self.device
        b = b.to(device=dev, dtype=torch.float64).contiguous()
        x = out if out is not None else torch.empty(self.n, dtype=torch.float64, device=dev)
        dw = diag_w.to(device=dev, dtype=torch.float64).contiguous() if diag_w is not None else None
        xh = torch.zeros((maxit, self.n), dtype=torch.float64, device=dev) if x_history else None
        rh = torch.zeros(maxit, dtype=torch.float64, device=dev) if relres_history else None
        sk = self._dense_sketch(sketch_matrix, s, self.m if method == "sflsqr" else self.n)
        sks = self._dense_sketch(sketch_matrix_stop, s, self.m)
        lr = self._lowrank(precond, lowrank_rank, lowrank_oversample, lowrank_power, lowrank_omega, lowrank_fp64)
        o = self._opts(s, zeta, seed, window, maxit, noise_norm, eta, precond, stop_rule, dw, irw_eps, vec_dtype,
                       xh, rh, orth_against, sk, sks, lr, sketch_apply, sketch_kind)
        info = N.Info()
        pinfo = ctypes.byref(info) if sync else None
        with torch.cuda.device(dev):
            mid = METHODS[method]
            if driver == "graph":
                fn = (self.lib.sflsqr_solve, self.lib.sflsmr_solve, self.lib.flsqr_solve)[mid]
                st = fn(self.handle, _ptr(b), ctypes.byref(o), _ptr(x), pinfo, _stream())
            elif driver == "profiled":
                kt = N.KernelTimes()
                st = self.lib.sfl_solve_profiled(self.handle, mid, _ptr(b), ctypes.byref(o),
                                                 _ptr(x), pinfo, ctypes.byref(kt), _stream())
            elif driver == "host_loop":
                st = self.lib.sfl_solve_host_loop(self.handle, mid, _ptr(b),
                                                  ctypes.byref(o), _ptr(x), pinfo, _stream())
            else:
                raise ValueError(driver)
        N.check(st, method)
        hist = {"x": xh, "relres": rh}
        if driver == "profiled":
            hist["kernel_ms"] = {c: kt.ms[i] for i, c in enumerate(N.KERNEL_CLASSES)}
            hist["kernel_launches"] = {c: kt.launches[i] for i, c in enumerate(N.KERNEL_CLASSES)}
        return x, (SolveInfo(info.iters, info.status, info.relres, info.tol) if sync else None), hist

    def solve_host(self, method: str, b: np.ndarray, *, s: int, zeta: int = 8, seed: int = 0, window: int = 2,
                   maxit: int = 100, noise_norm: float = 0.0, eta: float = 1.01, precond: str = "identity",
                   stop_rule: str = "residual", diag_w: torch.Tensor | None = None, irw_eps: float = 1e-4,
                   vec_dtype: str | None = None, x_out: np.ndarray | None = None, orth_against: str = "p",
                   sketch_apply: str = "auto"):
        """Same solve with host FP64 b and x (copies inside the call)."""
        if vec_dtype is None:
            vec_dtype = "f64" if self.value_dtype == "f64" else "f32"
        b = np.ascontiguousarray(b, dtype=np.float64)
        x = x_out if x_out is not None else np.empty(self.n, dtype=np.float64)
        dw = diag_w.to(device=self.device, dtype=torch.float64).contiguous() if diag_w is not None else None
        o = self._opts(s, zeta, seed, window, maxit, noise_norm, eta, precond, stop_rule, dw, irw_eps, vec_dtype,
                       None, None, orth_against, sketch_apply=sketch_apply)
        info = N.Info()
        fn = (self.lib.sflsqr_solve_host, self.lib.sflsmr_solve_host, self.lib.flsqr_solve_host)[METHODS[method]]
        with torch.cuda.device(self.device):
            st = fn(self.handle, b.ctypes.data_as(ctypes.c_void_p), ctypes.byref(o), x.ctypes.data_as(ctypes.c_void_p),
                    ctypes.byref(info), _stream())
        N.check(st, method + "_host")
        return x, SolveInfo(info.iters, info.status, info.relres, info.tol)


def _batched_opts(plan, s, zeta, seed, window, maxit, eta, precond, diag_w, spmm_tile=0, x_hist=None):
    dw = diag_w.to(device=plan.device, dtype=torch.float64).contiguous() if diag_w is not None else None
    vec = "f64" if plan.value_dtype == "f64" else "f32"
    o = plan._opts(s, zeta, seed, window, maxit, 0.0, eta, precond, "residual", dw, 0.0, vec, x_hist, None)
    o.spmm_tile = int(spmm_tile)
    return o, dw


def solve_batched(plan: Plan, B: torch.Tensor, noise_norms, *, s: int, zeta: int = 8, seed: int = 0, window: int = 2,
                  maxit: int = 100, eta: float = 1.01, precond: str = "identity", diag_w: torch.Tensor | None = None,
                  spmm_tile: int = 0, out: torch.Tensor | None = None, sync: bool = True,
                  x_history: bool = False):
    """Batched sFLSQR: B is (nrhs, m) (row r = b_r), noise_norms has nrhs entries.
    spmm_tile: RHS per CTA column of the SpMMs (8/16/32/64) or 0 = tuned.
    x_history: also return every right-hand side's iterate after every step,
    a (maxit, nrhs, n) tensor whose [k - 1, r] row is x_k of column r for
    k <= its stop step (zeros after it).
    Returns (X (nrhs, n), [SolveInfo per RHS] or None when sync=False), plus
    the history as a third item when x_history is set."""
    dev = plan.device
    B = B.to(device=dev, dtype=torch.float64).contiguous()
    R = int(B.shape[0])
    X = out if out is not None else torch.empty((R, plan.n), dtype=torch.float64, device=dev)
    noise = np.ascontiguousarray(np.broadcast_to(np.asarray(noise_norms, dtype=np.float64), (R,)))
    xh = torch.zeros((maxit, R, plan.n), dtype=torch.float64, device=dev) if x_history else None
    o, dw = _batched_opts(plan, s, zeta, seed, window, maxit, eta, precond, diag_w, spmm_tile, xh)
    infos = (N.Info * R)() if sync else None
    with torch.cuda.device(dev):
        st = plan.lib.sflsqr_solve_batched(plan.handle, R, _ptr(B), noise.ctypes.data_as(ctypes.c_void_p),
                                           ctypes.byref(o), _ptr(X), infos, _stream())
    N.check(st, "sflsqr_solve_batched")
    del dw
    infos = [SolveInfo(i.iters, i.status, i.relres, i.tol) for i in infos] if sync else None
    return (X, infos, xh) if x_history else (X, infos)


def batched_tiles(plan: Plan):
    """(A tile, A^T/B tile) the SpMM tuner picked for the last batch session."""
    return plan.lib.sfl_batched_tile(plan.handle, 0), plan.lib.sfl_batched_tile(plan.handle, 1)


def fixed_batched(plan: Plan, B: torch.Tensor, d: torch.Tensor | None = None, *, s: int, zeta: int = 8, seed: int = 0,
                  window: int = 2, maxit: int = 30, out: torch.Tensor | None = None):
    """Fixed-k batched sFLSQR (exactly maxit steps, no stop test) with
    tau = diag(d) (identity when d is None).  B: (nrhs, m).  Returns
    (X (nrhs, n), infos, forward id); the plan keeps the state for `adjoint`."""
    dev = plan.device
    B = B.detach().to(device=dev, dtype=torch.float64).contiguous()
    R = int(B.shape[0])
    X = out if out is not None else torch.empty((R, plan.n), dtype=torch.float64, device=dev)
    o, dw = _batched_opts(plan, s, zeta, seed, window, maxit, 1.01, "diag" if d is not None else "identity",
                          d.detach() if d is not None else None)
    infos = (N.Info * R)()
    with torch.cuda.device(dev):
        st = plan.lib.sflsqr_fixed_batched(plan.handle, R, _ptr(B), ctypes.byref(o), _ptr(X), infos, _stream())
    N.check(st, "sflsqr_fixed_batched")
    del dw
    return X, [SolveInfo(i.iters, i.status, i.relres, i.tol) for i in infos], plan.lib.sfl_fixed_calls(plan.handle)


def adjoint(plan: Plan, Xbar: torch.Tensor, want_d: bool = True):
    """Adjoint of the plan's latest fixed_batched call: (Bbar (nrhs, m), dbar (n) or None)."""
    dev = plan.device
    Xbar = Xbar.detach().to(device=dev, dtype=torch.float64).contiguous()
    R = int(Xbar.shape[0])
    Bbar = torch.empty((R, plan.m), dtype=torch.float64, device=dev)
    dbar = torch.empty(plan.n, dtype=torch.float64, device=dev) if want_d else None
    with torch.cuda.device(dev):
        st = plan.lib.sflsqr_adjoint_batched(plan.handle, R, _ptr(Xbar), _ptr(Bbar), _ptr(dbar), _stream())
    N.check(st, "sflsqr_adjoint_batched")
    return Bbar, dbar


class FixedKSolve(torch.autograd.Function):
    """X = sFLSQR_k(B, d) on the GPU, differentiable in B and d through the
    hand-written adjoint (the forward state, every basis vector included, is
    kept by the plan between forward and backward)."""

    @staticmethod
    def forward(ctx, plan, B, d, kw):
        X, infos, fid = fixed_batched(plan, B, d, **kw)
        ctx.plan, ctx.fid, ctx.has_d = plan, fid, d is not None
        ctx.infos = infos
        return X

    @staticmethod
    def backward(ctx, Xbar):
        plan = ctx.plan
        if plan.lib.sfl_fixed_calls(plan.handle) != ctx.fid:
            raise RuntimeError("the plan ran another fixed-k forward since this one; its state is gone")
        Bbar, dbar = adjoint(plan, Xbar, want_d=ctx.has_d and ctx.needs_input_grad[2])
        return None, Bbar if ctx.needs_input_grad[1] else None, dbar, None


def sflsqr_fixed_k(plan: Plan, B: torch.Tensor, d: torch.Tensor | None = None, **kw) -> torch.Tensor:
    """Differentiable fixed-k batched sFLSQR (see FixedKSolve); kw as fixed_batched."""
    return FixedKSolve.apply(plan, B, d, kw)


def sflsqr(plan: Plan, b, **kw):
    """Algorithm 1 (sFLSQR) on the GPU; see Plan.solve."""
    return plan.solve("sflsqr", b, **kw)


def sflsmr(plan: Plan, b, **kw):
    """Algorithm 2 (sFLSMR) on the GPU; see Plan.solve."""
    return plan.solve("sflsmr", b, **kw)


def sketch_export(seed: int, s: int, zeta: int, ncols: int, device=0):
    """(rows, signs) of the sparse-sign sketch the solvers draw, as int32 tensors (ncols, zeta)."""
    _require_cuda()
    lib = N.load()
    dev = torch.device("cuda", device) if isinstance(device, int) else torch.device(device)
    rows = torch.empty((ncols, zeta), dtype=torch.int32, device=dev)
    signs = torch.empty((ncols, zeta), dtype=torch.int32, device=dev)
    with torch.cuda.device(dev):
        N.check(lib.sfl_sketch_export(seed, s, zeta, ncols, _ptr(rows), _ptr(signs), _stream()), "sfl_sketch_export")
    return rows, signs


def sketch_apply(seed: int, s: int, zeta: int, v: torch.Tensor) -> torch.Tensor:
    """S v for the sparse-sign sketch (seed, s, zeta)."""
    _require_cuda()
    lib = N.load()
    v = v.to(dtype=torch.float64).contiguous()
    out = torch.empty(s, dtype=torch.float64, device=v.device)
    with torch.cuda.device(v.device):
        N.check(lib.sfl_sketch_apply(seed, s, zeta, _ptr(v), v.numel(), _ptr(out), _stream()), "sfl_sketch_apply")
    return out


def check_noalloc_args(s: int, v, out) -> None:
    """Argument checks of sketch_apply_noalloc, made before anything is
    launched: v must be a contiguous CUDA float64 vector, and out, when given,
    a contiguous CUDA float64 tensor on v's device with at least s elements
    (the kernel writes s doubles through its pointer).  Raises ValueError."""
    if not getattr(v, "is_cuda", False) or v.dtype != torch.float64 or not v.is_contiguous() or v.dim() != 1:
        raise ValueError("v must be a contiguous 1-D CUDA float64 tensor")
    if out is not None:
        if not getattr(out, "is_cuda", False) or out.dtype != torch.float64 or not out.is_contiguous():
            raise ValueError("out must be a contiguous CUDA float64 tensor")
        if out.device != v.device:
            raise ValueError(f"out is on {out.device}, v on {v.device}")
        if out.numel() < s:
            raise ValueError(f"out holds {out.numel()} elements, the sketch has s = {s} rows")


def sketch_apply_noalloc(seed: int, s: int, zeta: int, v: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
    """S v through the allocation-free entry point (s <= 1024), for callers
    that may not allocate device memory.  v must already be a contiguous CUDA
    float64 vector (no conversion is made).  The C entry point allocates
    nothing; this wrapper allocates only when `out` is omitted (the result
    tensor, through PyTorch's caching allocator), so pass a preallocated out
    for a call that allocates nothing at all."""
    check_noalloc_args(s, v, out)
    _require_cuda()
    lib = N.load()
    if out is None:
        out = torch.empty(s, dtype=torch.float64, device=v.device)
    with torch.cuda.device(v.device):
        N.check(lib.sfl_sketch_apply_noalloc(seed, s, zeta, _ptr(v), v.numel(), _ptr(out), _stream()),
                "sfl_sketch_apply_noalloc")
    return out
