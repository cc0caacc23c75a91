"""Planted-mistake checks: each test loads a copy of the oracle with one
plausible mistake written into its source (a dropped term, a wrong sign or
index, a transposed operand) and checks that the pins reject it.  The copy is
built on the CPU; the real oracle is never modified."""
import importlib.util
import os
import sys
import types

import numpy as np
import pytest
import scipy.sparse.linalg as spla

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = open(os.path.join(ROOT, "oracle", "sfl.py")).read()


def load_variant(src: str):
    """Import the oracle package with sfl.py replaced by `src`."""
    name = f"oracle_variant_{abs(hash(src))}"
    pkg = types.ModuleType(name)
    pkg.__path__ = [os.path.join(ROOT, "oracle")]
    sys.modules[name] = pkg
    spec = importlib.util.spec_from_file_location(f"{name}.sketch", os.path.join(ROOT, "oracle", "sketch.py"))
    sk = importlib.util.module_from_spec(spec)
    sys.modules[f"{name}.sketch"] = sk
    spec.loader.exec_module(sk)
    mod = types.ModuleType(f"{name}.sfl")
    mod.__package__ = name
    sys.modules[f"{name}.sfl"] = mod
    exec(compile(src, f"<{name}>", "exec"), mod.__dict__)
    return mod, sk


def pins_pass(sfl, sk) -> bool:
    """A compact run of the main pins; True when all of them hold."""
    rng = np.random.default_rng(10)
    U, _ = np.linalg.qr(rng.standard_normal((40, 25)))
    V, _ = np.linalg.qr(rng.standard_normal((25, 25)))
    A = (U * np.linspace(2, 0.3, 25)) @ V.T
    b = rng.standard_normal(40)
    ok = True
    # LSQR / LSMR special cases
    r = sfl.sflsqr(A, b, sk.IdentitySketch(40), maxit=6, ell=-1)
    x = spla.lsqr(A, b, atol=0, btol=0, conlim=0, iter_lim=6)[0]
    ok &= np.linalg.norm(r.x - x) <= 1e-8 * np.linalg.norm(x)
    r = sfl.sflsmr(A, b, sk.IdentitySketch(25), S_stop=sk.IdentitySketch(40), maxit=6, ell=-1)
    x = spla.lsmr(A, b, atol=0, btol=0, conlim=0, maxiter=6)[0]
    ok &= np.linalg.norm(r.x - x) <= 1e-8 * np.linalg.norm(x)
    # full space with window 2 and each flexible operator: dense sketched LS
    m, n = 12, 8
    A2 = rng.standard_normal((m, n))
    b2 = rng.standard_normal(m)
    S = sk.DenseSketch(rng.standard_normal((10, m)))
    Sn = sk.DenseSketch(rng.standard_normal((9, n)))
    for tau in (sfl.Identity(), sfl.FixedDiag(rng.uniform(0.5, 2, n)), sfl.Reweighting(1e-2)):
        r = sfl.sflsqr(A2, b2, S, maxit=n, ell=2, tau=tau)
        xr = np.linalg.lstsq(S.S @ A2, S.S @ b2, rcond=None)[0]
        ok &= r.iters == n and np.linalg.norm(r.x - xr) <= 1e-9 * np.linalg.norm(xr)
        r = sfl.sflsmr(A2, b2, Sn, S_stop=sk.IdentitySketch(m), maxit=n, ell=2, tau=tau)
        xr = np.linalg.lstsq(Sn.S @ A2.T @ A2, Sn.S @ A2.T @ b2, rcond=None)[0]
        ok &= r.iters == n and np.linalg.norm(r.x - xr) <= 1e-9 * np.linalg.norm(xr)
    # FGK relation and band with window 2
    S3 = sk.SparseSign(1, 31, 8, 40)
    r = sfl.sflsqr(A, b, S3, maxit=15, ell=2, tau=sfl.FixedDiag(rng.uniform(0.5, 1.5, 25)))
    ok &= np.linalg.norm(A @ r.Z - r.W @ r.H) <= 1e-13 * np.linalg.norm(A @ r.Z)
    k = r.Z.shape[1]
    ok &= all(r.H[i, j] == 0 for j in range(k) for i in range(k + 1) if not (j - 2 <= i <= j + 1))
    ATW = A.T @ r.W[:, :k]
    ok &= np.linalg.norm(ATW - r.P @ r.T) <= 1e-13 * np.linalg.norm(ATW)
    # window orthogonality: w_{k+1} against w_{k-2..k}, p_k against p_{k-2..k-1}
    ok &= all(abs(r.W[:, i] @ r.W[:, j]) <= 1e-13 for i in range(r.W.shape[1]) for j in range(max(0, i - 3), i))
    ok &= all(abs(r.P[:, i] @ r.P[:, j]) <= 1e-13 for i in range(k) for j in range(max(0, i - 2), i))
    # reweighting operator at step 2 (closed form of x_1)
    eps = 3e-3
    r = sfl.sflsqr(A, b, S3, maxit=3, ell=2, tau=sfl.Reweighting(eps))
    p1 = A.T @ b / np.linalg.norm(A.T @ b)
    z1 = eps ** 0.25 * p1
    c = S3.apply(A @ z1)
    x1 = (c @ S3.apply(b)) / (c @ c) * z1
    ok &= np.allclose(r.Z[:, 1] / r.P[:, 1], (x1 ** 2 + eps) ** 0.25, rtol=1e-12, atol=0)
    return bool(ok)


MUTATIONS = {
    "w_window_drops_last": ("for j in _window(k, ell, k):", "for j in _window(k, ell, k - 1):"),
    "mgs_sign": ("z = z - c * V[j - 1]", "z = z + c * V[j - 1]"),
    "window_off_by_one": ("lo = 1 if ell < 0 else max(1, k - ell)", "lo = 1 if ell < 0 else max(1, k - ell + 1)"),
    "sflsmr_drops_beta": ("s_Atb = beta0 * S_ls.apply(z)", "s_Atb = S_ls.apply(z)"),
    "sflsmr_drops_new_column": ("Mk = np.column_stack(SAtW + [Sz]) @ Hmat[:k + 1, :k]",
                                "Mk = np.column_stack(SAtW) @ Hmat[:k, :k]"),
    "reweight_exponent": ("np.power(x_prev * x_prev + self.eps, 0.25)", "np.power(x_prev * x_prev + self.eps, 0.5)"),
    "backsub_transposed": ("y[i] = (g[i] - R[i, i + 1:k] @ y[i + 1:]) / R[i, i]",
                           "y[i] = (g[i] - R[i + 1:k, i] @ y[i + 1:]) / R[i, i]"),
    "reflector_rhs_skipped": ("g[j:] -= beta * v * (v @ g[j:])", "pass"),
    "transposed_operator": ("rmatvec = (lambda v: A.T @ v) if AT is None", "rmatvec = (lambda v: (A @ A.T @ A).T @ v) if AT is None"),
    "h_not_recorded": ("Hmat[j - 1, k - 1] = h", "Hmat[j - 1, k - 1] = 0.0"),
}


def test_unmodified_oracle_passes_compact_pins():
    sfl, sk = load_variant(SRC)
    assert pins_pass(sfl, sk)


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(name):
    old, new = MUTATIONS[name]
    assert old in SRC, f"mutation anchor for {name} not found"
    sfl, sk = load_variant(SRC.replace(old, new, 1))
    with np.errstate(all="ignore"):
        try:
            caught = not pins_pass(sfl, sk)
        except Exception:
            caught = True
    assert caught, f"planted mistake {name} passed the pins"
