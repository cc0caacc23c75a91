"""Pins of the oracle's low-rank truncation operators (Section 1.2; the -RND
variants of Section 4.1) against closed forms and published bounds:

* a matrix built from a known SVD, U diag(sigma) V^T: the rank-r truncation is
  U_r diag(sigma_r) V_r^T, and its error is the Eckart-Young value
  sqrt(sum_{i>r} sigma_i^2) (Frobenius) and sigma_{r+1} (spectral);
* a rank-r input is returned unchanged; the operator is positively homogeneous
  and idempotent; row-major and column-stacking vectorisations give the same map;
* the randomized SVD is exact when rank(C) <= r + p (Gaussian test matrix);
  with many subspace-iteration steps it reaches the truncated SVD on a matrix
  with a spectral gap; it never beats the truncated SVD (Eckart-Young); and the
  mean range-finder error over Gaussian draws stays below the bound of Halko,
  Martinsson and Tropp (2011), eq. (1.9) (q = 0);
* planted mistakes in the truncation are rejected by these pins.
"""
import os
import types

import numpy as np

import oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def known_svd(m, n, sig, seed):
    rng = np.random.default_rng(seed)
    U, _ = np.linalg.qr(rng.standard_normal((m, len(sig))))
    V, _ = np.linalg.qr(rng.standard_normal((n, len(sig))))
    return U, np.asarray(sig, dtype=float), V, (U * sig) @ V.T


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_truncation_is_the_known_leading_terms():
    sig = np.geomspace(10.0, 0.01, 20)
    U, s, V, C = known_svd(30, 24, sig, 1)
    for r in (1, 5, 13):
        want = (U[:, :r] * s[:r]) @ V[:, :r].T
        got = O.truncated_svd(C, r)
        assert rel(got, want) <= 1e-12
        assert abs(np.linalg.norm(C - got) - np.sqrt(np.sum(s[r:] ** 2))) <= 1e-12 * np.linalg.norm(C)
        assert abs(np.linalg.norm(C - got, 2) - s[r]) <= 1e-12 * s[0]


def test_operator_properties():
    rng = np.random.default_rng(2)
    C = rng.standard_normal((16, 12))
    tau = O.LowRank(4, (16, 12))
    p = C.ravel()
    z = tau(p, None)
    assert np.linalg.matrix_rank(z.reshape(16, 12), tol=1e-10) == 4
    assert rel(tau(3.5 * p, None), 3.5 * z) <= 1e-13              # positively homogeneous
    assert rel(tau(z, None), z) <= 1e-12                           # idempotent
    # the column-stacking vectorisation of the paper gives the same map
    z_col = O.truncated_svd(C.T, 4).T.ravel()
    assert rel(z, z_col) <= 1e-12
    _, _, _, L = known_svd(16, 12, [3.0, 2.0, 1.0, 0.5], 3)        # rank 4: unchanged
    assert rel(tau(L.ravel(), None), L.ravel()) <= 1e-12


def test_randomized_svd_is_exact_below_its_sample_size():
    sig = np.array([9.0, 7.0, 5.0, 4.0, 3.0, 2.5, 2.0, 1.5, 1.0, 0.8, 0.5, 0.3])
    U, s, V, C = known_svd(40, 36, sig, 4)                          # rank 12 <= r + p
    Omega = np.random.default_rng(5).standard_normal((36, 14))
    for q in (0, 1, 2):
        got = O.randomized_svd_truncation(C, 6, Omega, q)
        assert rel(got, (U[:, :6] * s[:6]) @ V[:, :6].T) <= 1e-10


def test_randomized_svd_converges_to_the_truncation_with_subspace_iteration():
    sig = np.concatenate([np.geomspace(10.0, 5.0, 8), np.geomspace(0.5, 1e-3, 30)])   # gap after 8
    U, s, V, C = known_svd(60, 50, sig, 6)
    Omega = np.random.default_rng(7).standard_normal((50, 12))
    got = O.randomized_svd_truncation(C, 8, Omega, q=8)
    assert rel(got, (U[:, :8] * s[:8]) @ V[:, :8].T) <= 1e-10


def test_randomized_svd_obeys_eckart_young_and_the_hmt_bound():
    sig = np.geomspace(1.0, 1e-4, 60)
    U, s, V, C = known_svd(80, 70, sig, 8)
    r, p = 10, 6
    best_f = np.sqrt(np.sum(s[r:] ** 2))
    errs = []
    for t in range(200):
        Omega = np.random.default_rng(100 + t).standard_normal((70, r + p))
        Cr = O.randomized_svd_truncation(C, r, Omega, q=0)
        assert np.linalg.matrix_rank(Cr, tol=1e-12) <= r
        assert np.linalg.norm(C - Cr) >= best_f * (1 - 1e-12)          # no rank-r matrix beats the TSVD
        assert np.linalg.norm(C - Cr, 2) >= s[r] * (1 - 1e-12)
        Q, _ = np.linalg.qr(C @ Omega)                                   # range finder, rank r + p
        errs.append(np.linalg.norm(C - Q @ (Q.T @ C), 2))
    bound = (1 + 4 * np.sqrt(r + p) / (p - 1) * np.sqrt(min(C.shape))) * s[r]
    assert np.mean(errs) <= bound
    assert np.mean(errs) >= s[r + p] * (1 - 1e-12)                     # a rank-(r+p) projection


def _variant(old, new):
    src = open(os.path.join(ROOT, "oracle", "lowrank.py")).read()
    assert src.count(old) >= 1
    mod = types.ModuleType("lowrank_variant")
    mod.__dict__["Precond"] = O.sfl.Precond
    src = src.replace("from .sfl import Precond\n", "").replace(old, new)
    exec(compile(src, "<lowrank_variant>", "exec"), mod.__dict__)
    return mod


def _pins_pass(mod) -> bool:
    sig = np.geomspace(10.0, 0.01, 20)
    U, s, V, C = known_svd(30, 24, sig, 1)
    ok = rel(mod.truncated_svd(C, 5), (U[:, :5] * s[:5]) @ V[:, :5].T) <= 1e-12
    sig2 = np.array([9.0, 7.0, 5.0, 4.0, 3.0, 2.5, 2.0, 1.5, 1.0, 0.8, 0.5, 0.3])
    U, s, V, C = known_svd(40, 36, sig2, 4)
    Omega = np.random.default_rng(5).standard_normal((36, 14))
    ok &= rel(mod.randomized_svd_truncation(C, 6, Omega, 1), (U[:, :6] * s[:6]) @ V[:, :6].T) <= 1e-10
    return bool(ok)


def test_planted_mistakes_in_the_truncation_are_caught():
    assert _pins_pass(_variant("x", "x"))
    mistakes = [
        ("return (U[:, :r] * s[:r]) @ Vt[:r]", "return (U[:, :r] * s[:r]) @ Vt[1:r + 1]"),     # wrong index
        ("return (U[:, :r] * s[:r]) @ Vt[:r]", "return U[:, :r] @ Vt[:r]"),                   # dropped sigma
        ("B = Q.T @ C", "B = Q.T @ C.T.T[:, ::-1]"),                                          # permuted operand
        ("r = min(r, len(s))\n    return (Q", "r = min(r + 1, len(s))\n    return (Q"),       # off by one rank
    ]
    for old, new in mistakes:
        assert not _pins_pass(_variant(old, new)), new
